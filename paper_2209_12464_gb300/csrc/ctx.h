// Library handle (struct ruqlp_ctx) and the internal entry points shared by
// the synchronous API and the request loop of ruqlp_submit / ruqlp_poll.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/ruqlp.h"
#include "common.cuh"

namespace ruqlp {
struct Server;
}

struct ruqlp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  int max_slots = 8;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  ruqlp::DevStatus* status = nullptr;       // device
  ruqlp::DevStatus* status_host = nullptr;  // pinned host
  std::string err;
  // policy knobs (ruqlp_set_option)
  int orth_fp64 = 0;    // FP32/BF16 paths: CholeskyQR2 with FP64 Gram and Cholesky
  int orth_full = 0;    // 1: every orth() takes three CholeskyQR passes (else the
                        // intermediate ones take two)
  int bf16_simt = 0;    // 1: BF16 products on CUDA cores instead of tensor cores
  int orth_simt = 0;    // 1: orth() Grams and Q = Y R^{-1} on CUDA cores
  int batch_orth_tc = 0;  // 1: batched BF16 items with dp <= 80 take the tensor-core passes
  int orth_tsqr = 0;    // 1: every orth() is a Householder TSQR
  int tc_nsplit = 0;    // tensor-core products: column split (0 = tuned per shape)
  int test_withhold = 0;  // test hook: the next tensor-core products run out a wait
  bool tsqr_now = false;  // this run takes the TSQR orth() (fallback rerun)
  // the last single decomposition's arguments, for its TSQR rerun
  ruqlp_matrix last_A{};
  ruqlp_params last_prm{};
  ruqlp_outputs last_out{};
  // phase timing with CUDA events on the handle's stream (option "profile")
  bool profile = false;
  struct Span { int cat; cudaEvent_t a, b; };
  std::vector<Span> spans;
  std::vector<cudaEvent_t> pool;
  // batched decompositions, per batch signature (shapes, q, dtype, product
  // kernels, arena address): the captured launch sequence and the host image
  // of the tensor maps
  struct BatchEntry {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
    int seen = 0;
    int64_t launches = 0;           // kernels in the captured graph
    std::vector<uint8_t> maps;      // the tensor maps of every matrix
    std::vector<const void*> aptr;  // A each A map was encoded for
    std::vector<int64_t> alda;
  };
  std::vector<BatchEntry> batches;
  void* stage = nullptr;  // pinned staging of the batch metadata
  size_t stage_bytes = 0;
  int batch_graphs = 1;  // option "batch_graph"
  cudaStream_t cap_stream = nullptr;  // capture stream (the legacy stream cannot capture)
  // host-buffer entry: large copies split over these streams (more copy
  // engines), joined back into `stream` by events
  static constexpr int kCopyStreams = 4;
  cudaStream_t copy_streams[kCopyStreams] = {};
  cudaEvent_t copy_ev[kCopyStreams + 1] = {};
  // per profile phase (the kProfNames list of ruqlp_api.cu, which checks
  // that its length matches)
  static constexpr int kProfPhases = 10;
  int64_t prof_count[kProfPhases] = {};
  double prof_ms[kProfPhases] = {};
  // request loop of ruqlp_submit / ruqlp_poll (created on the first submit)
  ruqlp::Server* server = nullptr;
  std::mutex server_mu;
};


namespace ruqlp {

// A batched launch in flight on a handle's stream (the two halves of
// ruqlp_decompose_batch).
struct BatchRun {
  int count = 0;
  size_t off_status = 0, off_err = 0;
  // the items, for the TSQR rerun of any that CholeskyQR could not handle
  std::vector<ruqlp_matrix> A;
  std::vector<ruqlp_params> prm;
};

// Validate and launch one decomposition on h's stream and arena (returns
// before completion); single_end waits for it and reports flags and errors.
ruqlp_status single_begin(ruqlp_ctx* h, const ruqlp_matrix* A, const ruqlp_params* prm,
                          const ruqlp_outputs* out);
ruqlp_status single_end(ruqlp_ctx* h, ruqlp_outputs* out);
// Same for a batch (graphs: reuse or capture the launch sequence).
ruqlp_status batch_begin(ruqlp_ctx* h, int count, const ruqlp_matrix* A, const ruqlp_params* prm,
                         const ruqlp_outputs* out, bool graphs, BatchRun* run);
ruqlp_status batch_end(ruqlp_ctx* h, const BatchRun& run, ruqlp_outputs* out);
// Validation only (no device work); d receives k + p.
ruqlp_status check_request(ruqlp_ctx* h, const ruqlp_matrix* A, const ruqlp_params* prm,
                           const ruqlp_outputs* out, int* d);
// Workspace bytes of one decomposition alone, and of one item inside a batch
// (an upper bound of its share of the batch arena).
size_t single_bytes(const ruqlp_matrix* A, const ruqlp_params* prm);
size_t batch_item_bytes(const ruqlp_matrix* A, const ruqlp_params* prm);
// Whether the request loop batches this request: dense, FP32/BF16, d <= 256
// (the batched tensor-core product's widest N), at most 2^25 elements, no
// finish_paper.  Larger requests run alone on the single-matrix path.
bool batchable(const ruqlp_matrix* A, const ruqlp_params* prm);
void copy_options(const ruqlp_ctx* from, ruqlp_ctx* to);
ruqlp_status set_error(ruqlp_ctx* h, ruqlp_status s, const char* msg);
// Request loop teardown (waits for every submitted request).
void server_shutdown(ruqlp_ctx* h);

}  // namespace ruqlp
