// Request loop behind ruqlp_submit / ruqlp_poll: decompositions arrive at
// any time, are admitted as execution slots and HBM budget free up, and run
// concurrently on the device (continuous batching).
//
// One scheduler thread per handle owns `max_slots` slots; a slot is a child
// handle with its own stream and workspace arena.  Each pass of the loop
//   1. retires the slots whose work has completed (a CUDA event per launch),
//      publishing flags, status and completion time of their requests;
//   2. admits queued requests in arrival order into idle slots: a run of
//      consecutive batchable requests (small dense FP32/BF16, same dtype and
//      q) becomes one batched launch (ruqlp_decompose_batch's device path,
//      up to `max_batch` items); any other request runs alone; a launch is
//      admitted only while the arenas of all slots fit the budget;
//   3. sleeps until a submit arrives or ~20 us pass while work is in flight.
// The handle's mutex guards only the queue and the request table: the loop
// takes it to pick and pop requests and to publish results, and does its
// CUDA work (launches, completion handling, freeing idle arenas) without it,
// so ruqlp_submit / ruqlp_poll never wait behind a launch or a cudaFree.
// Requests that arrive while others run are admitted into the next idle
// slot, so their work overlaps on the device.  Because each item of a batch
// gets bitwise the result it gets alone, a request's result does not depend
// on what it was batched with.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ruqlp.h"
#include "ctx.h"

namespace ruqlp {

using Clock = std::chrono::steady_clock;

struct Request {
  ruqlp_matrix A;
  ruqlp_params prm;
  ruqlp_outputs* out = nullptr;  // caller's struct: flags written on completion
  ruqlp_outputs oc;              // copy used for the launch
  bool batch = false;
  size_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  ruqlp_status st = RUQLP_OK;
  std::string err;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// Owned by the scheduler thread; the request data a launch needs is copied
// in (the request table may rehash while the slot runs).
struct Slot {
  ruqlp_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false, batch = false;
  std::vector<uint64_t> ids;
  std::vector<ruqlp_matrix> A;
  std::vector<ruqlp_params> prm;
  std::vector<ruqlp_outputs> outs;
  BatchRun run;
};

struct Server {
  ruqlp_ctx* h = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot> slots;
  std::thread th;
  bool stop = false;
  uint64_t next_id = 1;
  int max_batch = 64;
  Clock::time_point t0 = Clock::now();
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

ruqlp_status make_slot(ruqlp_ctx* parent, Slot& s) {
  if (cudaSetDevice(parent->device) != cudaSuccess) return RUQLP_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess)
    return RUQLP_ERR_CUDA;
  if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess)
    return RUQLP_ERR_CUDA;
  ruqlp_config cfg{};
  cfg.device = parent->device;
  cfg.hbm_budget_bytes = 0;  // the loop enforces the parent's budget over all slots
  cfg.max_slots = 1;
  cfg.cuda_stream = s.stream;
  return ruqlp_create(&s.ctx, &cfg);
}

void free_slot(Slot& s) {
  if (s.ctx) ruqlp_destroy(s.ctx);
  if (s.ev) cudaEventDestroy(s.ev);
  if (s.stream) cudaStreamDestroy(s.stream);
  s.ctx = nullptr;
  s.ev = nullptr;
  s.stream = nullptr;
}

// Whether slot `k` may grow its arena to `need` bytes within the budget.
bool fits(Server& S, int k, size_t need) {
  const size_t budget = S.h->budget;
  if (budget == 0) return true;
  size_t total = 0;
  for (int i = 0; i < (int)S.slots.size(); ++i) {
    const size_t a = S.slots[i].ctx->arena_bytes;
    total += (i == k) ? std::max(a, need) : a;
  }
  return total <= budget;
}

// Release the arenas of idle slots other than k (to make room for k).
void trim_idle(Server& S, int k) {
  for (int i = 0; i < (int)S.slots.size(); ++i) {
    Slot& s = S.slots[i];
    if (i == k || s.busy || !s.ctx->arena) continue;
    cudaFree(s.ctx->arena);
    s.ctx->arena = nullptr;
    s.ctx->arena_bytes = 0;
    for (auto& g : s.ctx->batches)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    s.ctx->batches.clear();
  }
}

void finish_req(Server& S, uint64_t id, ruqlp_status st, uint32_t flags, const std::string& err,
                double t) {
  Request& r = S.reqs[id];
  r.st = st;
  r.err = err;
  r.oc.flags = flags;
  if (r.out) r.out->flags = flags;
  r.t_done = t;
  r.state = 2;
}

// A finished request's result, published under the mutex.
struct Done {
  uint64_t id;
  ruqlp_status st;
  uint32_t flags;
  std::string err;
  double t;
};

void publish(Server& S, std::vector<Done>& done) {
  if (done.empty()) return;
  std::lock_guard<std::mutex> g(S.mu);
  for (const Done& d : done) finish_req(S, d.id, d.st, d.flags, d.err, d.t);
  done.clear();
}

// 1. completions (no lock held: batch_end / single_end synchronise and may
// rerun a flagged item)
bool retire(Server& S) {
  std::vector<Done> done;
  for (auto& s : S.slots) {
    if (!s.busy) continue;
    const cudaError_t q = cudaEventQuery(s.ev);
    if (q == cudaErrorNotReady) continue;
    s.ctx->err.clear();
    if (s.batch) {
      const ruqlp_status st = batch_end(s.ctx, s.run, s.outs.data());
      const double t = S.now();
      for (size_t i = 0; i < s.ids.size(); ++i)
        done.push_back({s.ids[i], st, s.outs[i].flags, s.ctx->err, t});
    } else {
      const ruqlp_status st = single_end(s.ctx, &s.outs[0]);
      done.push_back({s.ids[0], st, s.outs[0].flags, s.ctx->err, S.now()});
    }
    s.busy = false;
    s.ids.clear();
  }
  const bool any = !done.empty();
  publish(S, done);
  return any;
}

// 2. admissions: pick under the mutex, launch without it
bool admit(Server& S) {
  bool any = false;
  for (;;) {
    int k = -1;
    for (int i = 0; i < (int)S.slots.size(); ++i)
      if (!S.slots[i].busy) { k = i; break; }
    if (k < 0) break;
    Slot& s = S.slots[k];
    std::vector<uint64_t> take;
    size_t need = 0;
    bool batch = false;
    {
      std::lock_guard<std::mutex> g(S.mu);
      if (S.queue.empty()) break;
      const Request& r0 = S.reqs[S.queue.front()];
      batch = r0.batch;
      if (batch) {
        for (size_t j = 0; j < S.queue.size() && (int)take.size() < S.max_batch; ++j) {
          const Request& r = S.reqs[S.queue[j]];
          if (!r.batch || r.prm.compute != r0.prm.compute || r.prm.q != r0.prm.q) break;
          if (!take.empty() && !fits(S, k, need + r.bytes)) break;
          take.push_back(S.queue[j]);
          need += r.bytes;
        }
        need += 65536;
      } else {
        take.push_back(S.queue.front());
        need = r0.bytes;
      }
    }
    if (!fits(S, k, need)) {
      trim_idle(S, k);  // cudaFree outside the mutex
      if (!fits(S, k, need)) break;  // wait for running work to free memory
    }
    // only this thread pops, so the picked requests are still at the front
    const double t = S.now();
    s.A.resize(take.size());
    s.prm.resize(take.size());
    s.outs.resize(take.size());
    {
      std::lock_guard<std::mutex> g(S.mu);
      for (size_t j = 0; j < take.size(); ++j) {
        S.queue.pop_front();
        Request& r = S.reqs[take[j]];
        s.A[j] = r.A;
        s.prm[j] = r.prm;
        s.outs[j] = r.oc;
        r.state = 1;
        r.t_start = t;
      }
    }
    copy_options(S.h, s.ctx);
    s.ctx->err.clear();
    s.ids = take;
    s.batch = batch;
    ruqlp_status st;
    if (batch)
      st = batch_begin(s.ctx, (int)take.size(), s.A.data(), s.prm.data(), s.outs.data(), false,
                       &s.run);
    else
      st = single_begin(s.ctx, &s.A[0], &s.prm[0], &s.outs[0]);
    if (st == RUQLP_OK && cudaEventRecord(s.ev, s.stream) != cudaSuccess) st = RUQLP_ERR_CUDA;
    if (st != RUQLP_OK) {
      // the launch failed as a whole: wait for whatever was queued, report
      cudaStreamSynchronize(s.stream);
      std::vector<Done> done;
      for (uint64_t id : take) done.push_back({id, st, 0u, s.ctx->err, S.now()});
      publish(S, done);
      s.ids.clear();
    } else {
      s.busy = true;
    }
    any = true;
  }
  return any;
}

void loop(Server* S) {
  cudaSetDevice(S->h->device);
  for (;;) {
    const bool r = retire(*S);
    const bool a = admit(*S);
    bool busy = false;
    for (auto& s : S->slots) busy = busy || s.busy;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop && !busy && S->queue.empty()) break;
    if (r || a) continue;
    if (busy) S->cv.wait_for(lk, std::chrono::microseconds(20));
    else S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
  }
}

Server* get_server(ruqlp_ctx* h, ruqlp_status* st) {
  std::lock_guard<std::mutex> g(h->server_mu);
  if (h->server) return h->server;
  Server* S = new Server();
  S->h = h;
  S->slots.resize(std::max(1, h->max_slots));
  for (auto& s : S->slots) {
    const ruqlp_status e = make_slot(h, s);
    if (e != RUQLP_OK) {
      for (auto& t : S->slots) free_slot(t);
      delete S;
      *st = e;
      return nullptr;
    }
  }
  S->th = std::thread(loop, S);
  h->server = S;
  return S;
}

}  // namespace

void server_shutdown(ruqlp_ctx* h) {
  Server* S = nullptr;
  {
    std::lock_guard<std::mutex> g(h->server_mu);
    S = h->server;
    h->server = nullptr;
  }
  if (!S) return;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  S->th.join();
  for (auto& s : S->slots) free_slot(s);
  delete S;
}

}  // namespace ruqlp

using namespace ruqlp;

extern "C" {

ruqlp_status ruqlp_submit(ruqlp_handle h, const ruqlp_matrix* A, const ruqlp_params* prm,
                          ruqlp_outputs* out, uint64_t* ticket) {
  if (!h) return RUQLP_ERR_INVALID;
  if (!ticket) return set_error(h, RUQLP_ERR_INVALID, "NULL ticket");
  *ticket = 0;
  int d = 0;
  ruqlp_status st = check_request(h, A, prm, out, &d);
  if (st != RUQLP_OK) return st;
  Request r;
  r.A = *A;
  r.prm = *prm;
  r.out = out;
  r.oc = *out;
  r.batch = batchable(A, prm);
  r.bytes = r.batch ? batch_item_bytes(A, prm) : single_bytes(A, prm);
  if (h->budget && r.bytes + (r.batch ? 65536 : 0) > h->budget)
    return set_error(h, RUQLP_ERR_BUDGET, "the request's workspace exceeds the HBM budget");
  Server* S = get_server(h, &st);
  if (!S) return set_error(h, st, "could not start the request loop");
  {
    std::lock_guard<std::mutex> g(S->mu);
    r.t_submit = S->now();
    const uint64_t id = S->next_id++;
    S->reqs.emplace(id, r);
    S->queue.push_back(id);
    *ticket = id;
  }
  S->cv.notify_all();
  return RUQLP_OK;
}

ruqlp_status ruqlp_poll_times(ruqlp_handle h, uint64_t ticket, ruqlp_request_times* times) {
  if (!h) return RUQLP_ERR_INVALID;
  Server* S;
  {
    std::lock_guard<std::mutex> g(h->server_mu);
    S = h->server;
  }
  if (!S) return set_error(h, RUQLP_ERR_INVALID, "unknown ticket");
  ruqlp_status st;
  std::string err;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return set_error(h, RUQLP_ERR_INVALID, "unknown ticket");
    Request& r = it->second;
    if (r.state != 2) return RUQLP_NOT_READY;
    if (times) {
      times->submit_s = r.t_submit;
      times->start_s = r.t_start;
      times->done_s = r.t_done;
    }
    st = r.st;
    err = r.err;
    S->reqs.erase(it);
  }
  if (st != RUQLP_OK) return set_error(h, st, err.c_str());
  return RUQLP_OK;
}

ruqlp_status ruqlp_poll(ruqlp_handle h, uint64_t ticket) {
  return ruqlp_poll_times(h, ticket, nullptr);
}

}  // extern "C"
