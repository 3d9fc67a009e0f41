"""RU-QLP benchmark: GB/s of A streamed on the dense 20000 x 20000 workload.

One step = one whole RU-QLP decomposition (Algorithm 1 + Algorithm 2,
Section III) of a device-resident A: sketch, q power steps with orth() after
every product, B^T = A^T Q and its QR.  The workload is the dense
20000 x 20000 matrix A = U diag(sigma) V^T + N with U, V Haar, sigma_i = 1
(i <= 200), 1e-2/(i-200) after, N iid N(0, 1e-12), k=200, p=20, q=2
(6 passes over A).  Metric: (2q+2) * bytes(A in the streamed dtype) / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype bf16|f32|f64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)
  python bench.py --workload batch [--dtype bf16|f32]   (512 uneven matrices:
      m log-uniform in [256, 4096], n in [128, 2048], k uniform in [8, 64],
      p=8, q=1, same spectrum form; one ruqlp_decompose_batch call per step)
  python bench.py --workload csr [--dtype f32|bf16]   (CSR 200000 x 100000,
      0.1 % uniform pattern, N(0,1) values + planted rank-100 term of scale 10,
      k=100, p=10, q=1; values in FP32 or BF16)
  python bench.py --workload csrlr   (the same pattern with N(0,1) values plus
      a rank-100 term X D Y^T kept as factors, D from 200 down to 2)
  python bench.py --workload serve [--duration S] [--rate R]   (Poisson
      arrivals at R/s: 95 % shaped like the batched workload, 5 % dense
      16384 x 8192 with k=256, p=16, q=2; BF16; 150 GB budget; p50/p99)

Under torchrun each rank runs its own replica of the workload (weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, K_RANK, P_OVER, Q_POW = 20000, 20000, 200, 20, 2
TAIL, NOISE = 1e-2, 1e-6
SEED = 20260 + 1
DT_BYTES = {"bf16": 2, "f32": 4, "f64": 8}
METRIC = "RU-QLP GB/s of A streamed vs HBM peak at fixed residual"
WORKLOAD = "dense 20000x20000, sigma_i=1 (i<=200) then 1e-2/(i-200), +N(0,1e-6^2); k=200 p=20 q=2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--dtype", default="bf16", choices=list(DT_BYTES))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--size", type=int, default=0, help="override m = n (testing only)")
    ap.add_argument("--workload", default="dense",
                    choices=["dense", "batch", "serve", "csr", "csrlr", "orth"],
                    help="dense: one 20000 x 20000 matrix (the metric's workload); batch: "
                         "512 matrices of uneven shapes in one batched call; serve: Poisson "
                         "arrivals through ruqlp_submit / ruqlp_poll; orth: ruqlp_orth of a "
                         "20000 x 220 FP32 matrix (the dense workload's sketch shape)")
    ap.add_argument("--duration", type=float, default=2.0,
                    help="seconds of arrivals (serve workload)")
    ap.add_argument("--rate", type=float, default=2000.0, help="arrivals per second (serve)")
    ap.add_argument("--count", type=int, default=512, help="batch size (batch workload)")
    ap.add_argument("--tune-file", default="",
                    help="product tuner cache (ruqlp_tune_file): read at start, measured "
                         "choices appended; pins the tuner's choices for a profiled rerun")
    ap.add_argument("--gen", default="haar", choices=["haar", "fast"],
                    help="haar: the workload's Haar U, V (torch.linalg.qr); fast: Gaussian "
                         "low-rank stand-in for profiling tools that cannot load torch.linalg")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(torch, dist, world, x, device):
    """The largest x over the ranks (the slowest rank sets the job's time);
    x itself on one rank."""
    if world <= 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units every rank processed (the same on each
    rank: weak scaling) over the slowest rank's time."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def make_inputs(torch, device, dtype, m, n, gen="haar"):
    """A in the streamed dtype, the FP32 original it was rounded from (for the
    residual), Omega (FP64) and the spectrum."""
    from paper_2209_12464_gb300 import workloads as wl
    sig = wl.spectrum_gap(min(m, n), K_RANK, TAIL)
    if gen == "haar":
        A32 = wl.dense_spectral_torch(SEED, m, n, sig, noise_std=NOISE, device=device,
                                      dtype=torch.float32)
    else:
        A32 = wl.dense_lowrank_gauss_torch(SEED, m, n, K_RANK, noise_std=NOISE, device=device)
    A = A32.to({"bf16": torch.bfloat16, "f32": torch.float32, "f64": torch.float64}[dtype])
    Om = wl.omega_torch(SEED + 1, n, K_RANK + P_OVER, device=device)
    return A, A32, Om, sig


def tc_traffic(m, n, d):
    """DRAM bytes per product launch from the committed ncu summary (a
    10240^2 capture scaled to the 20000^2 launch), for that workload only."""
    if (m, n, d) != (M, N, K_RANK + P_OVER):
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", "k_tc_gemm_dense10240_bf16.md")).read()
    except OSError:
        return None
    import re
    mt = re.search(r"traffic_bytes_per_launch_scaled_20000:\s*(\d+)", txt)
    return int(mt.group(1)) if mt else None


def residual_gpu(torch, A, Q, L, P):
    """||A - Q L P^T||_F / ||A||_F in FP64 on the device (measurement only)."""
    A64 = A.double()
    E = A64 - (Q.double() @ L.double()) @ P.double().T
    return float(torch.linalg.norm(E) / torch.linalg.norm(A64))


def cpu_baseline(dtype, rows):
    """Time the FP64 oracle, as it stands, on the leading `rows` rows of the
    workload (a bounded sample), in a spawned process using every host core."""
    code = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
import oracle
from paper_2209_12464_gb300 import workloads as wl
rows, n, k, p, q = %d, %d, %d, %d, %d
rng = np.random.default_rng(5)
sig = wl.spectrum_gap(rows, k, %r)
A, _, _, _ = wl.dense_spectral(11, rows, n, sig, noise_std=%r)
Om = wl.omega(12, n, k + p)
t0 = time.perf_counter()
oracle.ruqlp(A, Om, q)
t = time.perf_counter() - t0
print(json.dumps({"seconds": t}))
""" % (ROOT, rows, N, K_RANK, P_OVER, Q_POW, TAIL, NOISE)
    env = dict(os.environ)
    cores = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-400:]}
    t = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    gbytes = (2 * Q_POW + 2) * rows * N * DT_BYTES[dtype] / 1e9
    return {"value": gbytes / t, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "seconds": t,
            "sample": f"oracle.ruqlp (FP64 numpy, own Householder QR) on a {rows} x {N} row "
                      f"sample of the workload (same spectrum form, k={K_RANK}, p={P_OVER}, "
                      f"q={Q_POW}); bytes counted as (2q+2) x {rows}x{N} x {DT_BYTES[dtype]} B "
                      f"({dtype}) so the ratio is the time per decomposition"}


def oracle_full(A32, Om, q, L_gpu, resid_gpu):
    """The FP64 oracle, as it stands, on the whole workload matrix the GPU
    decomposed (the unrounded FP32 A, widened to FP64) and the same Omega, in a
    spawned process using every host core: its wall time (the CPU baseline on
    the full configuration) and the error of the GPU result against it --
    the residual ratio and max_i | |L_ii| - |L_ii^oracle| | / |L_11^oracle|."""
    import numpy as np
    tmp = tempfile.mkdtemp(prefix="ruqlp_oracle_")
    fa, fo, fr = (os.path.join(tmp, x) for x in ("A.npy", "Om.npy", "res.npz"))
    try:
        np.save(fa, A32.cpu().numpy())
        np.save(fo, Om.cpu().numpy())
        code = r"""
import sys, time, json
sys.path.insert(0, %r)
import numpy as np
import oracle
A = np.load(%r).astype(np.float64)
Om = np.load(%r)
t0 = time.perf_counter()
ref = oracle.ruqlp(A, Om, %d)
t = time.perf_counter() - t0
r0 = oracle.residual_fro(A, ref["Q"], ref["L"], ref["P"])
np.savez(%r, diag=np.diag(ref["L"]), r0=r0, seconds=t)
print(json.dumps({"seconds": t}))
""" % (ROOT, fa, fo, q, fr)
        env = dict(os.environ)
        cores = os.cpu_count() or 1
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(cores)
        env["CUDA_VISIBLE_DEVICES"] = ""
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=1800)
        if r.returncode != 0:
            return None, {"error": r.stderr[-400:]}
        z = np.load(fr)
        dg = np.abs(np.diag(L_gpu.double().cpu().numpy()))
        do = np.abs(z["diag"])
        r0 = float(z["r0"])
        acc = {"oracle_residual_fro": r0, "residual_ratio_to_oracle": resid_gpu / r0,
               "max_abs_diagL_dev_rel_L11": float(np.max(np.abs(dg - do)) / do[0]),
               "oracle": "oracle.ruqlp, FP64, same A (unrounded FP32 values) and Omega"}
        return float(z["seconds"]), acc
    finally:
        for x in (fa, fo, fr):
            if os.path.exists(x):
                os.remove(x)
        os.rmdir(tmp)


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each timed step is one whole decomposition of the workload's full-size
    matrix (built on the host: torch's CPU generator, the same shape and
    spectrum form as the GPU arm's matrix); the warm-up steps run a 300-row
    sample so the arm stays within a few minutes."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_baseline(args.dtype, 300)
    m = n = args.size or M
    code = r"""
import sys, time, json
sys.path.insert(0, %r)
import numpy as np, torch
import oracle
from paper_2209_12464_gb300 import workloads as wl
m, n, k, p, q, steps = %d, %d, %d, %d, %d, %d
sig = wl.spectrum_gap(min(m, n), k, %r)
A = wl.dense_spectral_torch(%d, m, n, sig, noise_std=%r, device="cpu").double().numpy()
Om = np.random.default_rng(%d).standard_normal((n, k + p))
secs = []
for _ in range(steps):
    t0 = time.perf_counter()
    oracle.ruqlp(A, Om, q)
    secs.append(time.perf_counter() - t0)
print(json.dumps({"seconds": secs}))
""" % (ROOT, m, n, K_RANK, P_OVER, Q_POW, max(args.steps, 1), TAIL, SEED, NOISE, SEED + 1)
    env = dict(os.environ)
    cores = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=3600)
    if r.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + r.stderr[-300:]}))
        return 0
    secs = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
    t = statistics.median(secs)
    gb = (2 * Q_POW + 2) * m * n * DT_BYTES[args.dtype] / 1e9
    v = gb / t
    sample = (f"the full workload: oracle.ruqlp (FP64 numpy, own Householder QR) on a {m} x {n} "
              f"matrix of the workload's form (k={K_RANK}, p={P_OVER}, q={Q_POW}); bytes counted "
              f"as (2q+2) x bytes(A in {args.dtype}) so the ratio is the time per decomposition")
    out = {"metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "m": m, "n": n, "k": K_RANK, "p": P_OVER, "q": Q_POW,
                      "l2": "inputs larger than L2 (host run)",
                      "warmup_sample_rows": 300},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": v,
                            "unit": "GB/s"},
           "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------
B_SEED, B_P, B_Q = 20260 + 3, 8, 1
B_WORKLOAD = ("batched: 512 dense matrices, m log-uniform [256,4096], n log-uniform [128,2048], "
              "k uniform [8,64], p=8, q=1, sigma_i=1 (i<=k) then 1e-2/(i-k)")


def two_part_roofline(prof, flops, nbytes, peaks):
    """The two-part last product B^T = A^T Q: two BF16 MMAs per A tile
    (2 x 2 x rows x cols x dp flop) over one pass of A (nbytes: A, both BF16
    parts of the skinny operand, the FP32 output).  Its roofline is the
    larger of the two times at peak: the tensor pipe (sustained BF16 peak:
    timed inside the step) for wide sketches, HBM for narrow ones."""
    cnt, tot = prof
    avg = tot / max(cnt, 1)
    tpk = peaks.get("bf16_tflops_sustained", 1700.0)
    hpk = peaks.get("hbm_gbs", 6800.0)
    if flops / (tpk * 1e12) >= nbytes / (hpk * 1e9):
        achieved = flops / (avg * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": tpk, "unit": "TFLOP/s",
                "frac": achieved / tpk, "alg_flops_per_launch": flops, "avg_launch_ms": avg,
                "launches": cnt,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"}
    achieved = nbytes / (avg * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hpk, "unit": "GB/s",
            "frac": achieved / hpk, "alg_bytes_per_launch": nbytes, "avg_launch_ms": avg,
            "launches": cnt, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}


def batch_inputs(torch, dev, count, dtype, gen):
    from paper_2209_12464_gb300 import workloads as wl
    shapes = wl.batch_shapes(B_SEED, count=count, p=B_P)
    A32, Om = [], []
    for i, (m, n, k, p) in enumerate(shapes):
        if gen == "haar":
            A32.append(wl.dense_spectral_torch(B_SEED + 1000 + i, m, n,
                                               wl.spectrum_gap(min(m, n), k, TAIL), device=dev))
        else:
            A32.append(wl.dense_lowrank_gauss_torch(B_SEED + 1000 + i, m, n, k, device=dev))
        Om.append(wl.omega_torch(B_SEED + 5000 + i, n, k + p, device=dev))
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32}[dtype]
    # rows start on 16-byte boundaries (what the tensor-map loads need)
    A = [wl.aligned_rows(a.to(tdt)) for a in A32]
    return shapes, A, A32, Om


def batch_cpu_baseline(dtype, count, items):
    """The FP64 oracle on the first `items` matrices of the batch (a bounded
    sample), in a spawned process using every host core."""
    code = r"""
import sys, time, json
sys.path.insert(0, %r)
import oracle
from paper_2209_12464_gb300 import workloads as wl
shapes = wl.batch_shapes(%d, count=%d, p=%d)[:%d]
mats = []
for i, (m, n, k, p) in enumerate(shapes):
    A, _, _, _ = wl.dense_spectral(31 + i, m, n, wl.spectrum_gap(min(m, n), k, %r))
    mats.append((A, wl.omega(77 + i, n, k + p)))
t0 = time.perf_counter()
for A, Om in mats:
    oracle.ruqlp(A, Om, %d)
t = time.perf_counter() - t0
el = sum(m * n for m, n, k, p in shapes)
print(json.dumps({"seconds": t, "elements": el, "items": len(shapes)}))
""" % (ROOT, B_SEED, count, B_P, items, TAIL, B_Q)
    env = dict(os.environ)
    cores = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-400:]}
    j = json.loads(r.stdout.strip().splitlines()[-1])
    gbytes = (2 * B_Q + 2) * j["elements"] * DT_BYTES[dtype] / 1e9
    return {"value": gbytes / j["seconds"], "unit": "GB/s", "cores": cores, "kind": "oracle",
            "seconds": j["seconds"], "decompositions_per_s": j["items"] / j["seconds"],
            "sample": f"oracle.ruqlp (FP64 numpy) on the first {j['items']} matrices of the "
                      f"batch (same shapes and spectrum form), bytes counted in {dtype}"}


def run_batch(args, torch, dev, local, world, rank, dist):
    from paper_2209_12464_gb300 import ruqlp
    if args.dtype not in ("bf16", "f32"):
        raise SystemExit("the batched workload runs in bf16 or f32")
    shapes, A, A32, Om = batch_inputs(torch, dev, args.count, args.dtype, args.gen)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    h = ruqlp.Handle(local, stream.cuda_stream)
    ks, ps = [s[2] for s in shapes], [s[3] for s in shapes]
    batch = h.prepare_batch(A, Om, ks, B_P, B_Q, ps=ps)
    for _ in range(max(args.warmup, 3)):
        batch.run()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ruqlp.ruqlp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    flags = 0
    for _ in range(args.steps):
        for f in batch.run():
            flags |= f
    e1.record(stream)
    torch.cuda.synchronize()
    launches = (ruqlp.ruqlp_launch_count() - l0) // max(args.steps, 1)
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    ms = max_over_ranks(torch, dist, world, ms, dev)
    passes = 2 * B_Q + 2
    elements = sum(m * n for m, n, k, p in shapes)
    bytes_a = elements * DT_BYTES[args.dtype]
    value = job_rate(world, passes * bytes_a / 1e9, ms * 1e-3)
    dps = job_rate(world, len(shapes), ms * 1e-3)

    # accuracy on a sample (relative residuals, FP64 on the device): the
    # batched result and the plain single-matrix FP32 path on the same
    # matrix values (for BF16, the BF16 values widened to FP32: equal inputs,
    # so the ratio isolates the BF16 arithmetic), and both against the
    # unrounded FP32 matrix (which adds the BF16 rounding of A itself)
    rng = __import__("numpy").random.default_rng(3)
    sample = sorted(rng.choice(len(shapes), 16, replace=False).tolist())
    res_b, res_1, res_bu, res_1u = [], [], [], []
    for i in sample:
        Q, L, P = batch.outs[i]
        Aw = A[i].float()  # the values the batched call saw
        res_b.append(residual_gpu(torch, Aw, Q, L, P))
        Q1, L1, P1, _ = h.decompose(Aw, Om[i], ks[i], ps[i], B_Q, out_dtype=torch.float32)
        res_1.append(residual_gpu(torch, Aw, Q1, L1, P1))
        res_bu.append(residual_gpu(torch, A32[i], Q, L, P))
        Q1, L1, P1, _ = h.decompose(A32[i], Om[i], ks[i], ps[i], B_Q, out_dtype=torch.float32)
        res_1u.append(residual_gpu(torch, A32[i], Q1, L1, P1))
    ratio = max(b / o for b, o in zip(res_b, res_1))
    ratio_u = max(b / o for b, o in zip(res_bu, res_1u))

    # the plain single-instance FP32 form: one ruqlp_decompose per matrix
    outs1 = [(torch.empty(m, k + p, device=dev), torch.empty(k + p, k + p, device=dev),
              torch.empty(n, k + p, device=dev)) for m, n, k, p in shapes]
    for i in range(len(shapes)):
        h.decompose(A32[i], Om[i], ks[i], ps[i], B_Q, outs=outs1[i])
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for i in range(len(shapes)):
        h.decompose(A32[i], Om[i], ks[i], ps[i], B_Q, outs=outs1[i])
    s1.record(stream)
    torch.cuda.synchronize()
    ms1 = s0.elapsed_time(s1)
    single = {"decompositions_per_s": len(shapes) / (ms1 * 1e-3), "ms_per_batch": ms1,
              "form": "ruqlp_decompose per matrix, FP32 A, FP32 compute"}
    del outs1

    # live per-phase timing (eager batched launches, CUDA events on the stream)
    h.set_option("profile", 1)
    for _ in range(2):
        batch.run()
    torch.cuda.synchronize()
    prof = {ph: h.profile(ph) for ph in ("ax", "atx", "orth", "step", "tc_ax", "tc_atx",
                                         "tc_atx2")}
    h.set_option("profile", 0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_mhz = ck.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    step_ms = prof["step"][1] / max(prof["step"][0], 1)
    common = {"phase_ms": {ph: prof[ph][1] / max(prof[ph][0], 1) for ph in prof},
              "phase_share": {ph: prof[ph][1] / max(prof["step"][1], 1e-9)
                              for ph in ("ax", "atx", "orth")},
              "eager_step_ms": step_ms}
    if prof["tc_ax"][0]:
        # the batched tcgen05 product: one pass over every A_i per launch.
        # Algorithmic bytes = sum_i A_i (BF16) + Bt_i (dp x K, BF16) + the
        # output (rows x dp, FP32); both orientations move the same bytes.
        dpad = [(k + p + 15) // 16 * 16 for m, n, k, p in shapes]
        alg = bytes_a + sum(dp * (2 * n + 4 * m) for (m, n, k, p), dp in zip(shapes, dpad))
        cnt = prof["tc_ax"][0] + prof["tc_atx"][0]
        avg = (prof["tc_ax"][1] + prof["tc_atx"][1]) / cnt
        achieved = alg / (avg * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": None,
                    "kernel": "k_btc_gemm (batched tcgen05 products over a tile list, one pass "
                              "over every A_i per launch; one-part skinny operand)",
                    "alg_bytes_per_launch": alg, "avg_launch_ms": avg, "launches": cnt,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", **common}
        if prof["tc_atx2"][0]:
            flops2 = 4.0 * sum(m * n * dp for (m, n, k, p), dp in zip(shapes, dpad))
            bytes2 = bytes_a + sum(dp * (4 * m + 4 * n) for (m, n, k, p), dp in zip(shapes, dpad))
            roofline["two_part_launch"] = two_part_roofline(prof["tc_atx2"], flops2, bytes2,
                                                            peaks)
    else:
        cnt = prof["ax"][0] + prof["atx"][0]
        avg = (prof["ax"][1] + prof["atx"][1]) / max(cnt, 1)
        flops = 2.0 * sum(m * n * (k + p) for m, n, k, p in shapes)
        alu_peak = 152 * 256 * sm_mhz * 1e6 / 1e12
        achieved = flops / (avg * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None,
                    "kernel": "k_bgemm (batched CUDA-core product, one pass over every A_i per "
                              "launch)",
                    "alg_flops_per_launch": flops, "avg_launch_ms": avg, "launches": cnt,
                    "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 x median SM clock",
                    **common}

    # end to end: pinned host inputs -> device, batched call, outputs -> host.
    # The batch's inputs and outputs each live in one packed buffer (every
    # item at a 256-byte aligned offset, A_i with its 16-byte row pitch), as
    # a caller holding a batch would keep them, so each direction is one
    # copy per buffer rather than one per item.
    e2e = None
    if not args.no_e2e:
        def pack(tensors, dtype):
            # one device buffer holding each 2-D tensor at an aligned offset
            es = torch.empty((), dtype=dtype).element_size()
            offs, tot = [], 0
            for t in tensors:
                offs.append(tot)
                tot += (t.shape[0] * t.stride(0) * es + 255) // 256 * 256
            buf = torch.empty(tot // es, dtype=dtype, device=dev)
            views = [buf.as_strided(tuple(t.shape), (t.stride(0), 1), o // es)
                     for t, o in zip(tensors, offs)]
            return buf, views
        Ad, Av = pack(A, A[0].dtype)
        for v, a in zip(Av, A):
            v.copy_(a)
        Omd, Omv = pack(Om, torch.float64)
        for v, o in zip(Omv, Om):
            v.copy_(o)
        outs_t = [(torch.empty(m, k + p, device=dev), torch.empty(k + p, k + p, device=dev),
                   torch.empty(n, k + p, device=dev)) for m, n, k, p in shapes]
        Od, Ov = pack([t for o in outs_t for t in o], torch.float32)
        outs_v = [tuple(Ov[3 * i:3 * i + 3]) for i in range(len(shapes))]
        be = h.prepare_batch(Av, Omv, ks, B_P, B_Q, ps=ps, outs=outs_v)
        Ah = Ad.cpu().pin_memory()
        Oh = Omd.cpu().pin_memory()
        Rh = torch.empty(Od.shape, dtype=Od.dtype).pin_memory()
        bi = Ah.numel() * Ah.element_size() + Oh.numel() * Oh.element_size()
        bo = Rh.numel() * Rh.element_size()
        be.run()  # first sighting of this batch's buffers
        be.run()
        ke = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            Ad.copy_(Ah, non_blocking=True)
            Omd.copy_(Oh, non_blocking=True)
            be.run()
            Rh.copy_(Od, non_blocking=True)
            torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / ke
        te = max_over_ranks(torch, dist, world, te, dev)
        e2e = {"value": job_rate(world, passes * bytes_a / 1e9, te), "unit": "GB/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": te * 1e3,
               "decompositions_per_s": job_rate(world, len(shapes), te),
               "layout": "inputs and outputs in one packed pinned buffer per kind (3 copies)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = batch_cpu_baseline(args.dtype, args.count, 24)
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": args.dtype, "data": "synthetic",
               "config": {"workload": B_WORKLOAD if args.gen == "haar" else
                          "Gaussian low-rank stand-in of the batched shapes (profiling)",
                          "count": len(shapes), "p": B_P, "q": B_Q, "passes": passes,
                          "bytes_A": bytes_a,
                          "l2": "inputs larger than L2 (%.0f MB of A vs 129 MB L2)" % (bytes_a / 1e6),
                          "parallelism": f"replicas x{world}"},
               "decompositions_per_s": dps,
               "single_fp32": single,
               "accuracy": {"sample": len(sample), "residual_fro_max": max(res_b),
                            "max_ratio_vs_single_fp32_same_values": ratio,
                            "max_ratio_vs_single_fp32_on_unrounded_A": ratio_u,
                            "flags": flags},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": ck}
        print(json.dumps(out))
    h.close()
    return 0



# ---------------------------------------------------------------------------
# serving workload
# ---------------------------------------------------------------------------
S_SEED = 20260 + 4
S_BIG = (16384, 8192, 256, 16, 2)
S_BUDGET = 150 * 10 ** 9


def run_serve(args, torch, dev, local, world, rank, dist):
    import numpy as np
    from paper_2209_12464_gb300 import ruqlp
    from paper_2209_12464_gb300 import workloads as wl
    # input pool (generation is not timed): 256 small matrices of the batched
    # workload's shapes and 4 big ones
    shapes = wl.batch_shapes(S_SEED, count=256, p=B_P)
    small = []
    for i, (m, n, k, p) in enumerate(shapes):
        if args.gen == "haar":
            A = wl.dense_spectral_torch(S_SEED + 100 + i, m, n, wl.spectrum_gap(min(m, n), k, TAIL),
                                        device=dev)
        else:
            A = wl.dense_lowrank_gauss_torch(S_SEED + 100 + i, m, n, k, device=dev)
        small.append((wl.aligned_rows(A.bfloat16()), wl.omega_torch(S_SEED + 600 + i, n, k + p,
                                                                     device=dev), k, p, B_Q))
    bm, bn, bk, bp, bq = S_BIG
    big = []
    for i in range(4):
        if args.gen == "haar":
            A = wl.dense_spectral_torch(S_SEED + 900 + i, bm, bn, wl.spectrum_gap(bn, bk, TAIL),
                                        device=dev, dtype=torch.bfloat16)
        else:
            A = wl.dense_lowrank_gauss_torch(S_SEED + 900 + i, bm, bn, bk, device=dev).bfloat16()
        big.append((A, wl.omega_torch(S_SEED + 950 + i, bn, bk + bp, device=dev), bk, bp, bq))
    torch.cuda.synchronize()
    h = ruqlp.Handle(local, torch.cuda.current_stream(dev).cuda_stream,
                     hbm_budget_bytes=S_BUDGET, max_slots=4)
    rng = np.random.default_rng(S_SEED)

    def run(nreq, rate, seed):
        arr = wl.poisson_arrivals(seed, rate, nreq)
        kinds = rng.random(nreq) < 0.05
        picks = rng.integers(0, 256, nreq)
        bigs = rng.integers(0, 4, nreq)
        tickets, pend = [], []
        t0 = time.perf_counter()
        for j in range(nreq):
            while time.perf_counter() - t0 < arr[j]:
                pend = [t for t in pend if not h.poll(t)]
            A, om, k, p, q = big[bigs[j]] if kinds[j] else small[picks[j]]
            t = h.submit(A, om, k, p, q)
            t.big = bool(kinds[j])
            t.bytes = A.shape[0] * A.shape[1] * 2 * (2 * q + 2)
            tickets.append(t)
            pend.append(t)
        while pend:
            pend = [t for t in pend if not h.poll(t)]
        return tickets

    run(max(100, int(0.1 * args.rate)), args.rate, S_SEED + 1)  # warm-up
    nreq = max(1, int(args.duration * args.rate))
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    l0 = ruqlp.ruqlp_launch_count()
    tickets = run(nreq, args.rate, S_SEED + 2)
    launches = ruqlp.ruqlp_launch_count() - l0
    ck = clocks.stop()
    lat = np.array([(t.times[2] - t.times[0]) * 1e3 for t in tickets])
    lat_b = np.array([(t.times[2] - t.times[0]) * 1e3 for t in tickets if t.big])
    lat_s = np.array([(t.times[2] - t.times[0]) * 1e3 for t in tickets if not t.big])
    wall = max(t.times[2] for t in tickets) - min(t.times[0] for t in tickets)
    dps = len(tickets) / wall
    gbs = sum(t.bytes for t in tickets) / wall / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    pct = lambda a, q_: float(np.percentile(a, q_)) if len(a) else None
    flags = 0
    for t in tickets:
        flags |= t.flags
    out = {"metric": "RU-QLP serving: decompositions/s with p50/p99 latency", "value": dps,
           "unit": "decompositions/s", "n_gpus": world, "steps": len(tickets),
           "warmup": max(100, int(0.1 * args.rate)), "ms_per_step": 1e3 / dps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic",
           "config": {"workload": "serving: Poisson arrivals %.0f/s for %.1f s; 95%% batched-"
                                  "workload shapes (q=1, p=8), 5%% dense 16384x8192 k=256 p=16 "
                                  "q=2; 150 GB budget, 4 slots" % (args.rate, args.duration),
                      "pool": "256 small + 4 big device-resident inputs",
                      "l2": "inputs larger than L2 (pool %.1f GB)" % (
                          sum(a[0].numel() * 2 for a in small + big) / 1e9),
                      "parallelism": f"replicas x{world}"},
           "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": float(lat.max()),
                          "small_p50": pct(lat_s, 50), "small_p99": pct(lat_s, 99),
                          "big_p50": pct(lat_b, 50), "big_p99": pct(lat_b, 99),
                          "n_small": int(len(lat_s)), "n_big": int(len(lat_b))},
           "offered_rate": args.rate, "accuracy": {"flags": flags},
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": gbs / hbm_peak, "traffic": None,
                        "kernel": "all: A bytes streamed (passes x bytes(A)) over the run's wall "
                                  "time (the load is latency-bound, not bandwidth-bound)",
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
           "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": ck}
    if rank == 0:
        print(json.dumps(out))
    h.close()
    return 0



# ---------------------------------------------------------------------------
# sparse workload
# ---------------------------------------------------------------------------
C_SEED = 20260 + 2
C_SHAPE = (200000, 100000, 1e-3, 100, 10, 1)  # m, n, density, k, p, q


def run_csr(args, torch, dev, local, world, rank, dist):
    import numpy as np
    from paper_2209_12464_gb300 import ruqlp
    from paper_2209_12464_gb300 import workloads as wl
    if args.dtype not in ("bf16", "f32"):
        raise SystemExit("the sparse workload runs with FP32 or BF16 values")
    m, n, dens, k, p, q = C_SHAPE
    lowrank = args.workload == "csrlr"
    if lowrank:
        A = wl.csr_lowrank(C_SEED, m, n, dens, 100, 200.0)
    else:
        A = wl.csr_uniform(C_SEED, m, n, dens, planted_rank=100, planted_scale=10.0)
    vdt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    rp = torch.from_numpy(A["rowptr"]).to(dev)
    ci = torch.from_numpy(A["colidx"]).to(dev)
    va = torch.from_numpy(A["values"]).to(vdt).to(dev)
    Om = wl.omega_torch(C_SEED + 1, n, k + p, device=dev)
    nnz = int(va.numel())
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    h = ruqlp.Handle(local, stream.cuda_stream)

    lr = None
    if lowrank:
        lr = tuple(torch.from_numpy(np.ascontiguousarray(A["lowrank"][key])).float().to(dev)
                   for key in ("X", "D", "Y"))
        torch.cuda.synchronize()

    def step():
        return h.decompose_csr(rp, ci, va, (m, n), Om, k, p, q, lowrank=lr)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ruqlp.ruqlp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    flags = 0
    for _ in range(args.steps):
        flags |= step()[3]
    e1.record(stream)
    torch.cuda.synchronize()
    launches = (ruqlp.ruqlp_launch_count() - l0) // max(args.steps, 1)
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    ms = max_over_ranks(torch, dist, world, ms, dev)
    passes = 2 * q + 2
    vbytes = va.element_size()
    bytes_a = nnz * (4 + vbytes) + (m + 1) * 4  # CSR of A (the CSC copy of A^T is the same size)
    value = job_rate(world, passes * bytes_a / 1e9, ms * 1e-3)
    h.set_option("profile", 1)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    prof = {ph: h.profile(ph) for ph in ("ax", "atx", "orth", "step")}
    h.set_option("profile", 0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    d = k + p
    dp = (d + 15) // 16 * 16
    # one SpMM launch streams the CSR (or CSC) once and writes rows x dp FP32;
    # the gathered skinny operand (n x dp or m x dp FP32) is read once from HBM
    # and then served from L2
    alg_ax = bytes_a + m * dp * 4 + n * dp * 4
    alg_atx = nnz * (4 + vbytes) + (n + 1) * 4 + n * dp * 4 + m * dp * 4
    cnt = prof["ax"][0] + prof["atx"][0]
    avg = (prof["ax"][1] + prof["atx"][1]) / max(cnt, 1)
    achieved = (alg_ax + alg_atx) / 2 / (avg * 1e-3) / 1e9
    gather = nnz * dp * 4  # each nonzero gathers one dp-row of the skinny operand (L2)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "kernel": "k_spmm (warp-per-row CSR/CSC product, one pass over A per launch)",
                "l2_gather_bytes_per_launch": gather,
                "l2_gather_gbs": gather / (avg * 1e-3) / 1e9,
                "note": "the skinny operand (<= 45 MB) stays in L2; every nonzero gathers a "
                        "dp-row of it, so the launch is bound by L2 gather bandwidth, not HBM",
                "alg_bytes_per_launch": (alg_ax + alg_atx) / 2, "avg_launch_ms": avg,
                "launches": cnt, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "phase_ms": {ph: prof[ph][1] / max(prof[ph][0], 1) for ph in prof},
                "phase_share": {ph: prof[ph][1] / max(prof["step"][1], 1e-9)
                                for ph in ("ax", "atx", "orth")}}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not lowrank:
        cpu = csr_cpu_baseline(args.dtype)
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": args.dtype, "data": "synthetic",
               "config": {"workload": ("CSR 200000x100000, uniform 0.1% pattern, N(0,1) values, "
                                       "plus a rank-100 term X D Y^T (D 200..2) as factors; "
                                       "k=100 p=10 q=1") if lowrank else
                                      ("CSR 200000x100000, uniform 0.1% pattern, N(0,1) values + "
                                       "planted rank-100 term of scale 10; k=100 p=10 q=1"),
                          "nnz": nnz, "passes": passes, "bytes_A": bytes_a,
                          "values": args.dtype,
                          "l2": "inputs larger than L2 (CSR %.0f MB vs 129 MB L2)" % (bytes_a / 1e6),
                          "parallelism": f"replicas x{world}"},
               "accuracy": {"flags": flags},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": None,
               "gpu_launches": launches, "clocks": ck}
        print(json.dumps(out))
    h.close()
    return 0


def csr_cpu_baseline(dtype):
    """The FP64 oracle (scipy.sparse products) on a 20000-row sample of the
    sparse workload's form, in a spawned process."""
    code = r"""
import sys, time, json
sys.path.insert(0, %r)
import oracle
from paper_2209_12464_gb300 import workloads as wl
A = wl.csr_uniform(7, 20000, 100000, 1e-3, planted_rank=100, planted_scale=10.0)
Om = wl.omega(8, 100000, 110)
t0 = time.perf_counter()
oracle.ruqlp(A, Om, 1)
t = time.perf_counter() - t0
print(json.dumps({"seconds": t, "nnz": int(A["values"].shape[0])}))
""" % (ROOT,)
    env = dict(os.environ)
    cores = os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(cores)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        return {"value": None, "error": r.stderr[-400:]}
    j = json.loads(r.stdout.strip().splitlines()[-1])
    vb = 2 if dtype == "bf16" else 4
    gbytes = 4 * (j["nnz"] * (4 + vb) + 20001 * 4) / 1e9
    return {"value": gbytes / j["seconds"], "unit": "GB/s", "cores": cores, "kind": "oracle",
            "seconds": j["seconds"],
            "sample": "oracle.ruqlp (FP64, scipy.sparse products, own Householder QR) on a "
                      "20000 x 100000 CSR of the same form (k=100, p=10, q=1)"}


def run_orth(args, torch, dev, local, world, rank, dist):
    """ruqlp_orth (shifted CholeskyQR3) of a seeded 20000 x 220 FP32 matrix
    with condition number about 1e3, the shape of the dense workload's
    sketch."""
    from paper_2209_12464_gb300 import ruqlp
    rows, d = M, K_RANK + P_OVER
    g = torch.Generator(device=dev)
    g.manual_seed(20000 + d)
    U = torch.randn(rows, d, generator=g, device=dev)
    # W = I + 0.1 N(0, 1/d): well conditioned (no torch.linalg, which a
    # profiler run cannot load)
    W = torch.eye(d, device=dev) + 0.1 * torch.randn(d, d, generator=g, device=dev) / d ** 0.5
    s = torch.logspace(0, -3, d, device=dev)
    Y = ((U * s[None, :]) @ W).contiguous()
    stream = torch.cuda.current_stream(dev)
    h = ruqlp.Handle(local, stream.cuda_stream)
    for _ in range(max(args.warmup, 3)):
        Q = h.orth(Y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        Q = h.orth(Y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    err = float(torch.max(torch.abs(Q.double().T @ Q.double() - torch.eye(d, device=dev,
                                                                        dtype=torch.float64))))
    if rank == 0:
        print(json.dumps({"metric": "ruqlp_orth time per call", "value": ms, "unit": "ms",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": {"workload": f"orth of a {rows} x {d} FP32 matrix, kappa ~1e3 "
                                                 "(three CholeskyQR passes)"},
                          "accuracy": {"max_abs_QtQ_minus_I": err}}))
    h.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as g
    g.build()
    from paper_2209_12464_gb300 import ruqlp
    if args.tune_file:
        ruqlp.ruqlp_tune_file(args.tune_file)
    if args.workload in ("batch", "serve", "csr", "csrlr", "orth"):
        fn = {"batch": run_batch, "serve": run_serve, "csr": run_csr,
              "csrlr": run_csr, "orth": run_orth}[args.workload]
        rc = fn(args, torch, dev, local, world, rank, dist)
        if world > 1:
            dist.destroy_process_group()
        return rc

    m = n = args.size or M
    k, p, q = K_RANK, P_OVER, Q_POW
    d = k + p
    A, A32, Om, sig = make_inputs(torch, dev, args.dtype, m, n, args.gen)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    h = ruqlp.Handle(local, stream.cuda_stream)
    od = torch.float64 if args.dtype == "f64" else torch.float32
    outs = (torch.empty(m, d, dtype=od, device=dev), torch.empty(d, d, dtype=od, device=dev),
            torch.empty(n, d, dtype=od, device=dev))

    def step():
        return h.decompose(A, Om, k, p, q, outs=outs)

    for _ in range(max(args.warmup, 3) if args.steps > 0 else args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ruqlp.ruqlp_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    flags = 0
    for _ in range(args.steps):
        flags |= step()[3]
    e1.record(stream)
    torch.cuda.synchronize()
    launches = (ruqlp.ruqlp_launch_count() - l0) // max(args.steps, 1)
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    ms = max_over_ranks(torch, dist, world, ms, dev)
    bytes_a = m * n * DT_BYTES[args.dtype]
    passes = 2 * q + 2
    value = job_rate(world, passes * bytes_a / 1e9, ms * 1e-3)

    # accuracy at this speed (FP64 measurement on the device, against the
    # unrounded A)
    Qo, Lo, Po = outs
    resid = residual_gpu(torch, A32, Qo, Lo, Po)
    # approximate Eckart-Young floor: spectrum tail plus the noise energy
    # outside a rank-d subspace ((m-d)(n-d) of its m n entries)
    floor = math.sqrt(float((sig[d:] ** 2).sum()) + (NOISE ** 2) * (m - d) * (n - d)) / math.sqrt(
        float((sig ** 2).sum()) + (NOISE ** 2) * m * n)

    # live per-phase timing of the dominant kernels (CUDA events on the
    # handle's stream, bracketing each launch)
    h.set_option("profile", 1)
    nprof = 2
    for _ in range(nprof):
        step()
    torch.cuda.synchronize()
    phases = ("ax", "atx", "orth", "step", "tc_ax", "tc_atx", "tc_atx2", "gram", "chol", "trsm")
    prof = {ph: h.profile(ph) for ph in phases}
    h.set_option("profile", 0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = ck.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    phase_ms = {ph: (prof[ph][1] / prof[ph][0] if prof[ph][0] else None) for ph in phases}
    share = {ph: prof[ph][1] / max(prof["step"][1], 1e-9) for ph in ("ax", "atx", "orth")}
    if args.dtype == "bf16" and prof["tc_ax"][0]:
        # the tcgen05 product kernel: one pass over A per launch.  Algorithmic
        # bytes = A (BF16) + the skinny operand (dp x K, BF16) + the output
        # (rows x dp, FP32); both orientations move the same bytes.
        dp = (d + 15) // 16 * 16
        alg = bytes_a + n * dp * 2 + m * dp * 4
        cnt = prof["tc_ax"][0] + prof["tc_atx"][0]
        avg = (prof["tc_ax"][1] + prof["tc_atx"][1]) / cnt
        achieved = alg / (avg * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": tc_traffic(m, n, d),
                    "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one "
                                      "k_tc_gemm launch captured at 10240 x 10240 and scaled by "
                                      "the units processed to the 20000 x 20000 launch "
                                      "(profiles/k_tc_gemm_dense10240_bf16.md); not measured "
                                      "in this run",
                    "kernel": "k_tc_gemm (tcgen05 A X / A^T Y, one pass over A per launch; "
                              "one-part skinny operand)",
                    "alg_bytes_per_launch": alg, "avg_launch_ms": avg, "launches": cnt,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "phase_ms": phase_ms, "phase_share": share}
        if prof["tc_atx2"][0]:
            roofline["two_part_launch"] = two_part_roofline(
                prof["tc_atx2"], 4.0 * m * n * dp, bytes_a + 4 * m * dp + 4 * n * dp, peaks)
    else:
        # CUDA-core products: FP32 (or FP64) multiply-add bound
        dom = max(("ax", "atx"), key=lambda ph: prof[ph][1])
        cnt, tot = prof[dom]
        avg = tot / max(cnt, 1)
        flops = 2.0 * m * n * d
        alu_peak = 152 * (4 if args.dtype == "f64" else 256) * sm_mhz * 1e6 / 1e12
        achieved = flops / (avg * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "traffic": None, "kernel": dom,
                    "peak_source": "derived: 152 SMs x 2 (FP64) or 128 (FP32) FMA/clk x 2 x "
                                   "median SM clock under load",
                    "phase_ms": phase_ms, "phase_share": share}

    # end to end through the host entry point (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        Ah = A.cpu().pin_memory()
        Omh = Om.cpu().pin_memory()
        ho = (torch.empty(m, d, dtype=od).pin_memory(), torch.empty(d, d, dtype=od).pin_memory(),
              torch.empty(n, d, dtype=od).pin_memory())
        h.decompose_host(Ah, Omh, k, p, q, ho)
        ke = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            h.decompose_host(Ah, Omh, k, p, q, ho)
        te = (time.perf_counter() - t0) / ke
        te = max_over_ranks(torch, dist, world, te, dev)
        bi = Ah.numel() * Ah.element_size() + Omh.numel() * 8
        bo = sum(x.numel() * x.element_size() for x in ho)
        e2e = {"value": job_rate(world, passes * bytes_a / 1e9, te), "unit": "GB/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": te * 1e3}

    cpu = None
    acc_oracle = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the FP64 oracle on the full workload: CPU baseline and per-result
        # error of this run's output against it
        secs, acc_oracle = oracle_full(A32, Om, q, outs[1], resid)
        if secs is not None:
            cores = os.cpu_count() or 1
            cpu = {"value": passes * bytes_a / 1e9 / secs, "unit": "GB/s", "cores": cores,
                   "kind": "oracle", "seconds": secs,
                   "sample": f"the full workload: oracle.ruqlp (FP64 numpy, own Householder "
                             f"QR) on the same {m} x {n} matrix and Omega; bytes counted as "
                             f"(2q+2) x bytes(A in {args.dtype}) so the ratio is the time per "
                             f"decomposition"}
        else:
            cpu = cpu_baseline(args.dtype, rows=2000)
    del A32

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": args.dtype, "data": "synthetic",
               "config": {"workload": WORKLOAD if args.gen == "haar" else
                          "Gaussian low-rank stand-in of the same shape (profiling)",
                          "m": m, "n": n, "k": k, "p": p, "q": q,
                          "passes": passes, "bytes_A": bytes_a,
                          "l2": "inputs larger than L2 (A is %.0f MB vs 129 MB L2)" % (bytes_a / 1e6),
                          "parallelism": f"replicas x{world}"},
               "accuracy": {"residual_fro": resid, "approx_floor_fro": floor,
                            "flags": flags, **acc_oracle},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": launches, "clocks": ck,
               "hbm_frac_of_measured": value / world / hbm_peak}
        print(json.dumps(out))
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
