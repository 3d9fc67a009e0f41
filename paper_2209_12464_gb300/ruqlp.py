"""Thin ctypes binding of libruqlp.so (include/ruqlp.h).

The ``ruqlp_*`` functions here have the names and arguments of the C ABI and
only marshal arguments; every step of RU-QLP runs in the library's CUDA
kernels.  ``decompose`` / ``decompose_host`` are conveniences that allocate
the outputs with torch and raise on a non-OK status.  There is no fallback:
if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libruqlp.so")

OK, NOT_READY, ERR_INVALID, ERR_BUDGET, ERR_CUDA, ERR_BREAKDOWN, ERR_TIMEOUT = range(7)
F64, F32, BF16 = 0, 1, 2
FLAG_SHIFTED, FLAG_RANKDEF, FLAG_TSQR = 0x1, 0x2, 0x4
STATUS_NAMES = {0: "OK", 1: "NOT_READY", 2: "ERR_INVALID", 3: "ERR_BUDGET", 4: "ERR_CUDA",
                5: "ERR_BREAKDOWN", 6: "ERR_TIMEOUT"}

c_int, c_int64, c_size_t, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_int64, ctypes.c_size_t,
                                                 ctypes.c_void_p, ctypes.c_char_p)


class Config(ctypes.Structure):
    _fields_ = [("device", c_int), ("hbm_budget_bytes", c_size_t), ("max_slots", c_int),
                ("cuda_stream", c_void_p)]


class Dense(ctypes.Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("ld", c_int64), ("dtype", c_int),
                ("data", c_void_p)]


class Csr(ctypes.Structure):
    _fields_ = [("m", c_int64), ("n", c_int64), ("nnz", c_int64), ("rowptr", c_void_p),
                ("colidx", c_void_p), ("values", c_void_p), ("dtype", c_int)]


class LowRank(ctypes.Structure):
    _fields_ = [("r", c_int64), ("X", c_void_p), ("D", c_void_p), ("Y", c_void_p)]


class Matrix(ctypes.Structure):
    _fields_ = [("is_csr", c_int), ("dense", Dense), ("csr", Csr), ("lr", LowRank)]


class Params(ctypes.Structure):
    _fields_ = [("k", c_int), ("p", c_int), ("q", c_int), ("compute", c_int),
                ("omega", c_void_p), ("finish_paper", c_int), ("omega_seed", ctypes.c_uint64)]


class Outputs(ctypes.Structure):
    _fields_ = [("Q", c_void_p), ("L", c_void_p), ("P", c_void_p), ("out_dtype", c_int),
                ("flags", ctypes.c_uint32)]


class RequestTimes(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "ruqlp_create": (c_int, [ctypes.POINTER(c_void_p), ctypes.POINTER(Config)]),
    "ruqlp_destroy": (c_int, [c_void_p]),
    "ruqlp_set_stream": (c_int, [c_void_p, c_void_p]),
    "ruqlp_set_option": (c_int, [c_void_p, c_char_p, c_int64]),
    "ruqlp_reserve": (c_int, [c_void_p, c_int64, c_int64, c_int, c_int, c_int64]),
    "ruqlp_workspace_bytes": (c_size_t, [c_int64, c_int64, c_int, c_int, c_int64]),
    "ruqlp_decompose": (c_int, [c_void_p, ctypes.POINTER(Matrix), ctypes.POINTER(Params),
                                ctypes.POINTER(Outputs)]),
    "ruqlp_decompose_batch": (c_int, [c_void_p, c_int, ctypes.POINTER(Matrix),
                                      ctypes.POINTER(Params), ctypes.POINTER(Outputs)]),
    "ruqlp_decompose_host": (c_int, [c_void_p, ctypes.POINTER(Matrix), ctypes.POINTER(Params),
                                     ctypes.POINTER(Outputs)]),
    "ruqlp_submit": (c_int, [c_void_p, ctypes.POINTER(Matrix), ctypes.POINTER(Params),
                             ctypes.POINTER(Outputs), ctypes.POINTER(ctypes.c_uint64)]),
    "ruqlp_poll": (c_int, [c_void_p, ctypes.c_uint64]),
    "ruqlp_poll_times": (c_int, [c_void_p, ctypes.c_uint64, ctypes.POINTER(RequestTimes)]),
    "ruqlp_omega": (c_int, [c_void_p, c_int64, c_int, ctypes.c_uint64, c_void_p]),
    "ruqlp_last_error": (c_char_p, [c_void_p]),
    "ruqlp_launch_count": (c_int64, []),
    "ruqlp_tune_file": (c_int, [c_char_p]),
    "ruqlp_sketch": (c_int, [c_void_p, ctypes.POINTER(Matrix), c_int, c_void_p, c_int64, c_int,
                             c_void_p, c_int64]),
    "ruqlp_orth": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_int64, c_int, c_void_p,
                           c_int64]),
    "ruqlp_gram": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_int64, c_int, c_void_p]),
    "ruqlp_gram_noalloc": (c_int, [c_void_p, c_int64, c_int, c_int64, c_int, c_void_p,
                                   c_void_p]),
    "ruqlp_profile": (c_int, [c_void_p, c_char_p, ctypes.POINTER(c_int64),
                              ctypes.POINTER(ctypes.c_double)]),
    "ruqlp_version": (c_char_p, []),
}


def lib():
    """Load libruqlp.so once; raise if it is missing (no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(_SIGS)


# ---- same-name wrappers of the C ABI --------------------------------------
def ruqlp_create(config):
    h = c_void_p()
    st = lib().ruqlp_create(ctypes.byref(h), ctypes.byref(config))
    return st, h


def ruqlp_destroy(h):
    return lib().ruqlp_destroy(h)


def ruqlp_set_stream(h, stream):
    return lib().ruqlp_set_stream(h, stream)


def ruqlp_set_option(h, name, value):
    return lib().ruqlp_set_option(h, name.encode(), int(value))


def ruqlp_reserve(h, m, n, d, compute, nnz=-1):
    return lib().ruqlp_reserve(h, m, n, d, compute, nnz)


def ruqlp_workspace_bytes(m, n, d, compute, nnz=-1):
    return lib().ruqlp_workspace_bytes(m, n, d, compute, nnz)


def ruqlp_decompose(h, A, prm, out):
    return lib().ruqlp_decompose(h, ctypes.byref(A), ctypes.byref(prm), ctypes.byref(out))


def ruqlp_decompose_batch(h, count, A, prm, out):
    """A, prm, out: ctypes arrays (Matrix * count, ...)."""
    return lib().ruqlp_decompose_batch(h, count, A, prm, out)


def ruqlp_decompose_host(h, A, prm, out):
    return lib().ruqlp_decompose_host(h, ctypes.byref(A), ctypes.byref(prm), ctypes.byref(out))


def ruqlp_submit(h, A, prm, out):
    """A, prm, out: ctypes structs the caller keeps alive until the poll."""
    t = ctypes.c_uint64()
    st = lib().ruqlp_submit(h, ctypes.byref(A), ctypes.byref(prm), ctypes.byref(out),
                            ctypes.byref(t))
    return st, t.value


def ruqlp_poll(h, ticket):
    return lib().ruqlp_poll(h, ticket)


def ruqlp_poll_times(h, ticket):
    tm = RequestTimes()
    st = lib().ruqlp_poll_times(h, ticket, ctypes.byref(tm))
    return st, (tm.submit_s, tm.start_s, tm.done_s)


def ruqlp_omega(h, n, d, seed, out):
    return lib().ruqlp_omega(h, n, d, seed, out)


def ruqlp_last_error(h):
    return lib().ruqlp_last_error(h).decode()


def ruqlp_version():
    return lib().ruqlp_version().decode()


def ruqlp_sketch(h, A, trans, X, ldx, d, Y, ldy):
    return lib().ruqlp_sketch(h, ctypes.byref(A), trans, X, ldx, d, Y, ldy)


def ruqlp_orth(h, Y, M, d, ldy, dtype, Q, ldq):
    return lib().ruqlp_orth(h, Y, M, d, ldy, dtype, Q, ldq)


def ruqlp_gram(h, Y, M, d, ldy, dtype, G):
    return lib().ruqlp_gram(h, Y, M, d, ldy, dtype, G)


def ruqlp_gram_noalloc(Y, M, d, ldy, dtype, G, stream):
    return lib().ruqlp_gram_noalloc(Y, M, d, ldy, dtype, G, stream)


def ruqlp_launch_count():
    return lib().ruqlp_launch_count()


def ruqlp_tune_file(path):
    return lib().ruqlp_tune_file(path.encode() if path else None)


def ruqlp_profile(h, phase):
    c = c_int64()
    ms = ctypes.c_double()
    st = lib().ruqlp_profile(h, phase.encode(), ctypes.byref(c), ctypes.byref(ms))
    return st, c.value, ms.value


# ---- conveniences over torch tensors ---------------------------------------
class RuqlpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dtype_code(t):
    import torch
    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[t]


class Batch:
    """ctypes arrays of one batched call, built once and reusable."""

    def __init__(self, handle, As, omegas, ks, p, q, out_dtype=None, ps=None, qs=None,
                 seeds=None, outs=None):
        import torch
        cnt = len(As)
        seeds = list(seeds) if seeds is not None else [0] * cnt
        od = out_dtype or torch.float32
        ps = list(ps) if ps is not None else [p] * cnt
        qs = list(qs) if qs is not None else [q] * cnt
        self.handle, self.count = handle, cnt
        self.M = (Matrix * cnt)()
        self.P = (Params * cnt)()
        self.O = (Outputs * cnt)()
        self.keep = [As]
        self.outs = []
        for i, (A, om, k) in enumerate(zip(As, omegas, ks)):
            if A.dim() != 2 or A.stride(1) != 1:
                raise ValueError("batch matrices must be 2-D row-major tensors")
            m, n = A.shape
            d = k + ps[i]
            om = om.contiguous() if om is not None else None
            self.keep.append(om)
            if outs is not None:  # caller-owned (Q, L, P), row-major, leading dimension d
                Q, L, P = outs[i]
                od = Q.dtype
            else:
                Q = torch.empty(m, d, dtype=od, device=A.device)
                L = torch.empty(d, d, dtype=od, device=A.device)
                P = torch.empty(n, d, dtype=od, device=A.device)
            self.M[i] = Matrix(0, Dense(m, n, A.stride(0), _dtype_code(A.dtype), A.data_ptr()),
                               Csr())
            self.P[i] = Params(k, ps[i], qs[i], _dtype_code(A.dtype),
                               om.data_ptr() if om is not None else None, 0, int(seeds[i]))
            self.O[i] = Outputs(Q.data_ptr(), L.data_ptr(), P.data_ptr(), _dtype_code(od), 0)
            self.outs.append((Q, L, P))

    def run(self):
        self.handle.check(ruqlp_decompose_batch(self.handle.h, self.count, self.M, self.P,
                                                self.O))
        return [self.O[i].flags for i in range(self.count)]


class Ticket:
    """A submitted request: its ticket id, the ctypes structs and tensors the
    library reads until completion, and the output tensors."""

    def __init__(self, tid, M, P, O, keep, outs):
        self.id, self.M, self.P, self.O, self.keep, self.outs = tid, M, P, O, keep, outs
        self.flags = None
        self.times = None


class Handle:
    """Owns one library handle bound to a device and stream."""

    def __init__(self, device=0, stream=None, hbm_budget_bytes=0, max_slots=0):
        cfg = Config(device, hbm_budget_bytes, max_slots, stream or None)
        st, h = ruqlp_create(cfg)
        if st != OK:
            raise RuqlpError(st, "ruqlp_create failed")
        self.h = h

    def check(self, st):
        if st != OK:
            raise RuqlpError(st, ruqlp_last_error(self.h))

    def set_stream(self, stream):
        self.check(ruqlp_set_stream(self.h, stream))

    def set_option(self, name, value):
        self.check(ruqlp_set_option(self.h, name, value))

    def profile(self, phase):
        st, c, ms = ruqlp_profile(self.h, phase)
        self.check(st)
        return c, ms

    def sketch(self, A, X, trans=False):
        """Y = A X (or A^T X) with the library's product kernel for A's dtype."""
        import torch
        m, n = A.shape
        K, Mout = (m, n) if trans else (n, m)
        d = X.shape[1]
        assert X.shape[0] == K
        Y = torch.empty(Mout, d, dtype=X.dtype, device=A.device)
        M = Matrix(0, Dense(m, n, A.stride(0), _dtype_code(A.dtype), A.data_ptr()), Csr())
        self.check(ruqlp_sketch(self.h, M, int(trans), X.data_ptr(), X.stride(0), d,
                                Y.data_ptr(), d))
        return Y

    def orth(self, Y):
        """Q with orthonormal columns, Y = Q R (R upper, positive diagonal)."""
        import torch
        M, d = Y.shape
        Q = torch.empty_like(Y)
        self.check(ruqlp_orth(self.h, Y.data_ptr(), M, d, Y.stride(0), _dtype_code(Y.dtype),
                              Q.data_ptr(), d))
        return Q

    def gram(self, Y):
        """G = Y^T Y (FP64) of a CUDA tensor Y (M x d, FP64 or FP32, row-major)."""
        import torch
        M, d = Y.shape
        G = torch.empty(d, d, dtype=torch.float64, device=Y.device)
        self.check(ruqlp_gram(self.h, Y.data_ptr(), M, d, Y.stride(0), _dtype_code(Y.dtype),
                              G.data_ptr()))
        return G

    def close(self):
        if self.h:
            ruqlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def omega(self, n, d, seed):
        """The library's Gaussian test matrix for a seed (ruqlp_omega): an
        n x d FP64 CUDA tensor."""
        import torch
        out = torch.empty(n, d, dtype=torch.float64, device="cuda")
        self.check(ruqlp_omega(self.h, n, d, seed, out.data_ptr()))
        return out

    def decompose(self, A, omega, k, p, q, out_dtype=None, outs=None, finish_paper=False,
                  seed=0):
        """RU-QLP of the CUDA tensor A (m x n, row-major) with the FP64 CUDA
        tensor omega (n x d), or omega=None: Omega generated on the device from
        seed.  Returns (Q, L, P, flags) as torch tensors."""
        import torch
        if A.dim() != 2 or A.stride(1) != 1:
            raise ValueError("A must be a 2-D row-major tensor")
        m, n = A.shape
        d = k + p
        omega = omega.contiguous() if omega is not None else None
        if out_dtype is None:
            out_dtype = torch.float64 if A.dtype == torch.float64 else torch.float32
        if outs is None:
            Q = torch.empty(m, d, dtype=out_dtype, device=A.device)
            L = torch.empty(d, d, dtype=out_dtype, device=A.device)
            P = torch.empty(n, d, dtype=out_dtype, device=A.device)
        else:
            Q, L, P = outs
        M = Matrix(0, Dense(m, n, A.stride(0), _dtype_code(A.dtype), A.data_ptr()), Csr())
        prm = Params(k, p, q, _dtype_code(A.dtype), omega.data_ptr() if omega is not None else None,
                     int(finish_paper), int(seed))
        out = Outputs(Q.data_ptr(), L.data_ptr(), P.data_ptr(), _dtype_code(out_dtype), 0)
        self.check(ruqlp_decompose(self.h, M, prm, out))
        return Q, L, P, out.flags

    def prepare_batch(self, As, omegas, ks, p, q, out_dtype=None, ps=None, qs=None,
                      seeds=None, outs=None):
        """Marshal a batch once (A_i, Omega_i, output tensors: new ones, or
        the caller's (Q, L, P) per item in outs); the returned object's run()
        calls ruqlp_decompose_batch and returns the flags."""
        return Batch(self, As, omegas, ks, p, q, out_dtype, ps, qs, seeds, outs)

    def decompose_batch(self, As, omegas, ks, p, q, out_dtype=None, ps=None, qs=None,
                        seeds=None):
        """Batched RU-QLP of CUDA tensors As[i] (m_i x n_i, one dtype) with FP64
        omegas[i] (n_i x (k_i + p_i)) or None (generated from seeds[i]); p, q
        are shared unless ps / qs give one per item.  Returns a list of
        (Q, L, P, flags)."""
        b = Batch(self, As, omegas, ks, p, q, out_dtype, ps, qs, seeds)
        flags = b.run()
        return [(Q, L, P, f) for (Q, L, P), f in zip(b.outs, flags)]

    def submit(self, A, omega, k, p, q, out_dtype=None, outs=None):
        """Queue one decomposition (ruqlp_submit); returns a Ticket."""
        import torch
        m, n = A.shape
        d = k + p
        omega = omega.contiguous()
        od = out_dtype or (torch.float64 if A.dtype == torch.float64 else torch.float32)
        if outs is None:
            outs = (torch.empty(m, d, dtype=od, device=A.device),
                    torch.empty(d, d, dtype=od, device=A.device),
                    torch.empty(n, d, dtype=od, device=A.device))
        Q, L, P = outs
        M = Matrix(0, Dense(m, n, A.stride(0), _dtype_code(A.dtype), A.data_ptr()), Csr())
        prm = Params(k, p, q, _dtype_code(A.dtype), omega.data_ptr(), 0)
        out = Outputs(Q.data_ptr(), L.data_ptr(), P.data_ptr(), _dtype_code(Q.dtype), 0)
        st, tid = ruqlp_submit(self.h, M, prm, out)
        self.check(st)
        return Ticket(tid, M, prm, out, (A, omega), outs)

    def poll(self, ticket):
        """True once the request has completed (its outputs are then final,
        ticket.flags and ticket.times set); raises on a failed request."""
        if ticket.times is not None:
            return True
        st, times = ruqlp_poll_times(self.h, ticket.id)
        if st == NOT_READY:
            return False
        ticket.times = times
        ticket.flags = ticket.O.flags
        self.check(st)
        return True

    def decompose_csr(self, rowptr, colidx, values, shape, omega, k, p, q, out_dtype=None,
                      lowrank=None):
        """RU-QLP of a CSR matrix given as CUDA tensors (rowptr, colidx int32;
        values float32 or bfloat16), optionally plus a low-rank term
        lowrank = (X, D, Y) (FP32 CUDA tensors, A = S + X D Y^T).  Returns
        (Q, L, P, flags)."""
        import torch
        m, n = shape
        d = k + p
        od = out_dtype or torch.float32
        dev = values.device
        Q = torch.empty(m, d, dtype=od, device=dev)
        L = torch.empty(d, d, dtype=od, device=dev)
        P = torch.empty(n, d, dtype=od, device=dev)
        M = Matrix(1, Dense(), Csr(m, n, values.numel(), rowptr.data_ptr(), colidx.data_ptr(),
                                   values.data_ptr(), _dtype_code(values.dtype)))
        if lowrank is not None:
            X, D, Y = (t.contiguous() for t in lowrank)
            M.is_csr = 2
            M.lr = LowRank(X.shape[1], X.data_ptr(), D.data_ptr(), Y.data_ptr())
        prm = Params(k, p, q, _dtype_code(values.dtype), omega.contiguous().data_ptr(), 0)
        out = Outputs(Q.data_ptr(), L.data_ptr(), P.data_ptr(), _dtype_code(od), 0)
        self.check(ruqlp_decompose(self.h, M, prm, out))
        return Q, L, P, out.flags

    def sketch_csr(self, rowptr, colidx, values, shape, X, trans=False, lowrank=None):
        """Y = A X (or A^T X) for a CSR A (plus an optional low-rank term
        (Xl, D, Yl), A = S + Xl D Yl^T) on the device; X float32."""
        import torch
        m, n = shape
        K, Mout = (m, n) if trans else (n, m)
        d = X.shape[1]
        Y = torch.empty(Mout, d, dtype=torch.float32, device=X.device)
        M = Matrix(1, Dense(), Csr(m, n, values.numel(), rowptr.data_ptr(), colidx.data_ptr(),
                                   values.data_ptr(), _dtype_code(values.dtype)))
        if lowrank is not None:
            Xl, Dl, Yl = (t.contiguous() for t in lowrank)
            M.is_csr = 2
            M.lr = LowRank(Xl.shape[1], Xl.data_ptr(), Dl.data_ptr(), Yl.data_ptr())
        self.check(ruqlp_sketch(self.h, M, int(trans), X.data_ptr(), X.stride(0), d,
                                Y.data_ptr(), d))
        return Y

    def decompose_host(self, A, omega, k, p, q, outs, seed=0):
        """Same with CPU tensors (pinned or pageable); outs = (Q, L, P) CPU
        tensors; omega=None generates Omega on the device from seed."""
        m, n = A.shape
        Q, L, P = outs
        M = Matrix(0, Dense(m, n, A.stride(0), _dtype_code(A.dtype), A.data_ptr()), Csr())
        prm = Params(k, p, q, _dtype_code(A.dtype), omega.data_ptr() if omega is not None else None,
                     0, int(seed))
        out = Outputs(Q.data_ptr(), L.data_ptr(), P.data_ptr(), _dtype_code(Q.dtype), 0)
        self.check(ruqlp_decompose_host(self.h, M, prm, out))
        return Q, L, P, out.flags


def decompose(A, omega, k, p, q, **kw):
    """One-shot RU-QLP on A's device and torch's current stream."""
    import torch
    dev = A.device.index or 0
    h = Handle(device=dev, stream=torch.cuda.current_stream(A.device).cuda_stream)
    try:
        return h.decompose(A, omega, k, p, q, **kw)
    finally:
        h.close()
