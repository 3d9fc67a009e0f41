"""Seeded synthetic inputs for RU-QLP (arXiv 2209.12464) tests and benchmarks.

This module only draws inputs: test matrices with a prescribed spectrum, the
Gaussian test matrix Omega, sparse CSR patterns, batched shape mixes and
Poisson arrival times.  It holds none of the method's arithmetic and imports
neither the CUDA binding nor the oracle, so both sides of a parity test can be
fed the same arrays from here.

Recipes (the dense ones follow Section V-B's construction A = U Sigma V^T
(+ noise) with U, V random orthonormal):
  * U, V are Haar-distributed: the Q factor of a seeded N(0,1) matrix with the
    sign of each column fixed so that diag(R) > 0 (Mezzadri 2007).
  * ``spectrum_gap(r, k, tail)``: sigma_i = 1 for i <= k, tail / (i - k) after.
  * ``lowrank_gap(n, k, mu)``: sigma decreasing linearly 1 -> 1e-10 over
    i = 1..n, zero beyond k, plus mu * sigma_k * A_N with A_N Gaussian
    normalised to ||A_N||_2 = 1 (LowRank{Large,Medium}Gap, Section V-B).
  * ``spectrum_decay(n, k, z)``: 1 (k times), then 2^-z, 3^-z, ...
    (LowRank{Slow,Fast}Decay, Section V-B).
  * Omega: iid N(0,1) (Section III-A step 1), float64, row-major n x d.
"""
from __future__ import annotations

import math

import numpy as np

MASTER_SEED = 20260


# ---------------------------------------------------------------------------
# spectra
# ---------------------------------------------------------------------------
def spectrum_gap(r, k, tail):
    """sigma_i = 1 for i <= k, then tail / (i - k) for i = k+1..r."""
    i = np.arange(1, r + 1, dtype=np.float64)
    s = np.ones(r)
    s[k:] = tail / (i[k:] - k)
    return s


def spectrum_rank(r, k):
    """sigma_i = 1 for i <= k, 0 beyond (an exactly rank-k matrix)."""
    s = np.zeros(r)
    s[:k] = 1.0
    return s


def spectrum_linear_rank(n, k):
    """Linear decrease from 1 to 1e-10 over i = 1..n, zero beyond k."""
    s = np.linspace(1.0, 1e-10, n)
    s[k:] = 0.0
    return s


def spectrum_decay(n, k, z):
    """1 (k times), then 2^-z, 3^-z, ..., (n-k+1)^-z."""
    s = np.ones(n)
    s[k:] = np.arange(2, n - k + 2, dtype=np.float64) ** (-float(z))
    return s


# ---------------------------------------------------------------------------
# dense matrices
# ---------------------------------------------------------------------------
def haar(rng, m, r):
    """m x r matrix with Haar-distributed orthonormal columns (numpy, float64)."""
    G = rng.standard_normal((m, r))
    Qf, Rf = np.linalg.qr(G)
    sgn = np.where(np.diag(Rf) < 0.0, -1.0, 1.0)
    return Qf * sgn[None, :]


def dense_spectral(seed, m, n, sigma, noise_std=0.0):
    """A = U diag(sigma) V^T (+ N(0, noise_std^2) iid noise), float64 numpy.

    U is m x r and V is n x r with r = len(sigma) <= min(m, n).  Returns
    (A, U, sigma, V) so tests can use the exact singular structure.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    if r > min(m, n):
        raise ValueError("len(sigma) must be <= min(m, n)")
    rng = np.random.default_rng(seed)
    U = haar(rng, m, r)
    V = haar(rng, n, r)
    A = (U * sigma[None, :]) @ V.T
    if noise_std:
        A = A + noise_std * rng.standard_normal((m, n))
    return A, U, sigma, V


def dense_spectral_torch(seed, m, n, sigma, noise_std=0.0, device="cuda",
                         dtype=None):
    """Large-size twin of ``dense_spectral`` built with torch on ``device``.

    Haar factors come from torch.linalg.qr of a seeded N(0,1) matrix in
    float32 (sign-fixed); A = U diag(sigma) V^T (+ noise) is formed in float32
    and returned in ``dtype`` (default float32).  Used where a numpy QR of the
    full size would take minutes (20000 x 20000); values differ from the
    numpy twin, and every parity check feeds the same returned tensor to both
    sides.
    """
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float32), device=device)
    r = sig.shape[0]

    def _haar(rows):
        G = torch.randn(rows, r, generator=g, device=device, dtype=torch.float32)
        Qf, Rf = torch.linalg.qr(G)
        sgn = torch.where(torch.diagonal(Rf) < 0, -1.0, 1.0)
        del G, Rf
        return Qf * sgn[None, :]

    U = _haar(m)
    U *= sig[None, :]
    V = _haar(n)
    A = U @ V.T
    del U, V
    if noise_std:
        A.add_(torch.randn(m, n, generator=g, device=device, dtype=torch.float32),
               alpha=float(noise_std))
    return A.to(dtype)


def dense_lowrank_gauss_torch(seed, m, n, k, tail_scale=1e-2, noise_std=0.0, device="cuda"):
    """Cheap stand-in with the same shape and a gapped spectrum, for profiling
    runs where torch.linalg is unavailable: A = G1 G2^T / sqrt(n) + tail_scale *
    G3 G4^T / sqrt(n) (G1, G2: k Gaussian columns; G3, G4: 2k columns) plus
    N(0, noise_std^2) noise, float32 on ``device``.  Its spectrum is not the
    Haar workload's; it is used only to time kernels."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f = 1.0 / math.sqrt(n)
    A = (torch.randn(m, k, generator=g, device=device) * f) @ torch.randn(k, n, generator=g, device=device)
    A.addmm_(torch.randn(m, 2 * k, generator=g, device=device) * (f * tail_scale),
             torch.randn(2 * k, n, generator=g, device=device))
    if noise_std:
        A.add_(torch.randn(m, n, generator=g, device=device), alpha=float(noise_std))
    return A


def lowrank_gap(seed, n, k, mu):
    """LowRank{Large,Medium}Gap of Section V-B: U Sigma V^T + mu sigma_k A_N."""
    sigma = spectrum_linear_rank(n, k)
    A, U, s, V = dense_spectral(seed, n, n, sigma)
    rng = np.random.default_rng(seed + 7919)
    AN = rng.standard_normal((n, n))
    AN /= np.linalg.norm(AN, 2)
    return A + mu * sigma[k - 1] * AN, U, s, V


def omega(seed, n, d):
    """Gaussian test matrix Omega, iid N(0,1), float64, n x d row-major."""
    return np.random.default_rng(seed).standard_normal((n, d))


def philox4x32_10(c, k):
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) on numpy uint32
    arrays: counter words c = (c0, c1, c2, c3), key k = (k0, k1); ten rounds of
    (hi0, lo0) = 0xD2511F53 c0, (hi1, lo1) = 0xCD9E8D57 c2,
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key += (0x9E3779B9,
    0xBB67AE85).  Returns the four output words."""
    m0, m1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    mask = np.uint64(0xFFFFFFFF)
    c = [np.asarray(x, dtype=np.uint32) for x in c]
    k0 = np.asarray(k[0], dtype=np.uint64)
    k1 = np.asarray(k[1], dtype=np.uint64)
    for _ in range(10):
        p0 = m0 * c[0].astype(np.uint64)
        p1 = m1 * c[2].astype(np.uint64)
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & mask).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & mask).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0.astype(np.uint32), lo1, hi0 ^ c[3] ^ k1.astype(np.uint32), lo0]
        k0 = (k0 + np.uint64(0x9E3779B9)) & mask
        k1 = (k1 + np.uint64(0xBB67AE85)) & mask
    return c


def omega_philox(seed, n, d):
    """Host twin of the library's device-generated Omega (float64 n x d):
    entry (i, j) takes counter (j, i mod 2^32, i >> 32, 0) and key
    (seed mod 2^32, seed >> 32); u = (x + 1/2) 2^-32 from the first two
    words; Omega_ij = sqrt(-2 ln u1) cos(2 pi u2)."""
    i = np.repeat(np.arange(n, dtype=np.uint64), d)
    j = np.tile(np.arange(d, dtype=np.uint64), n)
    s = np.uint64(seed)
    c = (j.astype(np.uint32), (i & np.uint64(0xFFFFFFFF)).astype(np.uint32),
         (i >> np.uint64(32)).astype(np.uint32), np.zeros(n * d, dtype=np.uint32))
    x = philox4x32_10(c, (np.full(n * d, int(s & np.uint64(0xFFFFFFFF)), dtype=np.uint32),
                          np.full(n * d, int(s >> np.uint64(32)), dtype=np.uint32)))
    u1 = (x[0].astype(np.float64) + 0.5) * 2.3283064365386963e-10
    u2 = (x[1].astype(np.float64) + 0.5) * 2.3283064365386963e-10
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)).reshape(n, d)


def omega_torch(seed, n, d, device="cuda"):
    """Device twin of ``omega`` for large n (float64 on ``device``)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn(n, d, generator=g, device=device, dtype=torch.float64)


# ---------------------------------------------------------------------------
# sparse matrices (CSR, int32 indices)
# ---------------------------------------------------------------------------
def csr_uniform(seed, m, n, density, planted_rank=0, planted_scale=0.0,
                chunk=1 << 20):
    """Uniform random CSR pattern with N(0,1) values plus an optional planted
    low-rank term restricted to the pattern.

    Each row draws Binomial(n, density) column indices uniformly (duplicates
    removed, columns sorted).  Values are z_ij + (planted_scale / sqrt(r))
    x_i^T y_j with x_i, y_j in R^r iid N(0,1), r = planted_rank, so the planted
    entries have standard deviation planted_scale.  Returns a dict with
    rowptr (int32, m+1), colidx (int32, nnz), values (float64), m, n.
    """
    rng = np.random.default_rng(seed)
    counts = rng.binomial(n, density, size=m).astype(np.int64)
    total = int(counts.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), counts)
    cols = rng.integers(0, n, size=total, dtype=np.int64)
    key = np.unique(rows * n + cols)
    rows = key // n
    cols = key - rows * n
    nnz = key.shape[0]
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    vals = rng.standard_normal(nnz)
    if planted_rank:
        X = rng.standard_normal((m, planted_rank))
        Yp = rng.standard_normal((n, planted_rank))
        c = planted_scale / math.sqrt(planted_rank)
        for s0 in range(0, nnz, chunk):
            s1 = min(nnz, s0 + chunk)
            vals[s0:s1] += c * np.einsum("ij,ij->i", X[rows[s0:s1]], Yp[cols[s0:s1]])
    if nnz >= 2 ** 31:
        raise ValueError("nnz exceeds int32 indexing")
    return {"rowptr": rowptr.astype(np.int32), "colidx": cols.astype(np.int32),
            "values": vals, "m": int(m), "n": int(n)}


def csr_lowrank(seed, m, n, density, r, scale, noise_values=1.0):
    """Sparse-plus-low-rank input A = S + X D Y^T: S a uniform CSR pattern
    (csr_uniform) with N(0, noise_values^2) values, X (m x r) and Y (n x r)
    with Haar-distributed orthonormal columns, D = diag(scale * (1, ..., 1/r))
    (linearly decreasing from scale to scale / r).  The low-rank term's
    singular values are D's; with scale well above ||S||_2 (about
    noise_values * sqrt(density) (sqrt(m) + sqrt(n))) the spectrum has a gap
    after r.  Returns the CSR dict with "lowrank" = {X, D, Y} (float64)."""
    A = csr_uniform(seed, m, n, density)
    A["values"] = A["values"] * noise_values
    rng = np.random.default_rng(seed + 101)
    X = haar(rng, m, r)
    Y = haar(rng, n, r)
    D = np.diag(scale * np.linspace(1.0, 1.0 / r, r))
    A["lowrank"] = {"X": X, "D": D, "Y": Y}
    return A


def csr_to_dense(A):
    """Dense float64 copy of a small CSR dict (test helper)."""
    D = np.zeros((A["m"], A["n"]))
    rp = A["rowptr"]
    for i in range(A["m"]):
        D[i, A["colidx"][rp[i]:rp[i + 1]]] = A["values"][rp[i]:rp[i + 1]]
    return D


# ---------------------------------------------------------------------------
# batched and served mixes
# ---------------------------------------------------------------------------
def batch_shapes(seed, count=512, m_range=(256, 4096), n_range=(128, 2048),
                 k_range=(8, 64), p=8):
    """Shapes of a batch: m, n log-uniform over the ranges, k uniform (ints).
    Returns a list of (m, n, k, p) with d = k + p < n and d <= m."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        k = min(k, n - p - 1, m - p)
        out.append((m, n, k, p))
    return out


def aligned_rows(A):
    """A copy of the 2-D torch tensor A whose rows start on 16-byte boundaries
    (leading dimension rounded up to a multiple of 16 bytes; the padding
    columns are zero and not part of the returned view)."""
    import torch
    m, n = A.shape
    per = max(1, 16 // A.element_size())
    ld = (n + per - 1) // per * per
    buf = torch.zeros(m, ld, dtype=A.dtype, device=A.device)
    buf[:, :n] = A
    return buf[:, :n]


def poisson_arrivals(seed, rate, count):
    """Arrival times (seconds) of a Poisson process with ``rate`` per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
