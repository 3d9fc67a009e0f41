"""Deterministic bounds of Section IV (Theorems 1, 2, 5 and Corollary 1),
restated for the right-sketch orientation used by the library and the oracle.

The library's RU-QLP of A with Omega (n x d) equals the paper's algorithm on
A' = A^T with Phi = Omega.  With A = U Sigma V^T the roles translate as
  Phi_hat_1 = V_k^T Omega,   Phi_hat_2 = V_perp^T Omega,
  paper theta_i (its Q vs U_k, exponent 2q+2)  ->  angle(P, V_k),
  paper phi_i   (its P vs V_k, exponent 2q+1)  ->  angle(Q, U_k),
  paper R_11, R_22                             ->  L_11^T, L_22^T,
  paper "P-based" error ||A' - A'P'P'^T||      ->  ||A - Q Q^T A||,
  paper "Q-based" error ||A' - Q'Q'^T A'||     ->  ||A - A P P^T||.
||Phi_hat_2 Phi_hat_1^+||_2 is evaluated as ||(I - V_k V_k^T) Omega (V_k^T Omega)^+||_2,
which needs no basis of the complement.
"""
from __future__ import annotations

import numpy as np


def omega_ratio_norm(Omega, Vk):
    O1 = Vk.T @ Omega
    O2 = Omega - Vk @ O1
    return float(np.linalg.norm(O2 @ np.linalg.pinv(O1), 2))


def deltas(sigma, k):
    """delta_i = sigma_{k+1} / sigma_i, i = 1..k (Section IV)."""
    return sigma[k] / sigma[:k]


def gamma(sigma):
    """gamma = sigma_min / sigma_1 over the full spectrum (Section IV)."""
    return float(sigma[-1] / sigma[0])


def sigma_perp(sigma, k, norm):
    tail = sigma[k:]
    return float(tail[0]) if norm == 2 else float(np.sqrt(np.sum(tail * tail)))


def thm1_lower(sigma, k, q, w):
    """Theorem 1 / Corollary 1: sigma_i(L_11) >= sigma_i / sqrt(1 + delta_i^(4q+4) w^2)."""
    dl = deltas(sigma, k)
    return sigma[:k] / np.sqrt(1.0 + dl ** (4 * q + 4) * w * w)


def thm1_upper_22(sigma, k, q, w, norm):
    """Theorem 1: ||L_22|| <= (1 + delta_k^(2q+1) w / (1 + gamma^(4q+4) w^2)) ||Sigma_perp||."""
    dk = sigma[k] / sigma[k - 1]
    g = gamma(sigma)
    return (1.0 + dk ** (2 * q + 1) * w / (1.0 + g ** (4 * q + 4) * w * w)) * sigma_perp(sigma, k, norm)


def thm2_sin_P(sigma, k, q, w):
    """Theorem 2 (paper theta_i, exponent 2q+2) -> sin angle(P, V_k)_i."""
    dl = deltas(sigma, k)
    x = dl ** (2 * q + 2) * w
    return x / np.sqrt(1.0 + x * x)


def thm2_sin_Q(sigma, k, q, w):
    """Theorem 2 (paper phi_i, exponent 2q+1) -> sin angle(Q, U_k)_i."""
    dl = deltas(sigma, k)
    return dl ** (2 * q + 1) * w / np.sqrt(1.0 + dl ** (4 * q + 2) * w * w)


def thm5_QQtA(sigma, k, q, w, norm):
    """Theorem 5 second bound (paper P-based) -> ||A - Q Q^T A||."""
    dk = sigma[k] / sigma[k - 1]
    g = gamma(sigma)
    return (1.0 + dk ** (2 * q) * w / (1.0 + g ** (4 * q + 2) * w * w)) * sigma_perp(sigma, k, norm)


def thm5_APPt(sigma, k, q, w, norm):
    """Theorem 5 first bound (paper Q-based) -> ||A - A P P^T||."""
    dk = sigma[k] / sigma[k - 1]
    g = gamma(sigma)
    return (1.0 + dk ** (2 * q + 1) * w / (1.0 + g ** (4 * q + 4) * w * w)) * sigma_perp(sigma, k, norm)
