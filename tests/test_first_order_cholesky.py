"""The first-order Cholesky factor that the last CholeskyQR pass takes for a
Gram close to the identity (CPU only: the mathematics the kernel relies on,
checked against LAPACK's Cholesky in FP64).

For G = I + E (E symmetric, e = max |E_ij|) the upper-triangular factor is
R = I + X with X + X^T = E - X^T X, so X = Phi(E) (the strict upper triangle
of E and half its diagonal) up to |X^T X| <= d e^2 entry by entry; and the
inverse of a 32 x 32 diagonal block I + X_KK is I - X_KK up to
|X_KK^2| <= 32 e^2.  The kernel takes this route when d e^2 <= 2^-25, below
FP32 rounding."""
import numpy as np
import pytest


def _phi(E):
    return np.triu(E, 1) + 0.5 * np.diag(np.diag(E))


@pytest.mark.parametrize("d", [1, 17, 64, 220, 288])
@pytest.mark.parametrize("e", [1e-3, 1e-5, 1e-7])
def test_first_order_factor_within_bound(d, e):
    rng = np.random.default_rng(d * 7 + int(-np.log10(e)))
    S = rng.uniform(-1.0, 1.0, (d, d))
    E = e * (S + S.T) / 2.0
    R = np.linalg.cholesky(np.eye(d) + E).T
    R1 = np.eye(d) + _phi(E)
    assert np.max(np.abs(R - R1)) <= d * e * e
    # the diagonal blocks' inverses to first order
    for K in range(0, d, 32):
        B = R1[K:K + 32, K:K + 32]
        X = B - np.eye(B.shape[0])
        assert np.max(np.abs(np.linalg.inv(B) - (np.eye(B.shape[0]) - X))) <= 32 * e * e * 1.01

