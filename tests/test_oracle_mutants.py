"""Plant plausible mistakes in copies of the oracle's steps (on the CPU) and
check that the pins catch every one.  This is the evidence that the pins are
not tautological: a dropped term, a wrong sign, a wrong index or a transposed
operand anywhere in the oracle fails at least one of them."""
import numpy as np
import pytest

import oracle
import pins
from oracle import ruqlp_oracle as ro


def _qr_mutant(kind):
    def qr(Y):
        W = np.array(Y, dtype=np.float64, copy=True)
        m, d = W.shape
        vs, betas = [], []
        for j in range(d):
            x = W[j:, j].copy()
            alpha = np.sqrt(x @ x)
            sgn = 1.0 if x[0] >= 0 else -1.0
            v = x
            v[0] = x[0] + sgn * alpha
            vtv = v @ v
            beta = 0.0 if vtv == 0 else (1.0 if kind == "beta" else 2.0) / vtv
            if beta:
                W[j:, j:] -= beta * np.outer(v, v @ W[j:, j:])
            vs.append(v)
            betas.append(beta)
        R = W[:d, :] if kind == "no-triu" else np.triu(W[:d, :])
        Q = np.zeros((m, d))
        Q[:d, :d] = np.eye(d)
        order = range(d) if kind == "forward-Q" else range(d - 1, -1, -1)
        for j in order:
            if betas[j]:
                Q[j:, :] -= betas[j] * np.outer(vs[j], vs[j] @ Q[j:, :])
        if kind != "no-sign-fix":
            f = np.where(np.diag(R) < 0, -1.0, 1.0)
            Q = Q * f[None, :]
            R = R * f[:, None]
        return Q, R
    return qr


@pytest.mark.parametrize("kind", ["beta", "no-triu", "forward-Q", "no-sign-fix"])
def test_qr_mutants_caught(kind):
    assert pins.check_qr(_qr_mutant(kind)) != []


def _svd_mutant(kind):
    def svd(A):
        if kind == "ascending":
            U, s, V = oracle.jacobi_svd(A)
            return U[:, ::-1], s[::-1], V[:, ::-1]
        if kind == "one-sweep":
            return oracle.jacobi_svd(A, max_sweeps=1)
        raise ValueError(kind)
    return svd


@pytest.mark.parametrize("kind", ["ascending", "one-sweep"])
def test_svd_mutants_caught(kind):
    assert pins.check_svd(_svd_mutant(kind)) != []


def _ruqlp_mutant(kind):
    def ruqlp(A, Omega, q, finish_paper=False):
        A = np.asarray(A, float)
        Y = A @ Omega
        Q = ro.orth(Y)
        loops = q - 1 if kind == "q-off-by-one" and q > 0 else q
        for _ in range(loops):
            Z = (A @ Q) if kind == "transposed-operand" and A.shape[0] == A.shape[1] else A.T @ Q
            Qt = ro.orth(Z)
            Y = A @ Qt
            Q = Y if kind == "no-final-orth" else ro.orth(Y)
        Bt = A.T @ (Y if kind == "sketch-not-basis" else Q)
        P, RB = ro.householder_qr(Bt)
        L = RB.copy() if kind == "L-not-transposed" else RB.T.copy()
        out = {"Q": Q, "L": L, "P": P, "RB": RB}
        if kind == "Q-drop-last-col":
            out["Q"] = Q.copy()
            out["Q"][:, -1] = 0.0
        if finish_paper:
            Pt, Rt = ro.householder_qr(out["L"])
            out["Qhat"] = Q @ Pt
            out["Rtilde"] = Rt
        return out
    return ruqlp


@pytest.mark.parametrize("kind", ["q-off-by-one", "transposed-operand", "sketch-not-basis",
                                  "L-not-transposed", "Q-drop-last-col", "no-final-orth"])
def test_ruqlp_mutants_caught(kind):
    fails = pins.check_ruqlp(_ruqlp_mutant(kind), oracle.ruqlp_paper, oracle.principal_sines,
                             oracle.jacobi_svd)
    assert fails != [], kind


def test_paper_form_mutant_caught():
    """A left-sketch Algorithm 1 that skips the first orth breaks the
    transposition identity."""
    def paper(A, Phi, q):
        Pbar = A.T @ Phi
        for _ in range(q):
            Pbar = ro.orth(A.T @ ro.orth(A @ Pbar))
        Q, R = ro.householder_qr(A @ Pbar)
        Pt, Rt = ro.householder_qr(R.T)
        return Q, Pbar @ Pt, Rt.T, R
    fails = pins.check_ruqlp(oracle.ruqlp, paper, oracle.principal_sines, oracle.jacobi_svd)
    assert any(f.startswith("transpose") for f in fails)
