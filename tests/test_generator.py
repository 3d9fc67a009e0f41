"""The host twin of the library's device Gaussian generator (Section III-A
step 1: Omega with iid N(0,1) entries; counter-based so both sides draw the
same matrix from a seed): Philox4x32-10 against its published known-answer
vectors, and the Box-Muller normals against the moments of N(0,1)."""
import json
import os

import numpy as np

from paper_2209_12464_gb300 import workloads as wl

KAT = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")))


def test_philox_known_answer_vectors():
    for v in KAT["vectors"]:
        c = [int(x, 16) for x in v["counter"]]
        k = [int(x, 16) for x in v["key"]]
        out = wl.philox4x32_10(c, k)
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_omega_normal_moments():
    Om = wl.omega_philox(20260, 4000, 250)  # 10^6 draws
    x = Om.ravel()
    n = x.size
    assert abs(x.mean()) <= 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) <= 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) <= 5 * np.sqrt(96.0 / n)
    # tail frequencies of the standard normal
    assert abs(np.mean(np.abs(x) > 1.959963984540054) - 0.05) <= 5 * np.sqrt(0.05 * 0.95 / n)
    # neighbouring entries in a row and in a column are uncorrelated
    assert abs(np.mean(Om[:, 1:] * Om[:, :-1])) <= 5 / np.sqrt(n)
    assert abs(np.mean(Om[1:, :] * Om[:-1, :])) <= 5 / np.sqrt(n)


def test_omega_depends_on_seed_and_position():
    a = wl.omega_philox(1, 50, 8)
    b = wl.omega_philox(2, 50, 8)
    c = wl.omega_philox(1, 60, 8)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, c[:50])  # entry (i, j) does not depend on n
    assert np.array_equal(wl.omega_philox(1, 50, 8), a)
    d = wl.omega_philox((1 << 40) + 7, 3, 4)  # both key words used
    assert not np.array_equal(d, wl.omega_philox(7, 3, 4))
