"""Host-side post-processing helpers (no GPU): the g_2 normalisation, the radial S(k) average and the tau
estimate of Eq. tau, on inputs whose answers are known in closed form."""
import math

import numpy as np

from paper_2304_09139_b300 import ssh


def test_g2_of_ideal_gas_counts_is_one():
    """Counts equal to an ideal gas's expectation in each shell give g_2 = 1 in every dimension."""
    for d in (1, 2, 3):
        N, L, n_ref, r_max, nb = 1000, 10.0, 100, 4.0, 40
        edges = np.arange(nb + 1) * (r_max / nb)
        vd = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
        expect = n_ref * (N - 1) / L ** d * vd * (edges[1:] ** d - edges[:-1] ** d)
        r, g = ssh.g2(expect, d, N, L, n_ref, r_max)
        assert np.allclose(g, 1.0, rtol=1e-12) and np.allclose(r, 0.5 * (edges[1:] + edges[:-1]))


def test_radial_structure_factor_and_tau():
    """S(k) = |n~|^2 / N averaged over shells of |k|; with S = 1 everywhere tau vanishes, and with S = 0 on a set
    it equals 2 M (2 pi / L)^d / ((2 pi / K)^d rho^2)."""
    L, N = 10.0, 64
    n = np.array([[1, 0], [0, 1], [1, 1], [2, 0], [1, -1]], dtype=np.int32)
    amp = 8.0  # |n~|^2 = 64 = N: S = 1 exactly
    C = np.stack([np.full(len(n), amp), np.zeros(len(n))], -1)
    S = np.zeros((len(n), 2))
    k, sb, cnt = ssh.structure_factor_radial(n, C, S, L, N, 4)
    assert cnt.sum() == len(n) and np.allclose(sb[cnt > 0], 1.0)
    K = 2 * math.pi / L * 2.0
    assert ssh.tau_estimate(n, C, S, L, N, K) == 0.0
    zero = np.zeros((len(n), 2))
    rho = N / L ** 2
    want = 2 * len(n) * (2 * math.pi / L) ** 2 / ((2 * math.pi / K) ** 2 * rho ** 2)
    assert math.isclose(ssh.tau_estimate(n, zero, zero, L, N, K), want, rel_tol=1e-12)
