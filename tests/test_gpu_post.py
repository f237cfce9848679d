"""Post-processing on the GPU (the supplement's Fig. S1: the linear S(k) and g_2(r) of quenched states): the pair
histogram behind g_2(r) against the oracle's brute force, bit for bit (its decisions are exact integers), and S(k)
beyond the exclusion region from a context with a larger cutoff."""
import math
import os

import numpy as np
import pytest

from paper_2304_09139_b300 import ssh, synth

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def built():
    from paper_2304_09139_b300 import _build
    _build.build()
    ssh.load()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return True


CASES = [
    # (label, d, N, n_ref, r_max as a fraction of L, nbins, seed)
    ("d2", 2, 3000, 3000, 0.45, 200, 21),
    ("d3", 3, 2000, 600, 0.49, 300, 22),
    ("d1", 1, 4000, 4000, 0.30, 1000, 23),
    # the d=2, N=10^4 workload, the largest bin count (shared-memory histogram beyond 48 KB)
    ("medium_d2", 2, 10_000, 800, 0.49, 4096, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pair_histogram_bit_exact(built, oracle_mod, case):
    label, d, N, n_ref, frac, nb, seed = case
    L = N ** (1 / d)
    s = synth.positions(seed, N, d)
    ctx = ssh.Context(d, N, L, chi=0.2)
    ctx.set_positions_frac(s)
    got = ctx.pair_histogram(n_ref, frac * L, nb)
    want = oracle_mod.pair_histogram(s, L, n_ref, frac * L, nb)
    assert np.array_equal(got, want), (label, np.abs(got.astype(np.int64) - want.astype(np.int64)).max())
    # an ideal gas: g_2 near 1 away from r = 0
    r, g = ssh.g2(got, d, N, L, n_ref, frac * L)
    assert abs(g[nb // 2:].mean() - 1.0) < 0.05, g[nb // 2:].mean()
    ctx.close()


def test_pair_histogram_lattice(built, oracle_mod):
    """The 16 x 16 square lattice (its counts pinned by Jacobi's two-square count in the oracle tests)."""
    g = np.arange(16) / 16.0
    s = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2) + 0.25 / 16
    ctx = ssh.Context(2, 256, 16.0, chi=0.1)
    ctx.set_positions_frac(s)
    assert np.array_equal(ctx.pair_histogram(256, 7.5, 30), oracle_mod.pair_histogram(s, 16.0, 256, 7.5, 30))
    ctx.close()


def test_pair_histogram_rejects_bad_arguments(built):
    ctx = ssh.Context(2, 100, 10.0, chi=0.3)
    for args in ((0, 1.0, 10), (101, 1.0, 10), (10, 5.0, 10), (10, 0.0, 10), (10, 1.0, 0), (10, 1.0, 5000)):
        with pytest.raises(ssh.SshError):
            ctx.pair_histogram(*args)
    ctx.close()


def test_structure_factor_beyond_the_exclusion_region(built, oracle_mod):
    """Quench the d=2, N=100 workload, then evaluate n~ on a K-mode set 2.5 times wider: S(k) vanishes (to the
    stopping threshold) on the constrained wavevectors and is of order 1 well beyond them; the radial average and
    the truncated order metric are finite."""
    cfg = synth.SMALL_D2
    ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    ctx.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
    r = ctx.minimize(max_steps=40000)
    assert r["status"] == 0
    hi, lo = ctx.positions_frac()
    inner = {tuple(v) for v in ctx.kset()}  # the exclusion set (chi mode may cut its outermost shell)
    kmax = 2 * math.pi / cfg.L * math.sqrt(float((ctx.kset().astype(np.float64) ** 2).sum(1).max()))
    wide = ssh.Context(cfg.d, cfg.N, cfg.L, K=2.5 * kmax)
    wide.set_positions_frac(hi, lo)
    wide.energy_grad(ssh.FX)
    C, S = wide.ntilde()
    n = wide.kset()
    kk = 2 * math.pi / cfg.L * np.sqrt((n.astype(np.float64) ** 2).sum(1))
    sk = ((C[:, 0] + C[:, 1]) ** 2 + (S[:, 0] + S[:, 1]) ** 2) / cfg.N
    mine = np.array([tuple(v) in inner for v in n])
    assert mine.sum() == len(inner) and sk[mine].max() <= 1.01e-36
    assert 0.2 < sk[kk > 1.5 * kmax].mean() < 5.0
    kb, sb, cnt = ssh.structure_factor_radial(n, C, S, cfg.L, cfg.N, 20)
    assert cnt.sum() == len(n) and np.all(np.isfinite(sb[cnt > 0]))
    assert math.isfinite(ssh.tau_estimate(n, C, S, cfg.L, cfg.N, kmax))
    # the oracle agrees on S(k) of the wide set
    ref = oracle_mod.phi_grad(hi, lo, n, cfg.L, want_force=False, want_cs=True, nthreads=NTHREADS)
    assert np.all(np.abs((C[:, 0] - ref["C"][:, 0]) + (C[:, 1] - ref["C"][:, 1])) <= 1e-28 * cfg.N)
    wide.close()
    ctx.close()
