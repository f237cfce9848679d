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
    sf = wide.structure_factor(20, K=kmax)
    assert sf["counts"].sum() == len(n) and np.all(np.isfinite(sf["mean"][sf["counts"] > 0]))
    assert math.isfinite(sf["tau"][0]) and sf["tau"][0] > 0
    # the oracle agrees on S(k) of the wide set
    ref = oracle_mod.phi_grad(hi, lo, n, cfg.L, want_force=False, want_cs=True, nthreads=NTHREADS)
    assert np.all(np.abs((C[:, 0] - ref["C"][:, 0]) + (C[:, 1] - ref["C"][:, 1])) <= 1e-28 * cfg.N)
    wide.close()
    ctx.close()


SF_CASES = [
    # (label, d, N, L, K cutoff in units of 2 pi / L, nbins, n2max (0: the set's largest), tau's K, seed)
    ("d2", 2, 1500, 1500 ** 0.5, 14.3, 9, 0, 1.0, 31),
    ("d3_partial", 3, 700, 700 ** (1 / 3), 5.2, 5, 20, 0.8, 32),
    ("d1", 1, 900, 900.0, 300.5, 17, 0, 2.0, 33),
    ("d4", 4, 300, 300 ** 0.25, 2.7, 4, 0, 1.5, 34),
]


@pytest.mark.parametrize("case", SF_CASES, ids=[c[0] for c in SF_CASES])
@pytest.mark.parametrize("prec", ["fx", "dd"])
def test_structure_factor_against_oracle(built, oracle_mod, case, prec):
    """Shell means of S(k) and tau (Eq. tau) from the GPU's evaluation against the oracle's binary128 values from
    its own n~ at the same positions.  Shell counts are exact integer decisions and must agree exactly.  The GPU's
    C, S are within 1e-28 N of the oracle's, so S(k) = |n~|^2 / N is within 1e-28 (4 sqrt(N S) + 1) and so is every
    shell mean (bound by the shell's largest S); tau moves by at most 2 (K L)^d / N^2 sum_k 2 |S - 1| dS."""
    label, d, N, L, kc, nb, n2max, Kt, seed = case
    s = synth.positions(seed, N, d)
    ctx = ssh.Context(d, N, L, K=2 * math.pi / L * kc)
    ctx.set_positions_frac(s)
    ctx.energy_grad(ssh.FX if prec == "fx" else ssh.DD)
    n = ctx.kset()
    sf = ctx.structure_factor(nb, n2max or None, Kt)
    sf2 = ctx.structure_factor(nb, n2max or None, Kt)
    assert all(np.array_equal(sf[k], sf2[k]) for k in sf), "repeated calls give the same bits"
    top = int((n.astype(np.int64) ** 2).sum(1).max()) if n2max == 0 else n2max
    counts, mean, tau = oracle_mod.structure_factor(s, None, n, L, nb, top, Kt, nthreads=NTHREADS)
    assert np.array_equal(sf["counts"], counts)
    ref = oracle_mod.phi_grad(s, None, n, L, want_force=False, want_cs=True, nthreads=NTHREADS)
    sk = ((ref["C"][:, 0] + ref["C"][:, 1]) ** 2 + (ref["S"][:, 0] + ref["S"][:, 1]) ** 2) / N
    dsk = 1e-28 * (4 * np.sqrt(N * sk) + 1) + 1e-30 * sk
    n2 = (n.astype(np.int64) ** 2).sum(1)
    E = [-(-(b * b * top) // (nb * nb)) for b in range(nb + 1)]
    for b in range(nb):
        sel = (n2 >= E[b]) & ((n2 < E[b + 1]) if b < nb - 1 else (n2 <= top))
        got = sf["mean"][b, 0] + sf["mean"][b, 1]
        want = mean[b, 0] + mean[b, 1]
        if not sel.any():
            assert got == 0.0 and want == 0.0
            continue
        assert abs((sf["mean"][b, 0] - mean[b, 0]) + (sf["mean"][b, 1] - mean[b, 1])) <= dsk[sel].max(), (b, got, want)
    scale = 2 * (Kt * L) ** d / N ** 2
    tol = scale * (2 * np.abs(sk - 1) * dsk + dsk ** 2).sum() + 1e-30 * (tau[0] + 1e-300)
    assert abs((sf["tau"][0] - tau[0]) + (sf["tau"][1] - tau[1])) <= tol, (sf["tau"], tau)
    assert np.allclose(sf["k_mid"], (np.arange(nb) + 0.5) * 2 * math.pi / L * math.sqrt(top) / nb, rtol=1e-14)
    ctx.close()


def test_structure_factor_rejects_bad_arguments(built):
    ctx = ssh.Context(2, 200, 200 ** 0.5, chi=0.3)
    ctx.set_positions_frac(synth.positions(5, 200, 2))
    with pytest.raises(ssh.SshError):
        ctx.structure_factor(4)            # no evaluation yet
    ctx.energy_grad(ssh.FX)
    for args in ((0,), (70000,), (4, -1), (4, 0, -1.0)):
        with pytest.raises(ssh.SshError):
            ctx.structure_factor(*args)
    ctx.close()


def test_structure_factor_over_an_explicit_wavevector_list(built, oracle_mod):
    """ssh_structure_factor over a context built from an explicit list in no particular order (ssh_create_kset):
    the shells follow |n|^2, not the list order, so the counts and means match the oracle's on the same list."""
    d, N = 2, 800
    L = N ** 0.5
    n = oracle_mod.kset(d, N, L, K=2 * math.pi / L * 9.5)
    n = n[np.random.default_rng(8).permutation(len(n))][: len(n) - 7]   # shuffled, a few dropped
    s = synth.positions(35, N, d)
    ctx = ssh.Context(d, N, L, kset=n)
    ctx.set_positions_frac(s)
    ctx.energy_grad(ssh.FX)
    sf = ctx.structure_factor(6, 80, 1.0)
    counts, mean, tau = oracle_mod.structure_factor(s, None, ctx.kset(), L, 6, 80, 1.0, nthreads=NTHREADS)
    assert np.array_equal(sf["counts"], counts)
    assert np.all(np.abs((sf["mean"][:, 0] - mean[:, 0]) + (sf["mean"][:, 1] - mean[:, 1])) <= 1e-26)
    assert abs((sf["tau"][0] - tau[0]) + (sf["tau"][1] - tau[1])) <= 1e-26 * max(1.0, tau[0])
    ctx.close()
