"""The paper's system size on the tensor-core path: d = 2, N = 2 x 10^6 at unit density, chi = 0.10
(M = 400000, 8 x 10^11 pairs per sum, one particle chunk) and chi = 0.40 (M = 1600000, several chunks), in the
launch configuration of a plain evaluation (Eqs. ntilde, energy and force of arXiv:2304.09139).

The oracle cannot sum every pair of a random configuration at this size, so two kinds of input are used.

Uniform random points (chi = 0.10): n~ on 48 sampled wavevectors against the binary128 oracle, each a full sum
over the 2 x 10^6 particles; Phi and S_max against the library's own (C, S); F against the integer-pipe
implementation within the normwise bound, and sum_j F_j = 0.

Columns (chi = 0.10 and 0.40): N = 128 x 15625 particles at (m / 128, y_i), m = 0..127, with 15625 random y_i,
and then 64 of them moved to random points.  Before the move the sum over m of e^{2 pi i n_1 m / 128} vanishes
unless 128 divides n_1 (a geometric series; the lattice closed form pinned in the oracle tests), and is 128
when it does, so n~(n) = 128 [128 | n_1] sum_i e^{2 pi i n_2 y_i} + sum over the moved particles of (new - old)
phasors, exactly.  The oracle evaluates each of those sums (15625 and 2 x 64 particles), so every n~(k) and the
force on 64 sampled particles (from the oracle's own (C, S) over all M wavevectors) are checked against it.
"""
import math
import os

import numpy as np
import pytest

from paper_2304_09139_b300 import ssh, synth

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 8
TOL = 1e-28


def ddv(x):
    return x[..., 0] + x[..., 1]


def ddiff(a, b):
    return (a[..., 0] - b[..., 0]) + (a[..., 1] - b[..., 1])


@pytest.fixture(scope="module")
def built():
    from paper_2304_09139_b300 import _build
    _build.build()
    ssh.load()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return True


def test_paper_scale_d2_sampled(built, oracle_mod):
    cfg = synth.PAPER_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    res = {}
    for impl in (ssh.FX_TENSOR, ssh.FX_INTEGER):
        ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=impl)
        assert ctx.fx_impl == impl
        n = ctx.kset()
        assert ctx.M == 400_000
        ctx.set_positions_frac(s)
        r = ctx.energy_grad(ssh.FX)
        C, S = ctx.ntilde()
        res[impl] = (r, C, S)
        ctx.close()
    N = cfg.N
    rng = np.random.default_rng(2_000_000)
    pick = np.sort(np.concatenate([[0, len(n) - 1], rng.choice(np.arange(1, len(n) - 1), 46, replace=False)]))
    Cr, Sr = oracle_mod.ntilde(s, None, n[pick], nthreads=NTHREADS)
    for impl, (r, C, S) in res.items():
        assert np.all(np.abs(ddiff(C[pick], Cr)) <= TOL * N), (impl, np.abs(ddiff(C[pick], Cr)).max())
        assert np.all(np.abs(ddiff(S[pick], Sr)) <= TOL * N), (impl, np.abs(ddiff(S[pick], Sr)).max())
    (rt, Ct, St), (ri, Ci, Si) = res[ssh.FX_TENSOR], res[ssh.FX_INTEGER]
    assert np.all(np.abs(ddiff(Ct, Ci)) <= 2 * TOL * N) and np.all(np.abs(ddiff(St, Si)) <= 2 * TOL * N)
    # the reduction: Phi = sum |n~|^2 and S_max = max |n~|^2 / N over the returned (C, S)
    a2 = ddv(Ct) ** 2 + ddv(St) ** 2
    phi, smax = float(rt["phi"].sum()), float(rt["smax"].sum())
    assert abs(phi - math.fsum(a2)) <= 1e-12 * phi
    assert abs(smax - a2.max() / N) <= 1e-12 * smax
    # the force of the two implementations, and sum_j F_j = 0
    Cabs = np.abs(ddv(Ci)) + np.abs(ddv(Si)) + math.sqrt(N)
    scale = TOL * 4 * math.pi / cfg.L * (np.abs(n).astype(np.float64) * Cabs[:, None]).sum(0)
    Ft = np.stack([rt["F_hi"], rt["F_lo"]], -1)
    Fi = np.stack([ri["F_hi"], ri["F_lo"]], -1)
    assert np.all(np.abs(ddiff(Ft, Fi)) <= 2 * scale[None, :]), (np.abs(ddiff(Ft, Fi)) / scale[None, :]).max()
    for F in (Ft, Fi):
        tot = np.array([math.fsum(np.concatenate([F[:, a, 0], F[:, a, 1]])) for a in range(cfg.d)])
        assert np.all(np.abs(tot) <= N * scale * 4), (tot, scale)


def _dd_add(a, b):
    """a + b for arrays of (hi, lo) pairs (TwoSum of the high words, then the low words)."""
    s = a[..., 0] + b[..., 0]
    bb = s - a[..., 0]
    e = (a[..., 0] - (s - bb)) + (b[..., 0] - bb) + a[..., 1] + b[..., 1]
    hi = s + e
    return np.stack([hi, e - (hi - s)], -1)


def _columns_configuration(N, q, seed, moved, mseed):
    """Particles (m / q, y_i) for m < q, i < N / q, then `moved` of them (indices drawn with mseed) moved to
    uniform random points: (positions, y, moved indices, their old positions)."""
    Q = N // q
    assert Q * q == N
    y = synth.positions(seed, Q, 1)[:, 0]
    s = np.stack([np.tile(np.arange(q) / q, Q), np.repeat(y, q)], -1)   # exact: q is a power of two
    idx = np.sort(np.random.default_rng(mseed).choice(N, moved, replace=False))
    old = s[idx].copy()
    s[idx] = synth.positions(mseed, moved, 2)
    return s, y, idx, old


def _columns_oracle(oracle_mod, n, y, q, new, old):
    """n~(k) of the columns configuration from the oracle: q sum_i e(n_2 y_i) on the wavevectors with q | n_1, plus
    the moved particles' new phasors minus their old ones."""
    M = len(n)
    C = np.zeros((M, 2))
    S = np.zeros((M, 2))
    col = np.nonzero(n[:, 0] % q == 0)[0]
    if len(col):
        c1, s1 = oracle_mod.ntilde(y[:, None], None, n[col, 1:2], nthreads=NTHREADS)
        C[col] = q * c1   # scaling (hi, lo) by a power of two is exact
        S[col] = q * s1
    cn, sn = oracle_mod.ntilde(new, None, n, nthreads=NTHREADS)
    co, so = oracle_mod.ntilde(old, None, n, nthreads=NTHREADS)
    C = _dd_add(_dd_add(C, cn), -co)
    S = _dd_add(_dd_add(S, sn), -so)
    return C, S


@pytest.mark.parametrize("cfg", [synth.PAPER_D2, synth.PAPER_D2_CHI40], ids=["chi0.10", "chi0.40"])
def test_paper_scale_d2_columns_against_oracle(built, oracle_mod, cfg):
    q = 128
    s, y, idx, old = _columns_configuration(cfg.N, q, cfg.seed, 64, cfg.seed + 100)
    ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    assert ctx.fx_impl == ssh.FX_TENSOR
    nchunk, _ = ctx.tc_chunks
    if cfg.chi >= 0.4:
        assert nchunk >= 2, nchunk   # the chunked path, as the paper-size evaluation at this chi runs it
    n = ctx.kset()
    ctx.set_positions_frac(s)
    r = ctx.energy_grad(ssh.FX)
    C, S = ctx.ntilde()
    ctx.close()
    N, M = cfg.N, len(n)
    Cr, Sr = _columns_oracle(oracle_mod, n, y, q, s[idx], old)
    assert np.all(np.abs(ddiff(C, Cr)) <= TOL * N), np.abs(ddiff(C, Cr)).max()
    assert np.all(np.abs(ddiff(S, Sr)) <= TOL * N), np.abs(ddiff(S, Sr)).max()
    a2 = ddv(Cr) ** 2 + ddv(Sr) ** 2
    phi, smax = float(r["phi"].sum()), float(r["smax"].sum())
    assert abs(phi - math.fsum(a2)) <= 1e-12 * phi
    assert abs(smax - a2.max() / N) <= 1e-12 * smax
    # F at the moved particles and at 56 others, against the oracle's force from its own (C, S)
    rng = np.random.default_rng(cfg.seed + 200)
    pick = np.unique(np.concatenate([idx[:8], rng.choice(N, 56, replace=False)]))
    Fr = oracle_mod.force_at(s[pick], None, n, cfg.L, Cr, Sr, nthreads=NTHREADS)
    Cabs = np.abs(ddv(Cr)) + np.abs(ddv(Sr)) + math.sqrt(N)
    scale = TOL * 4 * math.pi / cfg.L * (np.abs(n).astype(np.float64) * Cabs[:, None]).sum(0)
    F = np.stack([r["F_hi"], r["F_lo"]], -1)
    err = np.abs(ddiff(F[pick], Fr)) / scale[None, :]
    assert np.all(err <= 1.0), err.max()
    tot = np.array([math.fsum(np.concatenate([F[:, a, 0], F[:, a, 1]])) for a in range(cfg.d)])
    assert np.all(np.abs(tot) <= N * scale * 4), (tot, scale)
