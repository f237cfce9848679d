"""GPU parity: n~(k), Phi, S_max and F from the CUDA library against the binary128 oracle.

Eqs. ntilde, energy, structurefactor/smax and force of arXiv:2304.09139.  Every comparison is element by
element on the same seeded inputs, with normwise bounds (near a ground state n~ ~ 0, so relative error of
Phi alone is ill-conditioned):
  |dC_k|, |dS_k| <= tol N
  |dPhi|         <= tol * 4 max(Phi, M N)
  |dS_max|       <= tol * 4 (2 sqrt(N S_max) + 1)
  |dF_{j,a}|     <= tol * (4 pi / L) sum_k |n_a| (|C_k| + |S_k| + sqrt N)
with tol = 1e-28 for the double-double and fixed-point arithmetics and 1e-13 for plain FP64.
"""
import math
import os

import numpy as np
import pytest

from paper_2304_09139_b300 import ssh, synth

pytestmark = pytest.mark.gpu

TOL = {ssh.FP64: 1e-13, ssh.DD: 1e-28, ssh.FX: 1e-28}
PRECS = [ssh.FP64, ssh.DD, ssh.FX]
NTHREADS = os.cpu_count() or 8


def ddv(x):
    return x[..., 0] + x[..., 1]


def ddiff(a, b):
    """a - b for dd pairs, accurate when a ~ b: (hi - hi) is exact by Sterbenz, then the lo words."""
    return (a[..., 0] - b[..., 0]) + (a[..., 1] - b[..., 1])


@pytest.fixture(scope="module")
def built():
    from paper_2304_09139_b300 import _build
    _build.build()
    ssh.load()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return True


def check_parity(ctx, s_hi, s_lo, L, prec, ref, n, label=""):
    tol = TOL[prec]
    N, d = s_hi.shape
    M = len(n)
    r = ctx.energy_grad(prec)
    C, S = ctx.ntilde()
    # n~
    assert np.all(np.abs(ddiff(C, ref["C"])) <= tol * N), (label, np.abs(ddiff(C, ref["C"])).max())
    assert np.all(np.abs(ddiff(S, ref["S"])) <= tol * N), (label, np.abs(ddiff(S, ref["S"])).max())
    # Phi, S_max
    phi_ref = ddv(ref["phi"])
    assert abs(ddiff(r["phi"], ref["phi"])) <= tol * 4 * max(phi_ref, M * N), (label, r["phi"], ref["phi"])
    sm = ddv(ref["smax"])
    assert abs(ddiff(r["smax"], ref["smax"])) <= tol * 4 * (2 * math.sqrt(N * sm) + 1), (label, r["smax"], ref["smax"])
    # F (physical units)
    Cabs = np.abs(ddv(ref["C"])) + np.abs(ddv(ref["S"])) + math.sqrt(N)
    scale = tol * 4 * math.pi / L * (np.abs(n).astype(np.float64) * Cabs[:, None]).sum(0)  # [d]
    F = np.stack([r["F_hi"], r["F_lo"]], -1)
    err = np.abs(ddiff(F, ref["F"]))
    assert np.all(err <= scale[None, :]), (label, (err / scale[None, :]).max())
    return r


CASES = [
    # (label, d, N, L, chi, K, seed)
    ("small_d2", 2, 100, 1.0, 0.30, 0.0, 1),
    ("ragged_d2", 2, 333, 333 ** 0.5, 0.45, 0.0, 7),
    ("d1", 1, 257, 257.0, 0.45, 0.0, 8),
    # d = 1 on the tensor cores splits n = 2^b n1 + n2: M = 1800 spans several row and column tiles
    ("d1_wide", 1, 4000, 4000.0, 0.45, 0.0, 16),
    ("d3", 3, 300, 300 ** (1 / 3), 0.40, 0.0, 9),
    ("d3_kmode", 3, 150, 4.0, 0.0, 2 * math.pi * 3.3 / 4.0, 10),
    ("d4", 4, 120, 120 ** 0.25, 0.3, 0.0, 11),
    # four axes: about 150 canonical (n2, n3, n4) (three density row tiles), n1 in [0, 4] (two force column tiles
    # of 4 n1 x 4 axes), 700 particles (a ragged last particle tile)
    ("d4_tiles", 4, 700, 700 ** 0.25, 0.30, 0.0, 19),
    # |n| <= 7.5: about 880 canonical p (fourteen row tiles) and force K ranges of up to seven read-out chunks
    ("d4_wide_kmode", 4, 800, 800 ** 0.25, 0.0, 2 * math.pi * 7.5 / 800 ** 0.25, 20),
    ("fullbits_d4", 4, 300, 300 ** 0.25, 0.30, 0.0, -21),
    ("wide_d2", 2, 2000, 2000 ** 0.5, 0.45, 0.0, 12),
    # positions with full-mantissa bits and low words on every axis (as after minimiser moves); synthetic
    # draws are multiples of 2^-53, which makes every phase reduction exact and hides rounding in it
    ("fullbits_d2", 2, 700, 700 ** 0.5, 0.45, 0.0, -13),
    ("fullbits_d3", 3, 400, 400 ** (1 / 3), 0.40, 0.0, -14),
    # |n| <= 17.5: n1 in [0, 17] (two column tiles of the tensor-core density), about 480 canonical (n2, n3)
    # (eight row tiles), 1500 particles (a ragged last particle tile)
    ("d3_wide_kmode", 3, 1500, 1500 ** (1 / 3), 0.0, 2 * math.pi * 17.5 / 1500 ** (1 / 3), 15),
    # |n| <= 66.5: 67 canonical n2, the last row tile's three (n2 >= 64, n1 <= 18) run as the transposed tile
    ("d2_transposed", 2, 900, 30.0, 0.0, 2 * math.pi * 66.5 / 30.0, 17),
    # |n| <= 79.5: the transposed tile at its limits, 16 p in its 32 columns and n1 <= 47 filling its rows to 128
    ("d2_transposed_full", 2, 600, 25.0, 0.0, 2 * math.pi * 79.5 / 25.0, 18),
]


def impls(d):
    """(fx_impl, precisions to check) per context: the fixed point runs through both implementations."""
    return [(ssh.FX_INTEGER, PRECS), (ssh.FX_TENSOR, [ssh.FX])]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_against_oracle(built, oracle_mod, case):
    label, d, N, L, chi, K, seed = case
    s = synth.positions(abs(seed), N, d)
    # a few coordinates at the edges of the cell and a non-zero low word
    s[0, 0] = 0.0
    s[-1, -1] = 1.0 - 2.0 ** -53
    s_lo = np.zeros_like(s)
    s_lo[1::3, 0] = 2.0 ** -60
    if seed < 0:
        u = synth.uniform01(abs(seed) + 100, N * d).reshape(N, d)
        s = np.sqrt(s) * 0.999999937 + 1e-9 * u          # arbitrary low mantissa bits
        s[: N // 8] *= 0.01                                # many coordinates below 1/64
        s_lo = (u - 0.5) * 2.0 ** -53 * s
    ref = None
    for impl, precs in impls(d):
        ctx = ssh.Context(d, N, L, chi=chi, K=K, fx_impl=impl)
        n = ctx.kset()
        if ref is None:
            assert np.array_equal(n, oracle_mod.kset(d, N, L, chi=chi, K=K))
            ref = oracle_mod.phi_grad(s, s_lo, n, L, want_cs=True, nthreads=NTHREADS)
        ctx.set_positions_frac(s, s_lo)
        for prec in precs:
            check_parity(ctx, s, s_lo, L, prec, ref, n, label=f"{label}/{ssh.PREC_NAMES[prec]}/impl{impl}")
        ctx.close()


def test_parity_medium_d2_full(built, oracle_mod):
    """The d=2, N=10^4, chi=0.45 workload at full size: every output against the oracle."""
    cfg = synth.MEDIUM_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    ref = None
    for impl, precs in impls(cfg.d):
        ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=impl)
        n = ctx.kset()
        if ref is None:
            ref = oracle_mod.phi_grad(s, None, n, cfg.L, want_cs=True, nthreads=NTHREADS)
        ctx.set_positions_frac(s)
        for prec in precs:
            check_parity(ctx, s, None, cfg.L, prec, ref, n, label=f"medium/{ssh.PREC_NAMES[prec]}/impl{impl}")
        ctx.close()


def test_parity_medium_d4_full(built, oracle_mod):
    """The d=4, N=4096, chi=0.30 workload (M = 4914) at full size, in the launch configuration of its bench step
    (on the tensor cores: 11 density row tiles, the force K ranges split in two): every output of both fixed-point
    implementations and the dd path against the binary128 oracle."""
    cfg = synth.MEDIUM_D4
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    ref = None
    for impl, precs in impls(cfg.d):
        ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=impl)
        assert ctx.fx_impl == impl
        n = ctx.kset()
        if ref is None:
            assert np.array_equal(n, oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi))
            ref = oracle_mod.phi_grad(s, None, n, cfg.L, want_cs=True, nthreads=NTHREADS)
        ctx.set_positions_frac(s)
        for prec in precs:
            check_parity(ctx, s, None, cfg.L, prec, ref, n, label=f"medium_d4/{ssh.PREC_NAMES[prec]}/impl{impl}")
        ctx.close()


def test_parity_large_d3_full(built, oracle_mod):
    """The d=3, N=32768, chi=0.40 workload (M = 39320) at full size, in the launch configuration of a plain
    evaluation: every n~(k) against the binary128 oracle (each a full sum over the particles), and F on 64 sampled
    particles against the oracle's force at those particles from its own (C, S) over all M wavevectors, on both
    fixed-point implementations; the two implementations' forces also agree everywhere within the bound."""
    cfg = synth.LARGE_D3
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    res = {}
    for impl in (ssh.FX_TENSOR, ssh.FX_INTEGER):
        ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=impl)
        assert ctx.fx_impl == impl
        n = ctx.kset()
        ctx.set_positions_frac(s)
        r = ctx.energy_grad(ssh.FX)
        C, S = ctx.ntilde()
        res[impl] = (r, C, S)
        ctx.close()
    assert np.array_equal(n, oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi))
    Cr, Sr = oracle_mod.ntilde(s, None, n, nthreads=NTHREADS)
    tol, N = 1e-28, cfg.N
    for impl, (r, C, S) in res.items():
        assert np.all(np.abs(ddiff(C, Cr)) <= tol * N), (impl, np.abs(ddiff(C, Cr)).max())
        assert np.all(np.abs(ddiff(S, Sr)) <= tol * N), (impl, np.abs(ddiff(S, Sr)).max())
    rng = np.random.default_rng(20240)
    pick = np.sort(rng.choice(N, 64, replace=False))
    Fr = oracle_mod.force_at(s[pick], None, n, cfg.L, Cr, Sr, nthreads=NTHREADS)
    Cabs = np.abs(ddv(Cr)) + np.abs(ddv(Sr)) + math.sqrt(N)
    scale = tol * 4 * math.pi / cfg.L * (np.abs(n).astype(np.float64) * Cabs[:, None]).sum(0)
    for impl, (r, C, S) in res.items():
        F = np.stack([r["F_hi"], r["F_lo"]], -1)
        err = np.abs(ddiff(F[pick], Fr)) / scale[None, :]
        assert np.all(err <= 1.0), (impl, err.max())
    (rt, Ct, St), (ri, Ci, Si) = res[ssh.FX_TENSOR], res[ssh.FX_INTEGER]
    Ft = np.stack([rt["F_hi"], rt["F_lo"]], -1)
    Fi = np.stack([ri["F_hi"], ri["F_lo"]], -1)
    assert np.all(np.abs(ddiff(Ft, Fi)) <= 2 * scale[None, :]), (np.abs(ddiff(Ft, Fi)) / scale[None, :]).max()


@pytest.mark.parametrize("d,q,R", [(1, 64, 200.5), (2, 16, 20.5), (3, 8, 10.5)])
def test_lattice_closed_form_on_gpu(built, d, q, R):
    """N = q^d lattice points: n~(k) = 0 unless every n_a = 0 (mod q), where it is N (geometric sums).  Lattice
    phases sit on the axes, where products of rounded phasors are most delicate."""
    g = np.stack(np.meshgrid(*([np.arange(q) / q] * d), indexing="ij"), -1).reshape(-1, d)  # m / q: exact in binary
    N = len(g)
    for impl, precs in impls(d):
        ctx = ssh.Context(d, N, 1.0, K=2 * math.pi * R, fx_impl=impl)
        n = ctx.kset()
        ctx.set_positions_frac(g)
        mult = np.all(n % q == 0, axis=1)
        for prec in precs:
            ctx.energy_grad(prec)
            C, S = ctx.ntilde()
            tol = TOL[prec] * N
            assert np.all(np.abs(ddv(C[~mult])) <= tol) and np.all(np.abs(ddv(S[~mult])) <= tol)
            assert np.all(np.abs(ddv(C[mult]) - N) <= tol) and np.all(np.abs(ddv(S[mult])) <= tol)
        ctx.close()


def test_single_particle_on_gpu(built):
    """N = 1: |n~|^2 = 1 for every k, Phi = M, F = 0."""
    ctx = ssh.Context(3, 1, 2.0, K=2 * math.pi * 4 / 2.0)
    ctx.set_positions_frac(np.array([[0.1234, 0.5678, 0.9012]]))
    for prec in PRECS:
        r = ctx.energy_grad(prec)
        assert abs(ddv(r["phi"]) - ctx.M) <= TOL[prec] * 4 * ctx.M
        assert np.all(np.abs(r["F_hi"]) <= TOL[prec] * 1e3)


def test_repeat_is_bitwise_identical(built):
    """Fixed-order reductions: two evaluations of the same positions agree bit for bit, and so do the replayed
    evaluation graph and direct launches."""
    cfg = synth.MEDIUM_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    for impl, precs in impls(cfg.d):
        ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=impl)
        ctx.set_positions_frac(s)
        for prec in precs:
            a = ctx.energy_grad(prec)
            Ca, Sa = ctx.ntilde()
            b = ctx.energy_grad(prec)
            Cb, Sb = ctx.ntilde()
            assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["F_hi"], b["F_hi"])
            assert np.array_equal(a["F_lo"], b["F_lo"]) and np.array_equal(Ca, Cb) and np.array_equal(Sa, Sb)
            # evaluations replay a captured graph; with the profiler on the same kernels launch directly
            ctx.prof_enable(True)
            c = ctx.energy_grad(prec)
            ctx.prof_enable(False)
            assert np.array_equal(a["phi"], c["phi"]) and np.array_equal(a["F_hi"], c["F_hi"])
            assert np.array_equal(a["F_lo"], c["F_lo"])
        ctx.close()


def test_physical_positions_match_fractional(built):
    """ssh_set_positions (r in [0, L), divided by L in dd) agrees with the exact fractional entry."""
    d, N, L = 2, 500, 500 ** 0.5
    s = synth.positions(77, N, d)
    from fractions import Fraction
    r_hi = s * L
    r_lo = np.array([float(Fraction(x) * Fraction(L) - Fraction(y)) for x, y in zip(s.ravel(), r_hi.ravel())]).reshape(s.shape)
    for impl in (ssh.FX_INTEGER, ssh.FX_TENSOR):
        ctx = ssh.Context(d, N, L, chi=0.3, fx_impl=impl)
        ctx.set_positions_frac(s)
        a = ctx.energy_grad(ssh.FX)
        ctx.set_positions(r_hi, r_lo)
        b = ctx.energy_grad(ssh.FX)
        assert abs(ddiff(a["phi"], b["phi"])) <= 1e-26 * ctx.M * N
        # ssh_get_positions returns r = L s (dd): the given r to dd rounding
        ph, pl = ctx.positions()
        err = np.abs((ph - r_hi) + (pl - r_lo))
        assert err.max() <= 1e-29 * L, err.max()
        ctx.close()


def test_fx_impl_selection(built):
    with ssh.Context(2, 64, 8.0, chi=0.3, fx_impl=ssh.FX_TENSOR) as c:
        assert c.fx_impl == ssh.FX_TENSOR
    with ssh.Context(2, 64, 8.0, chi=0.3, fx_impl=ssh.FX_INTEGER) as c:
        assert c.fx_impl == ssh.FX_INTEGER
    with ssh.Context(3, 64, 4.0, chi=0.3) as c:
        assert c.fx_impl == ssh.FX_TENSOR        # the tensor-core path covers d = 1..4
    with ssh.Context(1, 64, 64.0, chi=0.3) as c:
        assert c.fx_impl == ssh.FX_TENSOR        # d = 1 on two lifted axes
    with ssh.Context(4, 64, 64 ** 0.25, chi=0.3) as c:
        assert c.fx_impl == ssh.FX_TENSOR
    with ssh.Context(4, 64, 64 ** 0.25, chi=0.3, fx_impl=ssh.FX_INTEGER) as c:
        assert c.fx_impl == ssh.FX_INTEGER
    # four axes with a component beyond 64 (the packed sub-vector's limit): the integer pipes serve the set
    far = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 65], [2, -1, 3, 1]], dtype=np.int32)
    with ssh.Context(4, 64, 64 ** 0.25, kset=far, fx_impl=ssh.FX_TENSOR) as c:
        assert c.fx_impl == ssh.FX_INTEGER
    with ssh.Context(4, 64, 64 ** 0.25, kset=far[[0, 1, 3]], fx_impl=ssh.FX_TENSOR) as c:
        assert c.fx_impl == ssh.FX_TENSOR
    with pytest.raises(ssh.SshError):
        ssh.Context(2, 64, 8.0, chi=0.3, fx_impl=7)


def test_bad_inputs_raise(built):
    ctx = ssh.Context(2, 10, 1.0, chi=0.3)
    with pytest.raises(ssh.SshError):
        ctx.energy_grad(ssh.FX)        # no positions yet
    s = synth.positions(1, 10, 2)
    s[3, 1] = float("nan")
    with pytest.raises(ssh.SshError) as e:
        ctx.set_positions_frac(s)
    assert e.value.status == 4
    with pytest.raises(ssh.SshError):
        ctx.eval(7)


def test_positions_wrap_exact(built):
    """Fractional positions are reduced into [0, 1) exactly as dd pairs: values already in [0, 1) with a zero
    low word pass unchanged (-0 becomes +0), and every other value is wrapped by its exact fraction."""
    from fractions import Fraction
    N, d = 16, 2
    hi = np.full((N, d), 0.375)
    lo = np.zeros((N, d))
    cases = [(-0.0, 0.0), (1.0, 0.0), (-3.25, 0.0), (0.5, 1e-20), (0.25, -1e-20), (0.0, -1e-30),
             (0.9999999999999999, 1e-17), (7.125, 2.0 ** -60), (-1e-300, 0.0), (0.0, -0.0), (0.7, 0.0),
             (2.0 ** -1074, 0.0)]
    for i, (h, l) in enumerate(cases):
        hi[i // d, i % d] = h
        lo[i // d, i % d] = l
    with ssh.Context(d, N, 1.0, chi=0.3) as ctx:
        ctx.set_positions_frac(hi, lo)
        gh, gl = ctx.positions_frac()
    for j in range(N):
        for a in range(d):
            x = Fraction(hi[j, a]) + Fraction(lo[j, a])
            f = x - (x.numerator // x.denominator)
            got = Fraction(gh[j, a]) + Fraction(gl[j, a])
            assert got == f, (hi[j, a], lo[j, a], gh[j, a], gl[j, a])
            assert 0 <= got < 1
            if lo[j, a] == 0.0 and 0.0 <= hi[j, a] < 1.0:   # unchanged, with +0 for -0
                assert gh[j, a] == hi[j, a] and gl[j, a] == 0.0
                assert math.copysign(1.0, gh[j, a]) == 1.0 and math.copysign(1.0, gl[j, a]) == 1.0


@pytest.mark.parametrize("d,N,L,chi,chunk", [(2, 10_000, 100.0, 0.45, 2048), (3, 3000, 3000 ** (1 / 3), 0.30, 1024),
                                              (1, 5000, 5000.0, 0.30, 1280), (4, 3000, 3000 ** 0.25, 0.30, 1024)])
def test_chunked_equals_unchunked(built, d, N, L, chi, chunk):
    """Particle chunks on the tensor-core path (ssh_opts.tc_chunk; the last chunk ragged, not a whole number of
    K-steps): the sums are exact integers, so n~, Phi, S_max and F are bit-identical to one chunk, and so is a
    FIRE segment.  At d = 3 and d = 4 these sizes also split the force K ranges (fewer particle-tile items than
    SMs), the same split in every chunk."""
    s = synth.positions(77 + d, N, d)
    out = {}
    for ch in (0, chunk):
        ctx = ssh.Context(d, N, L, chi=chi, fx_impl=ssh.FX_TENSOR, tc_chunk=ch)
        nc, size = ctx.tc_chunks
        if ch:
            assert size == chunk and nc == -(-N // chunk) and nc > 1
        else:
            assert nc == 1
        ctx.set_positions_frac(s)
        r = ctx.energy_grad(ssh.FX)
        C, S = ctx.ntilde()
        fp = ctx.min_defaults()
        fp.n_stages = 1
        fp.stage_prec[0] = ssh.FX
        fp.smax_target = 1e-300
        fp.max_steps = 1 << 40
        ctx.fire_begin(fp)
        ctx.fire_steps(ssh.FX, 20)
        out[ch] = (r, C, S, ctx.positions_frac())
        ctx.close()
    (ra, Ca, Sa, pa), (rb, Cb, Sb, pb) = out[0], out[chunk]
    for k in ("phi", "smax", "F_hi", "F_lo"):
        assert np.array_equal(ra[k], rb[k]), k
    assert np.array_equal(Ca, Cb) and np.array_equal(Sa, Sb)
    assert all(np.array_equal(x, y) for x, y in zip(pa, pb))


@pytest.mark.parametrize("d,N,L,chi", [(1, 300, 300.0, 0.45), (2, 500, 500 ** 0.5, 0.45), (3, 400, 400 ** (1 / 3), 0.40),
                                       (4, 120, 120 ** 0.25, 0.30)])
def test_weighted_parity(built, oracle_mod, d, N, L, chi):
    """Weights v~(k) in [0.25, 4] (every seventh exactly 1, which keeps the exact coefficient path): Phi = sum
    v~ |n~|^2 and F against the oracle in every arithmetic and both fixed-point implementations; n~ and S_max
    carry no weight.  The force bound weights each wavevector's term by its v~."""
    s = synth.positions(90 + d, N, d)
    ref = None
    for impl, precs in impls(d):
        ctx = ssh.Context(d, N, L, chi=chi, fx_impl=impl)
        n = ctx.kset()
        w = 0.25 + 3.75 * synth.uniform01(40 + d, len(n))
        w[::7] = 1.0
        if ref is None:
            ref = oracle_mod.phi_grad(s, None, n, L, want_cs=True, weights=w, nthreads=NTHREADS)
        ctx.set_positions_frac(s)
        ctx.set_weights(w)
        M = len(n)
        for prec in precs:
            tol = TOL[prec]
            r = ctx.energy_grad(prec)
            C, S = ctx.ntilde()
            assert np.all(np.abs(ddiff(C, ref["C"])) <= tol * N) and np.all(np.abs(ddiff(S, ref["S"])) <= tol * N)
            assert abs(ddiff(r["phi"], ref["phi"])) <= tol * 4 * w.max() * max(ddv(ref["phi"]), M * N), (prec, impl)
            sm = ddv(ref["smax"])
            assert abs(ddiff(r["smax"], ref["smax"])) <= tol * 4 * (2 * math.sqrt(N * sm) + 1)
            Cabs = np.abs(ddv(ref["C"])) + np.abs(ddv(ref["S"])) + math.sqrt(N)
            scale = tol * 4 * math.pi / L * (np.abs(n).astype(np.float64) * (w * Cabs)[:, None]).sum(0)
            F = np.stack([r["F_hi"], r["F_lo"]], -1)
            err = np.abs(ddiff(F, ref["F"]))
            assert np.all(err <= scale[None, :]), (prec, impl, (err / scale[None, :]).max())
        # back to unit weights: the unweighted results again
        ctx.set_weights(None)
        r1 = ctx.energy_grad(ssh.FX)
        ref1 = oracle_mod.phi_grad(s, None, n, L, want_force=False, nthreads=NTHREADS)
        assert abs(ddiff(r1["phi"], ref1["phi"])) <= 1e-28 * 4 * max(ddv(ref1["phi"]), M * N)
        ctx.close()


def test_weights_rejected_when_out_of_range(built):
    ctx = ssh.Context(2, 100, 1.0, chi=0.3)
    for bad in (-1.0, float("nan"), 2000.0):
        w = np.ones(ctx.M)
        w[3] = bad
        with pytest.raises(ssh.SshError):
            ctx.set_weights(w)
    ctx.close()


REGION_CASES = [
    # (label, d, N, axis weights or None, chi): anisotropic regions, and sets with gaps (every third vector of
    # the ball dropped), which leave holes in the columns of both fixed-point implementations
    ("aniso_d2", 2, 500, (1, 3), 0.30),
    ("aniso_d3", 3, 400, (1, 2, 5), 0.30),
    ("gaps_d2", 2, 700, None, 0.40),
    ("gaps_d1", 1, 400, None, 0.40),
    ("gaps_d3", 3, 300, None, 0.40),
]


@pytest.mark.parametrize("case", REGION_CASES, ids=[c[0] for c in REGION_CASES])
def test_region_parity(built, oracle_mod, case):
    """Contexts over a given wavevector set (ssh_create_kset): every output against the oracle on the same list,
    in every arithmetic and both fixed-point implementations."""
    label, d, N, w, chi = case
    L = N ** (1 / d)
    if w is not None:
        n = ssh.kset_region(d, N, L, w, chi=chi)
    else:
        ball = ssh.kset_build(d, N, L, chi=chi)
        n = ball[np.arange(len(ball)) % 3 != 1]
    s = synth.positions(60 + d, N, d)
    ref = oracle_mod.phi_grad(s, None, n, L, want_cs=True, nthreads=NTHREADS)
    for impl, precs in impls(d):
        ctx = ssh.Context(d, N, L, kset=n, fx_impl=impl)
        assert ctx.fx_impl == impl and np.array_equal(ctx.kset(), n)
        ctx.set_positions_frac(s)
        for prec in precs:
            check_parity(ctx, s, None, L, prec, ref, n, label=f"{label}/{ssh.PREC_NAMES[prec]}/impl{impl}")
        ctx.close()


@pytest.mark.parametrize("label, d, N, L, chi, K, want", [
    # the d = 2, N = 10^4, chi = 0.45 workload: 76 canonical n2 in two row tiles; the last one's 12 (n1 <= 40) run
    # transposed, so its three (row tile, column tile) pairs become one tile
    ("medium_d2", 2, 10_000, 100.0, 0.45, 0.0, {"row_tiles": 2, "col_tiles": 6, "tiles": 6, "transposed": 1}),
    ("d2_transposed", 2, 900, 30.0, 0.0, 2 * math.pi * 66.5 / 30.0, {"row_tiles": 2, "tiles": 6, "transposed": 1}),
    ("d2_transposed_full", 2, 600, 25.0, 0.0, 2 * math.pi * 79.5 / 25.0, {"row_tiles": 2, "transposed": 1}),
    # one row tile: nothing to transpose
    ("small_d2", 2, 100, 1.0, 0.30, 0.0, {"row_tiles": 1, "transposed": 0}),
    # |n| <= 80.5: 81 canonical n2, 17 in the last row tile, more than its 32 columns hold
    ("d2_no_transpose", 2, 600, 25.0, 0.0, 2 * math.pi * 80.5 / 25.0, {"row_tiles": 2, "transposed": 0}),
    ("d3", 3, 300, 300 ** (1 / 3), 0.40, 0.0, {"transposed": 0}),
])
def test_density_tile_plan(built, label, d, N, L, chi, K, want):
    """The density tile plan of the tensor-core path: which sets run their last row tile transposed."""
    with ssh.Context(d, N, L, chi=chi, K=K, fx_impl=ssh.FX_TENSOR) as ctx:
        plan = ctx.tc_plan
        assert all(plan[k] == v for k, v in want.items()), (label, plan)
