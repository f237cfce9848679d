"""Pins for the binary128 oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv:2304.09139 whose quantity it checks and the independent fact used:
closed forms (lattice sums, N = 1, N = 2), the brute-force pair form evaluated with mpmath at 40 digits,
translation invariance and Newton's third law for the force, finite differences of Phi, the exact
expectation E|n~|^2 = N for uniform points, inversion symmetry, and lattice-point counts from Jacobi's
two-square theorem.  A plausible slip in the oracle (a dropped term, a wrong sign, a transposed index,
a missing 2 pi) fails at least one of these.
"""
import math

import mpmath
import numpy as np
import pytest

from paper_2304_09139_b300 import synth

mpmath.mp.dps = 40


def dd(x):
    return float(x[..., 0]) + float(x[..., 1]) if np.ndim(x) == 1 else x[..., 0] + x[..., 1]


def mp_dd(x):
    return mpmath.mpf(float(x[0])) + mpmath.mpf(float(x[1]))


# ------------------------------------------------------------------ k-set (Definitions: k = 2 pi n / L, M, chi)

def jacobi_r2(q):
    """Number of integer (a, b) with a^2 + b^2 = q: 4 (d1(q) - d3(q)) (Jacobi's two-square theorem)."""
    if q == 0:
        return 1
    d1 = sum(1 for t in range(1, q + 1) if q % t == 0 and t % 4 == 1)
    d3 = sum(1 for t in range(1, q + 1) if q % t == 0 and t % 4 == 3)
    return 4 * (d1 - d3)


def jacobi_r4(q):
    """Number of integer (a, b, c, e) with a^2 + b^2 + c^2 + e^2 = q: 8 times the sum of the divisors of q that are
    not multiples of 4 (Jacobi's four-square theorem)."""
    if q == 0:
        return 1
    return 8 * sum(t for t in range(1, q + 1) if q % t == 0 and t % 4 != 0)


def brute_half_ball(d, r2max):
    R = int(math.isqrt(r2max))
    grid = np.stack(np.meshgrid(*([np.arange(-R, R + 1)] * d), indexing="ij"), -1).reshape(-1, d)
    n2 = (grid ** 2).sum(1)
    first_nz = np.array([next((c for c in row if c != 0), 0) for row in grid])
    keep = (n2 <= r2max) & (first_nz > 0)
    return grid[keep], n2[keep]


@pytest.mark.parametrize("r2max", [1, 2, 4, 5, 9, 25, 50, 65])
def test_kset_2d_shell_counts_match_jacobi(oracle_mod, r2max):
    K = 2 * math.pi * math.sqrt(r2max)  # L = 1 so |n| <= sqrt(r2max), boundary inclusive
    n = oracle_mod.kset(2, 10, 1.0, K=K)
    n2 = (n.astype(np.int64) ** 2).sum(1)
    for q in range(1, r2max + 1):
        assert (n2 == q).sum() * 2 == jacobi_r2(q), q   # inversion pairs: half of the shell is independent
    assert len(n) == (sum(jacobi_r2(q) for q in range(0, r2max + 1)) - 1) // 2


@pytest.mark.parametrize("r2max", [1, 3, 7, 12, 30])
def test_kset_4d_shell_counts_match_jacobi(oracle_mod, r2max):
    K = 2 * math.pi * math.sqrt(r2max)  # L = 1 so |n| <= sqrt(r2max), boundary inclusive
    n = oracle_mod.kset(4, 10, 1.0, K=K)
    n2 = (n.astype(np.int64) ** 2).sum(1)
    for q in range(1, r2max + 1):
        assert (n2 == q).sum() * 2 == jacobi_r4(q), q   # inversion pairs: half of the shell is independent
    assert len(n) == (sum(jacobi_r4(q) for q in range(0, r2max + 1)) - 1) // 2


@pytest.mark.parametrize("d,r2max", [(1, 16), (2, 30), (3, 12), (3, 27), (4, 6)])
def test_kset_matches_brute_force_order(oracle_mod, d, r2max):
    n = oracle_mod.kset(d, 10, 2.0, K=2 * math.pi * math.sqrt(r2max) / 2.0)
    g, n2 = brute_half_ball(d, r2max)
    order = np.lexsort(tuple(g[:, i] for i in range(d - 1, -1, -1)) + (n2,))
    assert np.array_equal(n, g[order])


def test_kset_half_space_and_inversion(oracle_mod):
    n = oracle_mod.kset(3, 32768, 32.0, chi=0.40)
    as_set = {tuple(r) for r in n.tolist()}
    assert len(as_set) == len(n)
    for r in n.tolist():
        first = next(c for c in r if c != 0)
        assert first > 0
        assert tuple(-c for c in r) not in as_set


def test_kset_chi_mode_counts(oracle_mod):
    # chi = M / (d (N - 1)) with M rounded half-even: 59.4 -> 59, 8999.1 -> 8999, 39320.4 -> 39320
    assert oracle_mod.chi_to_m(2, 100, 0.30) == 59
    assert oracle_mod.chi_to_m(2, 10_000, 0.45) == 8999
    assert oracle_mod.chi_to_m(3, 32_768, 0.40) == 39320
    assert oracle_mod.chi_to_m(1, 5, 0.375) == 2   # 1.5 -> 2 (half to even)
    assert oracle_mod.chi_to_m(1, 3, 0.25) == 0    # 0.5 -> 0 (half to even)
    n = oracle_mod.kset(2, 10_000, 100.0, chi=0.45)
    assert n.shape == (8999, 2)
    n2 = (n.astype(np.int64) ** 2).sum(1)
    assert np.all(np.diff(n2) >= 0)
    # every vector strictly inside the last (possibly partial) shell is present
    full, _ = brute_half_ball(2, int(n2.max()) - 1)
    assert len(full) == (n2 < n2.max()).sum()


# ------------------------------------------------------------------ n~(k), Phi, F: closed forms

@pytest.mark.parametrize("d,q", [(1, 7), (2, 5), (3, 3)])
def test_lattice_closed_form(oracle_mod, d, q):
    """N = q^d points at s = m/q: n~(k) = prod_a sum_m exp(2 pi i n_a m / q) is N when every n_a = 0 mod q
    and 0 otherwise (geometric sums)."""
    from fractions import Fraction
    hi1 = np.arange(q) / q
    lo1 = np.array([float(Fraction(m, q) - Fraction(float(hi1[m]))) for m in range(q)])  # s = m/q to ~2^-106
    mesh = lambda v: np.stack(np.meshgrid(*([v] * d), indexing="ij"), -1).reshape(-1, d)
    grid, grid_lo = mesh(hi1), mesh(lo1)
    N = len(grid)
    n = oracle_mod.kset(d, N, 1.0, K=2 * math.pi * (q + 0.5))
    C, S = oracle_mod.ntilde(grid, grid_lo, n)
    mult = np.all(n % q == 0, axis=1)
    assert mult.any() and (~mult).any()
    assert np.all(np.abs(dd(C[~mult])) <= 1e-30 * N)
    assert np.all(np.abs(dd(S[~mult])) <= 1e-30 * N)
    assert np.all(np.abs(dd(C[mult]) - N) <= 1e-30 * N)
    assert np.all(np.abs(dd(S[mult])) <= 1e-30 * N)


def test_single_particle(oracle_mod):
    """N = 1: |n~(k)|^2 = 1 for every k, so Phi = M and F = 0 (Eqs. energy, force)."""
    s = np.array([[0.123456789, 0.987654321]])
    n = oracle_mod.kset(2, 1, 3.0, K=2 * math.pi * 5 / 3.0)
    r = oracle_mod.phi_grad(s, None, n, 3.0)
    assert abs(dd(r["phi"]) - len(n)) <= 1e-30 * len(n)
    assert np.all(np.abs(dd(r["F"])) <= 1e-30)
    assert abs(dd(r["smax"]) - 1.0) <= 1e-30


def test_two_particles_closed_form(oracle_mod):
    """N = 2: |n~|^2 = 2 + 2 cos(k.(r1 - r2)) and F_1 = -F_2 = (4 pi / L) sum_k n sin(2 pi n.(s1 - s2))."""
    L = 2.5
    s = np.array([[0.1, 0.7], [0.65, 0.2]])
    s_lo = np.array([[1e-20, -3e-19], [2e-18, 0.0]])
    n = oracle_mod.kset(2, 2, L, K=2 * math.pi * 4.2 / L)
    r = oracle_mod.phi_grad(s, s_lo, n, L)
    sm = [[mpmath.mpf(float(s[j, a])) + mpmath.mpf(float(s_lo[j, a])) for a in range(2)] for j in range(2)]
    phi = mpmath.mpf(0)
    f1 = [mpmath.mpf(0), mpmath.mpf(0)]
    for k in n.tolist():
        th = 2 * mpmath.pi * sum(k[a] * (sm[0][a] - sm[1][a]) for a in range(2))
        phi += 2 + 2 * mpmath.cos(th)
        for a in range(2):
            f1[a] += k[a] * mpmath.sin(th)
    f1 = [4 * mpmath.pi / L * x for x in f1]
    assert abs(mp_dd(r["phi"]) - phi) <= 1e-30 * len(n)
    for a in range(2):
        assert abs(mp_dd(r["F"][0, a]) - f1[a]) <= 1e-29 * len(n) * 4.2
        assert abs(mp_dd(r["F"][1, a]) + f1[a]) <= 1e-29 * len(n) * 4.2


@pytest.mark.parametrize("d,N,seed", [(1, 9, 11), (2, 12, 12), (3, 7, 13)])
def test_pair_form_bruteforce(oracle_mod, d, N, seed):
    """|n~(k)|^2 = N + sum_{j != l} cos(k.(r_j - r_l)) and F_j = (4 pi/L) sum_k n sum_l sin(k.(r_j - r_l)),
    evaluated pair by pair with mpmath at 40 digits: independent of the collective-density form."""
    L = 1.7
    s = synth.positions(seed, N, d)
    n = oracle_mod.kset(d, N, L, chi=0.45)
    r = oracle_mod.phi_grad(s, None, n, L, want_cs=True)
    sm = [[mpmath.mpf(float(x)) for x in row] for row in s]
    phi = mpmath.mpf(0)
    F = [[mpmath.mpf(0)] * d for _ in range(N)]
    smax = mpmath.mpf(0)
    for k in n.tolist():
        a2 = mpmath.mpf(N)
        for j in range(N):
            for l in range(N):
                if j == l:
                    continue
                th = 2 * mpmath.pi * sum(k[a] * (sm[j][a] - sm[l][a]) for a in range(d))
                a2 += mpmath.cos(th)
                sn = mpmath.sin(th)
                for a in range(d):
                    F[j][a] += 4 * mpmath.pi / L * k[a] * sn
        phi += a2
        smax = max(smax, a2 / N)
    scale = len(n) * N
    assert abs(mp_dd(r["phi"]) - phi) <= 1e-30 * scale
    assert abs(mp_dd(r["smax"]) - smax) <= 1e-30 * N
    rk = max(math.sqrt(sum(c * c for c in row)) for row in n.tolist())
    for j in range(N):
        for a in range(d):
            assert abs(mp_dd(r["F"][j, a]) - F[j][a]) <= 1e-29 * scale * rk * 4 * math.pi / L


# ------------------------------------------------------------------ invariants

def test_force_sums_to_zero_and_translation_invariance(oracle_mod):
    """sum_j F_j = 0 (Phi depends only on differences) and Phi, |n~|, F are unchanged by a common shift."""
    cfg = synth.SMALL_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    n = oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    r = oracle_mod.phi_grad(s, None, n, cfg.L, want_cs=True)
    F = r["F"]
    # sum in extended precision: sort-free two-word sum is enough at this size
    tot = [mpmath.fsum([mp_dd(F[j, a]) for j in range(cfg.N)]) for a in range(cfg.d)]
    scale = 4 * math.pi / cfg.L * len(n) * 6.1 * cfg.N
    assert all(abs(t) <= 1e-30 * scale for t in tot)
    shift = np.array([0.3141592653589793, 0.2718281828459045])
    s2 = (s + shift) % 1.0
    s2_lo = (s + shift) - np.floor(s + shift) - s2   # exact remainder of the rounded sum
    r2 = oracle_mod.phi_grad(s2, s2_lo, n, cfg.L, want_cs=True)
    # the rounding of s + shift moves each point by <= 2**-53; compare at that level
    assert abs(dd(r2["phi"]) - dd(r["phi"])) <= 1e-10 * dd(r["phi"])
    a_old = dd(r["C"]) ** 2 + dd(r["S"]) ** 2
    a_new = dd(r2["C"]) ** 2 + dd(r2["S"]) ** 2
    assert np.allclose(a_new, a_old, rtol=1e-10, atol=1e-10)
    assert np.allclose(dd(r2["F"]), dd(F), rtol=1e-9, atol=1e-9 * np.abs(dd(F)).max())


def test_exact_shift_by_lattice_vector_is_bitwise(oracle_mod):
    """A shift by a whole period (s -> s + 1 on one axis, exact in binary128) leaves every output bitwise equal."""
    s = synth.positions(21, 30, 2)
    n = oracle_mod.kset(2, 30, 1.0, chi=0.4)
    r1 = oracle_mod.phi_grad(s, None, n, 1.0, want_cs=True)
    s_lo = np.zeros_like(s)
    s_shift = s.copy()
    s_shift[:, 1] += 1.0
    # s + 1 rounds in double; move the rounding error into the low word so the pair is exact
    s_lo[:, 1] = (s[:, 1] + 1.0) - s_shift[:, 1]
    s_lo[:, 1] = s[:, 1] - (s_shift[:, 1] - 1.0)
    r2 = oracle_mod.phi_grad(s_shift, s_lo, n, 1.0, want_cs=True)
    assert np.allclose(dd(r2["C"]), dd(r1["C"]), rtol=0, atol=1e-28)
    assert np.allclose(dd(r2["S"]), dd(r1["S"]), rtol=0, atol=1e-28)


def test_inversion_symmetry(oracle_mod):
    """S(k) = S(-k) (Definitions): n~(-k) is the complex conjugate of n~(k)."""
    s = synth.positions(31, 200, 3)
    n = oracle_mod.kset(3, 200, 5.0, chi=0.3)
    C1, S1 = oracle_mod.ntilde(s, None, n)
    C2, S2 = oracle_mod.ntilde(s, None, -n)
    assert np.all(np.abs(dd(C1) - dd(C2)) <= 1e-30 * 200)
    assert np.all(np.abs(dd(S1) + dd(S2)) <= 1e-30 * 200)


def test_finite_differences(oracle_mod):
    """F = -grad Phi (Eq. force): central differences in the fractional coordinate converge to -L F at
    second order (the error ratio between steps h and h/2 is about 4)."""
    cfg = synth.SMALL_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    n = oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    F = dd(oracle_mod.phi_grad(s, None, n, cfg.L)["F"])
    for j, a in [(0, 0), (17, 1), (99, 0)]:
        errs = []
        for h in (1e-5, 5e-6):
            lo_p = np.zeros_like(s)
            lo_m = np.zeros_like(s)
            lo_p[j, a] = h
            lo_m[j, a] = -h
            pp = oracle_mod.phi_grad(s, lo_p, n, cfg.L, want_force=False)["phi"]
            pm = oracle_mod.phi_grad(s, lo_m, n, cfg.L, want_force=False)["phi"]
            diff = (mp_dd(pp) - mp_dd(pm)) / (2 * h)
            errs.append(float(abs(diff + cfg.L * F[j, a])))
        assert errs[0] < 1e-6 * abs(cfg.L * F[j, a]) + 1e-3
        assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_uniform_points_mean_structure_factor(oracle_mod):
    """For i.i.d. uniform points E|n~(k)|^2 = N exactly, so mean_k S(k) is 1 within a few / sqrt(M)."""
    N, d = 2000, 2
    s = synth.positions(41, N, d)
    n = oracle_mod.kset(d, N, math.sqrt(N), chi=0.45)
    C, S = oracle_mod.ntilde(s, None, n)
    Sk = (dd(C) ** 2 + dd(S) ** 2) / N
    assert abs(Sk.mean() - 1.0) <= 5.0 / math.sqrt(len(n))
    # S(k) is close to Exp(1): the fraction above 3 is near e^-3 = 0.0498
    assert abs((Sk > 3).mean() - math.exp(-3)) < 0.02


# ------------------------------------------------------------------ the quench (Simulations: FIRE to the minimum)

def test_fire_quench_reaches_stealthy_ground_state(oracle_mod):
    """For chi < 1/2 a quench from a random start reaches a global minimum (Definitions / Simulations), so the
    binary128 FIRE run on the small d=2 workload must end with S_max <= 1e-36.  This pins the method, not a
    trajectory: only the final S_max is checked, recomputed by a fresh Phi evaluation."""
    cfg = synth.SMALL_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    n = oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    k2max = (2 * math.pi / cfg.L) ** 2 * float((n.astype(np.int64) ** 2).sum(1).max())
    dt_max = 1.0 / math.sqrt(2 * cfg.N * k2max)
    st, steps, sh, sl, smax, phi = oracle_mod.fire(s, None, n, cfg.L, dt0=dt_max / 10, dt_max=dt_max,
                                                   max_steps=5000, smax_target=1e-36)
    assert st == 0 and steps < 5000
    r = oracle_mod.phi_grad(sh, sl, n, cfg.L, want_force=False)
    assert dd(r["smax"]) <= 1e-36
    assert dd(r["phi"]) <= len(n) * cfg.N * 1e-36   # Phi = N sum_k S(k) <= N M S_max


# ------------------------------------------------------------------ weights v~(k) (Eqs. energy and force)

def test_weights_indicator_equals_smaller_set(oracle_mod):
    """Weight 1 on the first m wavevectors of the ordered set and 0 on the rest gives exactly the energy and force
    of the first m alone (a zero weight adds exact zeros), and weight 1 everywhere gives the unweighted values."""
    cfg = synth.SMALL_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    n = oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    m = 23
    w = np.zeros(len(n))
    w[:m] = 1.0
    a = oracle_mod.phi_grad(s, None, n, cfg.L, weights=w)
    b = oracle_mod.phi_grad(s, None, n[:m], cfg.L)
    assert np.array_equal(a["phi"], b["phi"]) and np.array_equal(a["F"], b["F"])
    full = oracle_mod.phi_grad(s, None, n, cfg.L)
    ones = oracle_mod.phi_grad(s, None, n, cfg.L, weights=np.ones(len(n)))
    assert np.array_equal(full["phi"], ones["phi"]) and np.array_equal(full["F"], ones["F"])
    assert np.array_equal(full["smax"], a["smax"])  # S(k) carries no weight


def test_weighted_finite_differences(oracle_mod):
    """With weights in [0.5, 2], F = -grad of the weighted Phi: central differences converge at second order."""
    cfg = synth.SMALL_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    n = oracle_mod.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    w = 0.5 + 1.5 * synth.uniform01(31, len(n))
    F = dd(oracle_mod.phi_grad(s, None, n, cfg.L, weights=w)["F"])
    for j, a in [(3, 0), (50, 1)]:
        errs = []
        for h in (1e-5, 5e-6):
            lo_p = np.zeros_like(s)
            lo_m = np.zeros_like(s)
            lo_p[j, a] = h
            lo_m[j, a] = -h
            pp = oracle_mod.phi_grad(s, lo_p, n, cfg.L, want_force=False, weights=w)["phi"]
            pm = oracle_mod.phi_grad(s, lo_m, n, cfg.L, want_force=False, weights=w)["phi"]
            diff = (mp_dd(pp) - mp_dd(pm)) / (2 * h)
            errs.append(float(abs(diff + cfg.L * F[j, a])))
        assert errs[0] < 1e-6 * abs(cfg.L * F[j, a]) + 1e-3
        assert 3.0 < errs[0] / errs[1] < 5.0, errs


# ------------------------------------------------------------------ pair histogram (g_2(r), supplement Fig. S1b)

def test_pair_histogram_square_lattice_closed_form(oracle_mod):
    """On a 16 x 16 square lattice of spacing 1 every particle has r_2(m) neighbours at squared distance m (Jacobi's
    two-square count) within half the box, so with bins of width 1/4 the counts are 256 sum r_2(m) over the m with
    floor(4 sqrt m) = b."""
    g = np.arange(16) / 16.0
    s = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2) + 0.25 / 16
    counts = oracle_mod.pair_histogram(s, 16.0, 256, 7.5, 30)
    want = np.zeros(30, dtype=np.int64)
    for m in range(1, 57):
        want[math.isqrt(16 * m)] += 256 * jacobi_r2(m)
    assert np.array_equal(counts.astype(np.int64), want)


def test_pair_histogram_chain_and_symmetry(oracle_mod):
    """A periodic chain of 32 points, spacing 1: two neighbours at each distance 1..15, in bins of width 1/2 at
    b = 2 m; and for random points the counts with n_ref = N are even (each unordered pair twice)."""
    s = (np.arange(32) + 0.5) / 32.0
    counts = oracle_mod.pair_histogram(s[:, None], 32.0, 32, 15.5, 31)
    want = np.zeros(31, dtype=np.int64)
    want[2:31:2] = 64
    assert np.array_equal(counts.astype(np.int64), want)
    r = synth.positions(5, 300, 2)
    c = oracle_mod.pair_histogram(r, 300 ** 0.5, 300, 0.45 * 300 ** 0.5, 50).astype(np.int64)
    assert np.all(c % 2 == 0) and c.sum() > 0


# ------------------------------------------------------------------ anisotropic exclusion regions (Conclusions)

def _k_for_r2(r2: float, L: float) -> float:
    """A cutoff K whose squared index radius (K L / 2 pi)^2 is r2 (chosen half-way between integers)."""
    return 2 * math.pi * math.sqrt(r2) / L


@pytest.mark.parametrize("d,w,axis,q", [(2, (1, 4), 1, 2), (2, (4, 1), 0, 2), (3, (1, 1, 9), 2, 3),
                                         (3, (9, 1, 1), 0, 3), (3, (1, 4, 1), 1, 2)])
def test_region_square_weight_is_the_ball_rescaled(oracle_mod, d, w, axis, q):
    """With weight q^2 on one axis and 1 on the others, sum_a w_a n_a^2 <= R^2 is the image of the ball's vectors
    whose component on that axis is a multiple of q, divided there by q: the norm is unchanged, division by q keeps
    the signs (so the half space) and the lexicographic order.  The ball comes from oracle.kset, pinned by Jacobi's
    counts and brute force.  A weight applied to the wrong axis, or divided instead of multiplied, fails."""
    L = 10.0
    K = _k_for_r2(300.5 if d == 2 else 60.5, L)
    ball = oracle_mod.kset(d, 100, L, K=K)
    keep = ball[:, axis] % q == 0
    want = ball[keep].copy()
    want[:, axis] //= q
    got = oracle_mod.kset_region(d, 100, L, w, K=K)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("w3,r2", [(3, 200), (5, 333), (7, 1000)])
def test_region_counts_by_columns(oracle_mod, w3, r2):
    """The points of n1^2 + w n2^2 <= r2 counted column by column, sum over n2 of 2 floor(sqrt(r2 - w n2^2)) + 1,
    give the full region; the half space holds (count - 1) / 2 of them, and the chi mode takes the first M of the
    K-mode list."""
    total = sum(2 * math.isqrt(r2 - w3 * b * b) + 1 for b in range(-math.isqrt(r2 // w3), math.isqrt(r2 // w3) + 1))
    L = 10.0
    got = oracle_mod.kset_region(2, 100, L, (1, w3), K=_k_for_r2(r2 + 0.5, L))
    assert len(got) == (total - 1) // 2
    q = (got.astype(np.int64) ** 2 * np.array([1, w3])).sum(1)
    assert np.all(np.diff(q) >= 0) and q.max() <= r2
    N = 200
    M = oracle_mod.chi_to_m(2, N, 0.2)
    chi_set = oracle_mod.kset_region(2, N, L, (1, w3), chi=0.2)
    assert len(chi_set) == M and np.array_equal(chi_set, got[:M])


# ------------------------------------------------------------------ force at chosen particles (Eq. force)

@pytest.mark.parametrize("d,weighted", [(2, False), (3, False), (2, True)])
def test_force_at_equals_the_full_force(oracle_mod, d, weighted):
    """force_at over every particle with the configuration's own (C, S) is the full force of phi_grad (pinned above by
    finite differences and the pair form), to the rounding of (C, S) to double-double."""
    N = 60
    L = N ** (1 / d)
    s = synth.positions(77 + d, N, d)
    n = oracle_mod.kset(d, N, L, chi=0.3)
    w = 0.5 + synth.uniform01(5, len(n)) if weighted else None
    r = oracle_mod.phi_grad(s, None, n, L, want_cs=True, weights=w)
    sel = np.array([0, 7, 31, N - 1])
    F = oracle_mod.force_at(s[sel], None, n, L, r["C"], r["S"], weights=w)
    scale = 4 * math.pi / L * (np.abs(n) * (np.abs(dd(r["C"])) + np.abs(dd(r["S"])) + math.sqrt(N))[:, None]).sum(0)
    assert np.all(np.abs(dd(F) - dd(r["F"][sel])) <= 1e-30 * scale[None, :])


def test_force_at_single_particle_is_zero(oracle_mod):
    """A lone particle feels no force from its own density: with (C, S) = (cos, sin) of its own phases,
    C sin - S cos = 0 term by term."""
    s = synth.positions(9, 1, 2)
    n = oracle_mod.kset(2, 50, 7.0, chi=0.4)
    C, S = oracle_mod.ntilde(s, None, n)
    F = oracle_mod.force_at(s, None, n, 7.0, C, S)
    assert np.all(np.abs(dd(F)) <= 1e-30 * len(n) * 4)


# ------------------------------------------------------------------ post-processing (Eq. tau; the supplement's Fig. S1)

def test_structure_factor_shell_counts_match_jacobi(oracle_mod):
    """Shell populations: shell b holds the half-space vectors with E_b <= |n|^2 < E_(b+1), E_b = ceil(b^2 R^2 /
    nbins^2); in d = 2 a value m >= 1 of |n|^2 has r_2(m) / 2 such vectors (Jacobi's two-square theorem)."""
    L, n2max, nb = 30.0, 400, 7
    n = oracle_mod.kset(2, 5000, L, K=2 * math.pi / L * math.sqrt(n2max + 30))
    s = synth.positions(71, 9, 2)
    counts, _, _ = oracle_mod.structure_factor(s, None, n, L, nb, n2max, 1.0)
    E = [-(-(b * b * n2max) // (nb * nb)) for b in range(nb + 1)]
    want = [sum(jacobi_r2(m) // 2 for m in range(max(E[b], 1), E[b + 1] if b < nb - 1 else n2max + 1))
            for b in range(nb)]
    assert counts.tolist() == want


def test_structure_factor_closed_forms(oracle_mod):
    """N = 1: S(k) = 1 for every k, so every shell's mean is 1 and tau (Eq. tau) vanishes.  A q x q lattice with
    every |n_a| < q: n~(k) = 0, S = 0, and tau = 2 (K L)^d M / N^2 (the integral of [0 - 1]^2 over 2 M cells of volume
    (2 pi / L)^d, divided by (2 pi / K)^d rho^2)."""
    L, K = 7.0, 1.3
    n = oracle_mod.kset(2, 1000, L, K=2 * math.pi / L * 5.5)
    n2max = int((n.astype(np.int64) ** 2).sum(1).max())
    counts, mean, tau = oracle_mod.structure_factor(np.array([[0.3141, 0.2718]]), None, n, L, 6, n2max, K)
    full = counts > 0
    assert counts.sum() == len(n) and full.sum() >= 4 and np.all(mean[~full] == 0)   # |n| < R / 6 holds no vector
    assert np.all(np.abs(mean[full, 0] - 1.0) + np.abs(mean[full, 1]) <= 1e-30)
    assert abs(tau[0]) + abs(tau[1]) <= 1e-50
    q = 8
    g = np.stack(np.meshgrid(np.arange(q), np.arange(q), indexing="ij"), -1).reshape(-1, 2) / q
    counts, mean, tau = oracle_mod.structure_factor(g, None, n, L, 6, n2max, K)
    assert np.all(np.abs(mean[:, 0]) <= 1e-30)
    want = mpmath.mpf(2) * (mpmath.mpf(K) * mpmath.mpf(L)) ** 2 * len(n) / q ** 4
    assert abs(mp_dd(tau) - want) <= 1e-30 * want


def test_structure_factor_two_particles(oracle_mod):
    """N = 2: |n~(k)|^2 = 2 + 2 cos(2 pi n.(s_1 - s_2)), so S(k) = 1 + cos(2 pi n.(s_1 - s_2)) (a closed form
    evaluated here in mpmath); the shell means and tau = 2 (K L)^d / 4 sum_k cos^2 follow, in every dimension."""
    for d, L, K, nb in ((1, 5.0, 2.0, 4), (2, 6.0, 1.1, 5), (3, 4.0, 0.7, 3)):
        n = oracle_mod.kset(d, 400, L, K=2 * math.pi / L * 4.2)
        s = synth.positions(80 + d, 2, d)
        n2 = (n.astype(np.int64) ** 2).sum(1)
        n2max = int(n2.max()) - 1          # the outermost shell left out of the shells, kept in tau
        counts, mean, tau = oracle_mod.structure_factor(s, None, n, L, nb, n2max, K)
        ds = [mpmath.mpf(float(s[0, a])) - mpmath.mpf(float(s[1, a])) for a in range(d)]
        sk = [1 + mpmath.cos(2 * mpmath.pi * sum(int(v[a]) * ds[a] for a in range(d))) for v in n]
        E = [-(-(b * b * n2max) // (nb * nb)) for b in range(nb + 1)]
        for b in range(nb):
            top = E[b + 1] if b < nb - 1 else n2max + 1
            sel = [sk[i] for i in range(len(n)) if E[b] <= n2[i] < top]
            assert counts[b] == len(sel)
            if sel:
                assert abs(mp_dd(mean[b]) - sum(sel) / len(sel)) <= 1e-30
        want = mpmath.mpf(2) * (mpmath.mpf(K) * mpmath.mpf(L)) ** d / 4 * sum((x - 1) ** 2 for x in sk)
        assert abs(mp_dd(tau) - want) <= 1e-30 * want


def test_g2_of_uniform_points_is_one(oracle_mod):
    """An ideal gas has g_2 = 1 at every r: uniform random points (pair counts from the exact histogram) give
    shell values near 1 in d = 1, 2, 3, which fixes the unit-ball volume and the density factor of the
    normalisation (a slip in either moves every shell by a constant factor)."""
    for d, N, nb in ((1, 4000, 8), (2, 3000, 8), (3, 3000, 6)):
        L = N ** (1 / d)
        s = synth.positions(90 + d, N, d)
        counts = oracle_mod.pair_histogram(s, L, 600, 0.45 * L, nb)
        r, g = oracle_mod.g2(counts, d, N, L, 600, 0.45 * L)
        assert np.allclose(r, (np.arange(nb) + 0.5) * 0.45 * L / nb)
        assert abs(g[1:].mean() - 1.0) < 0.02, (d, g)
        assert np.all(np.abs(g[1:] - 1.0) < 0.15), (d, g)
