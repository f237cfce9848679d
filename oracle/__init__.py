"""Oracle for the stealthy-hyperuniform energy, force and FIRE quench (arXiv:2304.09139).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / reference arm may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or calls it, and the two share no code.

The arithmetic lives in ``oracle.c`` (IEEE binary128 via libquadmath, one ``sincosq`` per
(k, particle) pair, index-order sums, OpenMP across k and across particles).  This module only
builds that file with gcc and marshals numpy arrays through ctypes.  Each wrapper names the
paper's equation it evaluates.

Parity pins for every function live in ``tests/test_oracle.py``.  The FIRE trajectory is
"parity unpinned" by design: trajectories are chaotic and the ground state is degenerate, so
minimised states are judged by S_max only.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_oracle.so (gcc, -O2, OpenMP, libquadmath)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lquadmath", "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


class FireParams(ctypes.Structure):
    _fields_ = [("dt0", ctypes.c_double), ("dt_max", ctypes.c_double), ("alpha_start", ctypes.c_double),
                ("f_alpha", ctypes.c_double), ("f_inc", ctypes.c_double), ("f_dec", ctypes.c_double),
                ("n_min", ctypes.c_int), ("max_steps", ctypes.c_int64), ("smax_target", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int32
            lib.oracle_chi_to_m.restype = i64
            lib.oracle_chi_to_m.argtypes = [ctypes.c_int, i64, d]
            lib.oracle_kset.restype = ctypes.c_int
            lib.oracle_kset.argtypes = [ctypes.c_int, i64, d, d, d, i64, P(i32), P(i64)]
            lib.oracle_ntilde.restype = ctypes.c_int
            lib.oracle_ntilde.argtypes = [ctypes.c_int, i64, P(d), P(d), i64, P(i32), P(d), P(d), ctypes.c_int]
            lib.oracle_phi_grad.restype = ctypes.c_int
            lib.oracle_phi_grad.argtypes = [ctypes.c_int, i64, d, P(d), P(d), i64, P(i32), P(d), P(d), P(d),
                                            P(d), P(d), ctypes.c_int]
            lib.oracle_phi_grad_w.restype = ctypes.c_int
            lib.oracle_phi_grad_w.argtypes = [ctypes.c_int, i64, d, P(d), P(d), i64, P(i32), P(d), P(d), P(d), P(d),
                                              P(d), P(d), ctypes.c_int]
            lib.oracle_force_at.restype = ctypes.c_int
            lib.oracle_force_at.argtypes = [ctypes.c_int, i64, d, P(d), P(d), i64, P(i32), P(d), P(d), P(d), P(d),
                                            ctypes.c_int]
            lib.oracle_fire.restype = ctypes.c_int
            lib.oracle_fire.argtypes = [ctypes.c_int, i64, d, P(d), P(d), i64, P(i32), P(FireParams), P(i64),
                                        P(d), P(d), ctypes.c_int]
            lib.oracle_structure_factor.restype = ctypes.c_int
            lib.oracle_structure_factor.argtypes = [ctypes.c_int, i64, d, P(d), P(d), i64, P(i32), ctypes.c_int, i64,
                                                    d, P(i64), P(d), P(d), ctypes.c_int]
            lib.oracle_g2.restype = ctypes.c_int
            lib.oracle_g2.argtypes = [ctypes.c_int, i64, d, i64, d, ctypes.c_int, P(ctypes.c_uint64), P(d), P(d)]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def chi_to_m(d: int, N: int, chi: float) -> int:
    """M = round-half-even(chi d (N-1)), the inverse of chi = M / (d (N-1)) (Definitions, Eq. for chi)."""
    return int(_load().oracle_chi_to_m(d, N, chi))


def kset(d: int, N: int, L: float, chi: float = 0.0, K: float = 0.0) -> np.ndarray:
    """Independent wavevectors n (k = 2 pi n / L) of the half-space, sorted by (|n|^2, lex) (Definitions)."""
    lib = _load()
    M = ctypes.c_int64(0)
    rc = lib.oracle_kset(d, N, L, chi, K, 0, None, ctypes.byref(M))
    if rc != 0:
        raise ValueError(f"oracle_kset rejected d={d} N={N} L={L} chi={chi} K={K} (rc={rc})")
    out = np.zeros((max(M.value, 1), d), dtype=np.int32)
    rc = lib.oracle_kset(d, N, L, chi, K, M.value, _ip(out), ctypes.byref(M))
    if rc != 0:
        raise RuntimeError(f"oracle_kset failed rc={rc}")
    return out[:M.value].copy()


def kset_region(d: int, N: int, L: float, axis_weights, chi: float = 0.0, K: float = 0.0) -> np.ndarray:
    """An anisotropic exclusion region by brute force (Definitions, with the ball |n|^2 <= R^2 replaced by
    sum_a w_a n_a^2 <= R^2): the half-space vectors (first non-zero component positive) of the region, ordered by
    that norm, then lexicographically; K mode keeps every one with norm <= (K L / 2 pi)^2 (1 + 1e-12), chi mode
    the first round-half-even(chi d (N - 1))."""
    import itertools
    import mpmath
    w = np.asarray(axis_weights, dtype=np.int64).reshape(d)

    def region(r2):
        R = [int(math.isqrt(r2 // int(w[a]))) + 1 for a in range(d)]
        pts = np.array(list(itertools.product(*[range(-R[a], R[a] + 1) for a in range(d)])), dtype=np.int64)
        q = (pts ** 2 * w[None, :]).sum(1)
        nz = pts != 0
        first = pts[np.arange(len(pts)), np.argmax(nz, axis=1)]
        keep = (q <= r2) & nz.any(1) & (first > 0)
        pts, q = pts[keep], q[keep]
        order = np.lexsort(tuple(pts[:, a] for a in range(d - 1, -1, -1)) + (q,))
        return pts[order]

    if K > 0:
        with mpmath.workdps(40):
            r2 = int(mpmath.floor((mpmath.mpf(K) * L / (2 * mpmath.pi)) ** 2 * (1 + mpmath.mpf("1e-12"))))
        out = region(r2)
    else:
        M = chi_to_m(d, N, chi)
        r2 = 1
        while True:
            out = region(r2)
            if len(out) >= M:
                break
            r2 *= 2
        out = out[:M]
    return out.astype(np.int32)


def pair_histogram(s_hi, L: float, n_ref: int, r_max: float, nbins: int) -> np.ndarray:
    """Ordered pairs (i < n_ref, j != i) by minimum-image distance (the pair correlation function's histogram, the
    supplement's Fig. S1b), decided in exact integers: coordinates floor(s 2^32), differences wrapped to the
    nearest image, squared distances summed exactly, bin b for E_b <= r2 < E_(b+1), E_b = ceil(b^2 q^2 / nbins^2),
    q = floor(r_max / L 2^32)."""
    s = np.asarray(s_hi, dtype=np.float64)
    s = s.reshape(s.shape[0], -1)
    u = np.floor(s * 2.0 ** 32).astype(np.int64)
    q = int(math.floor(r_max / L * 2.0 ** 32))
    E = np.array([-(-(b * b * q * q) // (nbins * nbins)) for b in range(nbins + 1)], dtype=object)
    Eu = np.array([int(x) for x in E], dtype=np.uint64)
    counts = np.zeros(nbins, dtype=np.int64)
    for i in range(n_ref):
        dx = (u[i][None, :] - u + 2 ** 31) % 2 ** 32 - 2 ** 31
        dx = np.delete(dx, i, axis=0)
        ok = np.all(np.abs(dx) < q, axis=1)
        r2 = (dx[ok].astype(np.uint64) ** 2).sum(1, dtype=np.uint64)
        r2 = r2[r2 < Eu[nbins]]
        b = np.searchsorted(Eu, r2, side="right") - 1
        counts += np.bincount(b, minlength=nbins)[:nbins]
    return counts.astype(np.uint64)


def structure_factor(s_hi, s_lo, n, L: float, nbins: int, n2max: int, K: float, nthreads: int = 0):
    """Shell averages of S(k) (Eq. structurefactor) over nbins shells of |n| up to sqrt(n2max), and the truncated
    order metric tau of Eq. tau over every wavevector of n and its mirror, with D = 1 / K; binary128 from the
    particles' own n~.  Shell b holds E_b <= |n|^2 < E_(b+1), E_b = ceil(b^2 n2max / nbins^2) (the last shell
    includes n2max).  Returns (counts int64 [nbins], mean S as [nbins, 2] (hi, lo), tau as (hi, lo))."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    d = n.shape[1]
    s_hi, s_lo = _pos(s_hi, s_lo, d)
    counts = np.zeros(nbins, dtype=np.int64)
    mean = np.zeros((nbins, 2))
    tau = np.zeros(2)
    rc = _load().oracle_structure_factor(d, s_hi.shape[0], L, _dp(s_hi), _dp(s_lo), n.shape[0], _ip(n), nbins,
                                         int(n2max), K, counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         _dp(mean), _dp(tau), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_structure_factor rc={rc}")
    return counts, mean, tau


def g2(counts, d: int, N: int, L: float, n_ref: int, r_max: float):
    """g_2(r) from pair counts (the supplement's Fig. S1b): each shell's count over an ideal gas's expectation,
    n_ref (N - 1) / L^d x the shell's volume.  Returns (shell centres, g_2)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    nb = len(c)
    r = np.zeros(nb)
    g = np.zeros(nb)
    rc = _load().oracle_g2(d, N, L, n_ref, r_max, nb, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _dp(r),
                           _dp(g))
    if rc != 0:
        raise RuntimeError(f"oracle_g2 rc={rc}")
    return r, g


def _pos(s_hi, s_lo, d):
    s_hi = np.ascontiguousarray(s_hi, dtype=np.float64).reshape(-1, d)
    s_lo = np.zeros_like(s_hi) if s_lo is None else np.ascontiguousarray(s_lo, dtype=np.float64).reshape(-1, d)
    return s_hi, s_lo


def ntilde(s_hi, s_lo, n, nthreads: int = 0):
    """(C_k, S_k) with n~(k) = C + iS = sum_j exp(+2 pi i n.s_j) (Eq. ntilde), each as an [M, 2] (hi, lo) array."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    d = n.shape[1]
    s_hi, s_lo = _pos(s_hi, s_lo, d)
    M = n.shape[0]
    C = np.zeros((max(M, 1), 2))
    S = np.zeros((max(M, 1), 2))
    rc = _load().oracle_ntilde(d, s_hi.shape[0], _dp(s_hi), _dp(s_lo), M, _ip(n), _dp(C), _dp(S), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_ntilde rc={rc}")
    return C[:M], S[:M]


def phi_grad(s_hi, s_lo, n, L: float, want_force: bool = True, want_cs: bool = False, nthreads: int = 0,
             weights=None):
    """Phi (Eq. energy, constant dropped), S_max (Eq. smax) and F (Eq. force) in binary128, optionally with a
    weight v~(k) >= 0 per wavevector (Phi = sum v~ |n~|^2, F = -grad Phi, S unweighted).

    Returns a dict with 'phi' and 'smax' as (hi, lo) pairs, 'F' as an [N, d, 2] array (or None), and
    'C', 'S' as [M, 2] arrays when want_cs.
    """
    n = np.ascontiguousarray(n, dtype=np.int32)
    d = n.shape[1]
    s_hi, s_lo = _pos(s_hi, s_lo, d)
    N, M = s_hi.shape[0], n.shape[0]
    phi = np.zeros(2)
    smax = np.zeros(2)
    F = np.zeros((max(N, 1), d, 2)) if want_force else None
    C = np.zeros((max(M, 1), 2)) if want_cs else None
    S = np.zeros((max(M, 1), 2)) if want_cs else None
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(M)
    rc = _load().oracle_phi_grad_w(d, N, L, _dp(s_hi), _dp(s_lo), M, _ip(n), _dp(w), _dp(phi), _dp(smax), _dp(F),
                                   _dp(C), _dp(S), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_phi_grad rc={rc}")
    out = {"phi": phi, "smax": smax, "F": None if F is None else F[:N]}
    if want_cs:
        out["C"], out["S"] = C[:M], S[:M]
    return out


def force_at(s_hi, s_lo, n, L: float, C, S, weights=None, nthreads: int = 0):
    """F (Eq. force, physical units) at the given particles, from given collective densities (C, S) as [M, 2]
    (hi, lo) arrays instead of the particles' own: the force on those particles inside a configuration whose
    n~(k) is C + iS.  Returns an [P, d, 2] array."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    d = n.shape[1]
    s_hi, s_lo = _pos(s_hi, s_lo, d)
    P_, M = s_hi.shape[0], n.shape[0]
    C = np.ascontiguousarray(C, dtype=np.float64).reshape(M, 2)
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(M, 2)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64).reshape(M)
    F = np.zeros((max(P_, 1), d, 2))
    rc = _load().oracle_force_at(d, P_, L, _dp(s_hi), _dp(s_lo), M, _ip(n), _dp(C), _dp(S), _dp(w), _dp(F), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_force_at rc={rc}")
    return F[:P_]


def fire(s_hi, s_lo, n, L: float, *, dt0: float, dt_max: float, alpha_start: float = 0.1, f_alpha: float = 0.99,
         f_inc: float = 1.1, f_dec: float = 0.5, n_min: int = 5, max_steps: int = 100000,
         smax_target: float = 1e-36, nthreads: int = 0):
    """FIRE quench (Bitzek et al. 2006, the paper's minimiser) in binary128 with the energy guard.

    Returns (status, steps, s_hi, s_lo, smax(hi, lo), phi(hi, lo)); status 0 = converged.
    """
    n = np.ascontiguousarray(n, dtype=np.int32)
    d = n.shape[1]
    s_hi, s_lo = _pos(s_hi, s_lo, d)
    s_hi, s_lo = s_hi.copy(), s_lo.copy()
    p = FireParams(dt0, dt_max, alpha_start, f_alpha, f_inc, f_dec, n_min, max_steps, smax_target)
    steps = ctypes.c_int64(0)
    smax = np.zeros(2)
    phi = np.zeros(2)
    st = _load().oracle_fire(d, s_hi.shape[0], L, _dp(s_hi), _dp(s_lo), n.shape[0], _ip(n), ctypes.byref(p),
                             ctypes.byref(steps), _dp(smax), _dp(phi), nthreads)
    if st < 0:
        raise RuntimeError(f"oracle_fire rc={st}")
    return st, steps.value, s_hi, s_lo, smax, phi
