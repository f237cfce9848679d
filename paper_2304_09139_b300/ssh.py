"""Python binding of the C ABI in include/ssh.h (ctypes, argument marshalling only).

Every step of the computation runs in the CUDA library libssh.so next to this file.  There is no
fallback: if the library is missing or cannot be loaded, every call raises.  Build it with
``python -m paper_2304_09139_b300._build`` (or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

FP64, DD, FX = 0, 1, 2
FX_AUTO, FX_INTEGER, FX_TENSOR = 0, 1, 2   # ssh_opts.fx_impl
MIN_FIRE, MIN_LBFGS = 0, 1                 # ssh_min_params.method
PREC_NAMES = {FP64: "fp64", DD: "dd", FX: "fx"}
KERNELS = ["twiddle", "ntilde", "nt_reduce", "finalize", "coef", "force", "f_reduce", "fire",
           "tc_prep", "tc_dens", "tc_finish", "tc_coef", "tc_force", "tc_tables"]

_STATUS = {0: "SSH_OK", 1: "SSH_EINVAL", 2: "SSH_ENOMEM", 3: "SSH_ECUDA", 4: "SSH_ENAN", 5: "SSH_ENOTCONV",
           6: "SSH_ETIMEOUT", 7: "SSH_EBUSY", 8: "SSH_ENOTFOUND"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libssh.so")

_lock = threading.Lock()
_lib = None


class MinParams(ctypes.Structure):
    """ssh_min_params (include/ssh.h); zero fields take the library defaults."""
    _fields_ = [("dt0", ctypes.c_double), ("dt_max", ctypes.c_double), ("alpha_start", ctypes.c_double),
                ("f_alpha", ctypes.c_double), ("f_inc", ctypes.c_double), ("f_dec", ctypes.c_double),
                ("n_min", ctypes.c_int), ("n_stages", ctypes.c_int), ("stage_prec", ctypes.c_int * 3),
                ("method", ctypes.c_int), ("stage_floor", ctypes.c_double * 3), ("stall_window", ctypes.c_int64 * 3),
                ("max_steps", ctypes.c_int64), ("smax_target", ctypes.c_double), ("chunk", ctypes.c_int64),
                ("max_seconds", ctypes.c_double)]


class MinResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("final_prec", ctypes.c_int), ("stages_used", ctypes.c_int),
                ("pad0", ctypes.c_int), ("steps", ctypes.c_int64), ("stage_steps", ctypes.c_int64 * 3),
                ("rejected", ctypes.c_int64), ("smax", ctypes.c_double * 2), ("phi", ctypes.c_double * 2),
                ("dt", ctypes.c_double), ("wall_s", ctypes.c_double), ("stage_wall_s", ctypes.c_double * 3)]

    def as_dict(self):
        return {"status": self.status, "final_prec": self.final_prec, "stages_used": self.stages_used,
                "steps": self.steps, "stage_steps": list(self.stage_steps), "rejected": self.rejected,
                "smax": list(self.smax), "phi": list(self.phi), "dt": self.dt, "wall_s": self.wall_s,
                "stage_wall_s": list(self.stage_wall_s)}


class ServerOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_slots", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64),
                ("chunk_steps", ctypes.c_int64), ("max_pairs_per_step", ctypes.c_int64), ("policy", ctypes.c_int),
                ("fx_impl", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("want_positions", ctypes.c_int), ("N", ctypes.c_int64),
                ("L", ctypes.c_double), ("chi", ctypes.c_double), ("K", ctypes.c_double),
                ("s_hi", ctypes.POINTER(ctypes.c_double)), ("s_lo", ctypes.POINTER(ctypes.c_double)),
                ("params", ctypes.POINTER(MinParams))]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("final_prec", ctypes.c_int), ("has_positions", ctypes.c_int),
                ("pad0", ctypes.c_int), ("steps", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("smax", ctypes.c_double * 2), ("phi", ctypes.c_double * 2), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {"status": self.status, "final_prec": self.final_prec, "has_positions": bool(self.has_positions),
                "steps": self.steps, "rejected": self.rejected, "smax": list(self.smax), "phi": list(self.phi),
                "t_submit": self.t_submit, "t_admit": self.t_admit, "t_done": self.t_done}


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "converged", "running", "queued",
                                              "hbm_used_bytes")]


class SshError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


P = ctypes.POINTER
c_d, c_i64, c_i32, c_int, c_vp = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p


def _sig(lib, name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args


def load():
    """Load libssh.so (raises OSError if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError(f"CUDA library not built: {LIB_PATH} is missing "
                              "(run python -m paper_2304_09139_b300._build)")
            lib = ctypes.CDLL(LIB_PATH)
            _sig(lib, "ssh_version", ctypes.c_char_p, [])
            _sig(lib, "ssh_last_error", ctypes.c_char_p, [])
            _sig(lib, "ssh_create", c_int, [c_int, c_i64, c_d, c_d, c_d, c_vp, P(c_vp)])
            _sig(lib, "ssh_destroy", None, [c_vp])
            _sig(lib, "ssh_get_dims", c_int, [c_vp, P(c_int), P(c_i64), P(c_i64), P(c_d)])
            _sig(lib, "ssh_get_kset", c_int, [c_vp, P(c_i64), P(c_i32)])
            _sig(lib, "ssh_get_fx_impl", c_int, [c_vp, P(c_int)])
            _sig(lib, "ssh_get_tc_chunks", c_int, [c_vp, P(c_int), P(c_i64)])
            _sig(lib, "ssh_get_tc_plan", c_int, [c_vp, P(c_int), P(c_int), P(c_int), P(c_int)])
            _sig(lib, "ssh_set_weights", c_int, [c_vp, P(c_d)])
            _sig(lib, "ssh_get_positions", c_int, [c_vp, P(c_d), P(c_d)])
            _sig(lib, "ssh_pair_histogram", c_int, [c_vp, c_i64, c_d, c_int, P(ctypes.c_uint64)])
            _sig(lib, "ssh_g2", c_int, [c_int, c_i64, c_d, c_i64, c_d, c_int, P(ctypes.c_uint64), P(c_d), P(c_d)])
            _sig(lib, "ssh_structure_factor", c_int, [c_vp, c_int, c_i64, c_d, P(c_i64), P(c_d), P(c_d), P(c_d)])
            _sig(lib, "ssh_create_kset", c_int, [c_int, c_i64, c_d, c_i64, P(c_i32), c_vp, P(c_vp)])
            _sig(lib, "ssh_kset_build_region", c_int, [c_int, c_i64, c_d, c_d, c_d, P(c_i32), c_i64, P(c_i32), P(c_i64)])
            _sig(lib, "ssh_kset_build", c_int, [c_int, c_i64, c_d, c_d, c_d, c_i64, P(c_i32), P(c_i64)])
            _sig(lib, "ssh_set_stream", c_int, [c_vp, c_vp])
            _sig(lib, "ssh_sync", c_int, [c_vp])
            _sig(lib, "ssh_set_positions", c_int, [c_vp, P(c_d), P(c_d)])
            _sig(lib, "ssh_set_positions_frac", c_int, [c_vp, P(c_d), P(c_d)])
            _sig(lib, "ssh_get_positions_frac", c_int, [c_vp, P(c_d), P(c_d)])
            _sig(lib, "ssh_energy_grad", c_int, [c_vp, c_int, P(c_d), P(c_d), P(c_d), P(c_d)])
            _sig(lib, "ssh_eval", c_int, [c_vp, c_int, c_int])
            _sig(lib, "ssh_get_results", c_int, [c_vp, P(c_d), P(c_d), P(c_d), P(c_d)])
            _sig(lib, "ssh_get_ntilde", c_int, [c_vp, P(c_d), P(c_d), P(c_d), P(c_d)])
            _sig(lib, "ssh_prof_enable", c_int, [c_vp, c_int])
            _sig(lib, "ssh_prof_read", c_int, [c_vp, c_int, P(c_d), P(c_i64)])
            _sig(lib, "ssh_set_wait_limit", c_int, [c_int, c_i64])
            _sig(lib, "ssh_gemm_counters", c_int, [c_int, c_int])
            _sig(lib, "ssh_gemm_counters_read", c_int, [c_int, P(ctypes.c_uint64)])
            _sig(lib, "ssh_pipe_rate", c_int, [c_int, c_int, P(c_d), P(c_d)])
            _sig(lib, "ssh_shard_words", c_int, [c_vp, P(c_i64), P(c_i64)])
            _sig(lib, "ssh_shard_density", c_int, [c_vp, c_vp])
            _sig(lib, "ssh_shard_finish", c_int, [c_vp, c_vp, c_int])
            _sig(lib, "ssh_shard_fire_begin", c_int, [c_vp, P(MinParams)])
            _sig(lib, "ssh_shard_step_dots", c_int, [c_vp, c_vp])
            _sig(lib, "ssh_shard_step_move", c_int, [c_vp, c_vp, c_vp])
            _sig(lib, "ssh_shard_step_finish", c_int, [c_vp, c_vp])
            _sig(lib, "ssh_ntilde_noalloc", c_int, [c_int, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                                   c_vp])
            _sig(lib, "ssh_min_defaults", c_int, [c_vp, P(MinParams)])
            _sig(lib, "ssh_minimize", c_int, [c_vp, P(MinParams), P(MinResult)])
            _sig(lib, "ssh_fire_begin", c_int, [c_vp, P(MinParams)])
            _sig(lib, "ssh_fire_steps", c_int, [c_vp, c_int, c_i64])
            _sig(lib, "ssh_fire_state", c_int, [c_vp, P(MinResult), P(c_int)])
            _sig(lib, "ssh_batch_create", c_int, [c_vp, P(c_vp)])
            _sig(lib, "ssh_batch_destroy", None, [c_vp])
            _sig(lib, "ssh_batch_add", c_int, [c_vp, c_int, c_i64, c_d, c_d, c_d, P(c_d), P(c_d), P(c_int)])
            _sig(lib, "ssh_batch_size", c_int, [c_vp, P(c_int), P(c_i64)])
            _sig(lib, "ssh_batch_member", c_int, [c_vp, c_int, P(c_vp)])
            _sig(lib, "ssh_batch_eval", c_int, [c_vp, c_int, c_int])
            _sig(lib, "ssh_batch_autotune", c_int, [c_vp, c_int, c_int, P(TuneReport)])
            _sig(lib, "ssh_batch_minimize", c_int, [c_vp, P(MinParams), c_i64, c_d, P(MinResult)])
            _sig(lib, "ssh_batch_begin", c_int, [c_vp, P(MinParams)])
            _sig(lib, "ssh_batch_steps", c_int, [c_vp, c_i64])
            _sig(lib, "ssh_batch_prof_enable", c_int, [c_vp, c_int])
            _sig(lib, "ssh_batch_prof_read", c_int, [c_vp, c_int, P(c_d), P(c_i64)])
            _sig(lib, "ssh_server_create", c_int, [P(ServerOpts), P(c_vp)])
            _sig(lib, "ssh_server_destroy", None, [c_vp])
            _sig(lib, "ssh_submit", c_int, [c_vp, P(Request), P(ctypes.c_uint64)])
            _sig(lib, "ssh_poll", c_int, [c_vp, ctypes.c_uint64, P(Result)])
            _sig(lib, "ssh_result_positions", c_int, [c_vp, ctypes.c_uint64, P(c_d), P(c_d)])
            _sig(lib, "ssh_release", c_int, [c_vp, ctypes.c_uint64])
            _sig(lib, "ssh_cancel", c_int, [c_vp, ctypes.c_uint64])
            _sig(lib, "ssh_server_get_stats", c_int, [c_vp, P(ServerStats)])
            _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        raise SshError(status, load().ssh_last_error().decode(errors="replace"))


def _dp(a):
    return None if a is None else a.ctypes.data_as(P(c_d))


def version() -> str:
    return load().ssh_version().decode()


def kset_build(d: int, N: int, L: float, chi: float = 0.0, K: float = 0.0) -> np.ndarray:
    """Host-only wavevector set (public order) with the library's own rules; no GPU needed."""
    lib = load()
    M = c_i64(0)
    _check(lib.ssh_kset_build(d, N, L, chi, K, 0, None, ctypes.byref(M)))
    out = np.zeros((max(M.value, 1), d), dtype=np.int32)
    _check(lib.ssh_kset_build(d, N, L, chi, K, M.value, out.ctypes.data_as(P(c_i32)), ctypes.byref(M)))
    return out[:M.value].copy()


def kset_region(d: int, N: int, L: float, axis_weights, chi: float = 0.0, K: float = 0.0) -> np.ndarray:
    """Host-only wavevectors of the anisotropic exclusion region sum_a w_a n_a^2 <= R^2 (integer w_a >= 1), in the
    order (that norm, lexicographic); pass the result to Context(..., kset=...)."""
    lib = load()
    w = np.ascontiguousarray(axis_weights, dtype=np.int32).reshape(d)
    wp = w.ctypes.data_as(P(c_i32))
    M = c_i64(0)
    _check(lib.ssh_kset_build_region(d, N, L, chi, K, wp, 0, None, ctypes.byref(M)))
    out = np.zeros((max(M.value, 1), d), dtype=np.int32)
    _check(lib.ssh_kset_build_region(d, N, L, chi, K, wp, M.value, out.ctypes.data_as(P(c_i32)), ctypes.byref(M)))
    return out[:M.value].copy()


def g2(counts, d: int, N: int, L: float, n_ref: int, r_max: float):
    """g_2(r) from pair_histogram counts (ssh_g2): (bin centres, g_2), each bin's count over the count an ideal gas
    of the same density gives in that shell."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    r = np.zeros(len(c))
    g = np.zeros(len(c))
    _check(load().ssh_g2(d, N, L, n_ref, r_max, len(c), c.ctypes.data_as(P(ctypes.c_uint64)), _dp(r), _dp(g)))
    return r, g


def ntilde_noalloc(d: int, N: int, M: int, s_hi_ptr: int, s_lo_ptr: int | None, n_ptr: int, C_hi_ptr: int,
                   C_lo_ptr: int, S_hi_ptr: int, S_lo_ptr: int, stream_ptr: int | None = None):
    """ssh_ntilde_noalloc with raw device pointers (allocation-free n~(k); enqueued, not synchronised)."""
    _check(load().ssh_ntilde_noalloc(d, N, M, s_hi_ptr, s_lo_ptr, n_ptr, C_hi_ptr, C_lo_ptr, S_hi_ptr, S_lo_ptr,
                                     stream_ptr))


PIPES = {"fp64_fma": 0, "fp32_fma": 1, "imad": 2, "imad_hi": 3, "dd_cmac": 4, "fx_cmul": 5}


def pipe_rate(kind: str, device: int = 0) -> tuple[float, float]:
    """ssh_pipe_rate: (operations per second, ms of the timed launch) of one pipe (a key of PIPES)."""
    r, ms = c_d(), c_d()
    _check(load().ssh_pipe_rate(device, PIPES[kind], ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value


def set_wait_limit(cycles: int, device: int = 0):
    """ssh_set_wait_limit: the tensor-core GEMM's wait limit in clock cycles on `device` (0: the default)."""
    _check(load().ssh_set_wait_limit(device, cycles))


GEMM_COUNTER_FIELDS = ("cycles", "producer_wait_stage", "mma_wait_operands", "mma_wait_accumulator", "mma_wait_item",
                       "epilogue_wait_accumulator", "epilogue_readout", "epilogue_math", "items", "ksteps",
                       "mma_thread_cycles", "t0_ns", "t1_ns")


def gemm_counters(enable: bool, device: int = 0):
    """ssh_gemm_counters: switch every tensor-core GEMM launch of the process to the counting instance (on) or back."""
    _check(load().ssh_gemm_counters(device, 1 if enable else 0))


def gemm_counters_read(device: int = 0) -> np.ndarray:
    """ssh_gemm_counters_read: uint64 [2][256][16], [0] the last density launch, [1] the last force launch, a row per
    CTA; the fields are GEMM_COUNTER_FIELDS."""
    out = np.zeros((2, 256, 16), dtype=np.uint64)
    _check(load().ssh_gemm_counters_read(device, out.ctypes.data_as(P(ctypes.c_uint64))))
    return out


def _rows(a, N, d):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(N, d)
    return a


class Context:
    """One configuration (d, N, L, chi | K) resident on the GPU.  Wraps ssh_create / ssh_destroy."""

    def __init__(self, d: int, N: int, L: float, chi: float = 0.0, K: float = 0.0, device: int = 0,
                 fx_impl: int = 0, tc_chunk: int = 0, kset=None, shard=None, _handle=None):
        """kset: an explicit [M, d] wavevector list (ssh_create_kset) in place of chi / K.  shard: (first, count), a
        particle shard of the configuration (ssh_opts.shard_first / shard_count; evaluate with the shard_* methods)."""
        lib = load()
        self._lib = lib
        self._owned = _handle is None
        self._h = c_vp()
        if _handle is None:
            sf, sn = shard if shard is not None else (0, 0)
            opts = (c_int * 8)(device, fx_impl, tc_chunk, sf, sn, 0, 0, 0)  # ssh_opts
            if kset is not None:
                n = np.ascontiguousarray(kset, dtype=np.int32).reshape(-1, d)
                _check(lib.ssh_create_kset(d, N, L, n.shape[0], n.ctypes.data_as(P(c_i32)), ctypes.cast(opts, c_vp),
                                           ctypes.byref(self._h)))
            else:
                _check(lib.ssh_create(d, N, L, chi, K, ctypes.cast(opts, c_vp), ctypes.byref(self._h)))
        else:
            self._h = _handle
        dd_, NN, MM, LL = c_int(), c_i64(), c_i64(), c_d()
        _check(lib.ssh_get_dims(self._h, ctypes.byref(dd_), ctypes.byref(NN), ctypes.byref(MM), ctypes.byref(LL)))
        self.d, self.N, self.M, self.L = dd_.value, NN.value, MM.value, LL.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h and self._owned:
            self._lib.ssh_destroy(self._h)
        self._h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def fx_impl(self) -> int:
        """FX_INTEGER or FX_TENSOR: the implementation of this context's fixed-point evaluations."""
        v = ctypes.c_int()
        _check(self._lib.ssh_get_fx_impl(self._h, ctypes.byref(v)))
        return v.value

    def set_weights(self, w=None):
        """Weights v~(k) in the order of kset() (None: all 1): Phi = sum v~ |n~|^2 and F = -grad Phi."""
        if w is None:
            _check(self._lib.ssh_set_weights(self._h, None))
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            if w.shape != (self.M,):
                raise ValueError(f"need {self.M} weights")
            _check(self._lib.ssh_set_weights(self._h, _dp(w)))

    def pair_histogram(self, n_ref: int, r_max: float, nbins: int) -> np.ndarray:
        """Counts of ordered pairs (i < n_ref, j != i) by minimum-image distance in nbins bins on [0, r_max)
        (ssh_pair_histogram; exact integer decisions); g2() turns them into g_2(r)."""
        out = np.zeros(nbins, dtype=np.uint64)
        _check(self._lib.ssh_pair_histogram(self._h, n_ref, r_max, nbins, out.ctypes.data_as(P(ctypes.c_uint64))))
        return out

    def structure_factor(self, nbins: int, n2max: int | None = None, K: float | None = None) -> dict:
        """Shell averages of S(k) and the order metric tau (Eq. tau) from the last evaluation
        (ssh_structure_factor): shells of |n| up to sqrt(n2max) (default: the largest |n|^2 of the set), tau with
        D = 1 / K (default: the largest |k| of the set).  Returns counts [nbins], mean [nbins, 2] (dd), tau (hi,
        lo) and k_mid [nbins]."""
        counts = np.zeros(nbins, dtype=np.int64)
        mean = np.zeros((nbins, 2))
        tau = np.zeros(2)
        k_mid = np.zeros(nbins)
        _check(self._lib.ssh_structure_factor(self._h, nbins, int(n2max or 0), float(K or 0.0),
                                              counts.ctypes.data_as(P(c_i64)),
                                              _dp(mean), _dp(tau), _dp(k_mid)))
        return {"counts": counts, "mean": mean, "tau": tau, "k_mid": k_mid}

    # ---- particle shards (ssh_shard_*): device buffers are passed as raw pointers (e.g. torch data_ptr())
    def shard_words(self) -> tuple[int, int]:
        """(int64 words of the density exchange, binary64 words of the dot-product exchange)."""
        a, b = c_i64(), c_i64()
        _check(self._lib.ssh_shard_words(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def shard_density(self, dens_out: int):
        _check(self._lib.ssh_shard_density(self._h, dens_out))

    def shard_finish(self, dens_total: int, want_force: bool = True):
        _check(self._lib.ssh_shard_finish(self._h, dens_total, 1 if want_force else 0))

    def shard_fire_begin(self, params: MinParams | None = None, **kw):
        p = params if params is not None else self.min_defaults()
        for k, v in kw.items():
            setattr(p, k, v)
        _check(self._lib.ssh_shard_fire_begin(self._h, ctypes.byref(p)))

    def shard_step_dots(self, dots_out: int):
        _check(self._lib.ssh_shard_step_dots(self._h, dots_out))

    def shard_step_move(self, dots_total: int, dens_out: int):
        _check(self._lib.ssh_shard_step_move(self._h, dots_total, dens_out))

    def shard_step_finish(self, dens_total: int):
        _check(self._lib.ssh_shard_step_finish(self._h, dens_total))

    @property
    def tc_chunks(self) -> tuple[int, int]:
        """(number of particle chunks, particles per chunk) of the tensor-core path; (0, 0) on the integer pipes."""
        n, c = c_int(), c_i64()
        _check(self._lib.ssh_get_tc_chunks(self._h, ctypes.byref(n), ctypes.byref(c)))
        return n.value, c.value

    @property
    def tc_plan(self) -> dict:
        """The tensor-core density tile plan (ssh_get_tc_plan): row tiles, column tiles, tiles in use, transposed."""
        v = [c_int() for _ in range(4)]
        _check(self._lib.ssh_get_tc_plan(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("row_tiles", "col_tiles", "tiles", "transposed"), (x.value for x in v)))

    def kset(self) -> np.ndarray:
        out = np.zeros((max(self.M, 1), self.d), dtype=np.int32)
        M = c_i64(0)
        _check(self._lib.ssh_get_kset(self._h, ctypes.byref(M), out.ctypes.data_as(P(c_i32))))
        return out[:self.M].copy()

    def set_stream(self, stream_ptr: int | None):
        _check(self._lib.ssh_set_stream(self._h, c_vp(stream_ptr) if stream_ptr else None))

    def sync(self):
        _check(self._lib.ssh_sync(self._h))

    def set_positions_frac(self, s_hi, s_lo=None):
        s_hi = _rows(s_hi, self.N, self.d)
        s_lo = _rows(s_lo, self.N, self.d)
        _check(self._lib.ssh_set_positions_frac(self._h, _dp(s_hi), _dp(s_lo)))

    def set_positions(self, r_hi, r_lo=None):
        r_hi = _rows(r_hi, self.N, self.d)
        r_lo = _rows(r_lo, self.N, self.d)
        _check(self._lib.ssh_set_positions(self._h, _dp(r_hi), _dp(r_lo)))

    def positions(self):
        """Current positions in physical units, r = L s, as (hi, lo) [N, d] arrays (ssh_get_positions)."""
        hi = np.zeros((self.N, self.d))
        lo = np.zeros((self.N, self.d))
        _check(self._lib.ssh_get_positions(self._h, _dp(hi), _dp(lo)))
        return hi, lo

    def positions_frac(self):
        hi = np.zeros((self.N, self.d))
        lo = np.zeros((self.N, self.d))
        _check(self._lib.ssh_get_positions_frac(self._h, _dp(hi), _dp(lo)))
        return hi, lo

    def eval(self, prec: int, want_force: bool = True):
        _check(self._lib.ssh_eval(self._h, prec, 1 if want_force else 0))

    def results(self, want_force: bool = True):
        phi = np.zeros(2)
        smax = np.zeros(2)
        Fh = np.empty((self.N, self.d)) if want_force else None   # every entry is written (or the call raises)
        Fl = np.empty((self.N, self.d)) if want_force else None
        _check(self._lib.ssh_get_results(self._h, _dp(phi), _dp(smax), _dp(Fh), _dp(Fl)))
        return {"phi": phi, "smax": smax, "F_hi": Fh, "F_lo": Fl}

    def energy_grad(self, prec: int, want_force: bool = True):
        """Phi, S_max (dd pairs) and F (physical units, hi and lo [N, d]) through ssh_energy_grad."""
        phi = np.zeros(2)
        smax = np.zeros(2)
        Fh = np.empty((self.N, self.d)) if want_force else None   # every entry is written (or the call raises)
        Fl = np.empty((self.N, self.d)) if want_force else None
        _check(self._lib.ssh_energy_grad(self._h, prec, _dp(phi), _dp(smax), _dp(Fh), _dp(Fl)))
        return {"phi": phi, "smax": smax, "F_hi": Fh, "F_lo": Fl}

    def prof_enable(self, on: bool = True):
        _check(self._lib.ssh_prof_enable(self._h, 1 if on else 0))

    def prof_read(self):
        """{kernel name: (total ms, launches)} since the last prof_enable."""
        ms = np.zeros(16)
        n = np.zeros(16, dtype=np.int64)
        _check(self._lib.ssh_prof_read(self._h, 16, _dp(ms), n.ctypes.data_as(P(c_i64))))
        return {KERNELS[i]: (float(ms[i]), int(n[i])) for i in range(len(KERNELS)) if n[i] > 0}

    def min_defaults(self) -> MinParams:
        p = MinParams()
        _check(self._lib.ssh_min_defaults(self._h, ctypes.byref(p)))
        return p

    def minimize(self, params: MinParams | None = None, stages=None, check: bool = False, **kw) -> dict:
        """Run ssh_minimize.  `stages` is a list of precisions (e.g. [FP64, DD]); keyword arguments set
        ssh_min_params fields.  Returns the result as a dict (its 'status' is the ssh_status code); with
        check=True a non-OK status raises."""
        p = params if params is not None else self.min_defaults()
        if stages is not None:
            p.n_stages = len(stages)
            for i, st in enumerate(stages):
                p.stage_prec[i] = st
        for k, v in kw.items():
            if k in ("stage_floor", "stall_window"):
                arr = getattr(p, k)
                for i, x in enumerate(v):
                    arr[i] = x
            else:
                setattr(p, k, v)
        r = MinResult()
        st = self._lib.ssh_minimize(self._h, ctypes.byref(p), ctypes.byref(r))
        if check:
            _check(st)
        return r.as_dict()

    def fire_begin(self, params: MinParams | None = None, **kw):
        p = params if params is not None else self.min_defaults()
        for k, v in kw.items():
            setattr(p, k, v)
        _check(self._lib.ssh_fire_begin(self._h, ctypes.byref(p)))

    def fire_steps(self, prec: int, nsteps: int):
        _check(self._lib.ssh_fire_steps(self._h, prec, nsteps))

    def fire_state(self) -> dict:
        r = MinResult()
        run = c_int(0)
        _check(self._lib.ssh_fire_state(self._h, ctypes.byref(r), ctypes.byref(run)))
        d = r.as_dict()
        d["running"] = bool(run.value)
        return d

    def ntilde(self):
        """(C, S) of the last evaluation, each an [M, 2] (hi, lo) array in public order."""
        ch, cl, sh, sl = (np.zeros(self.M) for _ in range(4))
        _check(self._lib.ssh_get_ntilde(self._h, _dp(ch), _dp(cl), _dp(sh), _dp(sl)))
        return np.stack([ch, cl], 1), np.stack([sh, sl], 1)


def _params(params, stages=None, **kw):
    p = params if params is not None else MinParams()
    if stages is not None:
        p.n_stages = len(stages)
        for i, st in enumerate(stages):
            p.stage_prec[i] = st
    for k, v in kw.items():
        if k in ("stage_floor", "stall_window"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


class TuneReport(ctypes.Structure):
    _fields_ = [("dens_pieces_pct", ctypes.c_int), ("force_bundles", ctypes.c_int), ("ms_default", ctypes.c_double),
                ("ms_tuned", ctypes.c_double), ("candidates", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class Batch:
    """Many configurations evaluated and minimised through the same launches (ssh_batch_*)."""

    def __init__(self, device: int = 0, fx_impl: int = 0):
        self._lib = load()
        self._h = c_vp()
        opts = (c_int * 8)(device, fx_impl, 0, 0, 0, 0, 0, 0)
        _check(self._lib.ssh_batch_create(ctypes.cast(opts, c_vp), ctypes.byref(self._h)))
        self._members = []

    def close(self):
        if self._h:
            for m in self._members:
                m._h = c_vp()
            self._lib.ssh_batch_destroy(self._h)
            self._h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, d, N, L, s_hi, s_lo=None, chi=0.0, K=0.0) -> int:
        s_hi = _rows(s_hi, N, d)
        s_lo = _rows(s_lo, N, d)
        slot = c_int(0)
        _check(self._lib.ssh_batch_add(self._h, d, N, L, chi, K, _dp(s_hi), _dp(s_lo), ctypes.byref(slot)))
        h = c_vp()
        _check(self._lib.ssh_batch_member(self._h, slot.value, ctypes.byref(h)))
        self._members.append(Context(0, 0, 0.0, _handle=h))
        return slot.value

    def autotune(self, prec: int = 2, reps: int = 5) -> dict:
        """ssh_batch_autotune: time the candidate work decompositions of the tensor-core GEMMs for this mix and keep
        the fastest (results are unchanged bit for bit)."""
        r = TuneReport()
        _check(self._lib.ssh_batch_autotune(self._h, prec, reps, ctypes.byref(r)))
        return {"dens_pieces_pct": r.dens_pieces_pct, "force_bundles": r.force_bundles, "ms_default": r.ms_default,
                "ms_tuned": r.ms_tuned, "candidates": r.candidates}

    def member(self, slot: int) -> Context:
        return self._members[slot]

    def size(self):
        n, pairs = c_int(0), c_i64(0)
        _check(self._lib.ssh_batch_size(self._h, ctypes.byref(n), ctypes.byref(pairs)))
        return n.value, pairs.value

    def eval(self, prec: int, want_force: bool = True):
        _check(self._lib.ssh_batch_eval(self._h, prec, 1 if want_force else 0))

    def minimize(self, params: MinParams | None = None, stages=None, chunk_steps: int = 0, max_seconds: float = 0.0,
                 **kw):
        n = self.size()[0]
        res = (MinResult * max(n, 1))()
        p = _params(params, stages, **kw)
        st = self._lib.ssh_batch_minimize(self._h, ctypes.byref(p), chunk_steps, max_seconds, res)
        return st, [res[i].as_dict() for i in range(n)]

    def begin(self, params: MinParams | None = None, stages=None, **kw):
        p = _params(params, stages, **kw)
        _check(self._lib.ssh_batch_begin(self._h, ctypes.byref(p)))

    def steps(self, nsteps: int):
        _check(self._lib.ssh_batch_steps(self._h, nsteps))

    def prof_enable(self, on: bool = True):
        _check(self._lib.ssh_batch_prof_enable(self._h, 1 if on else 0))

    def prof_read(self):
        ms = np.zeros(16)
        n = np.zeros(16, dtype=np.int64)
        _check(self._lib.ssh_batch_prof_read(self._h, 16, _dp(ms), n.ctypes.data_as(P(c_i64))))
        return {KERNELS[i]: (float(ms[i]), int(n[i])) for i in range(len(KERNELS)) if n[i] > 0}


class Server:
    """Continuous-batching minimisation service (ssh_server_*): submit, poll, collect."""

    def __init__(self, device: int = 0, max_slots: int = 256, hbm_budget_bytes: int = 64 << 30,
                 chunk_steps: int = 32, max_pairs_per_step: int = 0, fifo: bool = False, fx_impl: int = 0):
        self._lib = load()
        self._h = c_vp()
        o = ServerOpts(device, max_slots, hbm_budget_bytes, chunk_steps, max_pairs_per_step, 1 if fifo else 0,
                       fx_impl)
        _check(self._lib.ssh_server_create(ctypes.byref(o), ctypes.byref(self._h)))
        self._keep = {}

    def close(self):
        if self._h:
            self._lib.ssh_server_destroy(self._h)
            self._h = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, d, N, L, s_hi, s_lo=None, chi=0.0, K=0.0, params: MinParams | None = None,
               want_positions: bool = False) -> int:
        s_hi = _rows(s_hi, N, d)
        s_lo = _rows(s_lo, N, d)
        q = Request(d, 1 if want_positions else 0, N, L, chi, K, _dp(s_hi), _dp(s_lo),
                    ctypes.pointer(params) if params is not None else None)
        t = ctypes.c_uint64(0)
        _check(self._lib.ssh_submit(self._h, ctypes.byref(q), ctypes.byref(t)))
        self._keep[t.value] = (d, N)
        return t.value

    def poll(self, ticket: int):
        """The result dict when finished, None while queued or running."""
        r = Result()
        st = self._lib.ssh_poll(self._h, ticket, ctypes.byref(r))
        if st == 7:
            return None
        _check(st)
        return r.as_dict()

    def positions(self, ticket: int):
        d, N = self._keep[ticket]
        hi = np.zeros((N, d))
        lo = np.zeros((N, d))
        _check(self._lib.ssh_result_positions(self._h, ticket, _dp(hi), _dp(lo)))
        return hi, lo

    def release(self, ticket: int):
        _check(self._lib.ssh_release(self._h, ticket))

    def cancel(self, ticket: int):
        _check(self._lib.ssh_cancel(self._h, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(self._lib.ssh_server_get_stats(self._h, ctypes.byref(s)))
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}
