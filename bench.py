"""Throughput of the hot path: one FIRE step = Phi + force (+ minimiser update) on one configuration.

Metric: (k, particle) pairs per second per Phi+grad, pairs = M * N (one of the two sums of
Eqs. ntilde / force; the paper counts the work of one step as two such sums of M N terms).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fx|dd|fp64] [--impl ours|reference]
                  [--workload d2-n10000|d3-n32768]

Default workload: d = 2, N = 10^4 uniform random points (SplitMix64 seed 2) in a periodic square at unit
density (L = 100), chi = 0.45, so M = 8999.  Inputs are resident in HBM when the timed region starts;
L2 (126 MB) is flushed between timed steps by writing a 256 MiB buffer, outside the step's events.
Under torchrun every rank runs its own replica (independent configuration, seed 2 + rank): the path
shards by configuration with no collective; value = pairs of all ranks / max over ranks of the time.

--impl reference times the binary128 oracle (the only reference this method has) on the host cores,
each step a bounded sample of the same workload: the first M/8 wavevectors, all N particles, both sums.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Algorithmic integer multiply-add (IMAD pipe) instructions per (k, particle) pair in the fixed-point
# kernels: one truncated 128x128 top half is 16 32-bit multiply-adds; a complex multiply of first-quadrant
# phasors is three of them; the density kernel does one complex multiply per pair (48), the force kernel one
# (the phase recurrence) plus the two products of C sin - S cos (80).
FX_IMAD_PER_PAIR = {"ntilde": 48, "force": 80}
# Algorithmic FP64 instructions per pair on the double-double path (dd_mul = 8, dd_add = 20 flops as
# written in dd.cuh): density = complex dd multiply (4 mul + 2 add = 72) + complex accumulate (2 add = 40);
# force = complex multiply (72) + w = C sin - S cos (2 mul + 1 add = 36) + A += w, B += A (40).
DD_FP64_PER_PAIR = {"ntilde": 112, "force": 148}
# Tensor-core fixed point: every real product of two 2^-104 fixed-point values is 120 bf16 digit-pair products
# (2 FLOP each).  The density needs 2 real products per (k, particle) pair (4 real products serve k = (n1, p)
# and (n1, -p)), the force 2 d (G and the d - 1 weighted G^a, Re and Im, cos and sin terms, again for both
# signs of p).


def tc_flop_per_pair(d: int) -> dict:
    return {"tc_dens": 2 * 2 * 120, "tc_force": 2 * 2 * d * 120}


F64_FP64_PER_PAIR = {"ntilde": 6, "force": 8}


def pipe_rates_block(ssh, dev) -> dict:
    """Measured operation rates of the pipes the non-tensor arithmetics run on (ssh_pipe_rate: every SM busy with
    independent chains of one operation for about 100 ms, CUDA events, best of three), with the SM count read from
    the device and the SM clock sampled while they run.  The FP64 FMA and IMAD rates are the roofline denominators
    of the dd and integer fixed-point kernels; the nominal figures (unit counts x the maximum clock) are context."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    out = {"sm_count": props.multi_processor_count}
    with Clocks(dev) as clk:
        for kind in ("fp64_fma", "fp32_fma", "imad", "imad_hi", "dd_cmac", "fx_cmul"):
            r, ms = ssh.pipe_rate(kind, dev)
            out[kind] = {"ops_per_s": r, "ms": ms}
    out["clocks"] = clk.summary()
    sm, mhz = props.multi_processor_count, MEASURED.get("sm_max_mhz", 2032.0)
    out["nominal"] = {"fp64_fma": 2 * sm * mhz * 1e6, "imad": 64 * sm * mhz * 1e6,
                      "note": "unit counts x maximum SM clock: 2 FP64 FMA and 64 IMAD lanes per SM per clock"}
    return out


def _measured() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


MEASURED = _measured()


def _measured_bf16_peak() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1e12
    except (OSError, KeyError, ValueError):
        return 1.8e15   # one earlier B300 measurement, used only when the measured file is absent


BF16_PEAK = _measured_bf16_peak()

# The headline workload (the default) and the d = 3 one, selectable with --workload.
WORKLOADS = {"d2-n10000": dict(d=2, N=10_000, L=100.0, chi=0.45, seed=2),
             "d3-n32768": dict(d=3, N=32_768, L=32.0, chi=0.40, seed=3),
             "d4-n4096": dict(d=4, N=4096, L=8.0, chi=0.30, seed=44)}
WORKLOAD = WORKLOADS["d2-n10000"]

# DRAM bytes (read + write) per launch from one ncu capture of this workload (profiles/), valid only while
# the kernel's family of sources hashes to the value recorded with them; otherwise the traffic is reported as null.
NCU_TRAFFIC = {("d2-n10000", "fx", "force"): ("8c0684b40cfa", 35_871_488 + 24_064),
               ("d2-n10000", "fx", "ntilde"): ("8c0684b40cfa", 36_564_736 + 7_424),
               ("d2-n10000", "dd", "force"): ("8c0684b40cfa", 35_895_296 + 0),
               ("d2-n10000", "dd", "ntilde"): ("8c0684b40cfa", 36_669_184 + 512),
               ("d2-n10000", "fx-tensor", "tc_force"): ("44444e97309e", 74_682_624 + 2_351_104),
               ("d2-n10000", "fx-tensor", "tc_dens"): ("44444e97309e", 135_644_928 + 5_040_640),
               ("d3-n32768", "fx-tensor", "tc_force"): ("44444e97309e", 3_583_391_488 + 26_191_104),
               ("d3-n32768", "fx-tensor", "tc_dens"): ("44444e97309e", 3_008_975_360 + 8_591_872),
               ("d4-n4096", "fx-tensor", "tc_force"): ("44444e97309e", 191_571_968 + 4_759_296),
               ("d4-n4096", "fx-tensor", "tc_dens"): ("44444e97309e", 178_693_888 + 4_872_448)}


# The sources each family of kernels is built from: the integer fixed-point and dd kernels, and the tensor-core
# path.  A profile records the hash of its own family's sources.
KERNEL_SOURCES = {"fx": ("kernels.cu", "fx.cuh", "dd.cuh", "reduce.cuh"),
                  "tc": ("tc.cu", "tc.cuh", "fx.cuh", "dd.cuh", "reduce.cuh")}


def kernel_source_hash(family: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_2304_09139_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="fx", choices=["fx", "dd", "fp64"])
    ap.add_argument("--workload", default="d2-n10000", choices=sorted(WORKLOADS),
                    help="the timed configuration: d=2 N=10^4 chi=0.45 (default), d=3 N=32768 chi=0.40 or d=4 N=4096 chi=0.30")
    ap.add_argument("--fx-impl", default="auto", choices=["auto", "integer", "tensor"],
                    help="fixed-point implementation: integer pipes or exact-digit tensor-core GEMMs")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-minimize", action="store_true")
    ap.add_argument("--no-dd-ladder", action="store_true",
                    help="skip the FP64 -> dd and all-dd quenches of the d=2 N=100 and N=10^4 workloads (about 4 min)")
    ap.add_argument("--dd-seconds", type=float, default=300.0, help="wall limit of each dd-ladder quench")
    ap.add_argument("--no-floor", action="store_true", help="skip the quenches to the paper's 1e-50 floor")
    ap.add_argument("--no-d4", action="store_true", help="skip the d=4 block")
    ap.add_argument("--paper-full-quench", action="store_true",
                    help="also quench the paper's d=2 N=2x10^6 chi=0.10 system (an hour or more of GPU time)")
    ap.add_argument("--paper-full-quench-seconds", type=float, default=5400.0)
    ap.add_argument("--no-paper-quench", action="store_true", help="skip the d=2 N=2x10^5 chi=0.10 quenches (about 2 min)")
    ap.add_argument("--no-gemm-counters", action="store_true", help="skip the GEMM cycle-counter block")
    ap.add_argument("--minimize-seconds", type=float, default=150.0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the d=3, N=32768 block")
    ap.add_argument("--large-staged", action="store_true", help="also its staged FP64 -> fixed point quench (about 1 min)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-post", action="store_true", help="skip the pair-histogram (g_2) timing")
    ap.add_argument("--no-paper-scale", action="store_true",
                    help="skip the d=2 N=2x10^6 steps at chi=0.10 and 0.40 (each context holds about 200 GB)")
    ap.add_argument("--serve-seconds", type=float, default=45.0)
    ap.add_argument("--serve-method", default="lbfgs", choices=["lbfgs", "fire"],
                    help="minimiser of the serving requests")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seed(seed: int, rank: int) -> int:
    """Each rank quenches its own configuration (an independent replica): same sizes, its own draw."""
    return seed + rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The slowest rank's time: every rank holds the same per-GPU work, so the job ends with the last one."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(pairs_per_gpu: int, world: int, steps: int, tot_ms: float) -> float:
    """Whole-job throughput: the pairs all ranks processed over the slowest rank's time."""
    return pairs_per_gpu * world * steps / (tot_ms / 1e3)


class Clocks:
    """SM clock and clock-event (throttle) reasons sampled while the timed region runs: through NVML every
    millisecond from a thread (the device found by its PCI bus id), else nvidia-smi -lms 200."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"
    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.thread = None
        self.samples = []
        self.max_mhz = None

    class _Nvml:
        """The driver's NVML through ctypes (reads only): SM clock, maximum SM clock, clock-event reasons."""
        SM = 1  # NVML_CLOCK_SM

        def __init__(self, device: int):
            import ctypes
            import torch
            self.ct = ctypes
            self.lib = ctypes.CDLL("libnvidia-ml.so.1")
            if self.lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            p = torch.cuda.get_device_properties(device)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            self.h = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h)) != 0:
                raise OSError("no NVML device for " + bus.decode())
            self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

        def clock(self, fn="nvmlDeviceGetClockInfo"):
            v = self.ct.c_uint(0)
            if getattr(self.lib, fn)(self.h, self.SM, self.ct.byref(v)) != 0:
                raise OSError(fn)
            return float(v.value)

        def reasons(self):
            v = self.ct.c_ulonglong(0)
            if self.reasons_fn(self.h, self.ct.byref(v)) != 0:
                raise OSError("clock event reasons")
            return int(v.value)

    def _poll(self, nv):
        while not self.stop.is_set():
            try:
                self.samples.append((nv.clock(), nv.reasons()))
            except OSError:
                break
            time.sleep(0.001)

    def __enter__(self):
        import threading
        try:
            nv = self._Nvml(self.device)
            self.max_mhz = nv.clock("nvmlDeviceGetMaxClockInfo")
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(nv,), daemon=True)
            self.thread.start()
            return self
        except Exception:
            self.thread = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.thread:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        if self.thread is not None:
            if not self.samples:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "source": "nvml"}
            reasons = sorted(nm for nm, bit in self.REASONS.items() if any(r & bit for _, r in self.samples))
            return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.samples), "source": "nvml, 1 ms"}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0, "source": "nvidia-smi"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "source": "nvidia-smi, 200 ms"}


def cpu_sample(N, d, L, chi, seed, frac_k=8, nthreads=0, want_cs=False):
    """One bounded oracle Phi+grad sample: the first M/frac_k wavevectors, all particles, both sums.  With
    want_cs also the oracle's (C, S) of those wavevectors ([Ms, 2] dd pairs each)."""
    import oracle
    from paper_2304_09139_b300 import synth
    oracle.build()
    n = oracle.kset(d, N, L, chi=chi)
    Ms = max(1, len(n) // frac_k)
    s = synth.positions(seed, N, d)
    t = time.perf_counter()
    r = oracle.phi_grad(s, None, n[:Ms], L, nthreads=nthreads, want_cs=want_cs)
    dt = time.perf_counter() - t
    out = (Ms * N / dt, Ms, oracle.num_threads() if nthreads == 0 else nthreads)
    return out + ((r["C"], r["S"]),) if want_cs else out


def minimize_block(ssh, synth, w, dev, stream, with_dd=False, max_seconds=150):
    """Time full quenches of the workload from its random start to S_max <= 1e-36 (configs per hour): the
    library's default ladder (all fixed point on a tensor-core context) with FIRE (the paper's minimiser) and
    with L-BFGS, staged FP64 -> fixed point (the paper's cheap first stage), and all fixed point on the integer
    pipes; with_dd also FP64 -> dd and all-dd, the paper's own arithmetic (see dd_ladder_block)."""
    out = {}
    runs = [("default", None), ("lbfgs", None), ("fp64_then_fx", [ssh.FP64, ssh.FX]), ("all_fx", [ssh.FX]),
            ("all_fx_integer", [ssh.FX])]
    if with_dd:
        runs += [("fp64_then_dd", [ssh.FP64, ssh.DD]), ("all_dd", [ssh.DD])]
    for name, stages in runs:
        impl = ssh.FX_INTEGER if name == "all_fx_integer" else ssh.FX_AUTO
        c = ssh.Context(w["d"], w["N"], w["L"], chi=w["chi"], device=dev, fx_impl=impl)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(w["seed"], w["N"], w["d"]))
        r = c.minimize(stages=stages, max_steps=100000, max_seconds=max_seconds,
                       method=ssh.MIN_LBFGS if name == "lbfgs" else ssh.MIN_FIRE)
        ns = r["stages_used"]
        out[name] = {"converged": r["status"] == 0, "status": r["status"], "wall_s": r["wall_s"],
                     "steps": r["steps"], "stage_steps": r["stage_steps"][:ns],
                     "stage_wall_s": r["stage_wall_s"][:ns], "smax": r["smax"][0],
                     "configs_per_hour": 3600.0 / r["wall_s"] if r["status"] == 0 else 0.0}
        c.close()
    return out


def dd_ladder_block(ssh, synth, dev, stream, max_seconds=300.0):
    """The paper's precision ladder in its own arithmetic: FP64 descent to the FP64 floor, then the double-double
    polish, against double-double from the start, both with FIRE (the paper's minimiser) to S_max <= 1e-36 from
    the same random start, on the d=2 N=100 (chi=0.30) and N=10^4 (chi=0.45) workloads.  The staged ladder runs as
    its two stages (FP64 to S_max <= 1e-24 or its stall, then dd; FIRE restarts at a stage either way), and at the
    end of each stage that stage's arithmetic is compared with the binary128 oracle on 256 sampled wavevectors (the
    error of n~ over N).  Each final state is confirmed by the oracle's S_max over every wavevector (one
    evaluation), and configs per hour is 3600 / wall time of the quench."""
    import oracle
    oracle.build()
    out = {}
    for cfg, tag in ((synth.SMALL_D2, "d2_N100"), (synth.MEDIUM_D2, "d2_N10000")):
        blk = {"workload": f"d=2 N={cfg.N} L={cfg.L} chi={cfg.chi}, uniform random (SplitMix64 seed {cfg.seed}), FIRE"}
        for name in ("fp64_then_dd", "all_dd"):
            c = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
            c.set_stream(stream.cuda_stream)
            c.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
            n = c.kset()
            pick = np.sort(np.random.default_rng(7).choice(len(n), min(256, len(n)), replace=False))

            def stage_error(prec):
                c.energy_grad(prec, want_force=False)
                C, S = c.ntilde()
                hi, lo = c.positions_frac()
                ref = oracle.phi_grad(hi, lo, n[pick], cfg.L, want_force=False, want_cs=True)
                return float(max(np.abs((C[pick, 0] - ref["C"][:, 0]) + (C[pick, 1] - ref["C"][:, 1])).max(),
                                 np.abs((S[pick, 0] - ref["S"][:, 0]) + (S[pick, 1] - ref["S"][:, 1])).max()) / cfg.N)
            runs, errs = [], {}
            if name == "fp64_then_dd":
                runs.append(c.minimize(stages=[ssh.FP64], smax_target=1e-24, max_steps=200000, max_seconds=max_seconds))
                errs["fp64"] = stage_error(ssh.FP64)
                if runs[-1]["status"] in (0, 5):
                    runs.append(c.minimize(stages=[ssh.DD], max_steps=200000, max_seconds=max_seconds))
            else:
                runs.append(c.minimize(stages=[ssh.DD], max_steps=200000, max_seconds=max_seconds))
            errs["dd"] = stage_error(ssh.DD)
            hi, lo = c.positions_frac()
            c.close()
            ref = oracle.phi_grad(hi, lo, n, cfg.L, want_force=False)
            r = runs[-1]
            wall = sum(x["wall_s"] for x in runs)
            ok = r["status"] == 0 and len(runs) == (2 if name == "fp64_then_dd" else 1)
            blk[name] = {"converged": ok, "status": r["status"], "wall_s": wall,
                         "steps": sum(x["steps"] for x in runs), "stage_steps": [x["steps"] for x in runs],
                         "stage_wall_s": [x["wall_s"] for x in runs], "smax": r["smax"][0],
                         "oracle_smax": float(ref["smax"][0] + ref["smax"][1]),
                         "stage_error_vs_oracle": errs,
                         "configs_per_hour": 3600.0 / wall if ok else 0.0}
        a, b = blk["fp64_then_dd"], blk["all_dd"]
        blk["staged_over_all_dd_configs_per_hour"] = (a["configs_per_hour"] / b["configs_per_hour"]
                                                      if b["configs_per_hour"] > 0 else None)
        blk["stage_error_note"] = ("max |n~ - n~_oracle| / N over 256 sampled wavevectors at the end of each stage, in "
                                   "that stage's arithmetic (bounds: 1e-13 FP64, 1e-28 dd)")
        out[tag] = blk
    return out


def gemm_counters_block(ssh, synth, dev, stream):
    """Where the tensor-core GEMMs' time goes (ssh_gemm_counters: a counting instance of the kernel records, per CTA,
    clock64 cycles in each wait and phase): one evaluation of the d=2 N=10^4 and d=3 N=32768 workloads after three
    warm ones.  Fractions are of the mean CTA time; cycles per K-step divide the MMA thread's time outside its waits
    by its K-steps.  The counting instance spills a few registers, so its times run slightly above production."""
    f = {n: i for i, n in enumerate(ssh.GEMM_COUNTER_FIELDS)}
    out = {}
    for tag, cfg in (("d2_N10000", synth.MEDIUM_D2), ("d3_N32768", synth.LARGE_D3)):
        c = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        ssh.gemm_counters(True, dev)
        try:
            for _ in range(4):
                c.eval(ssh.FX)
            c.sync()
            rec = ssh.gemm_counters_read(dev).astype(np.float64)
        finally:
            ssh.gemm_counters(False, dev)
            c.close()
        blk = {}
        for kind, name in ((0, "density"), (1, "force")):
            r = rec[kind][rec[kind][:, f["cycles"]] > 0]
            tot = r[:, f["cycles"]].mean()
            waits = r[:, [f["mma_wait_operands"], f["mma_wait_accumulator"], f["mma_wait_item"]]].sum(1)
            blk[name] = {"ctas": int(len(r)), "cta_cycles_mean": tot, "cta_cycles_max": r[:, f["cycles"]].max(),
                         "span_us": (r[:, f["t1_ns"]].max() - r[:, f["t0_ns"]].min()) / 1e3,
                         "end_spread_us": (r[:, f["t1_ns"]].max() - r[:, f["t1_ns"]].min()) / 1e3,
                         "items_per_cta": r[:, f["items"]].mean(), "ksteps_per_cta": r[:, f["ksteps"]].mean(),
                         "mma_cycles_per_kstep": ((r[:, f["mma_thread_cycles"]] - waits) / r[:, f["ksteps"]]).mean(),
                         **{k: r[:, f[k]].mean() / tot for k in ("mma_wait_operands", "mma_wait_accumulator",
                                                                  "mma_wait_item", "producer_wait_stage",
                                                                  "epilogue_wait_accumulator", "epilogue_readout",
                                                                  "epilogue_math")}}
        out[tag] = blk
    return out


def paper_quench_block(ssh, synth, dev, stream, max_seconds=240.0):
    """A full quench toward the paper's size: d=2, N=2x10^5 (a tenth of the paper's 2x10^6) at unit density,
    chi=0.10 (M = 40000, 8x10^9 pairs per sum), from a uniform random start to S_max <= 1e-36 with FIRE (the
    paper's minimiser) and with L-BFGS, in the default fixed point on the tensor cores.  The final state's S(k) is
    confirmed by the binary128 oracle on 400 sampled wavevectors (a full evaluation would take the host minutes)."""
    import oracle
    oracle.build()
    cfg = synth.PAPER_D2_TENTH
    out = {"workload": f"d=2 N={cfg.N} L={cfg.L:.4f} chi={cfg.chi}, uniform random (SplitMix64 seed {cfg.seed})"}
    for method, name in ((ssh.MIN_FIRE, "fire"), (ssh.MIN_LBFGS, "lbfgs")):
        c = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        r = c.minimize(max_steps=1000000, max_seconds=max_seconds, method=method)
        hi, lo = c.positions_frac()
        n = c.kset()
        c.close()
        pick = np.sort(np.random.default_rng(3).choice(len(n), 400, replace=False))
        ref = oracle.phi_grad(hi, lo, n[pick], cfg.L, want_force=False)
        out[name] = {"converged": r["status"] == 0, "status": r["status"], "steps": r["steps"], "wall_s": r["wall_s"],
                     "ms_per_step": 1e3 * r["wall_s"] / max(1, r["steps"]), "smax": r["smax"][0],
                     "oracle_smax_400_sampled_k": float(ref["smax"][0] + ref["smax"][1]),
                     "configs_per_hour": 3600.0 / r["wall_s"] if r["status"] == 0 else 0.0}
    return out


def paper_full_quench_block(ssh, synth, dev, stream, max_seconds=5400.0, method_name="lbfgs"):
    """The paper's own system: d=2, N=2x10^6 at unit density, chi=0.10 (M = 400000), quenched from a uniform random
    start toward S_max <= 1e-36 in the default fixed point on the tensor cores (about 0.87 s per evaluation), for at
    most max_seconds.  Progress (steps, S_max, Phi, seconds) goes to stderr about once a minute and into the block;
    the final state's S(k) is checked by the binary128 oracle on 100 sampled wavevectors (2x10^8 pairs).  Not run by
    default: it holds the GPU for an hour or more."""
    import oracle
    oracle.build()
    cfg = synth.PAPER_D2
    c = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
    try:
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        p = c.min_defaults()
        p.method = ssh.MIN_LBFGS if method_name == "lbfgs" else ssh.MIN_FIRE
        p.max_steps = 10_000_000
        c.fire_begin(p)
        t0 = time.perf_counter()
        prog, last_print = [], 0.0
        st = c.fire_state()
        while st["running"] and time.perf_counter() - t0 < max_seconds:
            c.fire_steps(ssh.FX, 25)
            st = c.fire_state()
            el = time.perf_counter() - t0
            prog.append([round(el, 1), st["steps"], st["smax"][0], st["phi"][0]])
            if el - last_print > 60 or not st["running"]:
                print(f"paper_full_quench {el:.0f} s: {st['steps']} steps, S_max {st['smax'][0]:.3e}, Phi "
                      f"{st['phi'][0]:.3e}", file=sys.stderr, flush=True)
                last_print = el
        wall = time.perf_counter() - t0
        hi, lo = c.positions_frac()
        n = c.kset()
        pick = np.sort(np.random.default_rng(11).choice(len(n), 100, replace=False))
        ref = oracle.phi_grad(hi, lo, n[pick], cfg.L, want_force=False)
        return {"workload": f"d=2 N={cfg.N} L={cfg.L:.4f} chi={cfg.chi} M={c.M}, uniform random (SplitMix64 seed "
                            f"{cfg.seed}), {method_name}, fixed point on the tensor cores",
                "converged": st["status"] == 0 and not st["running"], "status": st["status"], "steps": st["steps"],
                "wall_s": wall, "smax": st["smax"][0], "phi": st["phi"][0],
                "oracle_smax_100_sampled_k": float(ref["smax"][0] + ref["smax"][1]),
                "progress_every_25_steps": prog[::8] + ([prog[-1]] if prog else [])}
    finally:
        c.close()


def d4_block(ssh, synth, dev, stream, pipes):
    """d = 4 (the paper covers d = 1-4): N = 4096 points at unit density, chi = 0.30 (M = 4914).  Per-kernel times
    of one fixed-point evaluation on the tensor cores (the default path; GEMM work against the measured bf16 rate)
    and on the integer pipes (against the measured IMAD rate), and quenches to S_max <= 1e-36 with the default
    ladder (FP64, then fixed point) and with L-BFGS."""
    N, d, chi, seed = 4096, 4, 0.30, 44
    L = N ** (1 / d)
    out = {"workload": f"d=4 N={N} L={L:.4f} chi={chi}, uniform random (SplitMix64 seed {seed})"}
    for tag, impl in (("tensor", ssh.FX_TENSOR), ("integer", ssh.FX_INTEGER)):
        c = ssh.Context(d, N, L, chi=chi, device=dev, fx_impl=impl)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(seed, N, d))
        pairs = c.M * c.N
        used = c.fx_impl
        for _ in range(3):
            c.eval(ssh.FX)
        c.sync()
        reps = 5
        c.prof_enable(True)
        for _ in range(reps):
            c.eval(ssh.FX)
        pr = c.prof_read()
        c.prof_enable(False)
        c.close()
        ms = {k: v[0] / reps for k, v in pr.items()}  # per evaluation (the two finishes share one record name)
        r = {"M": pairs // N, "fx_impl": "tensor" if used == ssh.FX_TENSOR else "integer", "eval_ms": sum(ms.values()),
             "per_kernel_ms": ms, "eval_pairs_per_s": pairs / (sum(ms.values()) * 1e-3)}
        if used == ssh.FX_TENSOR:
            r["bf16_frac_of_measured"] = {k: f * pairs / (ms[k] * 1e-3) / BF16_PEAK
                                          for k, f in tc_flop_per_pair(d).items() if k in ms}
        else:
            r["imad_frac_of_measured"] = {k: FX_IMAD_PER_PAIR[k] * pairs / (ms[k] * 1e-3) / pipes["imad"]["ops_per_s"]
                                          for k in FX_IMAD_PER_PAIR if k in ms}
        out[tag] = r
    for name, method in (("default", ssh.MIN_FIRE), ("lbfgs", ssh.MIN_LBFGS)):
        c = ssh.Context(d, N, L, chi=chi, device=dev)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(seed, N, d))
        r = c.minimize(max_steps=200000, max_seconds=120.0, method=method)
        c.close()
        out[name] = {"converged": r["status"] == 0, "steps": r["steps"], "wall_s": r["wall_s"], "smax": r["smax"][0],
                     "stage_steps": r["stage_steps"][:r["stages_used"]],
                     "configs_per_hour": 3600.0 / r["wall_s"] if r["status"] == 0 else 0.0}
    return out


def floor_block(ssh, synth, dev, stream):
    """The paper's accuracy floor (S_max ~ 1e-51 at the end of its quenches): the default fixed-point ladder quenched
    with FIRE and with L-BFGS to S_max <= 1e-50 from the random starts of the d=2 N=100 (chi=0.30) and N=10^4
    (chi=0.45) workloads, each final state confirmed by the binary128 oracle's S_max over every wavevector; and the
    lowest S_max this arithmetic reaches (target 1e-70, ended by the stall rule) on the N=10^4 workload."""
    import oracle
    oracle.build()
    out = {}
    runs = [(synth.SMALL_D2, "d2_N100", ssh.MIN_FIRE, 1e-50), (synth.SMALL_D2, "d2_N100", ssh.MIN_LBFGS, 1e-50),
            (synth.MEDIUM_D2, "d2_N10000", ssh.MIN_FIRE, 1e-50), (synth.MEDIUM_D2, "d2_N10000", ssh.MIN_LBFGS, 1e-50),
            (synth.MEDIUM_D2, "d2_N10000", ssh.MIN_FIRE, 1e-70)]
    for cfg, tag, method, target in runs:
        c = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        r = c.minimize(max_steps=1000000, max_seconds=60.0, smax_target=target, method=method)
        hi, lo = c.positions_frac()
        n = c.kset()
        c.close()
        ref = oracle.phi_grad(hi, lo, n, cfg.L, want_force=False)
        key = f"{tag}_{'lbfgs' if method == ssh.MIN_LBFGS else 'fire'}_{target:g}"
        out[key] = {"target": target, "converged": r["status"] == 0, "status": r["status"], "steps": r["steps"],
                    "wall_s": r["wall_s"], "smax": r["smax"][0], "oracle_smax": float(ref["smax"][0] + ref["smax"][1]),
                    "phi": r["phi"][0]}
    out["note"] = ("the 1e-70 run stops at the arithmetic's floor (stall rule, status SSH_ENOTCONV); its smax is the "
                   "lowest the fixed point reaches on this workload")
    return out


def dd_roofline_block(ssh, ctx, pairs, fp64_rate, cmac_rate):
    """The double-double kernels against the measured FP64 FMA rate: algorithmic FP64 instructions per pair
    (DD_FP64_PER_PAIR, counted from dd.cuh) x pairs / the kernel's mean event time (the library's profiler, on the
    launching stream), over three evaluations; the density kernel's pair rate also against the measured rate of its
    own inner operation (one complex dd multiply and add)."""
    ctx.eval(ssh.DD)
    ctx.sync()
    ctx.prof_enable(True)
    for _ in range(3):
        ctx.eval(ssh.DD)
    pr = ctx.prof_read()
    ctx.prof_enable(False)
    out = {"bound": "fp64", "unit": "FP64 instr/s", "peak": fp64_rate,
           "peak_source": "ssh_pipe_rate fp64_fma, measured in this run", "kernels": {}}
    for k in ("ntilde", "force"):
        if k not in pr:
            continue
        ms = pr[k][0] / pr[k][1]
        ach = DD_FP64_PER_PAIR[k] * pairs / (ms * 1e-3)
        out["kernels"][k] = {"ms": ms, "achieved": ach, "frac": ach / fp64_rate,
                             "fp64_per_pair": DD_FP64_PER_PAIR[k]}
    if "ntilde" in out["kernels"]:
        out["kernels"]["ntilde"]["frac_of_measured_cmac_rate"] = pairs / (out["kernels"]["ntilde"]["ms"] * 1e-3) / cmac_rate
    out["per_kernel_ms"] = {k: v[0] / v[1] for k, v in pr.items()}
    return out


def batched_block(ssh, synth, dev, steps=5, warmup=2, count=256):
    """One batched FIRE step over the 256-configuration mix (d in {2, 3}, N log-uniform in [64, 8192],
    chi in [0.10, 0.49]): every member's tiles share the same persistent launches."""
    import torch
    cfgs = synth.mixed_batch(4, count)
    b = ssh.Batch(device=dev)
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    n, pairs = b.size()
    b.begin(stages=[ssh.FX], smax_target=1e-300)
    b.steps(warmup)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    b.steps(steps)
    torch.cuda.synchronize(dev)   # the batch works on its own stream: a device-wide synchronisation
    t_default = (time.perf_counter() - t0) / steps
    # the autotuner picks the GEMMs' work decomposition for this mix; the timed steps below use it
    tune = b.autotune(ssh.FX, reps=3)
    b.steps(warmup)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    b.steps(steps)
    torch.cuda.synchronize(dev)
    t = (time.perf_counter() - t0) / steps
    b.prof_enable(True)           # then one profiled step for the per-kernel split
    b.steps(1)
    pr = b.prof_read()
    b.prof_enable(False)
    b.close()
    return {"configs": n, "pairs_per_step": pairs, "ms_per_step": t * 1e3, "pairs_per_s": pairs / t,
            "ms_per_step_default_decomposition": t_default * 1e3, "autotune": tune,
            "per_kernel_ms": {k: v[0] for k, v in pr.items()},
            "workload": "256 configurations, d in {2,3}, N log-uniform [64, 8192], chi U[0.10, 0.49], unit density, "
                        "fixed point, one batched FIRE step (graph replay)"}


def serving_summary(done, tickets, sub_t, sub_work, elapsed, window_s):
    """Latency and load figures of a serving run.  done: ticket -> result (status, steps, t_submit, t_done);
    tickets: every submitted ticket in order, sub_t its submission time and sub_work its M N (same order) in the run's
    clock; elapsed: the run's length.  p50 / p99 cover every submitted request, the unfinished ones censored at the
    end of the run (a lower bound on their latency); the _completed figures cover the finished ones only."""
    ok = [r for r in done.values() if r["status"] == 0]
    lat = sorted(r["t_done"] - r["t_submit"] for r in ok)
    pct = (lambda v, q: float(np.percentile(v, q)) if len(v) else None)
    cens = sorted([r["t_done"] - r["t_submit"] for r in done.values()] +
                  [elapsed - sub_t[t] for t in tickets if t not in done])
    n_sub = len(tickets)
    work = {t: w for t, w in zip(tickets, sub_work)}
    return {"submitted": n_sub, "completed": len(done), "converged": len(ok),
            "completion_fraction": len(done) / n_sub if n_sub else None,
            "p50_s": pct(cens, 50), "p99_s": pct(cens, 99), "latency": "every submitted request, unfinished ones "
            "censored at the end of the run (a lower bound)",
            "p50_completed_s": pct(lat, 50), "p99_completed_s": pct(lat, 99),
            "configs_per_hour": len(ok) / elapsed * 3600.0, "elapsed_s": elapsed,
            "offered_requests_per_s": n_sub / window_s, "sustained_requests_per_s": len(done) / elapsed,
            "offered_pairs_per_s": sum(sub_work) / window_s, "offered_pairs": "sum of M N over the submitted requests "
            "per second of arrivals (one evaluation of each)",
            "sustained_pairs_per_s": sum(work[t] * r["steps"] for t, r in done.items()) / elapsed,
            "sustained_pairs": "sum of M N x steps of the finished requests per second of the run"}


def serving_block(ssh, synth, dev, window_s=45.0, drain_s=30.0, count=2000, mean_gap=0.020, method="lbfgs"):
    # The offered load (about 50 requests/s of up to 1.3e9 pairs per step each) exceeds one GPU by far; the
    # server admits the smallest requests first under a cap on pairs per batched step, so the figures below
    # describe what one B300 sustains, and still_queued / still_running show the backlog.
    """Poisson arrivals (mean 50/s) of ensemble requests (d in {1,2,3}, N log-uniform in [64, 32768],
    chi in [0.10, 0.49]) submitted in real time for window_s seconds; latency = submit -> converged."""
    import threading
    cfgs, arrivals = synth.serving_requests(5, count, mean_gap)
    sv = ssh.Server(device=dev, max_slots=256, chunk_steps=32)
    params = ssh.MinParams()  # zero fields: the library's defaults
    params.method = ssh.MIN_LBFGS if method == "lbfgs" else ssh.MIN_FIRE
    tickets, sub_t, sub_work = [], {}, []
    t0 = time.perf_counter()
    stop = threading.Event()

    def feeder():
        for c, ta in zip(cfgs, arrivals):
            if ta > window_s or stop.is_set():
                break
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            t = sv.submit(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi, params=params)
            sub_t[t] = time.perf_counter() - t0
            sub_work.append(c.N * round(c.chi * c.d * (c.N - 1)))   # M N (M = round-half-even(chi d (N - 1)))
            tickets.append(t)

    th = threading.Thread(target=feeder)
    th.start()
    done = {}
    while time.perf_counter() - t0 < window_s + drain_s:
        for t in list(tickets):
            if t not in done:
                r = sv.poll(t)
                if r is not None:
                    done[t] = r
        time.sleep(0.05)
    stop.set()
    th.join()
    elapsed = time.perf_counter() - t0
    st = sv.stats()
    sv.close()
    out = serving_summary(done, tickets, sub_t, sub_work, elapsed, window_s)
    out.update({"still_running": st["running"], "still_queued": st["queued"], "minimiser": method,
                "workload": f"Poisson arrivals mean {1 / mean_gap:.0f}/s for {window_s:.0f} s (+{drain_s:.0f} s drain), "
                            "d in {1,2,3}, N log-uniform [64, 32768], chi U[0.10, 0.49]"})
    return out


def arm_config(w, M, world):
    """The config of both arms' lines (the same dict, so that the two lines describe one workload): the workload and
    its sizes, the L2 policy of the GPU arm's timed steps, the parallelism."""
    return {"workload": f"d={w['d']} N={w['N']} L={w['L']} chi={w['chi']} M={M}, uniform random (SplitMix64 seed "
                        f"{w['seed']}+rank)",
            "l2": "flushed between timed steps (256 MiB write, outside the step events)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    import oracle
    oracle.build()
    M_full = oracle.chi_to_m(w["d"], w["N"], w["chi"])
    times, pairs = [], None
    for i in range(args.warmup + args.steps):
        rate, Ms, cores = cpu_sample(w["N"], w["d"], w["L"], w["chi"], w["seed"])
        if i >= args.warmup:
            times.append(Ms * w["N"] / rate)
            pairs = Ms * w["N"]
    tot = sum(times)
    value = pairs * len(times) / tot
    sample = f"first {Ms} of M wavevectors x all {w['N']} particles, both sums, per step"
    line = {"impl": "reference", "metric": "dd (k,particle) pairs/s per Phi+grad", "value": value,
            "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "binary128", "data": "synthetic",
            "config": arm_config(w, M_full, world),
            "step": "one binary128 oracle Phi + force over the sample on the host cores",
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def post_block(ssh, synth, dev):
    """Post-processing on the GPU: the pair histogram behind g_2(r) (exact integer distances) for the d=2, N=10^4
    workload, every particle a reference, r_max = 0.49 L, 512 bins: ordered pairs per second (host round trip
    included: the call is synchronous)."""
    cfg = synth.MEDIUM_D2
    with ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev) as ctx:
        ctx.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        ctx.pair_histogram(cfg.N, 0.49 * cfg.L, 512)
        reps = 5
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.pair_histogram(cfg.N, 0.49 * cfg.L, 512)
        t = (time.perf_counter() - t0) / reps
    pairs = cfg.N * (cfg.N - 1)
    return {"workload": "pair histogram, d=2 N=10^4, n_ref=N, r_max=0.49 L, 512 bins", "ms": t * 1e3,
            "pairs_per_s": pairs / t}


def paper_scale_block(ssh, synth, dev, stream, flush, steps=2, warmup=1):
    """The paper's system size, d=2, N=2x10^6 at unit density, at chi=0.10 (M = 400000, 8x10^11 pairs per sum) and
    chi=0.40 (M = 1.6x10^6, 3.2x10^12 pairs): one device FIRE step each in the default fixed point on the tensor
    cores, with the per-kernel split, the GEMMs' fractions of the bf16 peak, the particle chunks the context
    chose and the device memory it holds.  Inputs are far larger than L2; L2 is flushed between steps all the
    same."""
    return {f"chi={cfg.chi:.2f}": paper_scale_step(ssh, synth, cfg, dev, stream, flush, steps, warmup)
            for cfg in (synth.PAPER_D2, synth.PAPER_D2_CHI40)}


def paper_scale_step(ssh, synth, cfg, dev, stream, flush, steps, warmup):
    import torch
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
    try:
        ctx.set_stream(stream.cuda_stream)
        ctx.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        torch.cuda.synchronize(dev)
        held = free0 - torch.cuda.mem_get_info(dev)[0]
        pairs = ctx.M * ctx.N
        fp = ctx.min_defaults()
        fp.n_stages = 1
        fp.stage_prec[0] = ssh.FX
        fp.smax_target = 1e-300
        fp.max_steps = 1 << 40
        fp.stall_window[0] = 1 << 40
        ctx.fire_begin(fp)
        for _ in range(warmup):
            ctx.fire_steps(ssh.FX, 1)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            ctx.fire_steps(ssh.FX, 1)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        ctx.prof_enable(True)
        for _ in range(steps):
            flush.zero_()
            ctx.fire_steps(ssh.FX, 1)
        prof = ctx.prof_read()
        ctx.prof_enable(False)
        # per step: a chunked context launches the preparation and both GEMMs once per chunk
        per_step = {k: v[0] / steps for k, v in prof.items()}
        out = {"workload": f"d=2 N={cfg.N} L={cfg.L:.4f} chi={cfg.chi} M={ctx.M}, uniform random (SplitMix64 seed "
                           f"{cfg.seed}); one FIRE step in fixed point, L2 flushed between timed steps",
               "fx_impl": "tensor" if ctx.fx_impl == ssh.FX_TENSOR else "integer",
               "particle_chunks": list(ctx.tc_chunks),
               "device_bytes_held": int(held),
               "step": {"ms": ms, "pairs_per_s": pairs / (ms * 1e-3), "per_kernel_ms_per_step": per_step,
                        "launches_per_step": {k: v[1] // steps for k, v in prof.items()}}}
        if ctx.fx_impl == ssh.FX_TENSOR:
            fl = tc_flop_per_pair(cfg.d)
            out["step"]["tensor_frac_of_measured_bf16_peak"] = {
                k: fl[k] * pairs / (per_step[k] * 1e-3) / BF16_PEAK for k in fl if k in per_step}
        return out
    finally:
        ctx.close()


def large_d3_block(ssh, synth, dev, stream, flush, steps=5, warmup=3, max_seconds=150.0, staged=True):
    """The d=3, N=32768, chi=0.40 workload (M = 39320): one device FIRE step in the library's default fixed
    point (per-kernel split and tensor roofline), one evaluation in every arithmetic, and full quenches to
    S_max <= 1e-36 with the default ladder and with the paper's staged FP64 -> fixed point ladder.  An all-dd
    quench (several hundred dd evaluations of about a second each) is not run; its projection is the measured
    dd evaluation time times the step count of the default quench, and is labelled as such."""
    import torch
    cfg = synth.LARGE_D3
    ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
    ctx.set_stream(stream.cuda_stream)
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    ctx.set_positions_frac(s)
    pairs = ctx.M * ctx.N
    out = {"workload": f"d=3 N={cfg.N} L={cfg.L} chi={cfg.chi} M={ctx.M}, uniform random (SplitMix64 seed "
                       f"{cfg.seed}); L2 flushed between timed steps",
           "fx_impl": "tensor" if ctx.fx_impl == ssh.FX_TENSOR else "integer"}
    fp = ctx.min_defaults()
    fp.n_stages = 1
    fp.stage_prec[0] = ssh.FX
    fp.smax_target = 1e-300
    fp.max_steps = 1 << 40
    fp.stall_window[0] = 1 << 40
    ctx.fire_begin(fp)
    for _ in range(warmup):
        ctx.fire_steps(ssh.FX, 1)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        ctx.fire_steps(ssh.FX, 1)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    ctx.prof_enable(True)
    for _ in range(steps):
        flush.zero_()
        ctx.fire_steps(ssh.FX, 1)
    prof = ctx.prof_read()
    ctx.prof_enable(False)
    out["step"] = {"ms": ms, "pairs_per_s": pairs / (ms * 1e-3),
                   "per_kernel_ms": {k: v[0] / v[1] for k, v in prof.items()},
                   "per_step_ms": {k: v[0] / steps for k, v in prof.items()}}
    if ctx.fx_impl == ssh.FX_TENSOR:
        fl = tc_flop_per_pair(cfg.d)
        out["step"]["tensor_frac_of_measured_bf16_peak"] = {
            k: fl[k] * pairs / (prof[k][0] / prof[k][1] * 1e-3) / BF16_PEAK for k in fl if k in prof}
    # one evaluation (Phi, S_max, F) in every arithmetic
    evals = {}
    for name, prec, reps in (("fx", ssh.FX, 3), ("fp64", ssh.FP64, 3), ("dd", ssh.DD, 1)):
        ctx.eval(prec)
        ctx.sync()
        t0 = time.perf_counter()
        for _ in range(reps):
            ctx.eval(prec)
        ctx.sync()
        evals[name] = (time.perf_counter() - t0) / reps
    with ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev, fx_impl=ssh.FX_INTEGER) as c2:
        c2.set_stream(stream.cuda_stream)
        c2.set_positions_frac(s)
        c2.eval(ssh.FX)
        c2.sync()
        t0 = time.perf_counter()
        for _ in range(2):
            c2.eval(ssh.FX)
        c2.sync()
        evals["fx_integer"] = (time.perf_counter() - t0) / 2
    out["eval_ms"] = {k: v * 1e3 for k, v in evals.items()}
    out["eval_pairs_per_s"] = {k: pairs / v for k, v in evals.items()}
    ctx.close()
    runs = [("default", None), ("lbfgs", None)] + ([("fp64_then_fx", [ssh.FP64, ssh.FX])] if staged else [])
    q = {}
    for name, stages in runs:
        c = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, device=dev)
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(s)
        r = c.minimize(stages=stages, max_steps=100000, max_seconds=max_seconds,
                       method=ssh.MIN_LBFGS if name == "lbfgs" else ssh.MIN_FIRE)
        ns = r["stages_used"]
        q[name] = {"converged": r["status"] == 0, "status": r["status"], "wall_s": r["wall_s"], "steps": r["steps"],
                   "stage_steps": r["stage_steps"][:ns], "stage_wall_s": r["stage_wall_s"][:ns], "smax": r["smax"][0],
                   "configs_per_hour": 3600.0 / r["wall_s"] if r["status"] == 0 else 0.0}
        c.close()
    if q["default"]["converged"]:
        q["all_dd_projected"] = {"wall_s": evals["dd"] * q["default"]["steps"],
                                 "basis": "projection, not a run: measured dd evaluation time x step count of "
                                          "the default quench"}
    out["minimize"] = q
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2304_09139_b300 import _build, ssh, synth
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    dev = local
    torch.cuda.set_device(dev)
    _build.build()
    prec = {"fx": ssh.FX, "dd": ssh.DD, "fp64": ssh.FP64}[args.prec]
    w = WORKLOADS[args.workload]
    fx_impl = {"auto": ssh.FX_AUTO, "integer": ssh.FX_INTEGER, "tensor": ssh.FX_TENSOR}[args.fx_impl]
    ctx = ssh.Context(w["d"], w["N"], w["L"], chi=w["chi"], device=dev, fx_impl=fx_impl)
    stream = torch.cuda.Stream(dev)          # a real (non-legacy) stream shared by torch and the library
    ctx.set_stream(stream.cuda_stream)
    torch.cuda.set_stream(stream)
    s = synth.positions(replica_seed(w["seed"], rank), w["N"], w["d"])
    ctx.set_positions_frac(s)
    pairs = ctx.M * ctx.N
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    pipes = pipe_rates_block(ssh, dev)   # roofline denominators of the non-tensor arithmetics, measured here

    # A step is one device FIRE step: twiddle tables, n~, reductions, Phi / S_max, force, the FIRE update,
    # the energy-guard acceptance and the convergence test.  The target is set out of reach so that no
    # timed step turns into a no-op.
    fp = ctx.min_defaults()
    fp.n_stages = 1
    fp.stage_prec[0] = prec
    fp.smax_target = 1e-300
    fp.max_steps = 1 << 40
    fp.stall_window[0] = 1 << 40
    ctx.fire_begin(fp)

    def step():
        ctx.fire_steps(prec, 1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    # timed region: the production path (each step replays the library's captured one-step graph)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(dev) as clk:
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    # per-kernel device times: the same number of steps again with the library's event profiler (direct
    # launches, an event pair around every kernel on the launching stream), L2 flushed between steps
    ctx.prof_enable(True)
    for i in range(args.steps):
        flush.zero_()
        step()
    prof = ctx.prof_read()
    ctx.prof_enable(False)
    tot_ms = max_over_ranks(tot_ms, dist, device=f"cuda:{dev}")
    value = job_value(pairs, world, args.steps, tot_ms)
    # every profiled id is one kernel, except "fire": its two event pairs per step cover 2 + 2 kernels
    launches = sum(n for k, n in ((k, v[1]) for k, v in prof.items()) if k != "fire") + \
        4 * prof.get("fire", (0, 0))[1] // 2

    # roofline of the dominant kernel (largest share of device time in the timed region)
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    per_launch_s = dom_ms / 1e3 / dom_n
    tensor = prec == ssh.FX and ctx.fx_impl == ssh.FX_TENSOR
    if tensor:
        # the dominant of the two contractions (the digit preparation is reported in per_kernel_ms)
        dom_name = max(("tc_dens", "tc_force"), key=lambda k: prof.get(k, (0.0, 1))[0])
        dom_ms, dom_n = prof[dom_name]
        per_launch_s = dom_ms / 1e3 / dom_n
        per_pair, peak, unit, bound, what = tc_flop_per_pair(w["d"]), BF16_PEAK, "FLOP/s", "tensor", "bf16"
    elif prec == ssh.FX:
        per_pair, peak, unit, bound, what = FX_IMAD_PER_PAIR, pipes["imad"]["ops_per_s"], "IMAD/s", "alu", "IMAD"
    elif prec == ssh.DD:
        per_pair, peak, unit, bound, what = DD_FP64_PER_PAIR, pipes["fp64_fma"]["ops_per_s"], "FP64 instr/s", "fp64", "FP64"
    else:
        per_pair, peak, unit, bound, what = F64_FP64_PER_PAIR, pipes["fp64_fma"]["ops_per_s"], "FP64 instr/s", "fp64", "FP64"
    roof = None
    if dom_name in per_pair:
        achieved = per_pair[dom_name] * pairs / per_launch_s
        roof = {"bound": bound, "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None,
                "traffic_unit": "bytes per launch (dram read + write, ncu)",
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops (cuBLAS bf16 GEMM, burst), of measured"
                                if what == "bf16" else
                                f"ssh_pipe_rate {'imad' if what == 'IMAD' else 'fp64_fma'} measured in this run, "
                                f"of measured"),
                "per_kernel_ms": {k: v[0] / v[1] for k, v in prof.items()},
                # per step: "fire" and "tc_finish" are two records a step (FIRE before and after the
                # evaluation; the density and the force finish)
                "per_step_ms": {k: v[0] / args.steps for k, v in prof.items()},
                "records_per_step": {k: v[1] // args.steps for k, v in prof.items()}}
        tr = NCU_TRAFFIC.get((args.workload, "fx-tensor" if tensor else args.prec, dom_name))
        if tr and tr[0] == kernel_source_hash("tc" if tensor else "fx"):
            roof["traffic"] = tr[1]

    # end to end through the public API with host buffers (positions in, Phi / S_max / F out)
    e2e_steps = max(3, args.steps // 2)
    s2 = synth.positions(w["seed"] + 1000 + rank, w["N"], w["d"])
    ctx.set_positions_frac(s2)
    ctx.energy_grad(prec)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        ctx.set_positions_frac(s2 if i % 2 == 0 else s)
        ctx.energy_grad(prec)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, device=f"cuda:{dev}")
    h2d = 2 * 8 * w["d"] * w["N"]
    d2h = 2 * 8 * w["d"] * w["N"] + 16 * 8

    variants = {}
    if not args.no_variants and rank == 0:
        for name, p in (("dd", ssh.DD), ("fp64", ssh.FP64), ("fx", ssh.FX)):
            if p == prec:
                continue
            ctx.eval(p)
            ctx.sync()
            t0 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                ctx.eval(p)
            ctx.sync()
            variants[name] = pairs / ((time.perf_counter() - t0) / reps)
        if prec == ssh.FX:
            # the other fixed-point implementation on the same positions
            other = ssh.FX_INTEGER if tensor else ssh.FX_TENSOR
            with ssh.Context(w["d"], w["N"], w["L"], chi=w["chi"], device=dev, fx_impl=other) as c2:
                c2.set_stream(stream.cuda_stream)
                c2.set_positions_frac(s)
                c2.eval(ssh.FX)
                c2.sync()
                t0 = time.perf_counter()
                for _ in range(3):
                    c2.eval(ssh.FX)
                c2.sync()
                variants["fx_integer" if tensor else "fx_tensor"] = pairs / ((time.perf_counter() - t0) / 3)

    line = {"metric": "dd (k,particle) pairs/s per Phi+grad", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("bf16 digit products (15 balanced 7-bit digits of 2^-104 fixed point), exact f32 "
                      "accumulation, q34.126 sums" if tensor else
                      {"fx": "q2.126 fixed point (4 x int32 limbs)", "dd": "double-double (2 x f64)",
                       "fp64": "f64"}[args.prec]),
            "fx_impl": ("tensor" if tensor else "integer") if prec == ssh.FX else None,
            "data": "synthetic",
            "config": arm_config(w, ctx.M, world),
            "step": "one device FIRE step: Phi + force + update + acceptance",
            "roofline": roof, "gpu_launches": launches, "wall_s": t_wall,
            "e2e": {"value": pairs * world / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clk.summary(), "variants_pairs_per_s": variants, "pipe_rates": pipes}
    if tensor:
        line["arithmetic_class"] = ("dd-class: every value a 2^-104 fixed-point number held as 15 exact bf16 digits, "
                                    "exact sums; the paper's literal double-double path is variants_pairs_per_s.dd, "
                                    "its roofline roofline_dd")
    if rank == 0 and not args.no_variants:
        line["roofline_dd"] = dd_roofline_block(ssh, ctx, pairs, pipes["fp64_fma"]["ops_per_s"],
                                                pipes["dd_cmac"]["ops_per_s"])
    # the further blocks run at N = 1 only (a multi-GPU run holds every GPU while rank 0 works)
    if rank == 0 and world == 1 and not args.no_minimize:
        line["minimize"] = minimize_block(ssh, synth, w, dev, stream, max_seconds=args.minimize_seconds)
        conv = line["minimize"].get("default", {})
        if conv.get("converged"):
            line["configs_per_hour"] = 3600.0 / conv["wall_s"]
        conv = line["minimize"].get("lbfgs", {})
        if conv.get("converged"):
            line["configs_per_hour_lbfgs"] = 3600.0 / conv["wall_s"]
    if rank == 0 and world == 1 and not args.no_batched:
        line["batched"] = batched_block(ssh, synth, dev)
    if rank == 0 and world == 1 and not args.no_large:
        line["large_d3"] = large_d3_block(ssh, synth, dev, stream, flush, max_seconds=args.minimize_seconds,
                                          staged=args.large_staged)
    if rank == 0 and world == 1 and not args.no_post:
        line["post"] = post_block(ssh, synth, dev)
    if rank == 0 and world == 1 and not args.no_paper_scale:
        line["paper_scale"] = paper_scale_block(ssh, synth, dev, stream, flush)
    if rank == 0 and world == 1 and not args.no_serve:
        line["serving"] = serving_block(ssh, synth, dev, window_s=args.serve_seconds, method=args.serve_method)
        line["p50_s"] = line["serving"]["p50_s"]
        line["p99_s"] = line["serving"]["p99_s"]
    if rank == 0 and world == 1 and not args.no_gemm_counters and tensor:
        line["gemm_counters"] = gemm_counters_block(ssh, synth, dev, stream)
    if rank == 0 and world == 1 and not args.no_paper_quench:
        line["paper_quench"] = paper_quench_block(ssh, synth, dev, stream)
    if rank == 0 and world == 1 and args.paper_full_quench:
        line["paper_full_quench"] = paper_full_quench_block(ssh, synth, dev, stream,
                                                            max_seconds=args.paper_full_quench_seconds)
    if rank == 0 and world == 1 and not args.no_d4:
        line["d4"] = d4_block(ssh, synth, dev, stream, pipes)
    if rank == 0 and world == 1 and not args.no_floor:
        line["floor"] = floor_block(ssh, synth, dev, stream)
    if rank == 0 and world == 1 and not args.no_dd_ladder:
        line["dd_ladder"] = dd_ladder_block(ssh, synth, dev, stream, max_seconds=args.dd_seconds)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, Ms, cores, (Cr, Sr) = cpu_sample(w["N"], w["d"], w["L"], w["chi"], w["seed"], want_cs=True)
        line["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                                "sample": f"one oracle Phi+grad over the first {Ms} of {ctx.M} wavevectors x all "
                                          f"{w['N']} particles (binary128, OpenMP)"}
        # accuracy of the timed arithmetic in this run: n~ of the same sample against the oracle's
        ctx.set_positions_frac(s)
        ctx.energy_grad(prec)
        C, S = ctx.ntilde()
        err = max(np.abs((C[:Ms, 0] - Cr[:, 0]) + (C[:Ms, 1] - Cr[:, 1])).max(),
                  np.abs((S[:Ms, 0] - Sr[:, 0]) + (S[:Ms, 1] - Sr[:, 1])).max()) / w["N"]
        line["accuracy"] = {"max_abs_dntilde_over_N": float(err), "bound": 1e-28 if prec != ssh.FP64 else 1e-13,
                            "against": f"the binary128 oracle on the cpu_baseline sample ({Ms} wavevectors x "
                                       f"{w['N']} particles), at the workload's seeded positions"}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
