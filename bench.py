"""Benchmark: uint64 primality tests per second on GB300.

Default workload (N=1): 2^24 uint64 values uniform in [2^49, 2^64) with the
even indices forced odd ("plain_large"); one step classifies the whole array
through the library (classify + sieve lookup + trial division + Miller-Rabin
base 2 + the other six bases).  Inputs are resident in HBM before the timed
region; the array (128 MiB) is larger than L2 and L2 is also flushed between
steps.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--workload plain_large|plain_small|plain_mixed]

Under torchrun (N > 1) every rank classifies its own 2^24-element shard (weak
scaling, no collective on the data path); rank 0 reports the max over ranks.
`--impl reference` times the CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import generators as wg  # noqa: E402

METRIC = "uint64 primality tests/s & % int-pipe roofline vs plain; serve p50/p99 ms"
UNIT = "tests/s"

# Algorithmic work per element of plain_large (2^24 values, seed 1, trial
# division by the 15 odd primes <= 53, sieve below 2^32), counted once over
# the whole array by the CPU oracle's work counter (binary left-to-right
# schedule of Sec. 2.4); tests/test_bench_constants.py re-derives them.
WORK_PLAIN_LARGE = {
    "trial_tests": 11.2492,       # divisibility tests (multiply-by-inverse)
    "mr64_elements": 0.2041,      # survivors entering the base-2 test
    "base2_squarings": 12.4367,
    "base2_doublings": 6.2259,
    "base2_passes": 0.0346,       # elements entering the six-base kernel
    "rest_squarings": 12.5845,
    "rest_multiplies": 6.3263,
}
# Integer multiply-pipe slots per operation of the library's Montgomery
# arithmetic in 2x32-bit limbs (csrc/arith.cuh, mont_mul_c / mont_sqr_c; one
# slot = one 32-bit low multiply-add; a 32x32->64 wide product occupies the
# pipe for two slots, as measured on this GPU):
#   multiplication: a*b 4 wide (8) + m = lo*n^-1 mod 2^64 1 wide + 2 low (4)
#                   + hi(m*n) from 3 wide (6; the m0*n0 product is not needed) = 18
#   squaring:       a*a 3 wide (6) + 4 + 6 = 16
#   divisibility test n * p^-1 mod 2^64: 1 wide + 2 low = 4
IMAD_SLOTS_PER_MULMOD = 18
IMAD_SLOTS_PER_SQUARING = 16
IMAD_SLOTS_PER_TRIAL_TEST = 4
IMAD_PER_SM_PER_CLK = 64                           # 32-bit IMAD issue rate per SM
SM_COUNT_GB300 = 152
SM_MAX_MHZ = 2070.0

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# the ncu capture of this workload whose kernel-source hash and tuning are
# recorded here; they hold for that build only and are reported as null for
# any other.
NCU_TRAFFIC = {
    "sources": "c81e2467fcb1e9a0",
    "tuning": {"classify_block": 256, "mr_block": 256, "blocks_per_sm": 32, "td_primes": 15, "chunk_log2": 24, "mont_impl": 9, "mont_impl_base2": 9, "batch_block": 128, "batch_tile_log2": 10, "batch_blocks_per_sm": 0, "base2_window": 1, "rest_test": 0, "small_max": 8192, "compact_min": 33, "sieve_cutover_log2": 32, "serve_short_max": 32768, "td_fold": 3, "base2_split": 1, "base2_ilp": 1, "rest_window": 3, "window_ratio16": 0, "base2_blocks_per_sm": 4, "pdl": 1, "td2_groups": 16, "dual_stream": 0, "host_chunk_log2": 22, "inplace_max_log2": 0, "serve_long_log2": 24, "rest_ilp": 2},
    "mr64_base2": 27.45e6, "mr64_rest": 46.06e6, "classify_u64": 145.76e6}


# The sources of the kernels whose DRAM traffic NCU_TRAFFIC records (device
# code and the launchers that size their grids).
KERNEL_SOURCES = ("arith.cuh", "tables.cuh", "device_common.cuh", "classify.cu", "mr.cu")


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_2108_04791_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="mine", choices=["mine", "reference"])
    p.add_argument("--workload", default="plain_large",
                   choices=["plain_large", "plain_small", "plain_mixed", "batched", "served",
                            "range_1e8", "range_unix2021", "range_2p64", "scalar_t4", "window"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-probe", action="store_true", help="skip the integer-rate probe")
    p.add_argument("--no-sub", action="store_true",
                   help="skip the batched and served sub-records of the default run")
    p.add_argument("--tune", default="", help="tuning overrides, e.g. mont_impl=1,td_primes=24")
    return p.parse_args()


def _apply_tune(ctx, args):
    if args.tune:
        ctx.set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(","))})


def _workload(name: str, rank: int) -> tuple[np.ndarray, str]:
    if name == "plain_large":
        n = 1 << 24
        v = wg.uniform_range(1, n, 1 << 49, 1 << 64, offset=rank * n)
        v[0::2] |= np.uint64(1)
        return v, "2^24 uint64 uniform in [2^49, 2^64), even indices odd, seed 1"
    if name == "plain_small":
        n = 100_000
        return wg.uniform_range(0, n, 0, 10**6, offset=rank * n), \
            "100,000 uint64 uniform in [0, 10^6), seed 0"
    n = 1 << 26
    return wg.plain_mixed(n, seed=2, offset=rank * n), \
        "2^26 uint64, bit length uniform in 2..64, seed 2"


def _config(workload: str, n: int, desc: str, world: int) -> dict:
    """The workload's config: the same dict in both arms of the benchmark."""
    l2 = ("input 128 MiB > L2 (126 MB); the GPU arm also writes a 256 MiB buffer "
          "between steps to flush L2" if workload == "plain_large" else
          "the GPU arm writes a 256 MiB buffer between steps to flush L2")
    return {"workload": workload, "elements": n, "description": desc, "l2": l2,
            "parallelism": f"dp{world} (independent shards)"}


# ---------------------------------------------------------------- distributed

def _dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if (args.impl == "mine" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks

def _gpu_uuid(index: int) -> str | None:
    """The CUDA device's UUID in nvidia-smi's form (GPU-...), or None."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(index).uuid)
    except Exception:  # no CUDA device, or a torch without the field
        return None
    return u if u.startswith("GPU-") else "GPU-" + u


# A separate process that reads the SM clock and the clock-event reasons of one
# GPU through the driver's NVML library (read-only queries) every millisecond
# and writes "time,MHz,reason bits" lines; it runs outside this interpreter, so
# it keeps sampling while the benchmark holds the interpreter lock.
_NVML_SAMPLER = r"""
import ctypes, sys, time
uuid, index, path = sys.argv[1], int(sys.argv[2]), sys.argv[3]
lib = ctypes.CDLL("libnvidia-ml.so.1")
if lib.nvmlInit_v2() != 0:
    sys.exit(1)
h = ctypes.c_void_p()
if (uuid == "-" or lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h))) and \
        lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)):
    sys.exit(1)
reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
    lib.nvmlDeviceGetCurrentClocksThrottleReasons
mx = ctypes.c_uint()
lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
c, r = ctypes.c_uint(), ctypes.c_ulonglong()
with open(path, "w", buffering=1) as f:
    f.write("max,%d\n" % mx.value)
    while True:
        if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c)) == 0:
            if reasons(h, ctypes.byref(r)) != 0:
                r.value = 0
            f.write("%.6f,%d,%d\n" % (time.time(), c.value, r.value))
        time.sleep(0.001)
"""

# nvmlClocksEventReasons bits
_NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class ClockSampler:
    """SM clock and throttle reasons while running: nvidia-smi every 50 ms (the
    sampler starts before the region and the region starts after its first
    sample), and, where the driver's NVML library loads, a separate process
    reading the same quantities every millisecond, so that regions of a few
    milliseconds still get samples of their own (begin()/end() mark the
    region; without marks every sample counts)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.uuid = _gpu_uuid(gpu_index)
        self.proc = None
        self.path = None
        self.nv_proc = None
        self.nv_path = None
        self.t_begin = self.t_end = None

    def begin(self):
        """Marks the start of the timed region."""
        self.t_begin = time.time()

    def end(self):
        """Marks its end (call it after the device has synchronised)."""
        self.t_end = time.time()

    def start(self):
        try:
            fd, self.nv_path = tempfile.mkstemp(suffix=".nvml")
            os.close(fd)
            self.nv_proc = subprocess.Popen(
                [sys.executable, "-c", _NVML_SAMPLER, self.uuid or "-", str(self.gpu), self.nv_path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.nv_proc = None
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", self.uuid or str(self.gpu), "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        t0 = time.time()  # both samplers running (or given up) before the region
        while time.time() - t0 < 3.0:
            smi_ok = self.proc is None or os.path.getsize(self.path) > 0
            nv_ok = self.nv_proc is None or self.nv_proc.poll() is not None or \
                os.path.getsize(self.nv_path) > 40
            if smi_ok and nv_ok:
                break
            time.sleep(0.01)

    def _stop_proc(self, p):
        if p is None:
            return
        p.terminate()
        try:
            p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            p.kill()

    def stop(self) -> dict:
        rows = []
        if self.proc is not None:
            self._stop_proc(self.proc)
            self.fh.close()
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        nv, nv_all, nv_max = [], 0, None
        if self.nv_proc is not None:
            self._stop_proc(self.nv_proc)
            with open(self.nv_path) as f:
                for line in f:
                    p = line.strip().split(",")
                    if p[0] == "max" and len(p) == 2:
                        nv_max = float(p[1])
                    elif len(p) == 3:
                        nv_all += 1
                        t = float(p[0])
                        if self.t_begin is None or self.t_end is None or \
                                self.t_begin <= t <= self.t_end:
                            nv.append((float(p[1]), int(p[2])))
            os.unlink(self.nv_path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = {names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"}
        if nv_max:
            mx.append(nv_max)
        if nv:
            for _, bits in nv:
                reasons |= {nm for b, nm in _NVML_REASONS.items() if bits & b}
            mhz = [c for c, _ in nv]  # the dense samples decide the median
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(reasons) or ["no samples"], "samples": 0}
        loaded = [m for m in mhz if m > 0.5 * max(mhz)]
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows) + len(nv),
                "sources": {"nvidia_smi": len(rows), "nvml": len(nv), "nvml_total": nv_all,
                            "nvml_window": "timed region" if self.t_end else "whole phase"}}


# ---------------------------------------------------------------- CPU oracle

def _cpu_model() -> str:
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _oracle_rate(vals: np.ndarray, target_s: float = 10.0, single_s: float = 2.0) -> dict:
    """Times the CPU oracle on bounded samples: all host cores, then one thread."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.isprime_u64(vals[:4096], threads=cores)
    t0 = time.perf_counter()
    cal = vals[: 1 << 18]
    oracle.isprime_u64(cal, threads=cores)
    rate = cal.size / max(time.perf_counter() - t0, 1e-9)
    n = int(min(vals.size, max(1 << 18, rate * target_s)))
    sample = vals[:n]
    t0 = time.perf_counter()
    oracle.isprime_u64(sample, threads=cores)
    dt = time.perf_counter() - t0
    # one thread, on a prefix sized to about single_s seconds
    t0 = time.perf_counter()
    oracle.isprime_u64(vals[: 1 << 14], threads=1)
    rate1 = (1 << 14) / max(time.perf_counter() - t0, 1e-9)
    n1 = int(min(vals.size, max(1 << 14, rate1 * single_s)))
    t0 = time.perf_counter()
    oracle.isprime_u64(vals[:n1], threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} elements of the workload, one pass, {cores} threads",
            "seconds": dt, "cpu_model": _cpu_model(),
            "single_thread": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first {n1} elements of the workload, one pass",
                              "seconds": dt1}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    vals, desc = _workload(args.workload, 0)
    import oracle
    cores = os.cpu_count() or 1
    chunk = 1 << 16  # the oracle's multi-threaded driver hands out 64 Ki-element chunks
    cal = vals[: cores * chunk]
    t0 = time.perf_counter()
    oracle.isprime_u64(cal, threads=cores)
    rate = cal.size / max(time.perf_counter() - t0, 1e-9)
    budget_s = 60.0
    # every step gives each core at least one chunk; the whole run stays near budget_s
    per_step = int(max(cores * chunk, min(vals.size, rate * budget_s / max(args.steps + args.warmup, 1))))
    per_step = min(per_step, vals.size)
    for w in range(args.warmup):
        oracle.isprime_u64(vals[:per_step], threads=cores)
    total = 0.0
    for k in range(args.steps):
        off = (k * per_step) % max(vals.size - per_step, 1)
        s = vals[off:off + per_step]
        t0 = time.perf_counter()
        oracle.isprime_u64(s, threads=cores)
        total += time.perf_counter() - t0
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": _config(args.workload, int(vals.size), desc, world),
            "sample_elements_per_step": per_step,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} consecutive elements of the workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_mine(args, world, rank, local):
    import torch
    import paper_2108_04791_gb300 as ipg

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    vals, desc = _workload(args.workload, rank)
    n = vals.size
    d_in = torch.from_numpy(vals.view(np.int64)).to(dev)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    ctx = ipg.Context.default(local)              # builds the resident sieve (untimed)
    _apply_tune(ctx, args)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (126 MB)

    for k in range(max(args.warmup, 3)):
        flush.fill_(k & 0xFF)  # the first fill loads torch's fill kernel (a quarter second
        ctx.isprime(d_in, out=out)  # of host time) here rather than in the timed region
    torch.cuda.synchronize(dev)

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # The timed pass runs without the library's per-kernel timing events (they
    # sit between the kernels on the stream and add their own gaps); a second
    # pass below takes the per-kernel times.
    launches0 = ctx.stats()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    _barrier(world)
    torch.cuda.synchronize(dev)
    clocks.begin()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                    # evict the previous step's lines from L2
        ev_s[k].record(stream)
        ctx.isprime(d_in, out=out)
        ev_e[k].record(stream)
    torch.cuda.synchronize(dev)
    clocks.end()
    _barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    launches = ctx.stats()["kernel_launches"] - launches0
    step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    total_s = _max_over_ranks(total_s, world, dev)
    value = n * world * args.steps / total_s
    # per-kernel times: a separate pass of the same steps with the library's
    # CUDA events around every launch (on the launching stream)
    k_steps = max(3, min(args.steps, 50))
    ctx.timing_reset()
    ctx.timing(True)
    for k in range(k_steps):
        flush.fill_(k & 0xFF)
        ctx.isprime(d_in, out=out)
    torch.cuda.synchronize(dev)
    ctx.timing(False)
    ktimes = ctx.timing_read()

    # ---- roofline: the whole step, and the dominant kernel
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms, dom_launches = ktimes[dom]
    roof = None
    imad_rate = None
    if not args.no_probe:
        imad_rate = ipg.int_rates(local)
    peak_ops = SM_COUNT_GB300 * IMAD_PER_SM_PER_CLK * SM_MAX_MHZ * 1e6
    if args.workload == "plain_large":
        w, stage2, schedule = _plain_large_work(ctx.tuning.as_dict())
        slots = {
            "classify_u64": WORK_PLAIN_LARGE["trial_tests"] * IMAD_SLOTS_PER_TRIAL_TEST,
            "mr64_base2": (stage2 * IMAD_SLOTS_PER_TRIAL_TEST
                           + w["base2_squarings"] * IMAD_SLOTS_PER_SQUARING),
            "mr64_rest": w["rest_squarings"] * IMAD_SLOTS_PER_SQUARING
            + w["rest_multiplies"] * IMAD_SLOTS_PER_MULMOD,
        }
        same = (NCU_TRAFFIC["sources"] == kernel_sources_hash()
                and NCU_TRAFFIC["tuning"] == ctx.tuning.as_dict())
        per_kernel = {k: slots[k] * n / (ktimes[k][0] / ktimes[k][1] / 1e3) / peak_ops
                      for k in slots if ktimes.get(k, (0, 0))[1]}
        step_slots = sum(slots.values())
        step_achieved = (n * world * args.steps / total_s) / world * step_slots
        dom_roof = None
        if dom in slots:
            dom_achieved = slots[dom] * n / (dom_ms / dom_launches / 1e3)
            dom_roof = {"kernel": dom, "achieved": dom_achieved / 1e12, "frac": dom_achieved / peak_ops,
                        "ms_per_launch": dom_ms / dom_launches,
                        "algorithmic_slots_per_element": slots[dom],
                        "traffic": NCU_TRAFFIC.get(dom) if same else None}
        traffic = (sum(NCU_TRAFFIC[k] for k in slots) if same else None)
        roof = {"bound": "alu", "achieved": step_achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "T int-mul slots/s", "frac": step_achieved / peak_ops, "traffic": traffic,
                "kernel": "whole step: classify_u64 + mr64_base2 + mr64_rest (one launch each)",
                "frac_dominant_kernel": dom_roof["frac"] if dom_roof else None,
                "dominant_kernel": dom_roof,
                "peak_source": "152 SMs x 64 IMAD/clk x 2070 MHz (derived; the probe measures "
                               "64 mad.lo.u32 lanes/clk/SM)",
                "algorithmic_slots_per_element": step_slots,
                "roofline_tests_per_s": peak_ops / step_slots,
                "schedule": schedule,
                "frac_by_kernel": per_kernel,
                "traffic_note": "DRAM bytes per step (sum of the three kernels) from the ncu "
                                "capture whose source hash and tuning match this build; "
                                "null otherwise"}
    kernels = {k: {"ms_per_step": v[0] / k_steps, "launches": v[1]}
               for k, v in ktimes.items() if v[1]}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(vals.view(np.int64)).pin_memory()
        h_out = torch.empty(n, dtype=torch.uint8).pin_memory()
        hv = h_in.numpy().view(np.uint64)
        ho = h_out.numpy()
        ke = max(3, min(args.steps, 50))
        for _ in range(2):
            ipg._check(ipg.lib().isprime_u64_host(ctx.handle, hv.ctypes.data, ho.ctypes.data, n,
                                                  ipg.ctypes.c_void_p(stream.cuda_stream)))
        _barrier(world)
        t0 = time.perf_counter()
        for _ in range(ke):
            ipg._check(ipg.lib().isprime_u64_host(ctx.handle, hv.ctypes.data, ho.ctypes.data, n,
                                                  ipg.ctypes.c_void_p(stream.cuda_stream)))
        dt = _max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": n * world * ke / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": n, "steps": ke}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = _oracle_rate(vals)

    # ---- the batched and served forms on this GPU (bounded sub-records)
    subs = {}
    if args.workload == "plain_large" and world == 1 and not args.no_sub:
        with_cpu = rank == 0 and not args.no_cpu_baseline
        subs["plain_small"] = plain_record(ctx, dev, "plain_small", max(20, min(args.steps * 10, 200)),
                                           with_cpu)
        subs["plain_mixed"] = plain_record(ctx, dev, "plain_mixed", max(5, min(args.steps, 20)),
                                           with_cpu)
        subs["batched"] = batched_record(ctx, dev, max(3, min(args.steps, 10)), 3, world, with_cpu)
        subs["served"] = served_record(ctx, dev, 3, world, rank, with_cpu)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": _config(args.workload, n, desc, world),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "kernels": kernels,
            "tuning": ctx.tuning.as_dict(),
            "wall_s_timed_region": wall, "int_rates": imad_rate, **subs,
        }
        print(json.dumps(line), flush=True)


def _golden_work(name: str) -> dict:
    """Per-element algorithmic work of a workload, counted once by the CPU
    oracle's work counter (tests/golden/make_work_counts.py wrote the file)."""
    with open(os.path.join(ROOT, "tests", "golden", "work_counts.json")) as f:
        return json.load(f)[name]


def _plain_large_work(tuning: dict) -> tuple[dict, float, str]:
    """The per-element work of plain_large under the schedule the tuning runs:
    (operation counts, second-stage trial tests, description).  With the
    base-2 kernel's second trial stage (td2_groups = G) the first stage still
    tests the odd primes <= 53 on every odd element, the base-2 kernel tests
    the next 3 G primes on that stage's survivors, and only the values no
    prime divides reach the base-2 test; the oracle's count at the larger
    trial bound gives the Miller-Rabin work of that schedule."""
    groups = int(tuning.get("td2_groups", 0))
    if not groups:
        return (WORK_PLAIN_LARGE, 0.0,
                "trial division by the 15 odd primes <= 53, then the bases of Eq. 4")
    g = _golden_work("plain_large_td2")["groups"][str(groups)]
    return (g["per_element"], 3 * groups * WORK_PLAIN_LARGE["mr64_elements"],
            f"trial division by the 15 odd primes <= 53 (classify), then by the next "
            f"{3 * groups} odd primes up to {g['td_bound']} on its survivors (base-2 kernel, "
            f"td2_groups = {groups}), then the bases of Eq. 4")


def _slots_per_element(w: dict) -> float:
    """Integer-pipe slots per element of the canonical schedule: trial
    division, base-2 squarings, and the six bases' squarings and products."""
    return (w["trial_tests"] * IMAD_SLOTS_PER_TRIAL_TEST
            + (w["base2_squarings"] + w["rest_squarings"]) * IMAD_SLOTS_PER_SQUARING
            + w["rest_multiplies"] * IMAD_SLOTS_PER_MULMOD)


def _alu_roofline(tests_per_s: float, work_name: str, note: str) -> dict:
    peak_ops = SM_COUNT_GB300 * IMAD_PER_SM_PER_CLK * SM_MAX_MHZ * 1e6
    g = _golden_work(work_name)
    slots = _slots_per_element(g["per_element"])
    achieved = tests_per_s * slots
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
            "unit": "T int-mul slots/s", "frac": achieved / peak_ops, "traffic": None,
            "algorithmic_slots_per_element": slots, "roofline_tests_per_s": peak_ops / slots,
            "work_source": f"oracle work counter over {g['elements']} elements ({work_name})",
            "peak_source": "152 SMs x 64 IMAD/clk x 2070 MHz (derived)", "note": note}


def _cpu_rate_on(vals: np.ndarray, target_s: float, what: str) -> dict:
    """The CPU oracle on all host cores over a bounded prefix of `vals`."""
    import oracle
    cores = os.cpu_count() or 1
    cal = vals[: 1 << 16]
    t0 = time.perf_counter()
    oracle.isprime_u64(cal, threads=cores)
    rate = cal.size / max(time.perf_counter() - t0, 1e-9)
    n = int(min(vals.size, max(1 << 16, rate * target_s)))
    t0 = time.perf_counter()
    oracle.isprime_u64(vals[:n], threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} values of {what}, one pass, {cores} threads", "seconds": dt}


def plain_record(ctx, dev, workload: str, steps: int, with_cpu: bool) -> dict:
    """A plain workload through isprime_u64_ctx (plain_small: 10^5 values below
    10^6, the launch-bound case; plain_mixed: 2^26 values of uniform bit
    length, plus its 2^20 doubles through isprime_f64_ctx): device time per
    call with inputs resident (L2 flushed between calls), the per-kernel times
    from a second pass, and end to end through isprime_u64_host."""
    import torch
    import paper_2108_04791_gb300 as ipg
    vals, desc = _workload(workload, 0)
    n = vals.size
    d_in = torch.from_numpy(vals.view(np.int64)).to(dev)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, k):
        for i in range(3):
            flush.fill_(i & 0xFF)
            fn()
        torch.cuda.synchronize(dev)
        tot = 0.0
        for i in range(k):
            flush.fill_(i & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
        return tot / k

    ms = timed(lambda: ctx.isprime(d_in, out=out), steps)
    ctx.timing_reset()
    ctx.timing(True)
    k_steps = max(3, min(steps, 20))
    for _ in range(k_steps):
        ctx.isprime(d_in, out=out)
    torch.cuda.synchronize(dev)
    ctx.timing(False)
    kt = ctx.timing_read()
    h_in = torch.from_numpy(vals.view(np.int64)).pin_memory()
    h_out = torch.empty(n, dtype=torch.uint8).pin_memory()
    hv, ho = h_in.numpy().view(np.uint64), h_out.numpy()
    L = ipg.lib()
    sh = ipg.ctypes.c_void_p(stream.cuda_stream)
    for _ in range(2):
        ipg._check(L.isprime_u64_host(ctx.handle, hv.ctypes.data, ho.ctypes.data, n, sh))
    ke = max(3, min(steps, 20))
    t0 = time.perf_counter()
    for _ in range(ke):
        ipg._check(L.isprime_u64_host(ctx.handle, hv.ctypes.data, ho.ctypes.data, n, sh))
    e2e_s = (time.perf_counter() - t0) / ke
    rec = {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "config": _config(workload, n, desc, 1),
           "kernels": {k: {"ms_per_step": v[0] / k_steps, "launches": v[1]} for k, v in kt.items()
                       if v[1]},
           "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": n, "steps": ke}}
    if workload == "plain_mixed":
        x = wg.mixed_doubles(1 << 20)
        d_x = torch.from_numpy(x).to(dev)
        o_x = torch.empty(x.size, dtype=torch.uint8, device=dev)
        ms_f = timed(lambda: ctx.isprime(d_x, out=o_x), steps)
        rec["doubles"] = {"value": x.size / (ms_f / 1e3), "unit": UNIT, "ms_per_step": ms_f,
                          "elements": int(x.size),
                          "description": "2^20 doubles holding integers uniform in [0, 2^53), "
                                         "through isprime_f64_ctx"}
        del d_x, o_x
    if with_cpu:
        rec["cpu_baseline"] = _cpu_rate_on(vals, 3.0, f"the {workload} array")
    del d_in, out, flush
    return rec


def batched_record(ctx, dev, steps: int, warm: int, world: int, with_cpu: bool) -> dict:
    """The batched workload (4096 ragged arrays, log-uniform sizes 1..2^20,
    25% primes near 2^64, 10% semiprimes) through one batched launch per step,
    against the same arrays through one plain call each."""
    import torch
    from workloads import torch_gen
    d_all, offs = torch_gen.batched_arrays(n_arrays=4096, max_size=1 << 20, seed=3, device=dev)
    n = d_all.numel()
    out_all = torch.empty(n, dtype=torch.uint8, device=dev)
    ins = [d_all[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    outs = [out_all[offs[i]:offs[i + 1]] for i in range(len(offs) - 1)]
    stream = torch.cuda.current_stream(dev)

    def timed(fn, k):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize(dev)
        _barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return _max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)

    launches0 = ctx.stats()["kernel_launches"]
    ctx.timing_reset()
    ctx.timing(True)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    t_batch = timed(lambda: ctx.isprime_batched(ins, outs), steps)
    clk = clocks.stop()
    ctx.timing(False)
    launches = ctx.stats()["kernel_launches"] - launches0
    kt = ctx.timing_read()
    k_plain = max(1, min(steps, 2))
    t_plain = timed(lambda: [ctx.isprime(x, out=o) for x, o in zip(ins, outs)], k_plain)
    value = n * world * steps / t_batch
    plain_value = n * world * k_plain / t_plain
    roof = _alu_roofline(value / world, "batched",
                         "whole launch (the batched kernel runs every stage); per-element work "
                         "of this exact batch")
    rec = {"value": value, "unit": UNIT, "steps": steps, "ms_per_step": 1e3 * t_batch / steps,
           "config": {"workload": "batched", "arrays": len(ins), "elements": int(n),
                      "description": wg.WORKLOADS["batched"],
                      "launch": "one CUDA-graph replay per step",
                      "l2": "2.3 GB of input per step > L2"},
           "plain_per_call": {"value": plain_value, "unit": UNIT, "steps": k_plain,
                              "calls_per_step": len(ins)},
           "speedup_vs_plain_calls": value / plain_value,
           "roofline": roof, "gpu_launches": launches, "clocks": clk,
           "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in kt.items()
                       if v[1]},
           "kernels_note": "the launches include the warm-up replays"}
    if with_cpu:
        rec["cpu_baseline"] = _cpu_rate_on(d_all[: 1 << 24].cpu().numpy().view(np.uint64), 4.0,
                                           "the batch (arrays in order)")
    del d_all, out_all, ins, outs
    return rec


def served_record(ctx, dev, warm: int, world: int, rank: int, with_cpu: bool,
                  n_requests: int = 20_000) -> dict:
    """The served workload: requests with exponential inter-arrival times
    (mean 200 us), log-uniform sizes 1..2^22, values drawn as in the batched
    workload, through the continuous-batching server (8 GB device budget).
    Request inputs are slices of a 2^27-value pool with that distribution in
    pinned host memory; outputs go to a pinned ring larger than the server can
    hold in flight.  Three runs over the same request stream: open loop at the
    arrival times (latency at 5,000 req/s), all requests offered at once
    (capacity), and one isprime_u64_host call per request, one after another
    (the per-call plain form)."""
    import torch
    import paper_2108_04791_gb300 as ipg
    from workloads import torch_gen
    arrivals, sizes, _ = wg.served_requests(n_requests=n_requests, max_size=1 << 22,
                                            rate_per_s=5000.0, seed=4 + 1000 * rank, values=False)
    pool_n = 1 << 27
    pool = torch_gen.served_values(pool_n, seed=4 + 1000 * rank, device=dev).cpu().pin_memory()
    pool_np = pool.numpy().view(np.uint64)
    ring_n = 1 << 31
    ring = torch.empty(ring_n, dtype=torch.uint8).pin_memory().numpy()
    starts = np.zeros(len(sizes), dtype=np.int64)
    np.cumsum(sizes[:-1], out=starts[1:])
    in_off = starts % (pool_n - (1 << 22))
    out_off = starts % (ring_n - (1 << 22))
    total = int(sizes.sum())
    srv = ipg.Server(ctx, mem_budget_bytes=8 << 30, n_slots=4)
    for _ in range(max(warm, 3)):  # graph recording, first touch of the arena
        srv.wait(srv.submit(pool_np[:1 << 20], out=ring[:1 << 20]))

    def run(paced: bool):
        srv.reset_stats()
        _barrier(world)
        t0 = time.perf_counter()
        tickets = []
        for i in range(len(sizes)):
            if paced:
                target = t0 + arrivals[i]
                while True:
                    now = time.perf_counter()
                    if now >= target:
                        break
                    if target - now > 2e-3:
                        time.sleep(target - now - 1e-3)
            a, o, m = int(in_off[i]), int(out_off[i]), int(sizes[i])
            tickets.append(srv.submit(pool_np[a:a + m], out=ring[o:o + m]))
        for t in tickets:
            srv.wait(t)
        return time.perf_counter() - t0, srv.stats()

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    wall_open, st_open = run(paced=True)
    wall_cap, st_cap = run(paced=False)
    clk = clocks.stop()
    srv.close()
    # per-call plain form on the same stream: one host-buffer call per request
    L = ipg.lib()
    s = ipg.ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for i in range(3):
        ipg._check(L.isprime_u64_host(ctx.handle, pool_np[:1 << 20].ctypes.data,
                                      ring[:1 << 20].ctypes.data, 1 << 20, s))
    _barrier(world)
    t0 = time.perf_counter()
    for i in range(len(sizes)):
        a, o, m = int(in_off[i]), int(out_off[i]), int(sizes[i])
        ipg._check(L.isprime_u64_host(ctx.handle, pool_np[a:].ctypes.data, ring[o:].ctypes.data,
                                      m, s))
    t_plain = _max_over_ranks(time.perf_counter() - t0, world, dev)
    cap = total / st_cap["span_s"]
    rec = {"value": cap * world, "unit": UNIT,
           "config": {"workload": "served", "requests": len(sizes), "elements": total,
                      "rate_req_per_s": 5000, "budget_bytes": 8 << 30, "slots": 4,
                      "description": wg.WORKLOADS["served"],
                      "inputs": "slices of a 2^27-value pool in pinned host memory"},
           "capacity": {"value": cap * world, "unit": UNIT, "span_s": st_cap["span_s"],
                        "how": "all requests submitted at once, in arrival order",
                        "p50_ms": st_cap["p50_ms"], "p99_ms": st_cap["p99_ms"],
                        "batches": st_cap["batches"]},
           "open_loop": {"tests_per_s": st_open["tests_per_s"], "p50_ms": st_open["p50_ms"],
                         "p99_ms": st_open["p99_ms"], "mean_ms": st_open["mean_ms"],
                         "max_ms": st_open["max_ms"], "batches": st_open["batches"],
                         "short_requests": st_open["short_requests"],
                         "p50_short_ms": st_open["p50_short_ms"],
                         "p99_short_ms": st_open["p99_short_ms"],
                         "p50_long_ms": st_open["p50_long_ms"], "p99_long_ms": st_open["p99_long_ms"],
                         "offered_tests_per_s": float(total / arrivals[-1]), "wall_s": wall_open},
           "plain_per_call": {"value": total * world / t_plain, "unit": UNIT, "seconds": t_plain,
                              "how": "one isprime_u64_host call per request, in order"},
           "capacity_vs_plain_calls": cap * world / (total * world / t_plain),
           "roofline": _alu_roofline(cap, "served_pool",
                                     "capacity run; per-element work of the 2^27-value pool the "
                                     "requests are sliced from (the stream covers it about 40 "
                                     "times); copies in and out are inside the span"),
           "e2e": {"value": cap * world, "unit": UNIT, "h2d_bytes_per_step": 8 * total,
                   "d2h_bytes_per_step": total, "step": "the whole request stream"},
           "clocks": clk}
    if with_cpu:
        rec["cpu_baseline"] = _cpu_rate_on(pool_np, 4.0, "the request pool")
    del pool, ring
    return rec


def run_batched(args, world, rank, local):
    import torch
    import paper_2108_04791_gb300 as ipg
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ctx = ipg.Context.default(local)
    _apply_tune(ctx, args)
    rec = batched_record(ctx, dev, max(args.steps, 1), max(args.warmup, 3), world,
                         with_cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if rank == 0:
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
                "steps": rec["steps"], "warmup": max(args.warmup, 3),
                "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic", **rec,
                "tuning": ctx.tuning.as_dict()}
        print(json.dumps(line), flush=True)


def run_served(args, world, rank, local):
    import torch
    import paper_2108_04791_gb300 as ipg
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ctx = ipg.Context.default(local)
    _apply_tune(ctx, args)
    rec = served_record(ctx, dev, args.warmup, world, rank,
                        with_cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    if rank == 0:
        n_req = rec["config"]["requests"]
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
                "steps": n_req, "warmup": max(args.warmup, 3),
                "ms_per_step": 1e3 * rec["capacity"]["span_s"] / n_req, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", **rec,
                "tuning": ctx.tuning.as_dict()}
        print(json.dumps(line), flush=True)


RANGES = {
    "range_1e8": (1, 10**8, "1:10^8 (Table 3's largest incrementing sequence)"),
    "range_unix2021": (1609477200, 3600 * 24 * 365 + 1, "the Unix seconds of 2021 (Table 5)"),
    "range_2p64": ((1 << 64) - (1 << 28), 1 << 28, "the last 2^28 integers below 2^64"),
}


def _measured_hbm_gbs() -> dict:
    """HBM copy bandwidth measured on this GPU type (MEASURED_PEAKS.json), else the
    earlier fallback measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return {"value": float(json.load(f)["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"value": 6800.0, "source": "fallback"}


def run_range(args, world, rank, local):
    """isprime_range over a window of consecutive integers (no input array)."""
    import torch
    import paper_2108_04791_gb300 as ipg

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    lo, count, desc = RANGES[args.workload]
    ctx = ipg.Context.default(local)
    out = torch.empty(count, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    steps, warm = max(args.steps, 1), max(args.warmup, 3)
    for _ in range(warm):
        ctx.isprime_range(lo, count, out=out)
    ctx.timing_reset()
    ctx.timing(True)
    torch.cuda.synchronize(dev)
    _barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.isprime_range(lo, count, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ctx.timing(False)
    t = _max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    kt = ctx.timing_read()
    value = count * world * steps / t
    primes = int(out.sum().item())
    # Roofline of the range kernel (the one below S expands the bitmap: 1 byte written and
    # 1/16 byte of bitmap read per value; above S the sieve kernel writes 1 byte per value).
    below = max(0, min(lo + count, 1 << 32) - lo)
    algo_bytes = count + below / 16
    rk_ms, rk_n = kt.get("range", (0.0, 0))
    peak = _measured_hbm_gbs()
    achieved = algo_bytes / (rk_ms / max(rk_n, 1) / 1e3) / 1e9 if rk_n else None
    range_roof = {"bound": "hbm", "achieved": achieved, "peak": peak["value"], "unit": "GB/s",
                  "frac": achieved / peak["value"] if achieved else None, "traffic": None,
                  "kernel": "range", "algorithmic_bytes_per_launch": algo_bytes,
                  "peak_source": peak["source"]}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": warm, "ms_per_step": 1e3 * t / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": args.workload, "lo": lo, "count": count, "description": desc,
                           "primes_found": primes},
                "roofline": range_roof,
                "kernels": {k: {"ms_per_step": v[0] / steps, "launches": v[1]} for k, v in kt.items()
                            if v[1]}}
        print(json.dumps(line), flush=True)


# isprime_fast's mean time per call for prime scalars of each bit size
# (Table 4; MATLAB R2020b on an i7-9750H): context, not a target.
TABLE4_ISPRIME_FAST_S = {4: 7.7654e-07, 8: 1.0120e-06, 16: 1.8106e-06, 24: 5.8244e-06,
                         32: 5.3932e-05, 36: 0.0002828, 40: 0.001766, 44: 0.005818, 48: 0.02718,
                         50: 0.0326, 52: 0.0431, 56: 0.0552, 60: 0.0755, 64: 0.1194}


def run_scalar(args, world, rank, local):
    """Latency of one-value calls (isprime_u64_scalar) on Table 4's inputs:
    100 primes of each bit size, every call synchronous, timed on the host
    around the C call; plus the device time of the one-warp kernel, and the
    one-launch path against the queue path for short device arrays."""
    import torch
    import paper_2108_04791_gb300 as ipg

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ctx = ipg.Context.default(local)
    L = ipg.lib()
    res = ipg.ctypes.c_uint8()
    pools = wg.load_primes_by_bits()
    reps = max(1, min(args.steps, 20))
    for b in pools:                                 # warm-up: every kernel and code path
        for v in pools[b][:max(args.warmup, 3)].tolist():
            L.isprime_u64_scalar(ctx.handle, v, ipg.ctypes.byref(res))
    clocks = ClockSampler(local)
    clocks.start()
    per_bits, all_us, found = {}, [], 0
    for b, vals in sorted(pools.items()):
        lat = []
        for _ in range(reps):
            for v in vals.tolist():
                t0 = time.perf_counter_ns()
                st = L.isprime_u64_scalar(ctx.handle, v, ipg.ctypes.byref(res))
                lat.append((time.perf_counter_ns() - t0) / 1e3)
                if st:
                    ipg._check(st)
                found += res.value
        lat.sort()
        all_us += lat
        per_bits[b] = {"p50_us": lat[len(lat) // 2], "p99_us": lat[int(len(lat) * 0.99)],
                       "mean_us": sum(lat) / len(lat),
                       "paper_isprime_fast_s": TABLE4_ISPRIME_FAST_S.get(b)}
    clk = clocks.stop()
    # device time of the warp kernel per bit size (CUDA events, separate pass)
    ctx.timing_reset()
    ctx.timing(True)
    for b, vals in sorted(pools.items()):
        ctx.timing_reset()
        for v in vals.tolist():
            L.isprime_u64_scalar(ctx.handle, v, ipg.ctypes.byref(res))
        ms, cnt = ctx.timing_read()["small"]
        per_bits[b]["kernel_us"] = 1e3 * ms / max(cnt, 1)
    ctx.timing(False)
    # short device arrays: one-launch warp path vs the queue path (device time per call)
    stream = torch.cuda.current_stream(dev)
    arrays = {}
    old = ctx.tuning.small_max
    for n in (1, 32, 256, 1024, 4096, 16384, 65536):
        v = wg.plain_mixed(n, seed=5)
        t = torch.from_numpy(v.view(np.int64)).to(dev)
        out = torch.empty(n, dtype=torch.uint8, device=dev)
        row = {}
        for name, sm in (("warp", 1 << 20), ("queue", 0)):
            ctx.set_tuning(small_max=sm)
            for _ in range(5):
                ctx.isprime(t, out=out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = 200
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(k):
                ctx.isprime(t, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            row[name + "_us"] = 1e3 * e0.elapsed_time(e1) / k
        arrays[n] = row
    ctx.set_tuning(small_max=old)
    all_us.sort()
    mean_us = sum(all_us) / len(all_us)
    if rank == 0:
        line = {"metric": METRIC, "value": 1e6 / mean_us, "unit": "tests/s (one value per call)",
                "n_gpus": world, "steps": reps, "warmup": args.warmup,
                "ms_per_step": mean_us * len(all_us) / reps / 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": "scalar_t4",
                           "description": "100 primes of each bit size of Table 4, one "
                                          "isprime_u64_scalar call per value, host-timed",
                           "calls": len(all_us), "primes_found": found},
                "latency": {"p50_us": all_us[len(all_us) // 2],
                            "p99_us": all_us[int(len(all_us) * 0.99)], "mean_us": mean_us},
                "per_bits": per_bits, "short_arrays_device_us": arrays, "clocks": clk,
                "tuning": ctx.tuning.as_dict()}
        print(json.dumps(line), flush=True)


def run_window(args, world, rank, local):
    """The per-call path choice: the window path (sieve [min, max], gather)
    against the queue path on arrays of N values spread over windows of
    W = N / density integers, at two magnitudes; device time per call of each
    arm (the window arm includes its min/max read-back)."""
    import torch
    import paper_2108_04791_gb300 as ipg
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ctx = ipg.Context.default(local)
    _apply_tune(ctx, args)
    stream = torch.cuda.current_stream(dev)
    rows = []
    reps = max(3, min(args.steps, 10))
    for lo in (1 << 40, (1 << 64) - (1 << 34)):
        for n in (1 << 20, 1 << 22, 1 << 24):
            for dens in (8.0, 2.0, 1.0, 0.5, 0.25, 0.125):
                w = max(int(n / dens), 16)
                rng = np.random.default_rng(n + w)
                v = (np.uint64(lo) + rng.integers(0, w, size=n, dtype=np.uint64)).astype(np.uint64)
                t = torch.from_numpy(v.view(np.int64)).to(dev)
                out = torch.empty(n, dtype=torch.uint8, device=dev)
                row = {"lo_log2": round(float(np.log2(float(lo))), 3), "n": n, "density": dens,
                       "window": int(v.max() - v.min()) + 1}
                for arm, r16 in (("window_ms", 4096), ("queue_ms", 0)):
                    ctx.set_tuning(window_ratio16=r16, small_max=0)
                    for _ in range(2):
                        ctx.isprime(t, out=out)
                    torch.cuda.synchronize(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(reps):
                        ctx.isprime(t, out=out)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    row[arm] = e0.elapsed_time(e1) / reps
                row["winner"] = "window" if row["window_ms"] < row["queue_ms"] else "queue"
                rows.append(row)
                del t, out
    ctx.set_tuning(window_ratio16=0)
    if rank == 0:
        best = max(rows, key=lambda r: r["queue_ms"] / r["window_ms"])
        line = {"metric": METRIC, "value": best["n"] / (best["window_ms"] / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": reps, "warmup": 2, "ms_per_step": best["window_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic",
                "config": {"workload": "window", "description": "N values uniform over a window "
                           "of N / density integers at 2^40 and near 2^64"},
                "crossover": rows, "tuning": ctx.tuning.as_dict()}
        print(json.dumps(line), flush=True)


def main():
    args = _parse()
    world, rank, local = _dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "served":
        run_served(args, world, rank, local)
    elif args.workload.startswith("range"):
        run_range(args, world, rank, local)
    elif args.workload == "scalar_t4":
        run_scalar(args, world, rank, local)
    elif args.workload == "window":
        run_window(args, world, rank, local)
    else:
        run_mine(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
