"""Benchmark: spMTTKRP along every mode of the 50M-nonzero 3-mode workload.

Workload (synthetic stand-in for the paper's FROSTT tensors): 3-mode COO
tensor 1,000,000 x 500,000 x 200,000, coordinates per mode truncated
Zipf(1.2) with repeated cells removed, 50M nonzeros, values U(0,1), int32
indices, R = 32 FP32 factors N(0,1).  One mode-specific copy per mode is
resident in HBM (the plan, built before timing, as the workload states).

A step is spMTTKRP along modes 0, 1, 2 (output clearing, the MTTKRP kernel,
the partition fix-up; Algorithm 1 over all modes).  The plan build (copy
sorting and partitioning) and one CP-ALS sweep are timed separately and
reported beside the step.

Metric: spMTTKRP HBM GB/s over all modes, B_d / t_d summed over modes with
B_d = nnz*(4N+4) + sum_{w != d} U_w*R*4 + I_d*R*4 (streamed records, each
distinct gathered factor row once, the output written once).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the method does not
shard; see the design notes) and rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spMTTKRP HBM GB/s & roofline %, all modes; CPD solves/s + p50/p99 latency"
UNIT = "GB/s"
WORKLOAD = "scale: 3-mode COO 1,000,000x500,000x200,000, 50M nnz, Zipf(1.2) coordinates " \
           "deduplicated, U(0,1) values, R=32 FP32 factors, MTTKRP along all 3 modes"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nnz", type=int, default=50_000_000,
                    help="nonzeros (the workload is 50M; smaller only for quick checks)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the batching comparison that the headline line carries")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the short serving comparison that the headline line carries")
    ap.add_argument("--workload", default="scale",
                    choices=["scale", "batching", "serving", "precision", "five", "schemes",
                             "lean", "fibre", "probe"],
                    help="scale (default, the headline line); the others print their "
                         "own JSON line")
    ap.add_argument("--tensors", type=int, default=512, help="batching: tensor count")
    ap.add_argument("--sweeps", type=int, default=20, help="batching/precision: ALS sweeps")
    ap.add_argument("--requests", type=int, default=200, help="serving: request count")
    ap.add_argument("--preset", default="scale", choices=["scale", "precision", "five"],
                    help="probe: the synthetic preset")
    ap.add_argument("--factor", default="fp32", choices=["fp32", "bf16"],
                    help="probe: factor storage type")
    ap.add_argument("--probe-sweeps", type=int, default=0, help="probe: CP-ALS sweeps")
    return ap.parse_args()


def dist_init(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(bytes_per_replica, ms_max, world):
    """Whole-job GB/s of `world` independent replicas: every rank processes
    the same workload, the job takes the slowest rank's time."""
    return world * bytes_per_replica / (ms_max * 1e-3) / 1e9


def algorithmic_bytes(dims, nnz, R, distinct, s_f=4):
    """B_d per mode: records + distinct gathered rows + output rows."""
    N = len(dims)
    out = []
    for d in range(N):
        b = nnz * (4 * N + 4)
        b += sum(distinct[w] * R * s_f for w in range(N) if w != d)
        b += dims[d] * R * 4
        out.append(b)
    return out


class ClockSampler:
    """SM clocks and throttle reasons sampled while the GPU works.

    NVML (the driver's libnvidia-ml, read through ctypes) is polled every
    ~2 ms from a thread, so that even a timed region of a few tens of
    milliseconds holds many samples; mark() brackets the timed region and
    stop() summarises the samples inside it.  Falls back to nvidia-smi at
    its own 200 ms period when NVML cannot be loaded.  Only reads settings."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock event reason bits of nvml.h
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    PERIOD_S = 0.002

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.thread = None
        self.lines = []
        self.samples = []  # (t, sm_mhz, max_mhz, reasons bits)
        self.window = None
        self.source = None
        self._stop = threading.Event()

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.gpu).uuid)
        except Exception:
            uuid = None
        if uuid:
            u = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            if lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0:
                return lib, h
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        return lib, h

    def _poll_nvml(self, lib, h):
        import ctypes
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            ok = (lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and
                  lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0)
            r = get_reasons(h, ctypes.byref(rs)) == 0
            if ok:
                self.samples.append((time.perf_counter(), float(clk.value), float(mx.value),
                                     int(rs.value) if r else 0))
            time.sleep(self.PERIOD_S)

    def start(self):
        try:
            lib, h = self._nvml_handle()
            self.source = "nvml"
            self.thread = threading.Thread(target=self._poll_nvml, args=(lib, h), daemon=True)
            self.thread.start()
            return
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        names = [0x8, 0x40, 0x20, 0x4]
        for line in self.proc.stdout:
            f = [x.strip() for x in line.strip().split(",")]
            if len(f) < 9:
                continue
            try:
                sm, mx = float(f[1]), float(f[2])
            except ValueError:
                continue
            bits = sum(b for b, v in zip(names, f[5:9]) if v.lower() == "active")
            self.samples.append((time.perf_counter(), sm, mx, bits))

    def mark(self, t0, t1):
        """Host times (perf_counter) that bracket the timed region."""
        self.window = (t0, t1)

    def stop(self):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.source:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock query unavailable"],
                    "samples": 0}
        sel = self.samples
        if self.window:
            t0, t1 = self.window
            inside = [x for x in self.samples if t0 <= x[0] <= t1]
            sel = inside or sel
        sm = [x[1] for x in sel]
        mx = [x[2] for x in sel]
        bits = 0
        for x in sel:
            bits |= x[3]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(n for b, n in self.REASONS.items() if bits & b),
                "samples": len(sm), "source": self.source,
                "window": "timed region" if self.window else "whole run"}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_sample(dims, idx, vals, Y, sample_nnz):
    import numpy as np
    n = int(sample_nnz)
    h_idx = [c[:n].cpu().numpy() for c in idx]
    h_vals = vals[:n].cpu().numpy()
    h_Y = [y.cpu().numpy().astype(np.float64) for y in Y]
    return h_idx, h_vals, h_Y


def time_oracle(dims, h_idx, h_vals, h_Y, R):
    """One pass of the oracle MTTKRP over all modes; returns (seconds, bytes)."""
    import numpy as np
    import oracle
    n = h_vals.size
    distinct = [int(np.unique(c).size) for c in h_idx]
    t0 = time.perf_counter()
    for d in range(len(dims)):
        oracle.mttkrp(dims, h_idx, h_vals, h_Y, d)
    dt = time.perf_counter() - t0
    return dt, sum(algorithmic_bytes(dims, n, R, distinct))


def host_info():
    """Core count and CPU model of the host the oracle runs on."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def time_oracle_omp(dims, h_idx, h_vals, h_Y, R):
    """One pass of the all-core OpenMP oracle over all modes; returns
    (seconds, bytes, threads used)."""
    import numpy as np
    import oracle
    n = h_vals.size
    distinct = [int(np.unique(c).size) for c in h_idx]
    t0 = time.perf_counter()
    used = 0
    for d in range(len(dims)):
        _, used = oracle.mttkrp_omp(dims, h_idx, h_vals, h_Y, d)
    dt = time.perf_counter() - t0
    return dt, sum(algorithmic_bytes(dims, n, R, distinct)), used


def cpu_baseline(dims, idx, vals, Y, R, target_s):
    """The oracle as it stands, single-threaded, on a prefix sample of the
    workload's nonzeros (the same tensor's first nonzeros in draw order), and
    beside it the same definition on all host cores (OpenMP, thread-private
    outputs added at the end) on the same sample."""
    probe = 1_000_000
    h = host_sample(dims, idx, vals, Y, probe)
    dt, _ = time_oracle(dims, *h, R)
    n = int(min(vals.numel(), max(probe, probe * target_s / max(dt, 1e-3))))
    h = host_sample(dims, idx, vals, Y, n)
    dt, b = time_oracle(dims, *h, R)
    sample = f"first {n} of the workload's nonzeros (draw order), all {len(dims)} modes"
    res = {"value": b / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{sample}, {dt:.1f} s single-threaded FP64",
           "sample_nnz": n, "seconds_all_modes": dt,
           "host": host_info()}
    try:
        time_oracle_omp(dims, *host_sample(dims, idx, vals, Y, 100_000), R)  # warm-up
        dto, bo, used = time_oracle_omp(dims, *h, R)
        res["openmp_all_cores"] = {"value": bo / dto / 1e9, "unit": UNIT, "cores": used,
                                   "seconds_all_modes": dto,
                                   "kind": "oracle (OpenMP, thread-private outputs)",
                                   "sample": f"{sample}, {dto:.2f} s on {used} threads FP64",
                                   "speedup_vs_single_thread": dt / dto}
    except Exception as e:  # a baseline report: never fail the bench line for it
        res["openmp_all_cores"] = {"unavailable": str(e)[:200]}
    return res


def arm_config(nnz, dims, R, world):
    """The `config` object of the headline line (both arms)."""
    return {"workload": WORKLOAD, "nnz": nnz, "dims": list(dims), "rank": R,
            "factor_dtype": "fp32", "policy": "balanced",
            "step": "spMTTKRP along modes 0,1,2 on resident mode copies",
            "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


REFERENCE_SECONDS = 120.0  # wall-time target of a whole reference run


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same metric/unit.
    Each step runs the oracle's MTTKRP along all modes on the workload's first
    n nonzeros, n sized from a probe so that warm-up plus the timed steps take
    about REFERENCE_SECONDS."""
    if rank != 0:
        return
    import synth
    import torch
    torch.set_num_threads(max(1, os.cpu_count() or 1))
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    dims, idx, vals, R, Y = synth.preset_torch("scale", nnz=args.nnz, device=dev)
    probe = min(args.nnz, 200_000)
    dt, _ = time_oracle(dims, *host_sample(dims, idx, vals, Y, probe), R)
    per_step = REFERENCE_SECONDS / max(1, args.steps + args.warmup)
    n = int(min(args.nnz, 2_000_000, max(20_000, probe * per_step / max(dt, 1e-6))))
    h = host_sample(dims, idx, vals, Y, n)
    for _ in range(args.warmup):
        time_oracle(dims, *h, R)
    tot_s, tot_b = 0.0, 0
    for _ in range(args.steps):
        dt, b = time_oracle(dims, *h, R)
        tot_s += dt
        tot_b += b
    v = tot_b / tot_s / 1e9
    sample = f"first {n} of the workload's nonzeros per step, all 3 modes, single-threaded FP64 oracle"
    cfg = arm_config(int(vals.numel()), dims, R, world)
    cfg["sample_nnz"] = n
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def main():
    args = parse()
    import torch
    rank, world, local = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import synth
    import paper_2503_18198_gb300 as spm
    spm.load()  # fails loudly if the CUDA library is missing
    if args.workload != "scale":
        if rank == 0:  # the extra workloads run on one GPU
            {"batching": run_batching, "serving": run_serving, "precision": run_precision,
             "five": run_precision, "schemes": run_schemes,
             "lean": run_lean, "fibre": run_fibre,
             "probe": run_probe}[args.workload](args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    dims, idx, vals, R, Y = synth.preset_torch("scale", nnz=args.nnz, device="cuda")
    N = len(dims)
    nnz = int(vals.numel())
    distinct = [int((torch.bincount(c.long(), minlength=dims[w]) > 0).sum())
                for w, c in enumerate(idx)]
    B = algorithmic_bytes(dims, nnz, R, distinct)
    stream = torch.cuda.current_stream()

    # P1 + P2: plan build (timed once, not part of the step)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = spm.spmttkrp_plan(dims, idx, vals, R)
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    outs = [torch.empty(dims[d], R, device="cuda") for d in range(N)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(evs=None):
        for d in range(N):
            if evs is not None:
                evs[d][0].record(stream)
            spm.spmttkrp_run(plan, d, Y, outs[d])
            if evs is not None:
                evs[d][1].record(stream)

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    per_mode = [0.0] * N
    t_begin = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()  # evict L2 between steps (outside the events)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(N)]
        step(evs)
        torch.cuda.synchronize()
        for d in range(N):
            per_mode[d] += evs[d][0].elapsed_time(evs[d][1])
    torch.cuda.synchronize()
    clocks.mark(t_begin, time.perf_counter())
    barrier(world)
    clk = clocks.stop()
    step_ms = sum(per_mode) / args.steps
    step_ms = max_over_ranks(step_ms, world)
    mode_ms = [m / args.steps for m in per_mode]
    value = replica_value(sum(B), step_ms, world)

    # the same steps back to back with no flush (the ALS regime, where the
    # next mode finds what the previous one left in L2), reported beside
    warm_steps = max(3, min(args.steps, 20))
    per_mode_warm = [0.0] * N
    for _ in range(warm_steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(N)]
        step(evs)
        torch.cuda.synchronize()
        for d in range(N):
            per_mode_warm[d] += evs[d][0].elapsed_time(evs[d][1])
    mode_ms_warm = [m / warm_steps for m in per_mode_warm]

    # roofline of the MTTKRP launches (the dominant kernel)
    peak, peak_kind = measured_peak()
    achieved = sum(B) / (sum(mode_ms) * 1e-3) / 1e9
    traffic = None
    traffic_small = None  # counters of a smaller case of the same kernel, reported beside
    tfile = os.path.join(ROOT, "profiles", "mttkrp_traffic.json")
    if os.path.exists(tfile):
        try:
            with open(tfile) as f:
                tj = json.load(f)
            # counters taken with the current kernel sources only; `traffic`
            # only from this workload (they do not scale with the nonzeros)
            if tj.get("kernel_digest") == kernel_digest():
                if tj.get("nnz") == nnz:
                    traffic = tj.get("bytes_per_launch")
                else:
                    traffic_small = {"nnz": tj.get("nnz"),
                                     "bytes_per_launch": tj.get("bytes_per_launch"),
                                     "over_algorithmic": tj.get("traffic_over_algorithmic"),
                                     "source": "profiles/mttkrp_traffic.json"}
        except (OSError, ValueError):
            traffic = None

    # e2e through the C ABI with host buffers (spmttkrp_run_all_host): the
    # factors come in from pinned host memory and the three outputs go back
    # every step, the copies overlapped with the modes' kernels.
    hY = [y.cpu().pin_memory() for y in Y]
    hout = [torch.empty(dims[d], R).pin_memory() for d in range(N)]
    h2d = sum(y.numel() * 4 for y in hY)
    d2h = sum(o.numel() * 4 for o in hout)

    def e2e_step():
        spm.spmttkrp_run_all_host(plan, hY, hout)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(3, min(args.steps, 10))
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world)
    e2e_value = replica_value(sum(B), e2e_ms, world)
    copy_rates = host_copy_rates(hY[0], hout[0], stream)

    # one CP-ALS sweep (P6 included) on the same plan, beside the step
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    fit = torch.empty(1, dtype=torch.float64, device="cuda")
    fac = [y.clone() for y in Y]
    spm.cpd_als_step(plan, fac, lam, fit)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    spm.cpd_als_step(plan, fac, lam, fit)
    a1.record(stream)
    torch.cuda.synchronize()
    als_ms = a0.elapsed_time(a1)

    launches_per_step = sum(1 + (1 if plan_kappa(spm, plan) > 1 else 0) +
                            (1 if distinct[d] < dims[d] else 0) for d in range(N))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(dims, idx, vals, Y, R, args.cpu_seconds)

    # the batching comparison beside the headline: BF16 batched CP-ALS
    # against the tuned plain per-tensor FP32 path on the 512-tensor workload
    batching = None
    if rank == 0 and world == 1 and not args.no_batching:
        del outs, flush, hY, hout, fac
        torch.cuda.empty_cache()
        res = batching_measure(args.tensors, args.sweeps)
        arms = res["arms"]
        batching = {
            "workload": "512 independent 3-mode COO tensors (dims log-uniform [100, 20000], "
                        "nnz log-uniform [1e3, 2e6]), R in {16, 32}, 20 CP-ALS sweeps each",
            "metric": "CPD solves/s", "unit": "solves/s",
            "bf16_batched": arms["bf16_batched"]["solves_per_s"],
            "fp32_batched": arms["fp32_batched"]["solves_per_s"],
            "fp32_per_tensor_tuned": arms["fp32_per_tensor"]["solves_per_s"],
            "speedup_bf16_batched_vs_fp32_per_tensor": res["speedup_bf16_batched_vs_fp32_per_tensor"],
            "fit_agreement": res["fit_agreement"],
            "ms_per_sweep": {k: arms[k].get("ms_per_sweep") for k in ("bf16_batched", "fp32_batched")},
            "batch_autotune_nnz_per_partition": {k: arms[k]["autotune"]["chosen"]
                                                 for k in ("bf16_batched", "fp32_batched")},
            "plain_kappa_autotuned": arms["fp32_per_tensor"]["kappa_autotuned"],
            "total_nnz": res["config"]["total_nnz"], "sweeps": res["config"]["sweeps"],
            "clocks": res["clocks"], "wall_s": round(res["wall_s"], 1)}

    # and the serving comparison on the first SERVING_REQUESTS requests of the
    # Poisson stream (p50/p99 time to solution, solves/s)
    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        torch.cuda.empty_cache()
        t_sv = time.perf_counter()
        sv = serving_measure(SERVING_REQUESTS)
        serving = {
            "workload": f"first {SERVING_REQUESTS} requests of the seeded Poisson stream "
                        "(200 requests/s; 3 or 4 modes, dims log-uniform [1e3, 1e6], nnz "
                        "log-uniform [1e4, 5e7], R in {8, 16, 32, 64}), tol 1e-4, <= 50 sweeps",
            "metric": "CPD solves/s + p50/p99 time to solution", "unit": "solves/s",
            "served_bf16": sv["served_bf16_continuous_batching"],
            "plain_fp32_per_tensor": sv["plain_fp32_per_tensor"],
            "speedup_solves_per_s": sv["speedup_solves_per_s"],
            "fit_agreement": sv["fit_agreement"], "total_nnz": sv["config"]["total_nnz"],
            "clocks": sv["clocks"], "wall_s": round(time.perf_counter() - t_sv, 1)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": arm_config(nnz, dims, R, world),
            "per_mode_ms": [round(m, 4) for m in mode_ms],
            "per_mode_roofline_frac": [round(b / (m * 1e-3) / 1e9 / peak, 4)
                                       for b, m in zip(B, mode_ms)],
            "l2_not_flushed": {"steps": warm_steps,
                               "per_mode_ms": [round(m, 4) for m in mode_ms_warm],
                               "GBs": sum(B) / (sum(mode_ms_warm) * 1e-3) / 1e9},
            "nnz_per_s_per_mode": [round(nnz / (m * 1e-3), 1) for m in mode_ms],
            "effective_gather_GBs": round(nnz * (N - 1) * R * 4 * N / (sum(mode_ms) * 1e-3) / 1e9, 1),
            "algorithmic_bytes_per_mode": B,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_smaller_case": traffic_small,
                         "kernel": "mttkrp_kernel (+ row zero-fill and partition fix-up of the same call)",
                         "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "host_copy_GBs": copy_rates},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
            "plan_ms": plan_ms,
            "als_sweep_ms": als_ms,
            "plan_bytes": spm.spmttkrp_plan_bytes(plan),
            "batching": batching,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    plan.destroy()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_lean(args, rank, world):
    """Memory-lean plans (one record copy plus per-mode positions into it)
    against full plans (one record copy per mode) on the scale and
    precision workloads: plan bytes, plan build time, spMTTKRP time per
    mode (FP32 factors, default partitions) and one CP-ALS sweep."""
    import torch
    import synth
    import paper_2503_18198_gb300 as spm
    stream = torch.cuda.current_stream()
    out = {}
    for name in ("scale", "precision"):
        dims, idx, vals, R, Y = synth.preset_torch(name, device="cuda")
        N = len(dims)
        out[name] = {}
        for arm, flags in (("full", 0), ("lean", spm.SPM_PLAN_LEAN)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan = spm.spmttkrp_plan(dims, idx, vals, R, flags)
            torch.cuda.synchronize()
            plan_ms = (time.perf_counter() - t0) * 1e3
            outs = [torch.empty(dims[d], R, device="cuda") for d in range(N)]
            ms = []
            for d in range(N):
                for _ in range(3):
                    spm.spmttkrp_run(plan, d, Y, outs[d])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(10):
                    spm.spmttkrp_run(plan, d, Y, outs[d])
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(round(e0.elapsed_time(e1) / 10, 4))
            fac = [y.clone() for y in Y]
            lam = torch.zeros(R, dtype=torch.float64, device="cuda")
            spm.cpd_als_step(plan, fac, lam)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            spm.cpd_als_step(plan, fac, lam)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name][arm] = {"plan_bytes": spm.spmttkrp_plan_bytes(plan), "plan_ms": plan_ms,
                              "mttkrp_ms_per_mode": ms, "als_sweep_ms": e0.elapsed_time(e1)}
            plan.destroy()
        f, l = out[name]["full"], out[name]["lean"]
        out[name]["bytes_ratio_full_over_lean"] = f["plan_bytes"] / l["plan_bytes"]
        out[name]["mttkrp_time_ratio_lean_over_full"] = (sum(l["mttkrp_ms_per_mode"]) /
                                                         sum(f["mttkrp_ms_per_mode"]))
        del idx, vals, Y
    print(json.dumps({"workload": "lean", "metric": "plan bytes and spMTTKRP ms, full vs lean",
                      "unit": "ms", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                      "results": out}), flush=True)


def run_probe(args, rank, world):
    """A fixed launch sequence for profiler captures: one plan of --preset at
    --nnz nonzeros with --factor storage, three warm-up spMTTKRP launches per
    mode, then one launch per mode (timed by CUDA events and printed), then
    --probe-sweeps CP-ALS sweeps (each timed).  Profilers select launches with
    -k / -s / -c on this order; the printed times are not bench values."""
    import torch
    import synth
    import paper_2503_18198_gb300 as spm
    dims, idx, vals, R, Y = synth.preset_torch(args.preset, nnz=args.nnz, device="cuda")
    N = len(dims)
    bf16 = args.factor == "bf16"
    plan = spm.spmttkrp_plan(dims, idx, vals, R,
                             spm.SPM_FACTOR_BF16 if bf16 else spm.SPM_FACTOR_FP32)
    fac = [y.to(torch.bfloat16 if bf16 else torch.float32).clone() for y in Y]
    outs = [torch.empty(d, R, device="cuda") for d in dims]
    for _ in range(3):
        for d in range(N):
            spm.spmttkrp_run(plan, d, fac, outs[d])
    torch.cuda.synchronize()
    ms = []
    for d in range(N):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        spm.spmttkrp_run(plan, d, fac, outs[d])
        e1.record()
        torch.cuda.synchronize()
        ms.append(round(e0.elapsed_time(e1), 4))
    lam = torch.empty(R, dtype=torch.float64, device="cuda")
    fit = torch.empty(1, dtype=torch.float64, device="cuda")
    sweep_ms = []
    for _ in range(args.probe_sweeps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        spm.cpd_als_step(plan, fac, lam, fit)
        e1.record()
        torch.cuda.synchronize()
        sweep_ms.append(round(e0.elapsed_time(e1), 4))
    print(json.dumps({"workload": "probe", "preset": args.preset, "factor": args.factor,
                      "dims": list(dims), "nnz": int(vals.numel()), "rank": R,
                      "mttkrp_ms_per_mode": ms, "als_sweep_ms": sweep_ms}))


def fibre_bytes(dims, nnz, R, distinct, nfib, s_f=4):
    """B_d of a fibre-layout copy: 8-byte entries (one per nonzero and one per
    fibre header), each distinct gathered row once, the output once."""
    N = len(dims)
    return [8 * (nnz + nfib[d]) + sum(distinct[w] * R * s_f for w in range(N) if w != d)
            + dims[d] * R * 4 for d in range(N)]


def run_fibre(args, rank, world):
    """Fibre-layout copies (N1) against record copies on the 50M-nonzero scale
    workload: spMTTKRP time per mode (L2 flushed before each timed run),
    plan bytes, fibre counts, GB/s on each layout's own bytes and on the
    record layout's bytes, nonzeros/s, and a sampled-row check of the fibre
    result against the record result."""
    import torch
    import synth
    import paper_2503_18198_gb300 as spm
    dims, idx, vals, R, Y = synth.preset_torch("scale", nnz=args.nnz, device="cuda")
    N = len(dims)
    nnz = int(vals.numel())
    distinct = distinct_counts(idx)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    peak, peak_kind = measured_peak()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    res, outs_all = {}, {}
    for arm, flags in (("record", 0), ("fibre", spm.SPM_PLAN_FIBRE)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = spm.spmttkrp_plan(dims, idx, vals, R, flags)
        torch.cuda.synchronize()
        plan_ms = (time.perf_counter() - t0) * 1e3
        outs = [torch.empty(dims[d], R, device="cuda") for d in range(N)]
        for _ in range(3):
            for d in range(N):
                spm.spmttkrp_run(plan, d, Y, outs[d])
        reps = 10
        ms = [0.0] * N
        for _ in range(reps):
            for d in range(N):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                spm.spmttkrp_run(plan, d, Y, outs[d])
                e1.record(stream)
                torch.cuda.synchronize()
                ms[d] += e0.elapsed_time(e1) / reps
        nfib = [spm.spmttkrp_plan_fibre_count(plan, d) for d in range(N)] if flags else None
        B_rec = algorithmic_bytes(dims, nnz, R, distinct)
        B_own = fibre_bytes(dims, nnz, R, distinct, nfib) if flags else B_rec
        res[arm] = {"plan_ms": plan_ms, "plan_bytes": spm.spmttkrp_plan_bytes(plan),
                    "ms_per_mode": [round(m, 4) for m in ms], "ms_all_modes": sum(ms),
                    "GBs_own_bytes": sum(B_own) / (sum(ms) * 1e-3) / 1e9,
                    "GBs_record_bytes": sum(B_rec) / (sum(ms) * 1e-3) / 1e9,
                    "roofline_frac_own_bytes": sum(B_own) / (sum(ms) * 1e-3) / 1e9 / peak,
                    "nnz_per_s_per_mode": [round(nnz / (m * 1e-3), 1) for m in ms],
                    "fibres_per_mode": nfib,
                    "algorithmic_bytes_per_mode": B_own}
        outs_all[arm] = outs
        plan.destroy()
    clk = clocks.stop()
    g = torch.Generator(device="cuda").manual_seed(0)
    diff = []
    for d in range(N):
        rows = torch.randint(0, dims[d], (4096,), device="cuda", generator=g)
        a, b = outs_all["fibre"][d][rows], outs_all["record"][d][rows]
        diff.append(float((a - b).norm() / b.norm().clamp_min(1e-30)))
    print(json.dumps({
        "workload": "fibre", "metric": "spMTTKRP ms per mode, fibre vs record copies",
        "unit": "ms", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": WORKLOAD, "nnz": nnz, "rank": R, "l2": "flushed before each run",
                   "peak": peak, "peak_source": peak_kind},
        "results": res, "speedup_fibre_over_record": res["record"]["ms_all_modes"] /
        res["fibre"]["ms_all_modes"],
        "sampled_rows_rel_diff_fibre_vs_record": diff, "clocks": clk}), flush=True)


SCHEME_SHAPES = [
    # (name, dims, nnz, Zipf exponents (None = uniform), rank)
    ("scale-20M", (1_000_000, 500_000, 200_000), 20_000_000, (1.2, 1.2, 1.2), 32),
    ("precision-30M", (20_000, 20_000, 5_000, 24), 30_000_000, (1.0, 1.0, 1.0, None), 64),
    ("uniform-20M", (100_000, 100_000, 100_000), 20_000_000, (None, None, None), 32),
    ("short-modes-20M", (200_000, 5_000, 64), 20_000_000, (1.1, 1.1, None), 32),
]


def run_schemes(args, rank, world):
    """The paper's load-balancing ablation (Sec. III-B): spMTTKRP time per
    mode under Scheme 1 only, Scheme 2 only and the adaptive rule (Scheme 1
    when I_d >= kappa), all at the paper's kappa = SM count, plus this
    build's default (cost-balanced work units, two partitions per SM).
    Reports geometric-mean speedups over all (shape, mode) pairs."""
    import math
    import torch
    import synth
    import paper_2503_18198_gb300 as spm
    sms = spm.spm_device_sm_count()
    pols = [("scheme1", spm.SPM_POLICY_SCHEME1 | spm.SPM_KAPPA(sms)),
            ("scheme2", spm.SPM_POLICY_SCHEME2 | spm.SPM_KAPPA(sms)),
            ("adaptive", spm.SPM_POLICY_ADAPTIVE | spm.SPM_KAPPA(sms)),
            ("balanced_1_per_sm", spm.SPM_POLICY_BALANCED | spm.SPM_KAPPA(sms)),
            ("balanced_default", spm.SPM_POLICY_BALANCED),
            ("balanced_autotuned", spm.SPM_POLICY_BALANCED)]
    stream = torch.cuda.current_stream()
    res = {}
    for si, (name, dims, nnz, alphas, R) in enumerate(SCHEME_SHAPES):
        dims, idx, vals = synth.coo_distinct_torch(dims, nnz, alphas, seed=40 + si, device="cuda")
        Y = synth.factors_torch(dims, R, seed=40 + si, device="cuda")
        outs = [torch.empty(dims[d], R, device="cuda") for d in range(len(dims))]
        res[name] = {}
        for pname, flags in pols:
            plan = spm.spmttkrp_plan(dims, idx, vals, R, flags)
            if pname == "balanced_autotuned":
                spm.spmttkrp_plan_autotune(plan, Y)
            ms = []
            for d in range(len(dims)):
                for _ in range(2):
                    spm.spmttkrp_run(plan, d, Y, outs[d])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(5):
                    spm.spmttkrp_run(plan, d, Y, outs[d])
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(round(e0.elapsed_time(e1) / 5, 4))
            res[name][pname] = {"ms_per_mode": ms,
                                "scheme_per_mode": [spm.spmttkrp_plan_scheme(plan, d)
                                                    for d in range(len(dims))]}
            plan.destroy()
        del idx, vals, Y, outs

    def geomean(a, b):
        logs = [math.log(x / y) for n in res for x, y in
                zip(res[n][a]["ms_per_mode"], res[n][b]["ms_per_mode"])]
        return math.exp(sum(logs) / len(logs))
    line = {"workload": "schemes", "metric": "spMTTKRP ms per mode by partitioning policy",
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "config": {"kappa_paper": sms, "shapes": [s[0] for s in SCHEME_SHAPES],
                       "factors": "fp32"},
            "results": res,
            "geomean_speedup": {
                "adaptive_over_scheme1": geomean("scheme1", "adaptive"),
                "adaptive_over_scheme2": geomean("scheme2", "adaptive"),
                "balanced_1_per_sm_over_adaptive": geomean("adaptive", "balanced_1_per_sm"),
                "balanced_default_over_adaptive": geomean("adaptive", "balanced_default"),
                "balanced_autotuned_over_adaptive": geomean("adaptive", "balanced_autotuned")}}
    print(json.dumps(line), flush=True)


def distinct_counts(idx):
    import torch
    return [int(torch.unique(c).numel()) for c in idx]


def batching_measure(n_tensors, S, with_clocks=True):
    """Batching workload: many small 3-mode tensors, S CP-ALS sweeps each.

    Arms (same tensors, same initial factors):
      * batched FP32 and batched BF16: spm_batch_autotune picks the
        nonzeros per partition, then one CUDA graph of a whole batched sweep
        (persistent per-class spMTTKRP launches fed by the (tensor,
        partition) work queue, batched ALS passes) is replayed S times;
      * plain per-tensor FP32: cpd_als_step on each tensor in turn, each
        tensor's partition count picked by spmttkrp_plan_autotune among the
        batch candidates' counts and one or two partitions per SM (so the
        comparison is batching against a tuned single-tensor path, not
        against a default partition count).
    solves/s = tensors / time of all their sweeps (inputs resident in HBM,
    plans built and tuned before timing).  The final fits of the batched arms
    are compared with the plain FP32 path's (agreement within 1e-3).
    Returns the result dict (arms, fit agreement, speedups, clocks)."""
    import numpy as np
    import torch
    import synth
    import paper_2503_18198_gb300 as spm
    t_start = time.perf_counter()
    specs = synth.batching_specs(n_tensors)
    tens = []
    for dims, nnz, R, seed in specs:
        dims, idx, vals = synth.tensor_torch(dims, nnz, seed, device="cuda")
        tens.append((dims, idx, vals, R, seed, distinct_counts(idx)))
    n = len(tens)
    total_nnz = sum(int(t[2].numel()) for t in tens)
    stream = torch.cuda.current_stream()
    sms = spm.spm_device_sm_count()

    def build(flags):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plans = [spm.spmttkrp_plan(d, i, v, R, flags) for d, i, v, R, _, _ in tens]
        torch.cuda.synchronize()
        return plans, (time.perf_counter() - t0) * 1e3

    def factors(dtype):
        return [[f.to(dtype).contiguous() for f in synth.factors_torch(d, R, seed, device="cuda")]
                for d, _, _, R, seed, _ in tens]

    def mttkrp_bytes(s_f):
        return sum(sum(algorithmic_bytes(d, int(v.numel()), R, u, s_f))
                   for d, _, v, R, _, u in tens)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    clocks = ClockSampler(torch.cuda.current_device()) if with_clocks else None
    if clocks:
        clocks.start()
    out = {}
    cands = (0, 1 << 13, 1 << 15, 1 << 17, 1 << 18, 1 << 19)
    for name, flags, dtype, s_f in (("fp32_batched", spm.SPM_FACTOR_FP32, torch.float32, 4),
                                    ("bf16_batched", spm.SPM_FACTOR_BF16, torch.bfloat16, 2)):
        plans, plan_ms = build(flags)
        facs = factors(dtype)
        chosen, cms = spm.spm_batch_autotune(plans, facs, cands, reps=3)
        lam = torch.zeros(sum(t[3] for t in tens), dtype=torch.float64, device="cuda")
        fits = torch.zeros(n, dtype=torch.float64, device="cuda")
        B = spm.spm_batch_create(plans, facs, lam, fits, tol=0.0, max_sweeps=S)
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                spm.spm_batch_sweep(B)
        stream.wait_stream(cs)
        ms = timed(lambda: [g.replay() for _ in range(S)])
        active, nsw = spm.spm_batch_status(B)
        assert all(x == S for x in nsw), nsw
        assert all(spm.spmttkrp_plan_status(p) == 0 for p in plans)
        best = cands.index(chosen)
        out[name] = {"solves_per_s": n / (ms * 1e-3), "ms_total": ms, "ms_per_sweep": ms / S,
                     "plan_build_ms": plan_ms,
                     "autotune": {"nnz_per_partition_candidates": list(cands),
                                  "mttkrp_all_modes_ms": [round(x, 4) for x in cms],
                                  "chosen": chosen},
                     "mttkrp_GBs": mttkrp_bytes(s_f) / (cms[best] * 1e-3) / 1e9,
                     "mttkrp_all_modes_ms": cms[best],
                     "launches_per_sweep_graph": "one graph"}
        out[name]["fits"] = fits.cpu().numpy()
        del g
        B.destroy()
        for p in plans:
            p.destroy()
        del facs
    # plain per-tensor FP32 path, each plan's partition count autotuned
    plans, plan_ms = build(spm.SPM_FACTOR_FP32)
    facs = factors(torch.float32)
    t0 = time.perf_counter()
    chosen_k = []
    for t, (d, _, v, R, _, _) in enumerate(tens):
        nz = int(v.numel())
        ks = sorted({max(1, min(65535, -(-nz // c))) for c in cands[1:]} | {sms, 2 * sms})
        k, _ = spm.spmttkrp_plan_autotune(plans[t], facs[t], ks, reps=2)
        chosen_k.append(k)
    tune_ms = (time.perf_counter() - t0) * 1e3
    lams = [torch.zeros(t[3], dtype=torch.float64, device="cuda") for t in tens]
    fits = torch.zeros(n, dtype=torch.float64, device="cuda")

    def plain():
        for t in range(n):
            for _ in range(S):
                spm.cpd_als_step(plans[t], facs[t], lams[t], fits[t:t + 1])
    ms = timed(plain)
    assert all(spm.spmttkrp_plan_status(p) == 0 for p in plans)
    out["fp32_per_tensor"] = {"solves_per_s": n / (ms * 1e-3), "ms_total": ms,
                              "plan_build_ms": plan_ms, "autotune_ms": tune_ms,
                              "kappa_autotuned": {"min": min(chosen_k), "max": max(chosen_k),
                                                  "median": int(np.median(chosen_k))},
                              "fits": fits.cpu().numpy()}
    for p in plans:
        p.destroy()
    del facs
    clk = clocks.stop() if clocks else None
    ref = out["fp32_per_tensor"]["fits"]
    agree = {}
    for name in ("fp32_batched", "bf16_batched"):
        dfit = np.abs(out[name].pop("fits") - ref)
        agree[name + "_vs_fp32_per_tensor"] = {
            "max_abs_dfit": float(dfit.max()), "within_1e-3": int((dfit <= 1e-3).sum()),
            "of": n}
    out["fp32_per_tensor"].pop("fits")
    return {
        "config": {"tensors": n, "total_nnz": total_nnz, "sweeps": S, "modes": 3,
                   "ranks": "16 or 32", "dims": "log-uniform [100, 20000]",
                   "nnz": "log-uniform [1e3, 2e6], at most half the cells",
                   "l2": "inputs (mode copies of all tensors) larger than L2"},
        "arms": out, "fit_agreement": agree,
        "speedup_bf16_batched_vs_fp32_per_tensor":
            out["bf16_batched"]["solves_per_s"] / out["fp32_per_tensor"]["solves_per_s"],
        "speedup_bf16_batched_vs_fp32_batched":
            out["bf16_batched"]["solves_per_s"] / out["fp32_batched"]["solves_per_s"],
        "clocks": clk, "wall_s": time.perf_counter() - t_start}


def run_batching(args, rank, world):
    """The batching workload's own JSON line (see batching_measure)."""
    res = batching_measure(args.tensors, args.sweeps)
    line = {"workload": "batching", "metric": "CPD solves/s", "unit": "solves/s",
            "value": res["arms"]["bf16_batched"]["solves_per_s"], "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic"}
    line.update(res)
    print(json.dumps(line), flush=True)


def run_serving(args, rank, world):
    """Serving workload: a seeded Poisson stream (mean 200 requests/s) of
    CP-ALS jobs (3 or 4 modes, dims log-uniform [1e3, 1e6], nnz log-uniform
    [1e4, 5e7], Zipf(1.1) coordinates, R in {8, 16, 32, 64}), each run until
    its fit changes by less than 1e-4 or 50 sweeps.

    Arms, on the same inputs (resident in HBM before the clock starts, the
    requests' COO arrays and initial factors) and the same arrival times:
      * served: the BF16 continuous-batching server (spm_server_*), 150 GB
        budget for plans and factors; arrivals are submitted in real time,
        the host loop steps the server and collects finished jobs;
      * plain: per-tensor FP32, one job at a time in arrival order
        (spmttkrp_plan, then cpd_als_step with the fit read back after each
        sweep until the same stopping rule).
    Time to solution = finish - arrival (host clock); solves/s = requests /
    (last finish - first arrival)."""
    print(json.dumps(serving_measure(args.requests)), flush=True)


SERVING_REQUESTS = 60  # the default line's serving comparison (the full workload: 200)


def serving_measure(n_requests, with_clocks=True):
    """The serving comparison of run_serving on the first n_requests of the
    seeded request stream; returns its JSON line as a dict."""
    import numpy as np
    import torch
    import synth
    import paper_2503_18198_gb300 as spm
    specs = synth.serving_specs(n_requests)
    tol, cap, budget = 1e-4, 50, 150 * 10**9
    reqs = []
    for t_arr, dims, nnz, R, seed in specs:
        dims, idx, vals = synth.tensor_torch(dims, nnz, seed, alpha=synth.SERVING_ALPHA,
                                             device="cuda", max_rounds=6)
        init = [f.contiguous() for f in synth.factors_torch(dims, R, seed, device="cuda")]
        reqs.append((t_arr, dims, idx, vals, R, init))
    torch.cuda.synchronize()
    n = len(reqs)
    total_nnz = sum(int(r[3].numel()) for r in reqs)
    clocks = ClockSampler(torch.cuda.current_device()) if with_clocks else None
    if clocks:
        clocks.start()

    # ---- served: continuous batching, BF16 factors
    S = spm.Server(budget, max_active=256, flags=spm.SPM_FACTOR_BF16,
                   nnz_per_partition=1 << 17)
    ids, done, peak, steps = [None] * n, {}, 0, 0
    t0 = time.perf_counter()
    nxt = 0
    while len(done) < n:
        now = time.perf_counter() - t0
        while nxt < n and reqs[nxt][0] <= now:
            t_arr, dims, idx, vals, R, init = reqs[nxt]
            ids[nxt] = S.submit(dims, idx, vals, R, init, tol=tol, max_sweeps=cap)
            nxt += 1
        running, queued = S.step()
        steps += 1
        peak = max(peak, S.usage()[0])
        t_now = time.perf_counter() - t0
        for k in range(nxt):
            if k in done:
                continue
            info = S.info(ids[k])
            if info.state in (spm.binding.SPM_JOB_DONE, spm.binding.SPM_JOB_FAILED):
                done[k] = (t_now - reqs[k][0], info.sweeps, info.fit, info.state)
                if info.state == spm.binding.SPM_JOB_DONE:
                    S.result(ids[k])
        if running == 0 and queued == 0 and nxt < n:
            time.sleep(max(0.0, reqs[nxt][0] - (time.perf_counter() - t0)))
    served_span = max(reqs[k][0] + done[k][0] for k in done) - reqs[0][0]
    S.destroy()
    failed = sum(1 for v in done.values() if v[3] != spm.binding.SPM_JOB_DONE)

    # ---- plain per-tensor FP32, one job at a time in arrival order
    plain = {}
    t0 = time.perf_counter()
    for k, (t_arr, dims, idx, vals, R, init) in enumerate(reqs):
        wait = t_arr - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        plan = spm.spmttkrp_plan(dims, idx, vals, R)
        fac = [f.clone() for f in init]
        lam = torch.zeros(R, dtype=torch.float64, device="cuda")
        fit = torch.zeros(1, dtype=torch.float64, device="cuda")
        prev, sw = -1e300, 0
        while True:
            spm.cpd_als_step(plan, fac, lam, fit)
            sw += 1
            f = float(fit.item())
            if abs(f - prev) < tol or sw >= cap:
                break
            prev = f
        plan.destroy()
        plain[k] = ((time.perf_counter() - t0) - t_arr, sw, f)
        del fac
    plain_span = max(reqs[k][0] + plain[k][0] for k in plain) - reqs[0][0]
    clk = clocks.stop() if clocks else None

    def summary(d, span):
        tts = np.array([v[0] for v in d.values()]) * 1e3
        return {"solves_per_s": len(d) / span, "span_s": span,
                "p50_time_to_solution_ms": float(np.percentile(tts, 50)),
                "p99_time_to_solution_ms": float(np.percentile(tts, 99)),
                "mean_sweeps": float(np.mean([v[1] for v in d.values()]))}
    served = summary(done, served_span)
    served.update({"failed": failed, "steps": steps, "peak_bytes": peak, "budget_bytes": budget})
    plain_s = summary(plain, plain_span)
    ok = [k for k in done if done[k][3] == spm.binding.SPM_JOB_DONE]
    dfit = np.array([abs(done[k][2] - plain[k][2]) for k in ok])
    line = {
        "workload": "serving", "metric": "CPD solves/s + p50/p99 time to solution",
        "unit": "solves/s", "value": served["solves_per_s"], "higher_is_better": True,
        "n_gpus": 1, "data": "synthetic",
        "config": {"requests": n, "rate_per_s": 200, "total_nnz": total_nnz,
                   "modes": "3 or 4", "ranks": "8/16/32/64", "tol": tol, "max_sweeps": cap,
                   "budget_GB": budget / 1e9, "served_factors": "bf16",
                   "plain_factors": "fp32"},
        "served_bf16_continuous_batching": served, "plain_fp32_per_tensor": plain_s,
        "speedup_solves_per_s": served["solves_per_s"] / plain_s["solves_per_s"],
        "fit_agreement": {"max_abs_dfit": float(dfit.max()) if dfit.size else None,
                          "within_1e-3": int((dfit <= 1e-3).sum()), "of": len(ok)},
        "clocks": clk}
    del reqs
    torch.cuda.empty_cache()
    return line


def run_precision(args, rank, world):
    """Precision workload: 4-mode 20,000 x 20,000 x 5,000 x 24 COO, 100M
    nonzeros (Zipf(1.0) x3 + uniform, lognormal values), R = 64, factors
    stored in FP32 or BF16 with FP32 accumulation; Gram/Cholesky in FP64.
    With --workload five the same measurement runs on the 5-mode preset
    (165,400 x 11,400 x 2 x 100 x 89, 26M nonzeros, R = 32).

    Reports per arm: spMTTKRP time and algorithmic GB/s per mode (inputs
    resident, larger than L2), the error of sampled output rows against the
    FP64 oracle (BF16: against the oracle on the same BF16-rounded factors --
    the accumulation error -- and on the FP32 factors -- the total error),
    and `sweeps` CP-ALS sweeps from the same initial factors (time per sweep,
    final fit, and the BF16 - FP32 fit difference)."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_2503_18198_gb300 as spm
    name_w = "five" if args.workload == "five" else "precision"
    dims, idx, vals, R, Y = synth.preset_torch(name_w, device="cuda")
    N = len(dims)
    nnz = int(vals.numel())
    distinct = distinct_counts(idx)
    idx_h = [c.cpu().numpy() for c in idx]
    vals_h = vals.cpu().numpy()
    Y_h = [y.cpu().numpy() for y in Y]
    Yb_h = [oracle.store_round(y, "bf16") for y in Y_h]
    rng = np.random.default_rng(7)
    rows = []
    for d in range(N):
        deg = np.bincount(idx_h[d], minlength=dims[d])
        heavy = np.argsort(-deg, kind="stable")[:4]
        nz = np.nonzero(deg)[0]
        rows.append(np.unique(np.concatenate([heavy, rng.choice(nz, min(96, nz.size), replace=False)]))
                    .astype(np.int32))
    ref32 = [oracle.mttkrp_rows(dims, idx_h, vals_h, Y_h, d, rows[d]) for d in range(N)]
    ref16 = [oracle.mttkrp_rows(dims, idx_h, vals_h, Yb_h, d, rows[d]) for d in range(N)]

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    peak, peak_kind = measured_peak()
    arms = {}
    fits = {}
    for name, flags, dtype, s_f in (("fp32", spm.SPM_FACTOR_FP32, torch.float32, 4),
                                    ("bf16", spm.SPM_FACTOR_BF16, torch.bfloat16, 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = spm.spmttkrp_plan(dims, idx, vals, R, flags)
        torch.cuda.synchronize()
        plan_ms = (time.perf_counter() - t0) * 1e3
        fac = [y.to(dtype).clone() for y in Y]  # never alias the preset factors
        kappa, kappa_ms = spm.spmttkrp_plan_autotune(plan, fac)  # 1 or 2 partitions per SM
        outs = [torch.empty(dims[d], R, device="cuda") for d in range(N)]
        B = algorithmic_bytes(dims, nnz, R, distinct, s_f)
        ms = []
        for d in range(N):
            for _ in range(3):
                spm.spmttkrp_run(plan, d, fac, outs[d])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(10):
                spm.spmttkrp_run(plan, d, fac, outs[d])
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1) / 10)
        err = {}
        for d in range(N):
            got = outs[d][torch.as_tensor(rows[d]).long().cuda()].double().cpu().numpy()
            if name == "fp32":
                err[f"mode{d}"] = rel(got, ref32[d])
            else:
                err[f"mode{d}"] = {"vs_oracle_same_bf16_factors": rel(got, ref16[d]),
                                   "vs_oracle_fp32_factors": rel(got, ref32[d])}
        lam = torch.zeros(R, dtype=torch.float64, device="cuda")
        fit = torch.zeros(1, dtype=torch.float64, device="cuda")
        fac = [y.to(dtype).clone() for y in Y]  # never alias the preset factors
        spm.cpd_als_step(plan, [f.clone() for f in fac], lam, fit)  # warm-up on a copy
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.sweeps):
            spm.cpd_als_step(plan, fac, lam, fit)
        e1.record(stream)
        torch.cuda.synchronize()
        als_ms = e0.elapsed_time(e1) / args.sweeps
        assert spm.spmttkrp_plan_status(plan) == 0
        fits[name] = float(fit.item())
        arms[name] = {
            "plan_ms": plan_ms, "plan_bytes": spm.spmttkrp_plan_bytes(plan),
            "kappa_autotuned": kappa, "kappa_candidates_ms_all_modes": [round(x, 4) for x in kappa_ms],
            "mttkrp_ms_per_mode": [round(m, 4) for m in ms],
            "mttkrp_GBs_per_mode": [round(b / (m * 1e-3) / 1e9, 1) for b, m in zip(B, ms)],
            "roofline_frac_per_mode": [round(b / (m * 1e-3) / 1e9 / peak, 4) for b, m in zip(B, ms)],
            "mttkrp_GBs_all_modes": sum(B) / (sum(ms) * 1e-3) / 1e9,
            "nnz_per_s_per_mode": [round(nnz / (m * 1e-3), 1) for m in ms],
            "algorithmic_bytes_per_mode": B,
            "sampled_row_rel_error": err,
            "als_ms_per_sweep": als_ms, "fit_after_sweeps": fits[name]}
        plan.destroy()
        del fac, outs
    clk = clocks.stop()
    # the FP64 oracle on the host cores: one MTTKRP pass over every mode on a
    # prefix sample, and that time scaled to all nonzeros (labelled as such)
    cpu = None
    if not args.no_cpu:
        cpu = cpu_baseline(dims, idx, vals, Y, R, min(args.cpu_seconds, 10.0))
        scale = nnz / cpu["sample_nnz"]
        cpu["extrapolated_to_all_nonzeros"] = {
            "mttkrp_all_modes_s_1_core": cpu["seconds_all_modes"] * scale,
            "mttkrp_all_modes_s_all_cores": (cpu["openmp_all_cores"].get("seconds_all_modes", 0.0)
                                             * scale) or None,
            "how": "sample time x (nnz / sample nonzeros): extrapolated, not measured"}
    line = {
        "workload": name_w, "metric": "spMTTKRP GB/s per mode, FP32 vs BF16 factors",
        "unit": "GB/s", "value": arms["bf16"]["mttkrp_GBs_all_modes"], "higher_is_better": True,
        "n_gpus": 1, "data": "synthetic",
        "config": {"dims": list(dims), "nnz": nnz, "rank": R, "sweeps": args.sweeps,
                   "coords": "Zipf(1.0) x3 + uniform" if name_w == "precision" else
                             "Zipf(1.1) x2 + uniform x3",
                   "values": "lognormal(0,1)" if name_w == "precision" else "U(0,1)",
                   "l2": "inputs larger than L2", "peak": peak, "peak_source": peak_kind,
                   "sampled_rows_per_mode": [int(r.size) for r in rows]},
        "arms": arms, "fit_bf16_minus_fp32": fits["bf16"] - fits["fp32"],
        "bf16_speedup_mttkrp": arms["fp32"]["mttkrp_GBs_all_modes"] and
            sum(arms["fp32"]["mttkrp_ms_per_mode"]) / sum(arms["bf16"]["mttkrp_ms_per_mode"]),
        "cpu_baseline": cpu,
        "clocks": clk}
    print(json.dumps(line), flush=True)


def host_copy_rates(h_in, h_out, stream):
    """This box's plain copy rates between pinned host memory and the device
    (one copy of the largest factor each way, after one untimed copy): the
    end-to-end figure depends on them.  None if the measurement fails."""
    import torch
    try:
        d_in = torch.empty_like(h_in, device="cuda")
        d_out = torch.empty_like(h_out, device="cuda")
        rates = {}
        for name, dst, src, n in (("h2d", d_in, h_in, h_in.numel() * 4),
                                  ("d2h", h_out, d_out, h_out.numel() * 4)):
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
            torch.cuda.synchronize()
            rates[name] = round(n / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1)
        del d_in, d_out
        return rates
    except Exception:  # a context report only: never fail the bench line for it
        return None


KERNEL_SOURCES = ("mttkrp_kernel.cuh", "mttkrp.cu", "mttkrp_inst.cuh", "common.cuh")


def kernel_digest():
    """sha256 over the MTTKRP kernel's sources (ties stored ncu counters to
    the code they were taken on)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2503_18198_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def plan_kappa(spm, plan):
    import torch
    off = torch.empty(65536 + 1, dtype=torch.int64, device="cuda")
    return spm.spmttkrp_plan_partition(plan, 0, off)


if __name__ == "__main__":
    main()
