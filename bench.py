"""Throughput of the fused CLB stream-and-collide sweep on GB300.

Workload: the L/H = 100 pressure-driven microchannel of Sec. 3.2 at
Ny = 256, Nx = 25601 (6,553,856 nodes), Kn_out = 0.1, p_in/p_out = 2.47,
populations stored as FP32 deviations (the headline) and, for comparison, in
FP64, FP16 (x 2^14) and BF16, each with the error of its mass flow and
pressure deviation against the FP64 oracle after the CPU-baseline steps.  One step = one fused sweep over every node; the timed region also holds
one FP64 observable reduction (mass flow, centreline pressure, profiles).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead.  With torchrun (N > 1) every rank runs its own
replica of the channel (the method does not shard across GPUs here) and the
value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX, NY, KN_OUT, RATIO = 25601, 256, 0.1, 2.47
METRIC = "D2Q9 CLB MLUPS and % HBM roofline, FP32-shifted vs FP64 at stated error"
WORKLOAD = "pressure-driven microchannel L/H=100, Ny=256 x Nx=25601 (6.55M nodes), Kn_out=0.1, p_in/p_out=2.47"
# sources of each sweep engine: a committed ncu summary is used only while the
# hash of its engine's sources is the one it records
DIRECT_SOURCES = ["paper_1603_01955_gb300/csrc/sweep.cu", "paper_1603_01955_gb300/csrc/clb_device.cuh",
                  "paper_1603_01955_gb300/csrc/clb_internal.h"]
TMA_SOURCES = DIRECT_SOURCES + ["paper_1603_01955_gb300/csrc/sweep_tma.cu",
                                "paper_1603_01955_gb300/csrc/tma_common.cuh"]


def sweep_source_hash(pipeline: int = 2) -> str:
    h = hashlib.sha256()
    for p in (DIRECT_SOURCES if pipeline <= 1 else TMA_SOURCES):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


def profiled_value(storage: str, pipeline: int, key: str):
    """A figure (`key: value` line) from the committed ncu summary of that
    engine, if it was taken on the current sweep sources (else None)."""
    kernel = "sweep" if pipeline <= 1 else "sweep_tma"
    path = os.path.join(ROOT, "profiles", f"{kernel}_{storage}_pressure_25601x256.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"sweep_source_sha256:\s*([0-9a-f]+)", text)
    m_val = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_hash or not m_val or m_hash.group(1) != sweep_source_hash(pipeline):
        return None
    return float(m_val.group(1))


def profiled_traffic(storage: str, pipeline: int):
    """DRAM bytes per sweep launch (ncu summary), or None."""
    return profiled_value(storage, pipeline, "traffic_bytes_per_launch")


def flops_block(clb, results, nodes):
    """Measured arithmetic rate of each timed sweep: floating-point operations
    per node update from the SASS counters in the committed ncu summary (None
    where no summary of that kernel on the current sources exists) times the
    sweeps' own node rate (nodes / sweep_us, the timed region of hbm_frac),
    against the fused multiply-add rate clb_peak_fma measures in the sweep's
    compute precision (FP64 for FP64 storage, FP32 otherwise)."""
    peaks = {"f32": clb.clb_peak_fma(clb.CLB_FP32_SHIFTED), "f64": clb.clb_peak_fma(clb.CLB_FP64)}
    out = {"peak_tflops": {k: round(v, 3) for k, v in peaks.items()}, "peak_kind": "measured (clb_peak_fma)"}
    for storage, r in results.items():
        ops = profiled_value(storage, r["pipeline"], "fp_ops_per_node")
        prec = "f64" if storage == "fp64" else "f32"
        entry = {"precision": prec, "fp_ops_per_node": ops}
        if ops is not None:
            tf = ops * nodes / (r["sweep_us"] * 1e-6) / 1e12
            entry.update(achieved_tflops=round(tf, 3), frac=round(tf / peaks[prec], 4))
        out[storage] = entry
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self._t:
                self._t.join(timeout=2)

    def summary(self):
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def gpu_id_for_smi(torch) -> str:
    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = getattr(props, "pci_bus_id", None)
        if bus is not None:
            dom = getattr(props, "pci_domain_id", 0)
            dev = getattr(props, "pci_device_id", 0)
            return f"{dom:08x}:{bus:02x}:{dev:02x}.0"
    except Exception:  # noqa: BLE001
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    first = vis.split(",")[0].strip() if vis else ""
    return first if first.isdigit() else str(torch.cuda.current_device())


def max_over_ranks(v: float, world: int, device: str) -> float:
    """Slowest rank's time (the contract's max over ranks)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(nodes: int, steps: int, t_max: float, world: int) -> float:
    """Whole-job throughput of independent replicas: every rank updates
    `nodes` nodes `steps` times; the job takes the slowest rank's time."""
    return world * nodes * steps / t_max / 1e6


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1603_01955_gb300 import clb

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()


    K, W = args.steps, args.warmup
    nodes = NX * NY
    sampler_id = gpu_id_for_smi(torch)
    results = {}
    clocks = None
    for storage in args.variants:
        ch = clb.Channel(NX, NY, KN_OUT, drive="pressure", drive_value=RATIO, storage=storage,
                         pipeline=args.pipeline)
        info = ch.info()
        stream = ch.stream
        with torch.cuda.stream(stream):
            ch.observables()  # first call: the reduction's buffers and the residual history
            ch.sync()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            # the clock sampler starts first (it waits for nvidia-smi), so that the
            # W warm-up steps run directly before the timed region: an idle GPU
            # takes about 1 us per sweep longer over a short region
            sampler = ClockSampler(sampler_id)
            with sampler:
                ch.step(W)
                barrier()
                torch.cuda.synchronize()
                e0.record(stream)
                ch.step(K)
                e1.record(stream)
                obs = ch.observables()
                e2.record(stream)
                torch.cuda.synchronize()
                barrier()
        t_total = e0.elapsed_time(e2) / 1e3
        t_sweeps = e0.elapsed_time(e1) / 1e3
        t_obs = e1.elapsed_time(e2) / 1e3
        t_total = max_over_ranks(t_total, world, "cuda")
        results[storage] = dict(
            pipeline=info["pipeline"],
            mlups=replica_mlups(nodes, K, t_total, world),
            ms_per_step=t_total / K * 1e3,
            sweep_us=t_sweeps / K * 1e6,
            observables_us=t_obs * 1e6,
            bytes_per_node=info["bytes_per_node"],
            mass_flow=obs["mass_flow"],
            clocks=sampler.summary(),
        )
        if storage == "fp32s":
            clocks = results[storage]["clocks"]
        ch.close()

    # end to end through the C ABI with host buffers: upload the initial state
    # from pinned host memory, K sweeps, read the observables back
    ch = clb.Channel(NX, NY, KN_OUT, drive="pressure", drive_value=RATIO, storage="fp32s", pipeline=args.pipeline)
    host_f = torch.empty((9, NY, NX), dtype=torch.float64, pin_memory=True)
    host_f.numpy()[...] = ch.state()
    import numpy as np

    prof = {k: np.zeros(NY) for k in ("ux", "uy")}
    cols = {k: np.zeros(NX) for k in ("pc", "dp", "m")}
    s = clb.clb_scalars()
    with torch.cuda.stream(ch.stream):
        clb.clb_set_state(ch.sim, host_f.data_ptr())
        ch.step(W)
        ch.sync()
        barrier()
        t0 = time.perf_counter()
        clb.clb_set_state(ch.sim, host_f.data_ptr())
        clb.clb_step(ch.sim, K)
        clb.clb_observables(ch.sim, -1, s, prof["ux"], prof["uy"], cols["pc"], cols["dp"], cols["m"])
        t_e2e = time.perf_counter() - t0
        barrier()
    t_e2e = max_over_ranks(t_e2e, world, "cuda")
    ch.close()
    h2d = host_f.numel() * 8
    d2h = (2 * NY + 3 * NX) * 8 + 7 * 8

    if rank != 0:
        return None
    f32 = results["fp32s"]
    peak, peak_kind = measured_peaks()
    achieved = f32["bytes_per_node"] * nodes / (f32["sweep_us"] * 1e-6) / 1e9
    traffic = profiled_traffic("fp32s", f32["pipeline"])
    line = {
        "metric": METRIC,
        "value": round(f32["mlups"], 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(f32["ms_per_step"], 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "nx": NX, "ny": NY, "kn_out": KN_OUT, "pressure_ratio": RATIO,
            "storage": "fp32s (deviations from w_i*rho_ref(x)), FP32 collide",
            "step": "one fused stream-collide sweep per step; one FP64 observable reduction per timed region",
            "l2": "no flush: each population buffer is 236 MB (FP32) / 472 MB (FP64), above the 129 MB L2",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "launch": engine_of(f32["pipeline"]),
        },
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": traffic,
            "peak_kind": peak_kind,
            "bytes_per_node": f32["bytes_per_node"],
            "kernel": engine_of(f32["pipeline"])["kernel"],
        },
        "variants": variants_block(results, nodes, peak),
        "flops": flops_block(clb, results, nodes),
        "e2e": {
            "value": round(replica_mlups(nodes, K, t_e2e, world), 1),
            "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": d2h / K,
            "note": "per timed region: upload of the FP64 initial state from pinned host memory, K sweeps, "
                    "observables back to host; bytes per step = bytes per region / K",
        },
        "gpu_launches": K + 1,  # K sweeps and one observable reduction
        "clocks": clocks,
    }
    if not args.no_batch:
        line["knudsen_sweep"] = knudsen_sweep_bench(clb, torch, args.batch_steps)
        line["small_channel"] = small_channel_bench(clb, torch, args.batch_steps)
        line["adjoint"] = adjoint_bench(clb, torch)
    if args.no_cpu_baseline or world > 1:
        line["cpu_baseline"] = None
    else:
        base, ref = cpu_baseline(args.cpu_steps, args.error_steps)
        line["cpu_baseline"] = base
        line["errors_vs_oracle"] = errors_vs_oracle(clb, args.variants, ref, args.error_steps)
    return line


def adjoint_bench(clb, torch):
    """The adjoint calibration workload of Sec. 3.1: periodic channel nx = 4,
    ny = 64, Kn = 0.1, G = 1e-6, 20,000 FP32 steps with a checkpoint every 141
    steps.  Wall time of the checkpointed forward pass and of one backward
    pass (which recomputes every segment), per step, for the default engine
    (the grid fits in shared memory: one block per pass) and for one launch
    per step; and the device memory of the states they keep: ceil(N/C)
    checkpoints + C + 1 segment states + 4 adjoint fields, each 9 nx ny FP32
    values."""
    import math

    nx, ny, kn, g, n, every = 4, 64, 0.1, 1e-6, 20000, 141
    out = {"workload": "periodic 4 x 64, Kn 0.1, G 1e-6, 20000 fp32 steps, checkpoint every 141"}
    for name, pipeline in (("resident", 0), ("launch_per_step", 1)):
        fg = clb.FlowGradient(nx, ny, kn, 2.0, -1.0, g, 1000, storage="fp32s", checkpoint_every=32,
                              pipeline=pipeline)  # warm-up
        fg.q_grad()
        fg.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fg = clb.FlowGradient(nx, ny, kn, 2.0, -1.0, g, n, storage="fp32s", checkpoint_every=every,
                              pipeline=pipeline)
        t1 = time.perf_counter()
        grad = fg.q_grad()
        t2 = time.perf_counter()
        q = fg.q_norm
        fg.close()
        out[name] = {"forward_ms": round((t1 - t0) * 1e3, 2), "forward_us_per_step": round((t1 - t0) / n * 1e6, 3),
                     "backward_ms": round((t2 - t1) * 1e3, 2),
                     "backward_us_per_step": round((t2 - t1) / n * 1e6, 3), "q_norm": q, "dq_d_r_a_g": grad}
    states = math.ceil(n / every) + every + 1 + 4
    out.update(state_bytes=states * 9 * nx * ny * 4, states_kept=states)
    return out


def knudsen_sweep_bench(clb, torch, steps):
    """The batched Knudsen sweep of Sec. 3.1 (48 periodic channels, Kn
    log-spaced over 0.01..10, ny cycling 16/32/64/128, nx = 4, G = 1e-6,
    FP32-shifted): aggregate MLUPS of the persistent, graph-replayed launch
    against one ordinary sweep launch per channel per step."""
    n = 48
    kn = [10 ** (-2 + 3 * k / (n - 1)) for k in range(n)]
    ny = [(16, 32, 64, 128)[k % 4] for k in range(n)]
    nx = [4] * n
    nodes = sum(a * b for a, b in zip(nx, ny))
    b = clb.Batch(nx, ny, kn, g=1e-6, storage="fp32s")
    b.step(1000)  # autotunes, then warms up
    b.stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    q = [o["q_norm"] for o in b.observables()]
    block = b.info()["block_x"]
    schedule = b.schedule()
    b.close()
    stream = torch.cuda.Stream()
    chans = [clb.Channel(nx[k], ny[k], kn[k], drive="body_force", drive_value=1e-6, storage="fp32s",
                         stream=stream) for k in range(n)]
    rounds = max(50, steps // 40)
    for c in chans:
        c.step(20)
    stream.synchronize()
    e0.record(stream)
    for _ in range(rounds):
        for c in chans:
            c.step(1)
    e1.record(stream)
    e1.synchronize()
    t_sep = e0.elapsed_time(e1) / 1e3
    for c in chans:
        c.close()
    i = min(range(n), key=lambda k: q[k])
    return {
        "workload": "48 periodic channels, Kn = 10^(-2+3k/47), ny cycling 16/32/64/128, nx = 4, G = 1e-6, fp32s",
        "nodes": nodes,
        "mlups_persistent": round(nodes * steps / t_batch / 1e6, 1),
        "us_per_step_persistent": round(t_batch / steps * 1e6, 3),
        "mlups_separate_launches": round(nodes * rounds / t_sep / 1e6, 1),
        "us_per_step_separate_launches": round(t_sep / rounds * 1e6, 3),
        "speedup": round((nodes * steps / t_batch) / (nodes * rounds / t_sep), 2),
        "block_x_tuned": block,
        "schedule_tuned": schedule,
        "steps": steps,
        "q_min_kn_after_steps": kn[i],
    }


def small_channel_bench(clb, torch, steps):
    """The 1601 x 16 pressure channel of Sec. 3.2 (L/H = 100, Kn_out = 0.1,
    ratio 2, FP32-shifted): each sweep takes a few microseconds, so launch
    overhead bounds it; MLUPS with the sweeps replayed from CUDA graphs in
    chunks of 64 and with one launch per step."""
    c = {"nx": 1601, "ny": 16, "kn_out": 0.1, "ratio": 2.0}
    nodes = c["nx"] * c["ny"]
    out = {"workload": "pressure channel 1601 x 16 (25,616 nodes), Kn_out 0.1, p_in/p_out 2, fp32s",
           "nodes": nodes, "steps": steps}
    for name, graph_steps in (("graphs", 64), ("launches", -1)):
        ch = clb.Channel(c["nx"], c["ny"], c["kn_out"], drive="pressure", drive_value=c["ratio"], storage="fp32s",
                         graph_steps=graph_steps)
        ch.step(256)
        ch.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ch.stream)
        ch.step(steps)
        e1.record(ch.stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        ch.sync()
        ch.close()
        out[f"mlups_{name}"] = round(nodes * steps / t / 1e6, 1)
        out[f"us_per_step_{name}"] = round(t / steps * 1e6, 3)
    out["speedup"] = round(out["mlups_graphs"] / out["mlups_launches"], 2)
    return out


def errors_vs_oracle(clb, variants, ref, steps):
    """Each storage variant after `steps` steps from the initial state, against
    the FP64 oracle run of the CPU-baseline leg continued to the same step."""
    import numpy as np

    out = {"steps": steps}
    x = np.arange(NX)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    dev = np.abs(ref["state"] - w * (RATIO + (1.0 - RATIO) * x / (NX - 1))[None, None, :]).max()
    for storage in variants:
        ch = clb.Channel(NX, NY, KN_OUT, drive="pressure", drive_value=RATIO, storage=storage)
        ch.step(steps)
        o = ch.observables()
        f = ch.state()
        ch.close()
        out[storage] = {
            "mass_flow_rel": abs(o["mass_flow"] - ref["mass_flow"]) / abs(ref["mass_flow"]),
            "dp_nonlin_abs_max": float(np.abs(o["dp_nonlin"] - ref["dp_nonlin"]).max()),
            "population_abs_max_over_max_deviation": float(np.abs(f - ref["state"]).max() / dev),
        }
        del f
    return out


# tile shapes of the TMA-staged sweep, pipelines 2 to 4: (consumer threads, nodes per thread, stages)
TMA_SHAPES = [(512, 2, 3), (128, 4, 2), (256, 4, 3)]


def engine_of(pipeline: int) -> dict:
    if pipeline <= 1:
        return {"pipeline": pipeline, "engine": "direct vector loads + warp shuffles", "vec": 4, "block_x": 128,
                "kernel": "sweep_kernel<float, pressure, 4>"}
    nc, v, st = TMA_SHAPES[pipeline - 2]
    return {"pipeline": pipeline, "engine": "TMA bulk copies into a shared-memory ring",
            "consumers": nc, "nodes_per_thread": v, "stages": st,
            "kernel": f"sweep_tma_kernel<float, pressure, {nc}, {v}, {st}>"}


def variants_block(results, nodes, peak):
    """Per storage: `mlups` over the whole timed region (K sweeps and one
    observable reduction read back to the host), `mlups_sweeps` over the
    sweeps alone (the timed region of `sweep_us` and `hbm_frac`), and the
    observable reduction's own time."""
    out = {}
    for storage, r in results.items():
        out[storage] = {"mlups": round(r["mlups"], 1), "mlups_sweeps": round(nodes / r["sweep_us"], 1),
                        "sweep_us": round(r["sweep_us"], 3), "observables_us": round(r["observables_us"], 1),
                        "pipeline": r["pipeline"],
                        "bytes_per_node": r["bytes_per_node"],
                        "hbm_frac": round(r["bytes_per_node"] * nodes / (r["sweep_us"] * 1e-6) / 1e9 / peak, 4),
                        "mass_flow": r["mass_flow"], "clocks": r["clocks"]}
    if "fp64" in results:
        out["fp32s_over_fp64"] = round(results["fp32s"]["mlups"] / results["fp64"]["mlups"], 3)
    return out


def oracle_sample_run(nx_sample: int, steps: int, threads: int = 0):
    import oracle

    p = oracle.OracleParams(nx=nx_sample, ny=NY, pressure=True, kn=KN_OUT, rho_in=RATIO, rho_out=1.0)
    s = oracle.OracleSim(p)
    t0 = time.perf_counter()
    s.step(steps, threads)
    dt = time.perf_counter() - t0
    return dt, oracle.threads_used()


def cpu_baseline(steps: int, error_steps: int):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample:
    `steps` time steps of the full benchmark channel (timed), continued
    untimed to `error_steps` for the error report, whose oracle state and
    observables are returned too.  Sub-entries time the same oracle on one
    core (a few steps of the same channel) and on the 1601 x 16 channel of
    Sec. 3.2 (all cores and one core)."""
    import oracle

    p = oracle.OracleParams(nx=NX, ny=NY, pressure=True, kn=KN_OUT, rho_in=RATIO, rho_out=1.0)
    s = oracle.OracleSim(p)
    t0 = time.perf_counter()
    s.step(steps, 0)
    dt = time.perf_counter() - t0
    cores = oracle.threads_used()
    if error_steps > steps:
        s.step(error_steps - steps, 0)
    obs = s.observables()
    ref = {"state": s.state(), "mass_flow": obs["mass_flow"], "dp_nonlin": obs["dp_nonlin"]}
    s.close()
    base = {"value": round(NX * NY * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} time steps of the full {NX}x{NY} channel from the initial state "
                      f"({dt:.1f} s, FP64, OpenMP over rows)"}
    subs = {}
    for name, nx, ny, n, threads in (("25601x256_one_core", NX, NY, 4, 1), ("1601x16_all_cores", 1601, 16, 2000, 0),
                                     ("1601x16_one_core", 1601, 16, 1000, 1)):
        q = oracle.OracleParams(nx=nx, ny=ny, pressure=True, kn=KN_OUT, rho_in=RATIO if ny == NY else 2.0,
                                rho_out=1.0)
        o = oracle.OracleSim(q)
        t0 = time.perf_counter()
        o.step(n, threads)
        t = time.perf_counter() - t0
        subs[name] = {"value": round(nx * ny * n / t / 1e6, 3), "unit": "MLUPS", "cores": oracle.threads_used(),
                      "sample": f"{n} steps of the {nx}x{ny} pressure channel ({t:.1f} s)"}
        o.close()
    base["more"] = subs
    return base, ref


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return None
    K, W = args.steps, args.warmup
    # size one reference step so that the whole run stays within ~2 minutes
    dt1, _ = oracle_sample_run(NX, 1)
    per_node = dt1 / (NX * NY)
    budget = 120.0 / max(K + W, 1)
    nx_s = int(max(4, min(NX, budget / (per_node * NY))))
    import oracle

    p = oracle.OracleParams(nx=nx_s, ny=NY, pressure=True, kn=KN_OUT, rho_in=RATIO, rho_out=1.0)
    s = oracle.OracleSim(p)
    s.step(W)
    t0 = time.perf_counter()
    s.step(K)
    dt = time.perf_counter() - t0
    cores = oracle.threads_used()
    mlups = nx_s * NY * K / dt / 1e6
    sample = (f"each step: one FP64 oracle time step of a {nx_s}x{NY} slice of the benchmark channel "
              f"(same cross-section, Kn_out and pressure ratio)")
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": round(mlups, 3),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(dt / K * 1e3, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "kn_out": KN_OUT, "pressure_ratio": RATIO},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-steps", type=int, default=200, help="timed oracle steps of the CPU baseline")
    ap.add_argument("--error-steps", type=int, default=1000,
                    help="steps after which every storage is compared with the oracle (>= --cpu-steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="fp32s,fp64,fp16s,bf16s", help="storages to time (fp32s first)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the launch-bound measurements (batched Knudsen sweep, 1601x16 channel)")
    ap.add_argument("--batch-steps", type=int, default=20000)
    ap.add_argument("--pipeline", type=int, default=0,
                    help="sweep engine for FP32/16-bit storage (clb_opts.pipeline; 0 = library default)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    args.error_steps = max(args.error_steps, args.cpu_steps)
    args.variants = [v for v in args.variants.split(",") if v]
    if not args.variants or args.variants[0] != "fp32s":
        ap.error("--variants must start with fp32s (the headline)")
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
