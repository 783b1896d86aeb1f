"""Throughput of the fused CLB stream-and-collide sweep on GB300.

Workload: the L/H = 100 pressure-driven microchannel of Sec. 3.2 at
Ny = 256, Nx = 25601 (6,553,856 nodes), Kn_out = 0.1, p_in/p_out = 2.47,
populations stored as FP32 deviations (the headline) and, for comparison, in
FP64.  One step = one fused sweep over every node; the timed region also holds
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
SWEEP_SOURCES = ["paper_1603_01955_gb300/csrc/sweep.cu", "paper_1603_01955_gb300/csrc/clb_device.cuh",
                 "paper_1603_01955_gb300/csrc/clb_internal.h"]


def sweep_source_hash() -> str:
    h = hashlib.sha256()
    for p in SWEEP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[float, str]:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


def profiled_traffic(storage: str):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current sweep source (else None)."""
    path = os.path.join(ROOT, "profiles", f"sweep_{storage}_pressure_25601x256.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"sweep_source_sha256:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != sweep_source_hash():
        return None
    return float(m_tr.group(1))


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

    def max_over_ranks(v: float) -> float:
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    K, W = args.steps, args.warmup
    nodes = NX * NY
    sampler_id = gpu_id_for_smi(torch)
    results = {}
    clocks = None
    for storage in args.variants:
        ch = clb.Channel(NX, NY, KN_OUT, drive="pressure", drive_value=RATIO, storage=storage)
        info = ch.info()
        stream = ch.stream
        with torch.cuda.stream(stream):
            ch.step(W)
            ch.observables()
            ch.sync()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            sampler = ClockSampler(sampler_id)
            with sampler:
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
        t_total = max_over_ranks(t_total)
        results[storage] = dict(
            mlups=world * nodes * K / t_total / 1e6,
            ms_per_step=t_total / K * 1e3,
            sweep_us=t_sweeps / K * 1e6,
            bytes_per_node=info["bytes_per_node"],
            mass_flow=obs["mass_flow"],
            clocks=sampler.summary(),
        )
        if storage == "fp32s":
            clocks = results[storage]["clocks"]
        ch.close()

    # end to end through the C ABI with host buffers: upload the initial state
    # from pinned host memory, K sweeps, read the observables back
    ch = clb.Channel(NX, NY, KN_OUT, drive="pressure", drive_value=RATIO, storage="fp32s")
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
    t_e2e = max_over_ranks(t_e2e)
    ch.close()
    h2d = host_f.numel() * 8
    d2h = (2 * NY + 3 * NX) * 8 + 7 * 8

    if rank != 0:
        return None
    f32 = results["fp32s"]
    f64 = results.get("fp64")
    peak, peak_kind = measured_peaks()
    achieved = f32["bytes_per_node"] * nodes / (f32["sweep_us"] * 1e-6) / 1e9
    traffic = profiled_traffic("fp32s")
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
            "launch": {"vec": 4, "block_x": 128},
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
            "kernel": "sweep_kernel<float, pressure, 4>",
        },
        "variants": variants_block(f32, f64, nodes, peak),
        "e2e": {
            "value": round(world * nodes * K / t_e2e / 1e6, 1),
            "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / K,
            "d2h_bytes_per_step": d2h / K,
            "note": "per timed region: upload of the FP64 initial state from pinned host memory, K sweeps, "
                    "observables back to host; bytes per step = bytes per region / K",
        },
        "gpu_launches": K + 2,
        "clocks": clocks,
    }
    line["cpu_baseline"] = cpu_baseline(args.cpu_seconds) if not args.no_cpu_baseline else None
    return line


def variants_block(f32, f64, nodes, peak):
    out = {"fp32s": {"mlups": round(f32["mlups"], 1), "sweep_us": round(f32["sweep_us"], 3),
                     "mass_flow": f32["mass_flow"]}}
    if f64 is not None:
        out["fp64"] = {"mlups": round(f64["mlups"], 1), "sweep_us": round(f64["sweep_us"], 3),
                       "mass_flow": f64["mass_flow"],
                       "hbm_frac": round(f64["bytes_per_node"] * nodes / (f64["sweep_us"] * 1e-6) / 1e9 / peak, 4),
                       "clocks": f64["clocks"]}
        out["fp32s_over_fp64"] = round(f32["mlups"] / f64["mlups"], 3)
    return out


def oracle_sample_run(nx_sample: int, steps: int, threads: int = 0):
    import oracle

    p = oracle.OracleParams(nx=nx_sample, ny=NY, pressure=True, kn=KN_OUT, rho_in=RATIO, rho_out=1.0)
    s = oracle.OracleSim(p)
    t0 = time.perf_counter()
    s.step(steps, threads)
    dt = time.perf_counter() - t0
    return dt, oracle.threads_used()


def cpu_baseline(seconds: float = 15.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample:
    full-length steps of the benchmark channel, as many as fit ~`seconds`."""
    dt1, _ = oracle_sample_run(NX, 1)
    steps = max(1, int(seconds / max(dt1, 1e-6)))
    dt, cores = oracle_sample_run(NX, steps)
    return {"value": round(NX * NY * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} time steps of the full {NX}x{NY} channel from the initial state "
                      f"({dt:.1f} s, FP64, OpenMP over rows)"}


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
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="fp32s,fp64", help="storages to time (fp32s first)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    args.variants = [v for v in args.variants.split(",") if v]
    if not args.variants or args.variants[0] != "fp32s":
        ap.error("--variants must start with fp32s (the headline)")
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
