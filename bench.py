"""Benchmark of the GB300 P-RSoXS hot path (Algorithm 1).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload p1-1024|p1-512|p2-2048|p0-small] [--precision 32|64]

One step = one photon energy of Algorithm 1: the morphology of the workload
(c components, seeded synthetic, resident in HBM) through polarisation, FFT,
Ewald projection and the detector-rotation average over the e-field angles
0:2:180 (91 angles).  The metric is voxel-angle throughput, the voxel count
times angles times energies per second, summed over ranks.  Multi-GPU runs
shard energies across ranks (independent units, no collective): weak scaling.

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # Sec. 6.1 voxel scaling, largest case (1024^2 x 128, 4 materials, 0:2:180)
    "p1-1024": dict(shape=(128, 1024, 1024), c=4, angles=(0.0, 2.0, 180.0)),
    "p1-512": dict(shape=(64, 512, 512), c=4, angles=(0.0, 2.0, 180.0)),
    # Sec. 6.2 material scaling (2048^2 x 64)
    "p2-2048": dict(shape=(64, 2048, 2048), c=4, angles=(0.0, 2.0, 180.0)),
    "p0-small": dict(shape=(16, 128, 128), c=4, angles=(0.0, 2.0, 180.0)),
    # P1's lateral size with a shorter stack: the same kernel shapes in ~3 GB,
    # small enough for full ncu captures
    "p1-1024-z32": dict(shape=(32, 1024, 1024), c=4, angles=(0.0, 2.0, 180.0)),
}
VOXEL_NM = 5.0
METRIC = "P-RSoXS voxel-angle throughput (restated from 'filtered H*X GDoF-vec/s')"
UNIT = "Gvoxel-angle/s"


FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64, nominal (no measured FP64 peak is available)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2209_13121_gb300 import rsx, synth

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    __graft_entry__.build()

    W = WORKLOADS[args.workload]
    nz, ny, nx = W["shape"]
    c = W["c"]
    prec = args.precision
    real = 4 if prec == 32 else 8
    n_ang = rsx.angle_count(*W["angles"])
    n_steps = args.warmup + args.steps
    # 150 energies over 270..320 eV (Sec. 6.1), sharded across ranks with no
    # data-path collective; each step is one energy of this rank's shard.
    from paper_2209_13121_gb300.shard import energy_shard
    energies_all = synth.energies_uniform(150)
    shard = energy_shard(150, rank, ws, "strided")
    mine = [energies_all[shard[i % len(shard)]] for i in range(n_steps)]
    K = synth.optical_constants(mine, c, seed=2)
    M = synth.morphology_random_torch((nz, ny, nx), c, seed=1, device="cuda",
                                      dtype=torch.float32 if prec == 32 else torch.float64)
    ctx = rsx.Context(nx, ny, nz, c, VOXEL_NM, precision=prec, algorithm=args.algorithm)
    ctx.set_morphology(M)
    ctx.set_optical_constants(mine, K)
    out = torch.empty((1, ny, nx), device="cuda", dtype=M.dtype)
    stream = torch.cuda.current_stream()

    def step(i):
        ctx.run(W["angles"], energy_indices=[i], out=out)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ctx.phase_times()  # discard
    ctx.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.warmup, n_steps):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    phases = ctx.phase_times()
    ctx.set_timing(False)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    N = nx * ny * nz
    units = N * n_ang * args.steps * ws
    value = units / (ms / 1e3) / 1e9

    # roofline of the dominant kernel (polarisation + x-FFT), timed live
    top = max(phases, key=lambda k: phases[k][0])
    peak, peak_kind = _peaks()
    cplx = 2 * real
    # the library fuses the y-FFT with the q_z bins for FP32 grids with
    # ny = 1024, nx a multiple of 16 and nz a power of two up to 1024: the
    # y-transformed fields are then read once and never written
    fused = (prec == 32 and ny == 1024 and nx % 16 == 0 and nz <= 1024
             and nz & (nz - 1) == 0)
    nf = 5 if args.algorithm == 3 else 3
    y_bytes = nf * cplx if fused else 2 * nf * cplx
    z_bytes = 0 if fused else nf * cplx  # the bins kernel then reads per-pixel data only
    if args.algorithm == 3:
        # per energy: x-FFT of the 5 N_t entries (read + write); y-FFT (+ q_z bins)
        per_voxel = {"pol_fftx": 2 * 5 * cplx, "ffty": y_bytes, "ewald": z_bytes,
                     "rotate": 0, "other": 0, "nt": c * 4 * real + 5 * cplx}
    else:
        src_bytes = c * 4 * real if args.algorithm == 1 else 5 * cplx  # M, or N_t's 5 entries
        per_voxel = {"pol_fftx": src_bytes + 3 * cplx, "ffty": y_bytes, "ewald": z_bytes,
                     "rotate": 0, "other": 0, "nt": c * 4 * real + 5 * cplx}
    bytes_per_voxel = per_voxel[top]
    t_ms, n_l = phases[top]
    if args.algorithm == 3 and top == "ewald":
        # the ewald phase mixes one q_z reduction per energy with light per-angle kernels
        n_l = args.steps
    achieved = (bytes_per_voxel * N * n_l) / (t_ms / 1e3) / 1e9 if bytes_per_voxel else None
    if args.algorithm == 3:
        # per-energy FFT work dominates; report the x-FFT of the five N_t entries
        top = "pol_fftx"
        t_ms, n_l = phases[top]
        bytes_per_voxel = per_voxel[top]
        achieved = (bytes_per_voxel * N * n_l) / (t_ms / 1e3) / 1e9 if n_l else None
    traffic = _traffic_from_profiles(args.workload, top, prec) if args.algorithm == 1 else None
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "alg_bytes_per_voxel": bytes_per_voxel,
                "launch_ms": t_ms / n_l if n_l else None}
    if prec == 64 and args.algorithm == 1:
        # FP64 runs on the FP64 units (a small fraction of the FP32 rate on
        # GB300): the x pass is bound by FP64 arithmetic, reported against
        # the nominal FP64 rate.  Algorithmic flops per voxel: 41 per
        # component (Eq. (polarization) in the closed form, sincos not
        # counted), 22 for p, 100 for the x-FFT of three fields.
        t_ms, n_l = phases["pol_fftx"]
        flops = 41 * c + 22 + 100
        ach = flops * N * n_l / (t_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": "pol_fftx", "achieved": ach,
                    "peak": FP64_NOMINAL_TFLOPS, "peak_kind": "nominal FP64",
                    "unit": "TFLOP/s", "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": None,
                    "alg_flops_per_voxel": flops, "launch_ms": t_ms / n_l}

    # end to end through the public API: host morphology in, host image out.
    # Two contexts on two streams: the next energy's morphology upload
    # (page-locked, asynchronous) overlaps the current energy's run; every
    # step still uploads its full morphology and reads its image back.
    e2e = None
    if not args.no_e2e:
        Mh = torch.empty(M.shape, dtype=M.dtype, pin_memory=True)
        Mh.copy_(M)
        Mh_np = Mh.numpy()
        out_t = torch.empty((1, ny, nx), dtype=M.dtype, pin_memory=True)
        host_out = out_t.numpy()
        del M
        ctx.close()
        torch.cuda.empty_cache()
        ctxs = [rsx.Context(nx, ny, nz, c, VOXEL_NM, precision=prec, algorithm=args.algorithm)
                for _ in range(2)]
        for cx in ctxs:
            cx.set_optical_constants(mine, K)
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]

        def e2e_steps(first, last):
            ctxs[first % 2].set_morphology(Mh_np, stream=streams[first % 2], async_copy=True)
            for i in range(first, last):
                if i + 1 < last:
                    j = (i + 1) % 2
                    ctxs[j].set_morphology(Mh_np, stream=streams[j], async_copy=True)
                ctxs[i % 2].run(W["angles"], energy_indices=[i], out=host_out,
                                stream=streams[i % 2])

        e2e_steps(0, args.warmup)
        torch.cuda.synchronize()
        # host-to-device bandwidth of this machine for the same pinned buffer
        # (outside the timed region; the end-to-end number depends on it)
        dbuf = torch.empty(Mh.shape, dtype=Mh.dtype, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dbuf.copy_(Mh, non_blocking=True)
        e1.record()
        e1.synchronize()
        h2d_gbs = Mh_np.nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9
        del dbuf
        torch.cuda.empty_cache()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_steps(args.warmup, n_steps)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": units / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(Mh_np.nbytes), "d2h_bytes_per_step": int(host_out.nbytes),
               "h2d_gbs": round(h2d_gbs, 1)}
        for cx in ctxs:
            cx.close()
    else:
        ctx.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == 32 else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: Algorithm {args.algorithm}, {nx}x{ny}x{nz} voxels, "
                                   f"c={c}, 91 e-field angles 0:2:180 per energy, one energy "
                                   f"per step (of 150 over 270-320 eV)",
                       "voxels": N, "components": c, "angles_per_energy": n_ang,
                       "precision": prec, "parallelism": f"energy-sharded x{ws}",
                       "l2": f"inputs larger than L2 (morphology {N * c * 4 * real / 1e9:.1f} GB)"},
            "roofline": roofline,
            "phases_ms": {k: round(v[0], 3) for k, v in phases.items()},
            "gpu_launches": int(sum(v[1] for v in phases.values())),
            "clocks": clk,
            "e2e": e2e,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(W, args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _traffic_from_profiles(workload, kernel, prec):
    """DRAM bytes per launch of this kernel and workload recorded from an ncu
    capture in profiles/traffic.txt (None when there is none)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split("#")[0].split()
                if len(parts) == 2 and parts[0] == f"{workload}/{kernel}/f{prec}":
                    return float(parts[1])
    except OSError:
        pass
    return None


def cpu_baseline(W, args, angles_sample=10):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    128 x 128 x 16 voxels with the same c, one energy, the first
    `angles_sample` angles of 0:2:180.  Voxel-angle/s scales linearly in N
    (Sec. 6.1), so the sample's throughput stands for the workload's."""
    import numpy as np

    from oracle import cyrsoxs_oracle as O
    from paper_2209_13121_gb300 import synth

    shape = (16, 128, 128)
    c = W["c"]
    M = synth.morphology_random(shape, c, seed=1, dtype=np.float64)
    K = synth.optical_constants([285.0], c, seed=2)
    alphas = O.angle_list(*W["angles"])[:angles_sample]
    t0 = time.perf_counter()
    acc = np.zeros(shape[1:])
    for a in alphas:
        acc += O.rotate_image(O.scatter_one_angle(M, K[0], 285.0, VOXEL_NM, a), a)
    dt = time.perf_counter() - t0
    units = math.prod(shape) * len(alphas)
    return {"value": units / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy oracle, {shape[2]}x{shape[1]}x{shape[0]} voxels, c={c}, "
                      f"1 energy x {len(alphas)} of the 91 angles, {dt:.1f} s"}


def run_reference(args):
    """The oracle timed as the reference arm: each step one bounded sample
    (see cpu_baseline) of the workload, rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(W, args, angles_sample=2)
    t0 = time.perf_counter()
    samples = [cpu_baseline(W, args, angles_sample=4) for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    vals = [s["value"] for s in samples]
    value = statistics.mean(vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (oracle on a bounded sample per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": samples[0]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="p1-1024", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--algorithm", type=int, default=1, choices=[1, 2, 3],
                    help="1: Algorithm 1 (headline); 2: Algorithm 2 (N_t); 3: Algorithm 2 "
                         "restated by linearity (five FFTs per energy), reported beside")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
