"""Benchmark of the GB300 P-RSoXS hot path (Algorithm 1).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--precision 32|64] [--algorithm 1|2|3]
                    [--components C] [--angle-batch K]
    python bench.py --cpu-report      # the oracle on this host, single and all cores

One step = one photon energy of Algorithm 1: the morphology of the workload
(c components, seeded synthetic, resident in HBM) through polarisation, FFT,
Ewald projection and the detector-rotation average over the e-field angles
0:2:180 (91 angles).  The metric is voxel-angle throughput, the voxel count
times angles times energies per second, summed over ranks.  Multi-GPU runs
shard energies across ranks (independent units, no collective): weak scaling.
With --gpus N > 1 and no torchrun environment, the script starts N ranks of
itself under torch.distributed.run (127.0.0.1 rendezvous).

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

# energies: (count, lo, hi) eV, uniform; one energy per step
WORKLOADS = {
    # Sec. 6.1 voxel scaling, largest case (1024^2 x 128, 4 materials, 0:2:180)
    "p1-1024": dict(shape=(128, 1024, 1024), c=4, angles=(0.0, 2.0, 180.0),
                    energies=(150, 270.0, 320.0)),
    "p1-512": dict(shape=(64, 512, 512), c=4, angles=(0.0, 2.0, 180.0),
                   energies=(150, 270.0, 320.0)),
    # Sec. 6.2 material scaling (2048^2 x 64, 9 energies; c swept 2..10 with
    # --components)
    "p2-2048": dict(shape=(64, 2048, 2048), c=4, angles=(0.0, 2.0, 180.0),
                    energies=(9, 270.0, 320.0)),
    # Sec. 5.1 sphere cases: the 2-D film (41 energies 270-310 eV, FP64
    # against FP32) and the 3-D stack at one energy
    "p3-2048-film": dict(shape=(1, 2048, 2048), c=2, angles=(0.0, 2.0, 180.0),
                         energies=(41, 270.0, 310.0)),
    "p4-2048": dict(shape=(128, 2048, 2048), c=2, angles=(0.0, 2.0, 180.0),
                    energies=(1, 285.0, 285.0)),
    "p0-small": dict(shape=(16, 128, 128), c=4, angles=(0.0, 2.0, 180.0),
                     energies=(150, 270.0, 320.0)),
    # P1's lateral size with a shorter stack: the same kernel shapes in ~3 GB,
    # small enough for full ncu captures
    "p1-1024-z32": dict(shape=(32, 1024, 1024), c=4, angles=(0.0, 2.0, 180.0),
                        energies=(150, 270.0, 320.0)),
    "p1-1024-z16": dict(shape=(16, 1024, 1024), c=4, angles=(0.0, 2.0, 180.0),
                        energies=(150, 270.0, 320.0)),
    # P1's stack depth (128 slices) on smaller lateral grids, for captures of
    # the z-first kernels at their P1 instantiation in a few GB: the
    # polarisation + z-FFT pass (any lateral size) and the 1024-row
    # selection pass
    "p1-512-z128": dict(shape=(128, 512, 512), c=4, angles=(0.0, 2.0, 180.0),
                        energies=(150, 270.0, 320.0)),
    "p1-1024x512-z128": dict(shape=(128, 1024, 512), c=2, angles=(0.0, 2.0, 180.0),
                             energies=(150, 270.0, 320.0)),
    # Sec. 5.2.2 grating geometry (E5): 1 nm voxels, 17 keV, the e-field at 0
    # only (no rotation), FP64 in the paper's comparison (--precision 64)
    "p5-1024x63": dict(shape=(63, 1024, 1024), c=2, angles=(0.0, 1.0, 0.0),
                       energies=(1, 17000.0, 17000.0), voxel_nm=1.0),
    "p5-1024x1": dict(shape=(1, 1024, 1024), c=2, angles=(0.0, 1.0, 0.0),
                      energies=(1, 17000.0, 17000.0), voxel_nm=1.0),
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


def gpu_local_cpus(index):
    """Host CPUs nearest to GPU `index` (the "CPU Affinity" column of
    nvidia-smi topo -m), or None when it cannot be read."""
    try:
        out = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True,
                             timeout=20).stdout
    except Exception:
        return None
    lines = [ln.rstrip() for ln in out.splitlines() if ln.strip()]
    header = next((ln for ln in lines if "CPU Affinity" in ln), None)
    row = next((ln for ln in lines if ln.split() and ln.split()[0] == f"GPU{index}"), None)
    if not header or not row:
        return None
    # columns are tab-separated; the header's first cell is empty
    hcols = [c.strip() for c in header.split("\t")]
    rcols = [c.strip() for c in row.split("\t")]
    try:
        spec = rcols[hcols.index("CPU Affinity")]
    except (ValueError, IndexError):
        return None
    cpus = set()
    for part in spec.split(","):
        part = part.strip()
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part.isdigit():
            cpus.add(int(part))
    return cpus or None


def pinned_near_gpu(shape, dtype, index):
    """A page-locked host tensor whose pages come from the memory nearest to
    GPU `index`: the allocation and first touch run with this process bound
    to the GPU's local CPUs (the default local-allocation policy then places
    the pages there), so host-to-device copies do not cross sockets.
    Returns (tensor, whether the binding applied)."""
    import torch
    cpus = gpu_local_cpus(index)
    old = None
    if cpus:
        try:
            old = os.sched_getaffinity(0)
            os.sched_setaffinity(0, cpus & set(range(os.cpu_count() or 1)) or old)
        except Exception:
            old = None
    try:
        t = torch.empty(shape, dtype=dtype, pin_memory=True)
        t.zero_()
    finally:
        if old is not None:
            os.sched_setaffinity(0, old)
    return t, old is not None


def _free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(n, argv):
    """Runs this script as n ranks under torch.distributed.run on this node
    (rendezvous on 127.0.0.1) and returns its exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={n}", "--master-addr=127.0.0.1", f"--master-port={_free_port()}",
           os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


class _Ranks:
    """The control plane of a multi-rank run: barrier and max over ranks.
    NCCL when every rank has its own GPU; gloo (CPU tensors) when ranks
    share a device or there is none (a functional check of the launch)."""

    def __init__(self, ws, backend):
        import torch.distributed as dist
        self.ws, self.backend, self.dist = ws, backend, dist
        if ws > 1:
            dist.init_process_group(backend)

    def barrier(self):
        if self.ws > 1:
            self.dist.barrier()

    def max(self, x):
        if self.ws == 1:
            return x
        import torch
        t = torch.tensor([float(x)], device="cuda" if self.backend == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.ws > 1:
            self.dist.destroy_process_group()


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2209_13121_gb300 import rsx, synth

    ws, rank, local = _dist()
    ndev = torch.cuda.device_count()
    dev = local % ndev
    ranks = _Ranks(ws, "nccl" if ws <= ndev else "gloo")
    torch.cuda.set_device(dev)
    if rank == 0:
        __graft_entry__.build()
    ranks.barrier()
    __graft_entry__.build()

    W = WORKLOADS[args.workload]
    nz, ny, nx = W["shape"]
    c = args.components or W["c"]
    prec = args.precision
    real = 4 if prec == 32 else 8
    n_ang = rsx.angle_count(*W["angles"])
    n_steps = args.warmup + args.steps
    # the workload's energies (Sec. 6.1: 150 over 270..320 eV), sharded
    # across ranks with no data-path collective; each step is one energy of
    # this rank's shard (repeated when the shard is shorter than the run).
    from paper_2209_13121_gb300.shard import energy_shard
    n_e, e_lo, e_hi = W["energies"]
    energies_all = synth.energies_uniform(n_e, e_lo, e_hi)
    shard = energy_shard(n_e, rank, ws, "strided")
    if len(shard) == 0:
        shard = [rank % n_e]
    mine = [energies_all[shard[i % len(shard)]] for i in range(n_steps)]
    K = synth.optical_constants(mine, c, seed=2)
    M = synth.morphology_random_torch((nz, ny, nx), c, seed=1, device="cuda",
                                      dtype=torch.float32 if prec == 32 else torch.float64)
    voxel_nm = W.get("voxel_nm", VOXEL_NM)
    ctx = rsx.Context(nx, ny, nz, c, voxel_nm, precision=prec, algorithm=args.algorithm,
                      angle_batch=args.angle_batch)
    angle_batch = ctx.angle_batch
    ctx.set_morphology(M)
    ctx.set_optical_constants(mine, K)
    zplan = [ctx.zfirst_plan(i) for i in range(n_steps)]
    out = torch.empty((1, ny, nx), device="cuda", dtype=M.dtype)
    stream = torch.cuda.current_stream()

    def step(i):
        ctx.run(W["angles"], energy_indices=[i], out=out)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ctx.phase_times()  # discard
    ctx.set_timing(True)
    clocks = ClockSampler(dev)
    clocks.start()
    ranks.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.warmup, n_steps):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    # the timed runs wrote device output asynchronously: a pipelined kernel
    # that ran out of a bounded wait would make them invalid (raises)
    ctx.check()
    ranks.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    phases = ctx.phase_times()
    ctx.set_timing(False)
    ms = ranks.max(ms)

    N = nx * ny * nz
    units = N * n_ang * args.steps * ws
    value = units / (ms / 1e3) / 1e9

    # roofline of the dominant kernel (polarisation + x-FFT), timed live
    top = max(phases, key=lambda k: phases[k][0])
    peak, peak_kind = _peaks()
    cplx = 2 * real
    # the library fuses the y-FFT with the q_z bins for FP32 grids with
    # ny = 512, 1024 or 2048, nx a power of two >= 16 and nz a power of two up
    # to 1024 (at least 4 for 2048 rows): the y-transformed fields are then
    # read once and never written
    fused = (prec == 32 and ny in (512, 1024, 2048) and nx >= 16 and nx & (nx - 1) == 0
             and nz <= 1024 and nz & (nz - 1) == 0 and (ny != 2048 or nz >= 4))
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
    kx = angle_batch if args.algorithm == 1 else 1
    if kx > 1:
        # the x pass reads the morphology once per batch of kx angles and
        # writes every angle's p: per launch, on average over the energy's
        # ceil(n_ang / kx) launches
        n_x = -(-n_ang // kx)
        per_voxel["pol_fftx"] = (src_bytes * n_x + 3 * cplx * n_ang) / n_x
    # the z-first path (rsx_zfirst_plan): per energy, ns q_z planes of the
    # nz slices are kept and kz angles share one read of the morphology.
    # Per launch: the polarisation + z-FFT pass reads M and writes kz x 3 x ns
    # planes; the x-FFT reads and writes them; the y-FFT + bin selection pass
    # reads one angle's 3 x ns planes (bins per pixel not counted)
    zplans = [zplan[i] for i in range(args.warmup, n_steps)]
    zfirst = args.algorithm == 1 and all(z[0] > 0 for z in zplans)
    if zfirst:
        npix = nx * ny
        tot = {"pol_fftx": 0.0, "fftx": 0.0, "ffty": 0.0}
        for ns_i, _, kz_i in zplans:
            n_pass = -(-n_ang // kz_i)
            tot["pol_fftx"] += n_pass * src_bytes * N + n_ang * 3 * ns_i * npix * cplx
            tot["fftx"] += n_ang * 2 * 3 * ns_i * npix * cplx
            tot["ffty"] += n_ang * 3 * ns_i * npix * cplx
        for k in tot:
            launches = phases[k][1]
            per_voxel[k] = tot[k] / (N * launches) if launches else 0.0
        per_voxel["ewald"] = 0
    per_voxel.setdefault("fftx", 0)
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
    # DRAM bytes per launch from an ncu capture of this kernel (the
    # multi-angle x pass is recorded per batch size)
    tkey = f"{top}-k{kx}" if (top == "pol_fftx" and kx > 1) else top
    if zfirst:
        tkey = f"zfirst-{top}"
    traffic = _traffic_from_profiles(args.workload, tkey, prec) if args.algorithm == 1 else None
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
        Mh, numa_bound = pinned_near_gpu(M.shape, M.dtype, dev)
        Mh.copy_(M)
        Mh_np = Mh.numpy()
        out_t = torch.empty((1, ny, nx), dtype=M.dtype, pin_memory=True)
        host_out = out_t.numpy()
        del M
        ctx.close()
        torch.cuda.empty_cache()
        ctxs = [rsx.Context(nx, ny, nz, c, voxel_nm, precision=prec, algorithm=args.algorithm,
                            angle_batch=args.angle_batch) for _ in range(2)]
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
        ranks.barrier()
        t0 = time.perf_counter()
        e2e_steps(args.warmup, n_steps)
        torch.cuda.synchronize()
        e2e_s = ranks.max(time.perf_counter() - t0)
        e2e = {"value": units / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(Mh_np.nbytes), "d2h_bytes_per_step": int(host_out.nbytes),
               "h2d_gbs": round(h2d_gbs, 1), "pinned_near_gpu": numa_bound}
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
                                   f"c={c}, {n_ang} e-field angle(s) {'%g:%g:%g' % W['angles']} "
                                   f"per energy, {voxel_nm:g} nm voxels, one energy "
                                   f"per step (of {n_e} over {e_lo:g}-{e_hi:g} eV)",
                       "voxels": N, "components": c, "angles_per_energy": n_ang,
                       "angle_batch": angle_batch,
                       "zfirst_planes": sorted({z[0] for z in zplans}) if zfirst else None,
                       "angles_per_pass": sorted({z[2] for z in zplans}) if zfirst else None,
                       "precision": prec, "parallelism": f"energy-sharded x{ws}",
                       "ranks_per_gpu": -(-ws // ndev),
                       "l2": f"inputs larger than L2 (morphology {N * c * 4 * real / 1e9:.1f} GB)"},
            "roofline": roofline,
            "phases_ms": {k: round(v[0], 3) for k, v in phases.items()},
            "gpu_launches": int(sum(v[1] for v in phases.values())),
            "clocks": clk,
            "e2e": e2e,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(W, args, c)
        print(json.dumps(line), flush=True)
    ranks.close()


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


def _oracle_angles(job):
    """Worker of the CPU baseline: the oracle's Algorithm 1 inner loop for a
    list of angles of one energy, summed (runs in a spawned process)."""
    shape, c, seed_m, seed_k, E, alphas = job
    import numpy as np

    from oracle import cyrsoxs_oracle as O
    from paper_2209_13121_gb300 import synth
    M = synth.morphology_random(shape, c, seed=seed_m, dtype=np.float64)
    K = synth.optical_constants([E], c, seed=seed_k)
    acc = np.zeros(shape[1:])
    for a in alphas:
        acc += O.rotate_image(O.scatter_one_angle(M, K[0], E, VOXEL_NM, a), a)
    return acc


def time_oracle(shape, c, angles_deg, n_angles, cores):
    """Wall time of the FP64 oracle (as it stands) over the first n_angles
    angles of one energy of a seeded morphology, on `cores` processes
    (spawned, each a share of the angles; cores = 1 runs in this process).
    Returns (voxel-angle/s in G units, seconds)."""
    import multiprocessing as mp

    import numpy as np

    from oracle import cyrsoxs_oracle as O
    alphas = list(O.angle_list(*angles_deg)[:n_angles])
    jobs = [(shape, c, 1, 2, 285.0, alphas[i::cores]) for i in range(cores)]
    jobs = [j for j in jobs if j[-1]]
    if cores == 1:
        t0 = time.perf_counter()
        _oracle_angles(jobs[0])
        dt = time.perf_counter() - t0
    else:
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            pool.map(_oracle_angles, [(shape, c, 1, 2, 285.0, alphas[:1])] * len(jobs))  # warm
            t0 = time.perf_counter()
            parts = pool.map(_oracle_angles, jobs)
            dt = time.perf_counter() - t0
        np.sum(parts, axis=0)
    return math.prod(shape) * len(alphas) / dt / 1e9, dt


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(W, args, c):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    128 x 128 x 16 voxels with the same c and one energy; all 91 angles on
    every host core (one spawned process per core, each a share of the
    angles), and 8 angles on one core beside it.  Voxel-angle/s scales
    linearly in N (Sec. 6.1), so the sample's throughput stands for the
    workload's."""
    shape = (16, 128, 128)
    cores = _host_cores()
    v_all, t_all = time_oracle(shape, c, W["angles"], 91, cores)
    v_one, t_one = time_oracle(shape, c, W["angles"], 8, 1)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": v_one,
            "sample": f"FP64 numpy oracle, {shape[2]}x{shape[1]}x{shape[0]} voxels, c={c}, 1 energy: "
                      f"91 angles on {cores} processes in {t_all:.1f} s; 8 angles on 1 core in "
                      f"{t_one:.1f} s"}


def cpu_report(args):
    """The oracle's CPU baselines: 128^2 x 16 and 256^2 x 32 (c = 4) and the
    2048^2 x 1 film (c = 2), one energy and the 91 angles of 0:2:180, on one
    core and on every host core; seconds per energy extrapolate linearly to
    the workloads' energy counts."""
    cores = _host_cores()
    rows = []
    for shape, c, n_one in (((16, 128, 128), 4, 91), ((32, 256, 256), 4, 23),
                            ((1, 2048, 2048), 2, 12)):
        v1, t1 = time_oracle(shape, c, (0.0, 2.0, 180.0), n_one, 1)
        va, ta = time_oracle(shape, c, (0.0, 2.0, 180.0), 91, cores)
        n = math.prod(shape)
        rows.append({"shape_zyx": shape, "components": c, "voxels": n,
                     "single_core": {"angles_timed": n_one, "s": round(t1, 2),
                                     "value": v1, "s_per_energy": round(n * 91 / v1 / 1e9, 2)},
                     "all_cores": {"cores": cores, "angles_timed": 91, "s": round(ta, 2),
                                   "value": va, "s_per_energy": round(ta, 2)}})
    print(json.dumps({"kind": "oracle CPU baselines", "unit": UNIT, "host_cores": cores,
                      "rows": rows}), flush=True)


def check_launcher(args):
    """The multi-rank control plane without a GPU: each rank (gloo) reports
    a different time, rank 0 prints the world size and the maximum."""
    ws, rank, _ = _dist()
    ranks = _Ranks(ws, "gloo")
    ranks.barrier()
    t = ranks.max(1.0 + rank)
    if rank == 0:
        print(json.dumps({"n_gpus": ws, "max_ms": t, "rank": rank}), flush=True)
    ranks.close()


def run_reference(args):
    """The oracle timed as the reference arm: each step one bounded sample
    (see cpu_baseline) of the workload, rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    c = args.components or W["c"]
    shape = (16, 128, 128)
    cores = _host_cores()
    for _ in range(args.warmup):
        time_oracle(shape, c, W["angles"], cores, cores)
    t0 = time.perf_counter()
    samples = [time_oracle(shape, c, W["angles"], 2 * cores, cores) for _ in range(args.steps)]
    dt = time.perf_counter() - t0
    value = statistics.mean(v for v, _ in samples)
    sample = (f"FP64 numpy oracle, 128x128x16 voxels, c={c}, 1 energy x {2 * cores} of the 91 "
              f"angles per step on {cores} processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (oracle on a bounded sample per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
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
    ap.add_argument("--angle-batch", type=int, default=0,
                    help="Algorithm 1: e-field angles per read of the morphology (0: the "
                         "library default)")
    ap.add_argument("--components", type=int, default=0,
                    help="material count c (0: the workload's; Sec. 6.2 sweeps 2..10)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-report", action="store_true",
                    help="time the oracle on this host (single core and all cores) and exit")
    ap.add_argument("--check-launcher", action="store_true",
                    help="run the multi-rank control plane only (gloo, no GPU)")
    args = ap.parse_args()
    if "WORLD_SIZE" in os.environ:
        if args.gpus not in (1, int(os.environ["WORLD_SIZE"])):
            raise SystemExit(f"--gpus {args.gpus} disagrees with WORLD_SIZE={os.environ['WORLD_SIZE']}")
    elif args.gpus > 1:
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]))
    if args.cpu_report:
        cpu_report(args)
    elif args.check_launcher:
        check_launcher(args)
    elif args.impl == "reference":
        if args.warmup < 3:
            print("note: fewer than 3 warm-up steps", file=sys.stderr)
        run_reference(args)
    else:
        if args.warmup < 3:
            print("note: fewer than 3 warm-up steps", file=sys.stderr)
        run_ours(args)


if __name__ == "__main__":
    main()
