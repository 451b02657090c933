"""Energy sharding with the library on every rank (Sec. 6.3: energies
distributed across GPUs, nothing exchanged on the data path).

Two ranks are spawned; each creates its own context, runs rsx_run on its own
energy shard, and the rows are gathered on rank 0 over gloo (the host
control plane).  On a one-GPU machine both ranks share cuda:0: their kernels
are independent launches of separate processes and never wait on one
another, so this is a functional check of the multi-rank path, not a
scaling measurement.  The gathered result must equal a single-process run
bit for bit, for block and strided shards."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPE, C, VOXEL = (4, 32, 64), 3, 5.0
ENERGIES = [272.0, 281.0, 285.0, 290.0, 301.0]
ANGLES = (0.0, 30.0, 150.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    from paper_2209_13121_gb300 import synth
    M = synth.morphology_random(SHAPE, C, seed=81, dtype=np.float32)
    K = synth.optical_constants(ENERGIES, C, seed=82)
    return M, K


def _rank(rank, ws, port, mode, outdir):
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_13121_gb300 import rsx
    from paper_2209_13121_gb300.shard import energy_shard, gather_rows

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    torch.cuda.set_device(rank % torch.cuda.device_count())
    M, K = _inputs()
    nz, ny, nx = SHAPE
    idx = energy_shard(len(ENERGIES), rank, ws, mode)
    with rsx.Context(nx, ny, nz, C, VOXEL, precision=32) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        rows = ctx.run(ANGLES, energy_indices=list(idx)) if len(idx) else np.zeros((0, ny, nx),
                                                                                  np.float32)
    full = gather_rows(rows, idx, len(ENERGIES))
    if rank == 0:
        np.save(os.path.join(outdir, f"gathered_{mode}.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["block", "strided"])
def test_two_ranks_drive_the_library_and_gather_the_single_process_result(tmp_path, mode):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp

    import __graft_entry__
    __graft_entry__.build()
    from paper_2209_13121_gb300 import rsx
    mp.start_processes(_rank, args=(2, _free_port(), mode, str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    got = np.load(tmp_path / f"gathered_{mode}.npy")
    M, K = _inputs()
    nz, ny, nx = SHAPE
    with rsx.Context(nx, ny, nz, C, VOXEL, precision=32) as ctx:
        ctx.set_morphology(torch.from_numpy(M).cuda())
        ctx.set_optical_constants(ENERGIES, K)
        ref = ctx.run(ANGLES)
    np.testing.assert_array_equal(got, ref)
