"""Multi-process path of the energy sharding, on CPU with the gloo backend.

Two ranks each compute the images of their own energies (with the CPU
oracle: these tests run without a GPU) and the rows are gathered on rank 0;
the result must equal the single-process run exactly, for block and strided
shards, including a rank that gets no energy."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2209_13121_gb300.shard import energy_shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, n_e, mode, outdir):
    import torch.distributed as dist

    from oracle import cyrsoxs_oracle as O
    from paper_2209_13121_gb300 import synth
    from paper_2209_13121_gb300.shard import energy_shard, gather_rows

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    E = list(np.linspace(270.0, 310.0, n_e))
    M = synth.morphology_random((2, 8, 8), 2, seed=3, dtype=np.float64)
    K = synth.optical_constants(E, 2, seed=4)
    idx = energy_shard(n_e, rank, ws, mode)
    rows = (O.run_alg1(M, K, E, 5.0, angles_deg=(0, 60, 120), energy_indices=list(idx))
            if len(idx) else np.zeros((0, 8, 8)))
    full = gather_rows(rows, idx, n_e)
    if rank == 0:
        np.save(os.path.join(outdir, f"gathered_{mode}.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode,n_e", [("block", 5), ("strided", 5), ("block", 1)])
def test_two_rank_shards_gather_to_single_process_result(tmp_path, mode, n_e):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, n_e, mode, str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    got = np.load(tmp_path / f"gathered_{mode}.npy")
    from oracle import cyrsoxs_oracle as O
    from paper_2209_13121_gb300 import synth
    E = list(np.linspace(270.0, 310.0, n_e))
    M = synth.morphology_random((2, 8, 8), 2, seed=3, dtype=np.float64)
    K = synth.optical_constants(E, 2, seed=4)
    ref = O.run_alg1(M, K, E, 5.0, angles_deg=(0, 60, 120))
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n,ws", [(150, 1), (150, 2), (150, 8), (7, 3), (2, 4), (0, 2)])
@pytest.mark.parametrize("mode", ["block", "strided"])
def test_shards_partition_the_energies(n, ws, mode):
    parts = [energy_shard(n, r, ws, mode) for r in range(ws)]
    allidx = np.concatenate(parts) if parts else np.array([], int)
    assert sorted(allidx.tolist()) == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        energy_shard(10, 2, 2)
