"""The multi-rank path on CPU (gloo, world size 2): ranks evaluate their own
shift streams of the same jobs (here with the oracle, standing in for each
rank's GPU), gather the per-shift sums and reduce the step time; the gathered
statistics equal one process evaluating all N x m shifts itself, and the
timing is the slowest rank's."""
import os

import numpy as np
import torch.multiprocessing as mp

import oracle
from paper_2305_19768_gb300 import dist as qdist
from paper_2305_19768_gb300 import qmc
from paper_2305_19768_gb300.inputs import workloads as w
from paper_2305_19768_gb300.inputs.lattice import lattice_for

N_RANKS, M, N_LAT = 2, 4, 1009


def _sums(seed):
    I = w.box_massless()
    out = []
    for s in range(len(I.sectors)):
        _, z = lattice_for(N_LAT, I.sectors[s].d)
        dl = oracle.shifts(seed, s, M, I.sectors[s].d)
        o, _, _ = oracle.shift_sums(oracle.SectorView(I, s, [-3.0, -2.0]), N_LAT, z, dl, -2, 3)
        out.append(o)
    return np.array(out)    # [sectors][m][orders][2]


def _worker(rank, port, result_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=N_RANKS)
    try:
        local = _sums(qdist.rank_seed(1, rank))
        allsums = qdist.gather_shift_sums(local)
        tmax = qdist.max_over_ranks(1.0 + rank)
        if rank == 0:
            np.save(os.path.join(result_dir, "all.npy"), allsums)
            np.save(os.path.join(result_dir, "tmax.npy"), np.array([tmax]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_shift_sums_and_time(tmp_path):
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(port, str(tmp_path)), nprocs=N_RANKS, start_method="spawn")
    allsums = np.load(tmp_path / "all.npy")
    assert float(np.load(tmp_path / "tmax.npy")[0]) == float(N_RANKS)
    expect = np.concatenate([_sums(qdist.rank_seed(1, r)) for r in range(N_RANKS)], axis=1)
    assert allsums.shape == (12, N_RANKS * M, 3, 2)
    assert np.array_equal(allsums, expect)
    # the ranks' shifts are distinct draws, and the statistics use all of them
    assert not np.array_equal(allsums[:, :M], allsums[:, M:])
    for sec in range(12):
        mean, var = qmc.qmc_shift_stats(allsums[sec])
        assert np.allclose(mean, allsums[sec].mean(axis=0), rtol=1e-14, atol=0)
