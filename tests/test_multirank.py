"""The multi-GPU path's host logic on two CPU ranks (gloo): frames are
sharded across ranks with distinct scatterer seeds and no data-path
collective; only the step time is reduced, as a max over ranks, and the
whole-job throughput counts every rank's frames."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from tidas_workloads import generators
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # this rank's first frame of scatterers
    pos, _ = generators.compound_speckle_frame(0, seed=bench.rank_seed_base(rank))
    gathered = [torch.zeros(8, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(pos[:4].ravel().copy()))
    # a step time per rank, reduced as the bench reduces it
    ms = [4.0 + rank, 8.0 - 3 * rank]
    red = bench.max_over_ranks(torch, ms, world, "cpu")
    value = bench.whole_job_mpix_s(64, 524288, world, red[0])
    np.save(os.path.join(out_dir, "rank%d.npy" % rank),
            np.array([red[0], red[1], value] + [float(v) for g in gathered for v in g]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_reduce_the_step_time(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    # both ranks see the same reduced times: the max over ranks
    np.testing.assert_array_equal(r0[:3], r1[:3])
    assert r0[0] == 5.0 and r0[1] == 8.0
    # weak scaling: 2 x 64 frames of 512 x 1024 pixels in the slowest rank's 5 ms
    assert r0[2] == pytest.approx(2 * 64 * 524288 / 5e-3 / 1e6)
    # the ranks' frames come from different scatterer draws
    first0, first1 = r0[3:11], r0[11:19]
    assert not np.allclose(first0, first1)
    np.testing.assert_array_equal(r0[3:], r1[3:])


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, [3.5, 1.0], 1, "cpu") == [3.5, 1.0]
    assert bench.rank_seed_base(0) != bench.rank_seed_base(1)
