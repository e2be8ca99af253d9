"""N > 1 path on CPU: two gloo ranks each evaluate their shard of sun
directions (RNG counter offset by the shard start) with the FP64 oracle and
all-gather; the union equals the unsharded evaluation bit for bit."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2602_10712_gb300.shard import shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import oracle
    import workloads as W
    from paper_2602_10712_gb300.shard import gather_items, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, rho, _, com = W.config1()
    sun = W.fibonacci_directions(7)
    a, b = shard_range(7, rank, world)
    ft, _ = oracle.force(m.verts, m.tris, m.group, rho, sun[a:b], com, nx=48, K=3, sun_base=a, threads=2)
    full = gather_items(ft, 7, rank, world)
    if rank == 0:
        np.save(out_path, full)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 7, 100):
        for w in (1, 2, 3, 8):
            parts = [shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in parts) - min(b - a for a, b in parts) <= 1


def test_two_gloo_ranks_equal_unsharded(tmp_path):
    import oracle
    import workloads as W
    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    full = np.load(out)
    m, rho, _, com = W.config1()
    ref, _ = oracle.force(m.verts, m.tris, m.group, rho, W.fibonacci_directions(7), com, nx=48, K=3, threads=2)
    assert np.array_equal(full, ref)


def test_reflectance_projection():
    """The design loop's projection keeps rho_s, rho_d >= 0 and
    rho_s + rho_d <= 1 and leaves admissible values unchanged."""
    import numpy as np
    from paper_2602_10712_gb300.design import _project_rho
    r = np.array([[0.2, 0.3], [0.9, 0.4], [-0.1, 0.5], [1.2, -0.3], [0.6, 0.6]])
    p = _project_rho(r)
    assert np.all(p >= 0.0) and np.all(p.sum(axis=1) <= 1.0 + 1e-12)
    assert np.allclose(p[0], r[0])
