"""The multi-GPU path is independent replicas (one faux-shock box per rank,
no data-path collective): bench.py's whole-job throughput sums the particles
of every rank and divides by the slowest rank's time. Checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, lr, dist = bench.dist_setup(world, backend="gloo")
    # rank k pushed 1000 + 10 k particles per step for 5 steps in 2 + k ms
    v, t = bench.replica_value(1000.0 + 10 * r, 5, 2.0 + r, dist)
    dist.barrier()
    out.put((r, w, v, t))
    dist.destroy_process_group()


def test_two_gloo_replicas_sum_particles_over_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, v, t in res:
        assert w == 2
        assert t == 3.0                                  # the slower rank
        assert v == pytest.approx((1000 + 1010) * 5 / 3e-3)


def test_single_process_is_one_replica():
    import bench
    v, t = bench.replica_value(1000.0, 5, 2.0, None)
    assert t == 2.0 and v == pytest.approx(1000 * 5 / 2e-3)
