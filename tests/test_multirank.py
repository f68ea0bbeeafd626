"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2): each
rank renders its own seeded views, the per-Gaussian gradients of the
data-parallel step are summed across ranks with one all-reduce of the flat
gradient buffer (the step's only exchange), the timing is the maximum over
ranks, the value is the whole-job pixel rate, and only rank 0 reports."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup(None, backend="gloo")
    cams = [c.as_array().tolist() for c in bench.cameras_for(r, n_views=2)]
    bench.barrier(w)
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w)  # rank 1 is the slow one
    value = bench.weak_value(ms, w, 1000, 4)
    # gradients of 7 Gaussians (SH degree 3): rank r's own are r + 1 + index
    import torch
    flat, g = bench.flat_grads(7, 16, "cpu")
    flat.copy_(torch.arange(flat.numel(), dtype=torch.float32) + (r + 1))
    bench.reduce_grads(flat, w)
    q.put((r, w, cams, ms, value, flat.numpy().copy(), tuple(g["g_sh"].shape), g["g_logit"].numpy().copy()))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, cams0, ms0, v0, f0, sh0, lg0), (r1, w1, cams1, ms1, v1, f1, sh1, lg1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert cams0 != cams1                     # every rank its own views
    assert ms0 == ms1 == 15.0                 # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)
    import numpy as np
    n = 7 * 59
    want = 2 * np.arange(n, dtype=np.float32) + 3  # (i + 1) + (i + 2)
    assert f0.shape == (n,) and np.array_equal(f0, want) and np.array_equal(f1, want)
    assert sh0 == sh1 == (7, 16, 3)
    assert np.array_equal(lg0, want[7 * 10:7 * 11])  # logit block after mean, log-scale, quaternion


_NAMES = (("g_mean", "mean"), ("g_log_scale", "log_scale"), ("g_quat", "quat"), ("g_logit", "logit"),
          ("g_sh", "sh"))


def _oracle_scene():
    from paper_2508_03180_gb300 import synth
    sc = synth.make_scene(30, 4, synth._box(-0.5, 0.5), 0.15, 0.4, 3, seed=5)
    return sc, synth.sphere_cameras(2, 3.0, 24, 20, seed0=11)


def _oracle_view_grads(sc, cam, rank):
    import numpy as np
    import oracle
    g = np.random.default_rng(100 + rank).standard_normal((3, cam.H, cam.W))
    return oracle.render_and_grad(sc, cam.as_array(), g)[2]


def _oracle_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    w, r, _ = bench.dist_setup(None, backend="gloo")
    sc, cams = _oracle_scene()
    pg = _oracle_view_grads(sc, cams[r], r)  # this rank's view only
    flat, gr = bench.flat_grads(sc.G, 16, "cpu")
    for k, name in _NAMES:
        gr[k].copy_(torch.from_numpy(pg[name].reshape(gr[k].shape)).float())
    bench.reduce_grads(flat, w)
    q.put((r, {k: v.numpy().copy() for k, v in gr.items()}))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_gradient_buffer_sums_the_ranks_views():
    """Each of two gloo ranks writes the oracle's parameter gradients of its
    own view into the data-parallel flat buffer; after the one all-reduce
    every rank holds the gradients of the two-view loss (the oracle's sum over
    both views) in the renderer's output layout."""
    import socket
    import numpy as np
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    sc, cams = _oracle_scene()
    both = [_oracle_view_grads(sc, cams[r], r) for r in range(2)]
    for k, name in _NAMES:
        want = both[0][name] + both[1][name]
        assert np.abs(want).max() > 0, name
        for r in range(2):
            got = res[r][k].astype(np.float64).reshape(want.shape)
            assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max(), (r, name)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.weak_value(1000.0, 1, 2_000_000, 10) == pytest.approx(20.0)
    import torch
    flat, _ = bench.flat_grads(3, 16, "cpu")
    flat.fill_(2.0)
    bench.reduce_grads(flat, 1)  # one rank: no collective, unchanged
    assert torch.all(flat == 2.0)


def test_serving_at_equal_p99_picks_the_highest_rate_within_each_target():
    import bench
    rows = [{"offered_rps": 200.0, "p99_ms": 1.0, "fps": 200.0}, {"offered_rps": 2500.0, "p99_ms": 2.3, "fps": 2490.0},
            {"offered_rps": 3000.0, "p99_ms": 1.9, "fps": 2990.0}, {"offered_rps": 5000.0, "p99_ms": 14.0, "fps": 4300.0}]
    got = bench.at_p99(rows, slos=(2.0, 5.0, 20.0, 0.5))
    assert got["2ms"]["offered_rps"] == 3000.0 and got["5ms"]["offered_rps"] == 3000.0
    assert got["20ms"] == {"offered_rps": 5000.0, "fps": 4300.0, "p99_ms": 14.0}
    assert got["0.5ms"] is None
