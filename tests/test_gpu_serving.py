"""Continuous-batching serving loop: results are the same alone and in a
mixed batch (as graph replays and as plain launch chains), a batch whose
(tile, cell) pairs overflow the captured buffers is re-run after they grow,
admission respects the HBM budget, and the host-side error paths (queue
full, unknown ticket, timeout) behave."""
import time

import numpy as np
import pytest
import torch

from paper_2508_03180_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scenes():
    return [synth.scene_small(seed=1, n_cells=800), synth.scene_small(seed=2, n_cells=1500, sh_degree=3)]


def _ctx(**cfg):
    from paper_2508_03180_gb300.renderer import Context
    return Context(**cfg)


@pytest.mark.parametrize("graphs", [True, False])
def test_same_result_alone_and_in_a_mixed_batch(scenes, graphs):
    c = _ctx()
    sids = [c.upload_scene(s) for s in scenes]
    cams = [synth.sphere_cameras(1, 3.0, W, H, seed0=i)[0] for i, (W, H) in
            enumerate([(64, 48), (128, 72), (33, 17), (200, 120), (96, 96), (160, 90)])]
    # reference: each view alone through dgs_render
    ref = []
    for i, cam in enumerate(cams):
        img, _, _ = c.render(sids[i % 2], [cam])
        ref.append(img.clone())
    torch.cuda.synchronize()
    c.serve_start(max_batch=8, graphs=graphs)
    outs = [torch.zeros_like(r) for r in ref]
    tickets = [c.submit(sids[i % 2], cam, outs[i]) for i, cam in enumerate(cams)]
    results = [c.poll(t, -1) for t in tickets]
    # the same requests again: graphs of these scene sets are replayed
    outs2 = [torch.zeros_like(r) for r in ref]
    results += [c.poll(c.submit(sids[i % 2], cam, outs2[i]), -1) for i, cam in enumerate(cams)]
    stats = c.serve_stats()
    c.serve_stop()
    if graphs:
        assert 1 <= stats["graphs_captured"] < stats["batches"]
    else:
        assert stats["graphs_captured"] == 0
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in results)
    assert max(r.batch_size for r in results) > 1, "requests submitted together should share a batch"
    for o, o2, r in zip(outs, outs2, ref):
        assert torch.equal(o, r)
        assert torch.equal(o2, r)
    # host outputs too
    c.serve_start(max_batch=4, graphs=graphs)
    host = [np.zeros(r.numel(), np.float32) for r in ref[:3]]
    ht = [c.submit(sids[i % 2], cams[i], torch.from_numpy(host[i])) for i in range(3)]
    for t in ht:
        assert c.poll(t, -1).status == 0
    c.serve_stop()
    for h, r in zip(host, ref[:3]):
        assert np.array_equal(h, r.cpu().numpy())
    c.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_neural_scenes_served_alone_and_mixed(scenes, graphs):
    """Neural-cell scenes in serving: batches that mix two neural scenes (one
    on the tensor-core decode, one wider on the CUDA-core decode) with an
    explicit scene return exactly the image dgs_render gives each view alone;
    each composition of neural scenes is its own captured graph."""
    c = _ctx()
    neural = [synth.neural_scene(n_cells=700, K=10, F=32, H=32, seed=3),
              synth.neural_scene(n_cells=500, K=6, F=20, H=36, seed=4)]
    sids = [c.upload_scene(scenes[0])] + [c.upload_scene(n) for n in neural]
    cams = [synth.sphere_cameras(1, 3.0, W, H, seed0=20 + i)[0] for i, (W, H) in
            enumerate([(64, 48), (128, 72), (33, 17), (200, 120), (96, 96), (160, 90), (80, 64), (120, 40)])]
    which = [1, 0, 2, 1, 1, 2, 0, 2]
    ref = []
    for cam, w in zip(cams, which):
        img, _, _ = c.render(sids[w], [cam])
        ref.append(img.clone())
    torch.cuda.synchronize()
    c.serve_start(max_batch=8, graphs=graphs)
    results, outs = [], []
    for rnd in range(2):  # the second round replays the captured graphs
        o = [torch.zeros_like(r) for r in ref]
        ts = [c.submit(sids[w], cam, o[i]) for i, (cam, w) in enumerate(zip(cams, which))]
        results += [c.poll(t, -1) for t in ts]
        outs.append(o)
    # only neural scenes in a batch
    o3 = [torch.zeros_like(ref[i]) for i in (0, 2, 3)]
    ts = [c.submit(sids[which[i]], cams[i], o3[j]) for j, i in enumerate((0, 2, 3))]
    results += [c.poll(t, -1) for t in ts]
    stats = c.serve_stats()
    c.serve_stop()
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in results), [r.status for r in results]
    assert max(r.batch_size for r in results) > 1
    if graphs:
        assert stats["graphs_captured"] >= 1
    for o in outs:
        for a, r in zip(o, ref):
            assert torch.equal(a, r)
    for a, i in zip(o3, (0, 2, 3)):
        assert torch.equal(a, ref[i])
    c.close()


def test_pair_overflow_grows_buffers_and_reruns():
    # thousands of large cells over a 48x32 view: far more (tile, cell) pairs
    # per tile than the initial estimate that sizes the captured buffers
    c = _ctx()
    scene = synth.scene_small(seed=7, n_cells=3000)
    sid = c.upload_scene(scene)
    cams = [synth.sphere_cameras(1, 2.2, 48, 32, seed0=s)[0] for s in range(3)]
    ref = [c.render(sid, [cam])[0].clone() for cam in cams]
    _, _, st = c.render(sid, [cams[0]], stats=True)
    assert st.sort_length > 200 * 6, "the scene must be dense enough to overflow"
    torch.cuda.synchronize()
    c.serve_start(max_batch=1)
    outs = [torch.zeros_like(r) for r in ref]
    rs = [c.poll(c.submit(sid, cam, o), -1) for cam, o in zip(cams, outs)]
    stats = c.serve_stats()
    c.serve_stop()
    assert all(r.status == 0 for r in rs)
    assert stats["overflow_retries"] >= 1
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    c.close()


def test_admission_respects_budget(scenes):
    # a budget that fits roughly one request at a time forces batches of one
    c = _ctx(hbm_budget_bytes=64 << 20)
    sid = c.upload_scene(scenes[0])
    c.serve_start(max_batch=8)
    cams = synth.sphere_cameras(6, 3.0, 1920, 1080, seed0=3)
    outs = [torch.zeros(3 * 1920 * 1080, device="cuda") for _ in cams]
    ts = [c.submit(sid, cam, o) for cam, o in zip(cams, outs)]
    rs = [c.poll(t, -1) for t in ts]
    c.serve_stop()
    assert all(r.status == 0 for r in rs)
    assert max(r.batch_size for r in rs) == 1
    c.close()


def test_poll_timeout_and_errors(scenes):
    from paper_2508_03180_gb300 import _lib as L
    # a budget below one request: one chain in flight, one view per chain, so
    # a burst of 4K renders of a 2M-Gaussian scene must back up the queue
    c = _ctx(hbm_budget_bytes=1)
    sid = c.upload_scene(synth.scene_small(seed=3, n_cells=250_000))
    with pytest.raises(L.DgsError):
        c.submit(sid, synth.small_camera(), torch.zeros(3 * 256 * 256, device="cuda"))  # serving not started
    c.serve_start(max_batch=2, queue_cap=2)
    out = torch.zeros(3 * 3840 * 2160, device="cuda")
    cam = synth.small_camera(3840, 2160)
    tickets = []
    busy = False
    for _ in range(64):
        try:
            tickets.append(c.submit(sid, cam, out))
        except L.DgsError as e:
            assert e.code == L.DGS_ERR_BUSY
            busy = True
            break
    assert busy, "a queue of capacity 2 must refuse a burst of 64 requests"
    r0 = c.poll(tickets[-1], 0)
    assert r0 is None or r0.status == 0  # 0 timeout: just a check
    for t in tickets:
        if r0 is not None and t == tickets[-1]:
            continue
        assert c.poll(t, -1).status == 0
    with pytest.raises(L.DgsError):
        c.poll(tickets[0], 0)  # consumed
    with pytest.raises(L.DgsError):
        c.poll(123456789, 0)  # never issued
    c.serve_stop()
    c.close()


def test_requests_arriving_during_a_render_join_later_batches(scenes):
    c = _ctx()
    sid = c.upload_scene(scenes[1])
    c.serve_start(max_batch=8)
    cams = synth.sphere_cameras(24, 3.0, 1280, 720, seed0=50)
    outs = [torch.zeros(3 * 1280 * 720, device="cuda") for _ in cams]
    ts = []
    for cam, o in zip(cams, outs):
        ts.append(c.submit(sid, cam, o))
        time.sleep(0.0005)
    rs = [c.poll(t, -1) for t in ts]
    c.serve_stop()
    assert all(r.status == 0 for r in rs)
    starts = sorted({round(r.t_start_ms, 6) for r in rs})
    assert len(starts) >= 2  # more than one batch ran
    c.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_mixed_cells_per_gaussian_and_view_dependent_v(graphs):
    # K = 8 and K = 10 scenes in one batch take the blend's generic-K path;
    # the third scene has a view-dependent v_n
    c = _ctx()
    scs = [synth.scene_small(seed=5, n_cells=600),
           synth.make_scene(500, 10, synth._box(-1.0, 1.0), 0.02, 0.1, 1, seed=6),
           synth.with_view_dependent_v(synth.scene_small(seed=7, n_cells=700), degree=2, seed=1)]
    sids = [c.upload_scene(s) for s in scs]
    cams = [synth.sphere_cameras(1, 3.0, W, H, seed0=20 + i)[0] for i, (W, H) in
            enumerate([(64, 48), (80, 60), (50, 70), (96, 40), (64, 64), (40, 40)])]
    ref = [c.render(sids[i % 3], [cam])[0].clone() for i, cam in enumerate(cams)]
    torch.cuda.synchronize()
    c.serve_start(max_batch=8, graphs=graphs)
    outs = [torch.zeros_like(r) for r in ref]
    ts = [c.submit(sids[i % 3], cam, outs[i]) for i, cam in enumerate(cams)]
    rs = [c.poll(t, -1) for t in ts]
    c.serve_stop()
    assert all(r.status == 0 for r in rs)
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    c.close()


def test_empty_scene_in_a_served_batch():
    from paper_2508_03180_gb300.renderer import Context
    bg = (0.1, 0.2, 0.3)
    c = Context(bg=bg)
    sids = [c.upload_scene(synth.scene_small(n_cells=0)), c.upload_scene(synth.scene_small(seed=9, n_cells=300))]
    cams = [synth.small_camera(48, 32), synth.small_camera(64, 40), synth.small_camera(16, 16)]
    ref = [c.render(sids[i % 2], [cam])[0].clone() for i, cam in enumerate(cams)]
    torch.cuda.synchronize()
    c.serve_start(max_batch=4)
    outs = [torch.zeros_like(r) for r in ref]
    rs = [c.poll(c.submit(sids[i % 2], cam, outs[i]), -1) for i, cam in enumerate(cams)]
    c.serve_stop()
    assert all(r.status == 0 for r in rs)
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    for ch in range(3):
        assert torch.all(outs[0].view(3, -1)[ch] == bg[ch])
    c.close()


def test_cancel_queued_and_running_requests_leaves_the_others_intact(scenes):
    """Cancelling requests, newest first, while the queue is long: each one
    still queued or in a batch on the GPU completes with DGS_ERR_CANCELLED
    (the newest, cancelled right after its submission behind a long queue,
    certainly does); one that had already finished keeps status 0 and its
    image.  Every request not cancelled, including those batched with a
    cancelled one, returns exactly the image dgs_render gives it alone."""
    from paper_2508_03180_gb300 import _lib as L
    c = _ctx()
    sids = [c.upload_scene(s) for s in scenes]
    cams = [synth.sphere_cameras(1, 3.0, 1280, 720, seed0=50 + i)[0] for i in range(60)]
    ref = []
    for i, cam in enumerate(cams):
        img, _, _ = c.render(sids[i % 2], [cam])
        ref.append(img.clone())
    torch.cuda.synchronize()
    c.serve_start(max_batch=4)
    outs = [torch.zeros_like(r) for r in ref]
    tickets = [c.submit(sids[i % 2], cam, outs[i]) for i, cam in enumerate(cams)]
    cancel = set(range(1, 60, 3))
    for i in sorted(cancel, reverse=True):
        c.cancel(tickets[i])
    results = [c.poll(t, 10_000_000) for t in tickets]
    # cancelled after it finished: the result keeps its own status
    t_late = c.submit(sids[0], cams[0], outs[0])
    time.sleep(0.5)
    c.cancel(t_late)
    late = c.poll(t_late, 10_000_000)
    with pytest.raises(L.DgsError) as ei:
        c.cancel(t_late)  # consumed by the poll
    assert ei.value.code == L.DGS_ERR_NOT_FOUND
    c.serve_stop()
    torch.cuda.synchronize()
    assert late is not None and late.status == 0
    assert results[max(cancel)].status == L.DGS_ERR_CANCELLED
    n_cancelled = 0
    for i, r in enumerate(results):
        assert r is not None, i
        if i in cancel and r.status == L.DGS_ERR_CANCELLED:
            n_cancelled += 1
            continue
        assert r.status == 0, (i, r.status)
        assert torch.equal(outs[i], ref[i]), i
    print(f"{n_cancelled} of {len(cancel)} cancellations took effect")
    c.close()
