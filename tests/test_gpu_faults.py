"""Failure detection without a GPU fault (the library's debugging and
fault-injection calls, include/dgs.h):

* a radix-sort look-back wait made to run out (the first partition withholds
  its counts, a short poll limit) ends the kernels, returns DGS_ERR_TIMEOUT,
  and the same context then sorts and renders correctly;
* an injected device-allocation failure returns DGS_ERR_OOM from a scene
  upload and from a render, and the context stays usable;
* a host-side fault in the serving worker completes every open request with
  DGS_ERR_WORKER at once (no poll blocks), submit refuses new requests, and
  serving restarts;
* guard words next to device buffers report an overwrite (made on the host,
  inside the allocation) and pass again once that buffer is released;
* the tensor-core decode's completion wait made to run out (no products
  issued, a short limit) ends the kernel, the next call on the context
  returns DGS_ERR_TIMEOUT, and the context then renders the neural scene
  exactly as before.
"""
import time

import numpy as np
import pytest
import torch

from paper_2508_03180_gb300 import _lib as L
from paper_2508_03180_gb300 import synth
from paper_2508_03180_gb300.renderer import Context

pytestmark = pytest.mark.gpu


def _render(ctx, sid, cams):
    img, _, _ = ctx.render(sid, cams)
    torch.cuda.synchronize()
    return img.cpu()


def _reference_image(scene, cams):
    ref = Context()
    try:
        sid = ref.upload_scene(scene)
        return _render(ref, sid, cams)
    finally:
        ref.close()


def test_sort_wait_runs_out_and_the_context_stays_usable():
    ctx = Context()
    n, bits = 100_003, 32  # 33 partitions: 32 of them wait on the first
    g = torch.Generator().manual_seed(1)
    keys = torch.randint(0, 2 ** 31, (n,), generator=g, dtype=torch.int64).to(torch.int32)
    vals = torch.arange(n, dtype=torch.int32)
    try:
        L.dgs_debug_inject_fault(ctx.ctx, L.DGS_FAULT_SORT_WAIT, 1)
        for call in ("ctx", "noalloc"):
            k, v = keys.cuda(), vals.cuda()
            t0 = time.monotonic()
            with pytest.raises(L.DgsError) as ei:
                if call == "ctx":
                    ctx.sort_pairs(k, v, bits)
                else:
                    L.dgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), n, bits, 0)
            torch.cuda.synchronize()
            assert ei.value.code == L.DGS_ERR_TIMEOUT, str(ei.value)
            assert time.monotonic() - t0 < 10.0
    finally:
        L.dgs_debug_inject_fault(ctx.ctx, L.DGS_FAULT_SORT_WAIT, 0)
    try:
        k, v = keys.cuda(), vals.cuda()
        ctx.sort_pairs(k, v, bits)
        torch.cuda.synchronize()
        order = np.argsort(keys.numpy().view(np.uint32), kind="stable")
        assert np.array_equal(v.cpu().numpy(), order.astype(np.int32))
        scene = synth.scene_small(n_cells=400)
        cams = [synth.small_camera(64, 48)]
        sid = ctx.upload_scene(scene)
        assert torch.equal(_render(ctx, sid, cams), _reference_image(scene, cams))
    finally:
        ctx.close()


def test_injected_allocation_failure_returns_oom():
    scene = synth.scene_small(n_cells=300)
    cams = [synth.small_camera(80, 40)]
    ref = _reference_image(scene, cams)
    ctx = Context()
    try:
        L.dgs_debug_inject_fault(None, L.DGS_FAULT_ALLOC, 1)
        with pytest.raises(L.DgsError) as ei:
            ctx.upload_scene(scene)
        assert ei.value.code == L.DGS_ERR_OOM
        sid = ctx.upload_scene(scene)  # the next allocation succeeds
        L.dgs_debug_inject_fault(None, L.DGS_FAULT_ALLOC, 1)
        with pytest.raises(L.DgsError) as ei:
            ctx.render(sid, cams)  # a fresh context: the render must allocate its workspace
        assert ei.value.code == L.DGS_ERR_OOM
        assert torch.equal(_render(ctx, sid, cams), ref)
    finally:
        L.dgs_debug_inject_fault(None, L.DGS_FAULT_ALLOC, 0)
        ctx.close()


def test_serving_worker_fault_fails_open_requests_and_restarts():
    scene = synth.scene_small(n_cells=300)
    cams = synth.sphere_cameras(6, 3.0, 64, 48, seed0=3)
    ctx = Context()
    try:
        sid = ctx.upload_scene(scene)
        ctx.serve_start(max_batch=4)
        outs = [torch.zeros(3 * 64 * 48, device="cuda") for _ in cams]
        L.dgs_debug_inject_fault(ctx.ctx, L.DGS_FAULT_SERVE_WORKER, 1)
        tickets = []
        for c, o in zip(cams, outs):  # the worker may stop after the first submission
            try:
                tickets.append(ctx.submit(sid, c, o))
            except L.DgsError as e:
                assert e.code == L.DGS_ERR_WORKER, str(e)
        assert tickets, "the first submission reaches a live worker"
        t0 = time.monotonic()
        for t in tickets:
            r = ctx.poll(t, 10_000_000)  # bounded: 10 s at most
            assert r is not None, "poll blocked on a request of a stopped worker"
            assert r.status == L.DGS_ERR_WORKER
        assert time.monotonic() - t0 < 10.0
        with pytest.raises(L.DgsError) as ei:
            ctx.submit(sid, cams[0], outs[0])
        assert ei.value.code == L.DGS_ERR_WORKER
        ctx.serve_stop()
        ctx.serve_start(max_batch=4)
        t = ctx.submit(sid, cams[0], outs[0])
        r = ctx.poll(t, 10_000_000)
        assert r is not None and r.status == L.DGS_OK
        torch.cuda.synchronize()
        assert torch.equal(outs[0].cpu(), _render(ctx, sid, [cams[0]]))
    finally:
        ctx.close()


def test_guard_words_report_an_overwrite():
    L.dgs_debug_guards(True)
    ctx = Context()
    try:
        L.dgs_debug_inject_fault(None, L.DGS_FAULT_GUARD, 1)
        ctx.upload_scene(synth.scene_small(n_cells=50))
        with pytest.raises(L.DgsError) as ei:
            L.dgs_debug_check_guards()
        assert ei.value.code == L.DGS_ERR_GUARD
        assert "after its end" in str(ei.value)
    finally:
        L.dgs_debug_inject_fault(None, L.DGS_FAULT_GUARD, 0)
        ctx.close()  # releases the overwritten buffer
    assert L.dgs_debug_check_guards() >= 0


def test_tensor_core_wait_runs_out_and_the_context_stays_usable():
    from oracle import decode as odec
    F, H, K = 32, 32, 10
    sc = synth.neural_scene(n_cells=600, K=K, F=F, H=H, seed=5)
    cams = [synth.small_camera(96, 64), synth.sphere_cameras(1, 3.0, 80, 60, seed0=4)[0]]
    ctx = Context()
    try:
        sid = ctx.upload_scene(sc)
        ref = _render(ctx, sid, cams)
        g = dict(g_mlp=torch.zeros(odec.packed_size(F, H, K), device="cuda"))
        L.dgs_debug_inject_fault(ctx.ctx, L.DGS_FAULT_TC_WAIT, 1)
        try:
            t0 = time.monotonic()
            img, state, _ = ctx.render(sid, cams, want_state=True)  # asynchronous: returns before the wait ends
            torch.cuda.synchronize()
            elapsed = time.monotonic() - t0
        finally:
            L.dgs_debug_inject_fault(ctx.ctx, L.DGS_FAULT_TC_WAIT, 0)
        assert elapsed < 5.0, elapsed
        with pytest.raises(L.DgsError) as ei:
            ctx.backward(state, torch.ones_like(img), g)  # the completed chain's status is seen here
        assert ei.value.code == L.DGS_ERR_TIMEOUT and "tensor-core" in str(ei.value), str(ei.value)
        ctx.release_state(state)
        assert torch.equal(_render(ctx, sid, cams), ref)
        _, state2, _ = ctx.render(sid, cams, want_state=True)
        ctx.backward(state2, torch.ones_like(img), g)
        torch.cuda.synchronize()
        assert g["g_mlp"].abs().max() > 0
        ctx.release_state(state2)
    finally:
        ctx.close()
