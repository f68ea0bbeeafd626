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
  inside the allocation) and pass again once that buffer is released.
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
