"""dgs_sort_pairs_noalloc -- the sort for callers that cannot allocate
device memory (a process whose caching allocator already holds the free
memory, or a loop that forbids allocation after start-up) -- gives the same
result as dgs_sort_pairs, on two calls in a row that share its fixed
scratch array, leaves the device's free memory unchanged once its first
call has loaded that array, and refuses sizes beyond its fixed maximum.

This file is collected last on purpose: it runs after every other test in a
full run, and it also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_ITEMS = 1 << 20


def _inputs(n, bits, seed):
    g = torch.Generator().manual_seed(seed)
    keys = torch.randint(0, 2 ** 31, (n,), generator=g, dtype=torch.int64)
    keys[: n // 4] = keys[0]  # long runs of equal keys: stability is visible
    keys = (keys & ((1 << bits) - 1)).to(torch.int32)
    vals = torch.arange(n, dtype=torch.int32)
    return keys, vals


@pytest.mark.parametrize("n,bits", [(300_007, 32), (MAX_ITEMS, 13), (4097, 8)])
def test_noalloc_sort_matches_sort_pairs_twice(n, bits):
    from paper_2508_03180_gb300 import _lib as L
    from paper_2508_03180_gb300.renderer import Context
    ctx = Context()
    keys, vals = _inputs(n, bits, seed=n + bits)
    # existing entry point (context-owned scratch)
    k_ref, v_ref = keys.cuda(), vals.cuda()
    ctx.sort_pairs(k_ref, v_ref, bits)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the second call sees the scratch left by the first
        k, v = keys.cuda(), vals.cuda()
        L.dgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), n, bits, stream)
        torch.cuda.synchronize()
        assert torch.equal(k, k_ref)
        assert torch.equal(v, v_ref)
    # and both agree with a stable host sort
    order = np.argsort(keys.numpy().astype(np.uint32), kind="stable")
    assert np.array_equal(v_ref.cpu().numpy(), order.astype(np.int32))
    ctx.close()


def test_noalloc_sort_rejects_more_than_its_maximum():
    from paper_2508_03180_gb300 import _lib as L
    k = torch.zeros(MAX_ITEMS + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros_like(k)
    with pytest.raises(L.DgsError) as ei:
        L.dgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), MAX_ITEMS + 1, 32, 0)
    assert ei.value.code == L.DGS_ERR_CAPACITY
    assert "1048576" in str(ei.value)


def test_noalloc_sort_allocates_nothing_after_its_first_call():
    """The call's defining property: once the first call on the device has
    loaded the scratch array and the sort's kernels (the caller's set-up),
    further calls of the largest size leave the device's free memory as it
    was.  Inputs are created before the readings, and nothing else touches
    the device between them."""
    from paper_2508_03180_gb300 import _lib as L
    keys, vals = _inputs(MAX_ITEMS, 32, seed=7)
    k, v = keys.cuda(), vals.cuda()
    stream = torch.cuda.current_stream().cuda_stream
    L.dgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), MAX_ITEMS, 32, stream)  # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        L.dgs_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), MAX_ITEMS, 32, stream)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    order = np.argsort(keys.numpy().astype(np.uint32), kind="stable")
    assert np.array_equal(v.cpu().numpy(), order.astype(np.int32))
