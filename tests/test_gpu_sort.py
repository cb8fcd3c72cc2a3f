"""The one-sweep radix sort behind the tile lists (gs_sort_u32) vs numpy's
stable sort, and the bounded device wait of its look-back: a pass whose
first tile never publishes gives up, reports GS_ERR_TIMEOUT and leaves the
context usable (no fault, no hang)."""
import ctypes
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_10154_gb300 as gsmod
    from paper_2408_10154_gb300 import build
    build.build()
    return gsmod


@pytest.fixture(scope="module")
def ctx(gs):
    c = gs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,bits", [(5, 8), (2048, 16), (10007, 32), (300_000, 20), (1_000_003, 32)])
def test_sort_matches_stable_numpy_sort(gs, ctx, n, bits):
    rng = np.random.default_rng(n + bits)
    # few distinct values in the low bits (stability), random high bits
    keys = (rng.integers(0, 1 << 32, n, dtype=np.uint64) & 0xFFFFFF00).astype(np.uint32) | rng.integers(
        0, 7, n).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    masked = keys & np.uint32(0xFFFFFFFF if bits == 32 else (1 << bits) - 1)
    order = np.argsort(masked, kind="stable")
    k = torch.as_tensor(keys.view(np.int32)).cuda()
    v = torch.as_tensor(vals.view(np.int32)).cuda()
    gs.gs_sort_u32(ctx, k, v, bits)
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys[order])


def test_bounded_wait_gives_up_and_the_context_survives(gs, ctx):
    n = 20_000
    k = torch.randint(0, 1 << 30, (n,), dtype=torch.int32, device="cuda")
    v = torch.arange(n, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    st = ctx._lib.gs_selftest_bounded_wait(ctx.handle, ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                           n, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 5, (st, ctx._lib.gs_last_error(ctx.handle))  # GS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the device and the context still work
    k2 = torch.randint(0, 1 << 30, (n,), dtype=torch.int32, device="cuda")
    v2 = torch.arange(n, dtype=torch.int32, device="cuda")
    gs.gs_sort_u32(ctx, k2, v2, 32)
    kk = k2.cpu().numpy().view(np.uint32).astype(np.int64)
    assert (np.diff(kk) >= 0).all()
