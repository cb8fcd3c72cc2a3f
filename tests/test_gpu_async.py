"""The stream-ordered registration calls (gs_register_async,
gs_register_batch_async): device outputs, a device status word, no host
synchronisation once a plan shape's list size is known, and results equal to
the synchronous calls bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2408_10154_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GS_ERR_CAPACITY = 7


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_10154_gb300 as gsmod
    from paper_2408_10154_gb300 import build
    build.build()
    O.build()
    return gsmod


@pytest.fixture(scope="module")
def ctx(gs):
    c = gs.Context(0)
    yield c
    c.close()


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def room_edge(gs, ctx, n_views):
    c = synth.room_150k()
    src = gs.Gaussians.from_numpy(c["gaussians"])
    tgt = gs.gs_transform(ctx, src, c["T_gt"])
    I = dev(np.stack([np.eye(3, 4)] * n_views).reshape(n_views, 12))
    rs = gs.gs_render(ctx, src, I, c["src_cams"][:n_views])
    rt = gs.gs_render(ctx, tgt, I, c["tgt_cams"][:n_views])
    sv = list(zip(c["src_cams"][:n_views], [x.contiguous() for x in gs.split_views(rs["rgb"], c["src_cams"][:n_views], 3)],
                  [x.contiguous() for x in gs.split_views(rs["depth"], c["src_cams"][:n_views], 1)]))
    tv = list(zip(c["tgt_cams"][:n_views], [x.contiguous() for x in gs.split_views(rt["rgb"], c["tgt_cams"][:n_views], 3)],
                  [x.contiguous() for x in gs.split_views(rt["depth"], c["tgt_cams"][:n_views], 1)]))
    return src, tgt, sv, tv


def test_async_registration_chains_two_edges_without_host_sync(gs, ctx):
    # two room-size loop edges of different shapes (8 + 8 and 4 + 4
    # keyframes, 100 iterations): the synchronous calls give the reference
    # and let the context learn each shape's list size; then both edges are
    # enqueued back to back on one stream.  The host gets control back before
    # the GPU is done (an event recorded after the second call is still
    # pending), and after one synchronisation every output equals the
    # synchronous call's bit for bit.
    a = room_edge(gs, ctx, 8)
    b = room_edge(gs, ctx, 4)
    ref = [gs.gs_register(ctx, *e, 100) for e in (a, b)]
    torch.cuda.synchronize()
    oa = gs.gs_register_async(ctx, *a, 100)
    ob = gs.gs_register_async(ctx, *b, 100)
    ev = torch.cuda.Event()
    ev.record()
    pending = not ev.query()
    torch.cuda.synchronize()
    assert pending, "the asynchronous calls waited for the GPU"
    for o, (T, conf, eps, est) in zip((oa, ob), ref):
        assert int(o["status"].item()) == 0
        np.testing.assert_array_equal(o["T"].cpu().numpy(), T)
        assert float(o["conf"].item()) == conf
        np.testing.assert_array_equal(o["eps"].cpu().numpy()[:len(eps)], eps)
        np.testing.assert_array_equal(o["est"].cpu().numpy()[:len(eps)], est)


def _problem(gs, n, W, H, f, n_src, n_tgt, seed):
    c = synth.small_case(n, W, H, f, n_views=max(n_src + n_tgt, 2), seed=seed, ls_mean=-3.3)
    og = O.Gaussians.from_dict(c["gaussians"])
    oq = O.transform(og, c["T_gt"])
    cams_p = c["cams"][:n_src]
    cams_q = synth.moved_cameras(c["cams"][n_src:n_src + n_tgt], c["T_gt"]) if n_tgt else []
    im = lambda g, cam: O.render(g, np.eye(3, 4), cam)
    sv = [(cam, dev(im(og, cam)["rgb"].astype(np.float32)), dev(im(og, cam)["depth"].astype(np.float32)))
          for cam in cams_p]
    tv = [(cam, dev(im(oq, cam)["rgb"].astype(np.float32)), dev(im(oq, cam)["depth"].astype(np.float32)))
          for cam in cams_q]
    src = gs.Gaussians.from_numpy(c["gaussians"])
    tgt = gs.Gaussians(*[dev(x) for x in (oq.means4, oq.log_scales4, oq.quats4, oq.logits, oq.rgb4)])
    return src, tgt, sv, tv


def test_async_batch_equals_synchronous_batch(gs, ctx):
    probs = [_problem(gs, 900, 96, 64, 80.0, 1, 2, 31), _problem(gs, 300, 64, 40, 50.0, 2, 0, 32),
             _problem(gs, 1500, 120, 90, 100.0, 2, 1, 33)]
    T, conf, eps = gs.gs_register_batch(ctx, probs, 15)
    o = gs.gs_register_batch_async(ctx, probs, 15)
    torch.cuda.synchronize()
    assert int(o["status"].item()) == 0
    np.testing.assert_array_equal(o["T"].cpu().numpy(), T)
    np.testing.assert_array_equal(o["conf"].cpu().numpy(), conf)
    np.testing.assert_array_equal(o["eps"].cpu().numpy()[:len(eps)], eps)


def test_async_registration_reports_outgrown_lists_in_its_status(gs, ctx):
    # lists sized at half the duplicates an earlier call saw: the first
    # iteration outgrows them; the asynchronous call does not redo the edge,
    # it reports GS_ERR_CAPACITY in its status word (the synchronous call
    # redoes it with more room)
    src, tgt, sv, tv = _problem(gs, 1500, 120, 90, 100.0, 2, 1, 34)
    gs.gs_register(ctx, src, tgt, sv, tv, 5)
    o = gs.gs_register_async(ctx, src, tgt, sv, tv, 5, gs.default_options(list_headroom=0.5))
    torch.cuda.synchronize()
    assert int(o["status"].item()) == GS_ERR_CAPACITY
    ok = gs.gs_register_async(ctx, src, tgt, sv, tv, 5)
    torch.cuda.synchronize()
    assert int(ok["status"].item()) == 0


def test_async_rejects_bad_arguments(gs, ctx):
    # the host checks run before anything is enqueued: a missing status word
    # or output, and a problem without keyframes, are refused
    import ctypes
    src, tgt, sv, tv = _problem(gs, 300, 64, 40, 50.0, 1, 1, 35)
    T = torch.empty(12, dtype=torch.float64, device="cuda")
    conf = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    s, t = src.c_struct(), tgt.c_struct()
    views = gs.gsreg._views(sv)
    lib, h = ctx._lib, ctx.handle
    opt = gs.default_options()
    P = ctypes.c_void_p
    args = lambda Tp, cp, stp, nsv: (h, ctypes.byref(s), ctypes.byref(t), views, nsv, None, 0, ctypes.byref(opt), 5,
                                     Tp, cp, None, None, stp, gs.gsreg._stream())
    assert lib.gs_register_async(*args(P(T.data_ptr()), P(conf.data_ptr()), None, 1)) == 1
    assert lib.gs_register_async(*args(None, P(conf.data_ptr()), P(st.data_ptr()), 1)) == 1
    assert lib.gs_register_async(*args(P(T.data_ptr()), P(conf.data_ptr()), P(st.data_ptr()), 0)) == 1


def test_fp32_probe_measures_the_device(gs, ctx):
    tflops, sms = gs.gs_probe_fp32(ctx)
    props = torch.cuda.get_device_properties(0)
    assert sms == props.multi_processor_count
    # 128 FP32 lanes x 2 flops per FMA per SM per cycle: the probe lands
    # below that bound at the highest clock and well above a tenth of it
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.1 * bound < tflops < bound, (tflops, bound)
