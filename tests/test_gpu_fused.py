"""The fused registration compositing (the forward and the adjoint of a tile
in one CTA, option fuse_compositing = 1) against the two kernels (0): every
output of gs_register, gs_register_batch and the exposure and counting
variants is bit-equal, on short tile lists (the adjoint walks the forward's
staging), lists longer than one forward batch (restaged chunk by chunk), the
needle / threshold-opacity stress case and the full-size room edge."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2408_10154_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float32).contiguous()


def needles():
    c = synth.small_case(1500, 300, 200, 200.0, n_views=2, seed=21, ls_mean=-3.2, ls_std=0.3)
    g = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    rng = np.random.default_rng(21)
    g["log_scales4"][:, 0] += 1.5
    g["log_scales4"][:, 1] -= 2.5
    near = rng.random(len(g["logits"])) < 0.5
    g["logits"][near] = rng.normal(-5.55, 0.15, int(near.sum()))
    return g, c["cams"]


CASES = {
    "ragged_100x70": lambda: (lambda c: (c["gaussians"], c["cams"]))(
        synth.small_case(700, 100, 70, 70.0, n_views=3, seed=9, ls_mean=-3.5)),
    "needles_300x200": needles,
    # lists longer than one forward batch (256) and than two
    "dense_400": lambda: (lambda c: (c["gaussians"], c["cams"]))(
        synth.small_case(400, 64, 48, 200.0, n_views=2, seed=31, ls_mean=-3.0, ls_std=0.2, half=0.05)),
    "dense_3000": lambda: (lambda c: (c["gaussians"], c["cams"]))(
        synth.small_case(3000, 64, 48, 200.0, n_views=2, seed=31, ls_mean=-3.0, ls_std=0.2, half=0.05)),
    # alphas at the 0.99 clamp on the left half only
    "saturated_160x120": lambda: (lambda c: (c["gaussians"], c["cams"]))(synth.saturated_case()),
    # needles across the whole image whose conics are too ill-conditioned
    # for the fast walk
    "giant_needles_120x90": lambda: (lambda c: (c["gaussians"], c["cams"]))(synth.giant_needles_case()),
}


def views_of(gd, cams, seed, angle=1.5, trans=0.02):
    og = O.Gaussians.from_dict(gd)
    T = synth.about_point(synth.random_rigid(np.random.default_rng(seed), angle, trans), O.centroid(og))
    out = []
    for cam in cams:
        r = O.render(og, T, cam)
        out.append((cam, dev(r["rgb"].astype(np.float32)), dev(r["depth"].astype(np.float32))))
    return out


def both(gs, ctx, fn, **kw):
    return [fn(gs.default_options(fuse_compositing=f, **kw)) for f in (1, 0)]


def assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("case", list(CASES))
def test_fused_registration_equals_two_kernels(gs, ctx, case):
    gd, cams = CASES[case]()
    g = gs.Gaussians.from_numpy(gd)
    views = views_of(gd, cams, 41)
    half = max(1, len(views) // 2)
    a, b = both(gs, ctx, lambda o: gs.gs_register(ctx, g, g, views[:half], views[half:], 12, o))
    assert_same(a, b)


def test_fused_room_edge_equals_two_kernels(gs, ctx):
    c = synth.room_150k()
    src = gs.Gaussians.from_numpy(c["gaussians"])
    tgt = gs.gs_transform(ctx, src, c["T_gt"])
    I = dev(np.stack([np.eye(3, 4)] * 3).reshape(3, 12))
    rs = gs.gs_render(ctx, src, I, c["src_cams"][:3])
    rt = gs.gs_render(ctx, tgt, I, c["tgt_cams"][:3])
    sv = list(zip(c["src_cams"][:3], [x.contiguous() for x in gs.split_views(rs["rgb"], c["src_cams"][:3], 3)],
                  [x.contiguous() for x in gs.split_views(rs["depth"], c["src_cams"][:3], 1)]))
    tv = list(zip(c["tgt_cams"][:3], [x.contiguous() for x in gs.split_views(rt["rgb"], c["tgt_cams"][:3], 3)],
                  [x.contiguous() for x in gs.split_views(rt["depth"], c["tgt_cams"][:3], 1)]))
    for sched in (1, 4):  # one CTA per tile; the persistent queue, longest lists first
        a, b = both(gs, ctx, lambda o: gs.gs_register(ctx, src, tgt, sv, tv, 10, o), tile_schedule=sched)
        assert_same(a, b)


def test_fused_exposure_and_counting_variants(gs, ctx):
    gd, cams = CASES["ragged_100x70"]()
    g = gs.Gaussians.from_numpy(gd)
    views = views_of(gd, cams, 42)
    a, b = both(gs, ctx, lambda o: gs.gs_register(ctx, g, g, views[:1], views[1:], 12, o), exposure=1)
    assert_same(a, b)
    counts = []
    for f in (1, 0):
        res = gs.gs_register(ctx, g, g, views[:1], views[1:], 6, gs.default_options(fuse_compositing=f, profile=2))
        st = gs.gsreg.gs_stats_t()
        ctx.check(ctx._lib.gs_ctx_stats(ctx.handle, ctypes.byref(st)))
        counts.append((res, st.pairs, st.contributing, list(st.phase_ms)))
    assert_same(counts[0][0], counts[1][0])
    assert counts[0][1:3] == counts[1][1:3] and counts[0][2] > 0
    # fused: the forward phase holds the fused kernel, the backward phase is empty
    assert counts[0][3][2] > 0 and counts[0][3][3] < 0.1 * counts[0][3][2]
    assert counts[1][3][3] > 0


def test_fused_batch_equals_two_kernels(gs, ctx):
    probs = []
    for seed, (n, W, H, f) in enumerate([(900, 96, 64, 80.0), (300, 64, 40, 50.0), (1500, 120, 90, 100.0)]):
        c = synth.small_case(n, W, H, f, n_views=3, seed=50 + seed, ls_mean=-3.3)
        og = O.Gaussians.from_dict(c["gaussians"])
        oq = O.transform(og, c["T_gt"])
        im = lambda g_, cam: O.render(g_, np.eye(3, 4), cam)
        cq = synth.moved_cameras(c["cams"][1:], c["T_gt"])
        sv = [(cam, dev(im(og, cam)["rgb"].astype(np.float32)), dev(im(og, cam)["depth"].astype(np.float32)))
              for cam in c["cams"][:1]]
        tv = [(cam, dev(im(oq, cam)["rgb"].astype(np.float32)), dev(im(oq, cam)["depth"].astype(np.float32)))
              for cam in cq]
        src = gs.Gaussians.from_numpy(c["gaussians"])
        tgt = gs.Gaussians(*[dev(x) for x in (oq.means4, oq.log_scales4, oq.quats4, oq.logits, oq.rgb4)])
        probs.append((src, tgt, sv, tv))
    a, b = both(gs, ctx, lambda o: gs.gs_register_batch(ctx, probs, 10, o))
    assert_same(a, b)


def test_fused_option_is_checked(gs, ctx):
    gd, cams = CASES["ragged_100x70"]()
    g = gs.Gaussians.from_numpy(gd)
    views = views_of(gd, cams, 43)
    with pytest.raises(Exception):
        gs.gs_register(ctx, g, g, [], views, 2, gs.default_options(fuse_compositing=2))


def one_tile(n, seed):
    # n faint, wide splats in front of a 16x16 camera: every one lands on the
    # frame's only tile, and pixels stay far from opaque, so the walks run
    # the whole list -- list lengths at the fused kernel's chunk (64) and
    # staging (256) boundaries
    c = synth.small_case(n, 16, 16, 20.0, n_views=1, seed=seed, ls_mean=-1.6, ls_std=0.1, half=0.2)
    g = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    g["logits"][:] = np.random.default_rng(seed).normal(-4.0, 0.2, len(g["logits"]))
    return g, c["cams"]


@pytest.mark.parametrize("n", [63, 64, 65, 128, 255, 256, 257, 300])
def test_fused_at_list_length_boundaries(gs, ctx, n):
    gd, cams = one_tile(n, 70 + n)
    og = O.Gaussians.from_dict(gd)
    _, _, ranges = O.bin_tiles(og, np.eye(3, 4)[None], cams, O.DEFAULT_OPT)
    assert int((ranges[:, 1] - ranges[:, 0]).max()) == n
    g = gs.Gaussians.from_numpy(gd)
    views = views_of(gd, cams, 80 + n, angle=1.0, trans=0.01)
    a, b = both(gs, ctx, lambda o: gs.gs_register(ctx, g, g, [], views, 6, o))
    assert_same(a, b)
    la, ga = gs.gs_register_gradient(ctx, g, g, [], views)
    lb, gb = gs.gs_register_gradient(ctx, g, g, [], views, gs.default_options(fuse_compositing=0))
    np.testing.assert_array_equal(ga, gb)
    np.testing.assert_array_equal(la, lb)
