"""The registration hot path's adjoint against the oracle, directly:
gs_register_gradient runs one registration iteration (the fused forward +
adjoint, or the two kernels) without the update and returns each keyframe's
loss and pose gradient.  The oracle renders the same submap at the starting
pose, takes the L1 colour + depth loss (Sec. 3.2) or the tracking loss
(Eq. 2, Supp. A), and runs its FP64 adjoint with that loss's gradient
images about the moving submap's centroid.  Bars: the pose gradient within
1e-3 relative, the loss within the FP32 render's rounding."""
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


def small(*a, **k):
    c = synth.small_case(*a, **k)
    return c["gaussians"], c["cams"]


def one_tile(n, seed):
    # n faint, wide splats on a 16x16 frame's only tile: lists of exactly n
    # entries walked to the end (n = 65: two adjoint chunks; n = 257: more
    # than one forward batch, restaged chunk by chunk)
    c = synth.small_case(n, 16, 16, 20.0, n_views=1, seed=seed, ls_mean=-1.6, ls_std=0.1, half=0.2)
    g = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    g["logits"][:] = np.random.default_rng(seed).normal(-4.0, 0.2, len(g["logits"]))
    return g, c["cams"]


CASES = {
    "one_tile_65": lambda: one_tile(65, 135),
    "one_tile_257": lambda: one_tile(257, 327),
    "plain_2k": lambda: (lambda c: (c["gaussians"], c["cams"]))(synth.plain_2k()),
    "ragged_100x70": lambda: small(700, 100, 70, 70.0, n_views=3, seed=9, ls_mean=-3.5),
    "needles_300x200": needles,
    "dense_3000": lambda: small(3000, 64, 48, 200.0, n_views=2, seed=31, ls_mean=-3.0, ls_std=0.2, half=0.05),
    "saturated_160x120": lambda: (lambda c: (c["gaussians"], c["cams"]))(synth.saturated_case()),
    "room_full_size": lambda: (lambda c: (c["gaussians"], c["src_cams"][:2]))(synth.room_150k()),
}


def targets(og, cams, seed):
    T = synth.about_point(synth.random_rigid(np.random.default_rng(seed), 2.0, 0.03), O.centroid(og))
    out = []
    for cam in cams:
        r = O.render(og, T, cam)
        out.append((cam, r["rgb"].astype(np.float32), r["depth"].astype(np.float32)))
    return out


def check(gs, ctx, gd, cams, seed, opt, tracking=False):
    og = O.Gaussians.from_dict(gd)
    g = gs.Gaussians.from_numpy(gd)
    tg = targets(og, cams, seed)
    views = [(cam, dev(rgb), dev(dep)) for cam, rgb, dep in tg]
    loss, grad = gs.gs_register_gradient(ctx, g, g, [], views, opt)
    piv = O.centroid(og)
    for k, (cam, rgb, dep) in enumerate(tg):
        r = O.render(og, np.eye(3, 4), cam)
        if tracking:
            t = O.track_loss(r, rgb, dep)
            L, gr, gdp = t["loss"], t["g_rgb"], t["g_depth"]
        else:
            L, gr, gdp = O.loss(r["rgb"], r["depth"], rgb, dep)
        ref = O.backward(og, np.eye(3, 4), cam, gr, gdp, pivot=piv, params=False)["twist"]
        err = np.linalg.norm(grad[k] - ref) / np.linalg.norm(ref)
        assert err <= 1e-3, (k, err, grad[k], ref)
        assert loss[k] == pytest.approx(L, rel=1e-4), (k, loss[k], L)


@pytest.mark.parametrize("fuse", [1, 0])
@pytest.mark.parametrize("case", list(CASES))
def test_registration_gradient_matches_oracle(gs, ctx, case, fuse):
    gd, cams = CASES[case]()
    check(gs, ctx, gd, cams, 60, gs.default_options(fuse_compositing=fuse))


def test_registration_gradient_of_the_tracking_loss_matches_oracle(gs, ctx):
    gd, cams = CASES["ragged_100x70"]()
    check(gs, ctx, gd, cams, 61, gs.default_options(tracking_loss=1), tracking=True)


def test_registration_gradient_is_the_first_step_of_gs_register(gs, ctx):
    # the loss it returns is the residual a 0-iteration registration reports
    gd, cams = CASES["ragged_100x70"]()
    og = O.Gaussians.from_dict(gd)
    g = gs.Gaussians.from_numpy(gd)
    views = [(cam, dev(rgb), dev(dep)) for cam, rgb, dep in targets(og, cams, 62)]
    loss, _ = gs.gs_register_gradient(ctx, g, g, views[:1], views[1:])
    _, _, eps, _ = gs.gs_register(ctx, g, g, views[:1], views[1:], 0)
    np.testing.assert_array_equal(loss, eps)


def test_registration_gradient_of_reverse_keyframes_matches_oracle(gs, ctx):
    # keyframes of P localised in Q: the submap that moves is Q (= T P), its
    # render at P's keyframe cameras is compared with P's images, and the
    # gradient is Q's twist about Q's centroid
    gd, cams = CASES["ragged_100x70"]()
    og = O.Gaussians.from_dict(gd)
    T = synth.about_point(synth.random_rigid(np.random.default_rng(63), 2.0, 0.03), O.centroid(og))
    oq = O.transform(og, T)
    src = gs.Gaussians.from_numpy(gd)
    tgt = gs.Gaussians(*[dev(a) for a in (oq.means4, oq.log_scales4, oq.quats4, oq.logits, oq.rgb4)])
    ims = []
    for cam in cams:
        r = O.render(og, np.eye(3, 4), cam)
        ims.append((cam, r["rgb"].astype(np.float32), r["depth"].astype(np.float32)))
    views = [(cam, dev(rgb), dev(dep)) for cam, rgb, dep in ims]
    loss, grad = gs.gs_register_gradient(ctx, src, tgt, views, [])
    piv = O.centroid(oq)
    for k, (cam, rgb, dep) in enumerate(ims):
        r = O.render(oq, np.eye(3, 4), cam)
        L, gr, gdp = O.loss(r["rgb"], r["depth"], rgb, dep)
        ref = O.backward(oq, np.eye(3, 4), cam, gr, gdp, pivot=piv, params=False)["twist"]
        err = np.linalg.norm(grad[k] - ref) / np.linalg.norm(ref)
        assert err <= 1e-3, (k, err, grad[k], ref)
        assert loss[k] == pytest.approx(L, rel=1e-4), (k, loss[k], L)


def test_registration_gradient_with_exposure_and_counting(gs, ctx):
    # the exposure variant (gain 1, offset 0 at the start) and the counting
    # variant of the fused kernel give the plain gradient
    gd, cams = CASES["ragged_100x70"]()
    g = gs.Gaussians.from_numpy(gd)
    og = O.Gaussians.from_dict(gd)
    views = [(cam, dev(rgb), dev(dep)) for cam, rgb, dep in targets(og, cams, 64)]
    base = gs.gs_register_gradient(ctx, g, g, [], views)
    for kw in (dict(exposure=1), dict(profile=2), dict(exposure=1, profile=2)):
        got = gs.gs_register_gradient(ctx, g, g, [], views, gs.default_options(**kw))
        np.testing.assert_array_equal(got[0], base[0])
        np.testing.assert_array_equal(got[1], base[1])
