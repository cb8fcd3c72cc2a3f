"""Adjoint to every Gaussian parameter (gs_render_backward with parameter
gradients, config 'differentiation check') vs the FP64 oracle's analytic
adjoint, which finite differences pin (tests/test_oracle_pins.py).  Bar:
per parameter group, ||g_gpu - g_oracle|| / ||g_oracle|| <= 1e-3."""
import numpy as np
import pytest

import oracle as O
from paper_2408_10154_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_10154_gb300 as gs
    from paper_2408_10154_gb300 import autograd, build
    build.build()
    O.build()
    ctx = gs.Context(0)
    yield gs, autograd, ctx
    ctx.close()


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


GROUPS = (("means", "means4", 3), ("log_scales", "log_scales4", 3), ("quats", "quats4", 4), ("logits", "logits", 1),
          ("rgb", "rgb4", 3))


def check(env, gd, cams, poses, seed, subset=None):
    gs, autograd, ctx = env
    og = O.Gaussians.from_dict(gd)
    g = gs.Gaussians.from_numpy(gd)
    rng = np.random.default_rng(seed)
    P = dev(poses.reshape(-1, 12))
    out = gs.gs_render(ctx, g, P, cams)
    cr = [rng.standard_normal((3, int(c[5]), int(c[4]))).astype(np.float32) for c in cams]
    cd = [rng.standard_normal((int(c[5]), int(c[4]))).astype(np.float32) for c in cams]
    ca = [rng.standard_normal((int(c[5]), int(c[4]))).astype(np.float32) for c in cams]
    piv = np.stack([O.centroid(og).astype(np.float32)] * len(cams))
    cat = lambda xs: dev(np.concatenate([x.reshape(-1) for x in xs]))
    pg, gr = gs.gs_render_backward(ctx, g, P, cams, out["t_final"], out["last"], cat(cr), cat(cd), cat(ca),
                                   dev(piv), params=True)
    ref = {k: 0.0 for k, _, _ in GROUPS}
    for c, cam in enumerate(cams):
        b = O.backward(og, poses[c].astype(np.float32).astype(np.float64), cam, cr[c].astype(np.float64),
                       cd[c].astype(np.float64), ca[c].astype(np.float64), pivot=piv[c].astype(np.float64))
        for k, _, _ in GROUPS:
            ref[k] = ref[k] + b[k]
        tw = b["twist"]
        assert np.linalg.norm(pg[c].cpu().numpy() - tw) <= 1e-3 * np.linalg.norm(tw)
    idx = np.arange(og.n) if subset is None else subset
    for k, key, K in GROUPS:
        got = gr[key].cpu().numpy()
        got = got[idx] if key == "logits" else got[idx, :K]
        want = ref[k][idx]
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= 1e-3, (k, err)


def test_parameter_adjoint_500_exhaustive(env):
    c = synth.small_case(500, 64, 48, 56.0, n_views=2, seed=1003, ls_mean=-3.0)
    poses = np.stack([synth.random_rigid(np.random.default_rng(3), 3.0, 0.03) for _ in range(2)])
    check(env, c["gaussians"], c["cams"], poses, 4)


def test_parameter_adjoint_300k_subset(env):
    # the differentiation-check workload at full size (300k Gaussians,
    # 1200x680), one keyframe, a random 1 % of the Gaussians compared
    c = synth.diff_check_300k()
    rng = np.random.default_rng(1003)
    sub = rng.choice(c["gaussians"]["means4"].shape[0], 3000, replace=False)
    poses = np.stack([synth.random_rigid(rng, 5.0, 0.05)])
    check(env, c["gaussians"], c["cams"][:1], poses, 5, subset=np.sort(sub))


def test_autograd_function_matches_render_backward(env):
    gs, autograd, ctx = env
    c = synth.small_case(300, 48, 32, 40.0, n_views=1, seed=8)
    g = gs.Gaussians.from_numpy(c["gaussians"])
    leaves = [t.clone().requires_grad_(True) for t in (g.means4, g.log_scales4, g.quats4, g.logits, g.rgb4)]
    gg = gs.Gaussians(*leaves)
    P = dev(np.eye(3, 4).reshape(1, 12))
    rgb, depth, alpha = autograd.rasterize(ctx, gg, P, c["cams"])
    w = torch.randn_like(rgb)
    (w * rgb).sum().backward()
    out = gs.gs_render(ctx, g, P, c["cams"])
    _, gr = gs.gs_render_backward(ctx, g, P, c["cams"], out["t_final"], out["last"], w, torch.zeros_like(depth),
                                  torch.zeros_like(alpha), params=True)
    for leaf, key in zip(leaves, ("means4", "log_scales4", "quats4", "logits", "rgb4")):
        assert torch.equal(leaf.grad, gr[key])


@pytest.mark.parametrize("n,W,H,f,views", [(500, 64, 48, 56.0, 2), (3000, 160, 120, 140.0, 3)])
def test_saved_forward_equals_render_and_backward(env, n, W, H, f, views):
    # gs_render_saved + gs_render_backward_saved (the adjoint from the kept
    # projection and tile lists, no second binning) against gs_render +
    # gs_render_backward: the same renders and gradients, bit for bit
    gs, autograd, ctx = env
    c = synth.small_case(n, W, H, f, n_views=views, seed=n, ls_mean=-3.0)
    g = gs.Gaussians.from_numpy(c["gaussians"])
    rng = np.random.default_rng(n)
    poses = np.stack([synth.random_rigid(rng, 3.0, 0.03) for _ in range(views)])
    P = dev(poses.reshape(-1, 12))
    out = gs.gs_render(ctx, g, P, c["cams"])
    o2, sv = gs.gs_render_saved(ctx, g, P, c["cams"])
    for k in ("rgb", "depth", "alpha"):
        assert torch.equal(out[k], o2[k]), k
    npx = sum(int(cam[4]) * int(cam[5]) for cam in c["cams"])
    cr, cd, ca = (dev(rng.standard_normal(3 * npx)), dev(rng.standard_normal(npx)), dev(rng.standard_normal(npx)))
    piv = dev(np.stack([O.centroid(O.Gaussians.from_dict(c["gaussians"]))] * views))
    pg1, gr1 = gs.gs_render_backward(ctx, g, P, c["cams"], out["t_final"], out["last"], cr, cd, ca, piv, params=True)
    for _ in range(2):  # the saved state serves more than one adjoint
        pg2, gr2 = gs.gs_render_backward_saved(ctx, sv, cr, cd, ca, piv, params=True)
        assert torch.equal(pg1, pg2)
        for k in gr1:
            assert torch.equal(gr1[k], gr2[k]), k
    sv.close()
