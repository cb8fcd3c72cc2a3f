"""Frame-to-model tracking loss (Eq. 2 with the masks of Supp. A) on the GPU
vs the oracle: rendered FP32 depth, per-view median and inlier mask
bit-exact; loss within 1e-5 relative; cotangents, where the sign of the
error is unambiguous, within 1e-4 relative (the weight alpha^3 comes from
the FP32 transmittance, whose rounding after ~100 contributors reaches
~1e-5 absolute: 3e-5 / alpha relative in alpha^3 for alpha >= 0.3);
tracking registration trajectories within 0.5 mm / 0.01 deg; served
tracking requests equal gs_register with the same options."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2408_10154_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda().contiguous()


def track_hyper():
    hp = json.load(open(os.path.join(GOLDEN, "tracking_hyperparams.json")))
    return hp["lr_rotation"]["ScanNet"], hp["lr_translation"]["ScanNet"]


def targets(og, cams, rng):
    """Targets rendered by the oracle at perturbed poses, with a block of
    pixels without input depth and a few depth outliers."""
    out = []
    for cam in cams:
        r = O.render(og, synth.random_rigid(rng, 2.0, 0.02), cam)
        trgb = r["rgb"].astype(np.float32)
        tdep = r["depth32"].copy()
        H, W = tdep.shape
        tdep[: H // 5, : W // 4] = 0.0
        idx = rng.choice(H * W, max(H * W // 100, 1), replace=False)
        tdep.reshape(-1)[idx] += 3.0
        out.append((trgb, tdep))
    return out


@pytest.mark.parametrize("case", ["ragged", "needles", "room_640x480"])
def test_track_loss_parity(gs, ctx, case):
    if case == "ragged":
        c = synth.small_case(700, 100, 70, 70.0, n_views=3, seed=9, ls_mean=-3.5)
        gd, cams = c["gaussians"], c["cams"]
    elif case == "needles":
        c = synth.small_case(1500, 300, 200, 200.0, n_views=2, seed=21, ls_mean=-3.2, ls_std=0.3)
        gd, cams = c["gaussians"], c["cams"]
    else:
        # a served tracking frame: 640 x 480 (f = 320) from a room keyframe's
        # pose against the 150k-Gaussian room submap
        c = synth.room_150k()
        w2c = np.asarray(c["src_cams"][0][6:], np.float64).reshape(3, 4)
        gd, cams = c["gaussians"], np.stack([synth.camera(320.0, 320.0, 320.0, 240.0, 640, 480, w2c)])
    og = O.Gaussians.from_dict(gd)
    g = gs.Gaussians.from_numpy(gd)
    rng = np.random.default_rng(11)
    poses = np.stack([synth.random_rigid(rng, 3.0, 0.03) for _ in cams])
    tg = targets(og, cams, rng)
    P = dev(poses.reshape(-1, 12))
    out = gs.gs_render(ctx, g, P, cams)
    t_rgb = dev(np.concatenate([t[0].reshape(-1) for t in tg]))
    t_dep = dev(np.concatenate([t[1].reshape(-1) for t in tg]))
    loss, d_rgb, d_dep, inl, med = gs.gs_track_loss(ctx, cams, out["rgb"], out["depth"], out["t_final"], t_rgb, t_dep,
                                                    0.6)
    dep = [v.cpu().numpy() for v in gs.split_views(out["depth"], cams, 1)]
    inl = [v.cpu().numpy() for v in gs.split_views(inl, cams, 1)]
    grgb = [v.cpu().numpy() for v in gs.split_views(d_rgb, cams, 3)]
    gdep = [v.cpu().numpy() for v in gs.split_views(d_dep, cams, 1)]
    loss, med = loss.cpu().numpy(), med.cpu().numpy()
    for k, cam in enumerate(cams):
        r = O.render(og, np.asarray(poses[k], np.float32).astype(np.float64), cam)
        np.testing.assert_array_equal(dep[k].view(np.uint32), r["depth32"].view(np.uint32))
        ref = O.track_loss(r, tg[k][0], tg[k][1], 0.6)
        assert med[k] == np.float32(ref["median"])
        np.testing.assert_array_equal(inl[k].astype(bool), ref["inlier"])
        assert 0.05 < ref["inlier"].mean() < 1.0
        assert abs(loss[k] - ref["loss"]) <= 1e-5 * abs(ref["loss"])
        # cotangents where the sign of the error is unambiguous
        ec = np.abs(r["rgb"] - tg[k][0])
        m = ec > 1e-4
        np.testing.assert_allclose(grgb[k][m], ref["g_rgb"][m], rtol=1e-4, atol=1e-7)
        ed = np.abs(r["depth"] - tg[k][1])
        m = ed > 1e-4
        np.testing.assert_allclose(gdep[k][m], ref["g_depth"][m], rtol=1e-4, atol=1e-7)


def _rot_err(P, T):
    R = np.asarray(P)[:, :3].T @ np.asarray(T)[:, :3]
    return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2)))), float(
        np.linalg.norm(np.asarray(P)[:, 3] - np.asarray(T)[:, 3]))


def tracking_problem(gs, seed):
    c = synth.plain_2k()
    og = O.Gaussians.from_dict(c["gaussians"])
    T = synth.about_point(synth.random_rigid(np.random.default_rng(seed), 0.69, 0.0134),
                          synth.centroid(c["gaussians"]))
    cam = c["cams"][1]
    tr = O.render(og, T, cam)
    g = gs.Gaussians.from_numpy(c["gaussians"])
    return og, g, cam, tr["rgb"].astype(np.float32), tr["depth32"], T


def track_options(gs):
    lr, lt = track_hyper()
    return gs.default_options(tracking_loss=1, lambda_c=0.6, lr_rot=lr, lr_trans=lt)


def test_tracking_registration_matches_oracle(gs, ctx):
    og, g, cam, trgb, tdep, T = tracking_problem(gs, 77)
    opt = track_options(gs)
    iters = 15
    Tg, conf, eps, _ = gs.gs_register(ctx, g, g, [], [(cam, dev(trgb), dev(tdep))], iters, opt)
    hyper = [float(np.float32(v)) for v in (opt.lr_rot, opt.lr_trans, opt.beta1, opt.beta2, opt.adam_eps,
                                            opt.lr_final)]
    Po, eps_o, _ = O.register_view(og, cam, trgb, tdep, iters, hyper=hyper, track_lambda_c=float(np.float32(0.6)))
    ang, dt = _rot_err(Tg, Po)
    assert ang < 0.01 and dt < 5e-4, (ang, dt)
    assert abs(eps[0] - eps_o) <= 1e-3 * eps_o + 1e-6
    # and the pose moved toward the ground truth
    assert _rot_err(Tg, T)[0] < _rot_err(np.eye(3, 4), T)[0]


def test_served_tracking_equals_gs_register(gs, ctx):
    og, g, cam, trgb, tdep, T = tracking_problem(gs, 78)
    view = [(cam, dev(trgb), dev(tdep))]
    topt = track_options(gs)
    ref_t = gs.gs_register(ctx, g, g, [], view, 12, topt)
    ref_r = gs.gs_register(ctx, g, g, [], view, 9)
    srv = gs.Server(0, max_round_iters=4)
    a = srv.submit(g, g, [], view, 12, topt)
    b = srv.submit(g, g, [], view, 9)  # registration loss, server defaults
    while srv.counts()[0] or srv.counts()[1]:
        srv.step()
    for rid, ref in ((a, ref_t), (b, ref_r)):
        res = srv.poll(rid)
        np.testing.assert_array_equal(res["T"], ref[0])
        np.testing.assert_array_equal(res["eps"][:1], ref[2])
    srv.close()
    # a batch mixing the two losses equals the separate calls
    Tb, _, eb = gs.gs_register_batch(ctx, [(g, g, [], view, topt), (g, g, [], view)], 12)
    np.testing.assert_array_equal(Tb[0], ref_t[0])
    np.testing.assert_array_equal(Tb[1], gs.gs_register(ctx, g, g, [], view, 12)[0])


def test_exposure_registration_matches_oracle(gs, ctx):
    # a keyframe whose colours carry another exposure (gain e^0.15, offset
    # -0.03): pose and exposure registered together (Supp. B) on the GPU and
    # in the oracle follow the same trajectory
    c = synth.plain_2k()
    og = O.Gaussians.from_dict(c["gaussians"])
    g = gs.Gaussians.from_numpy(c["gaussians"])
    cam = c["cams"][0]
    tr = O.render(og, c["T_gt"], cam)
    t_rgb = (math.exp(0.15) * tr["rgb"] - 0.03).astype(np.float32)
    t_dep = tr["depth"].astype(np.float32)
    opt = gs.default_options(exposure=1)
    iters = 20
    Tg, conf, eps, _ = gs.gs_register(ctx, g, g, [], [(cam, dev(t_rgb), dev(t_dep))], iters, opt)
    hyper = [float(np.float32(v)) for v in (opt.lr_rot, opt.lr_trans, opt.beta1, opt.beta2, opt.adam_eps,
                                            opt.lr_final)]
    Po, eps_o, _, ab = O.register_view(og, cam, t_rgb, t_dep, iters, hyper=hyper,
                                       lr_exposure=float(np.float32(opt.lr_exposure)))
    ang, dt = _rot_err(Tg, Po)
    assert ang < 0.01 and dt < 5e-4, (ang, dt)
    assert abs(eps[0] - eps_o) <= 2e-3 * eps_o + 1e-6, (eps[0], eps_o)
    # without compensation the residual stays higher
    _, _, eps_plain, _ = gs.gs_register(ctx, g, g, [], [(cam, dev(t_rgb), dev(t_dep))], iters)
    assert eps_plain[0] > 1.2 * eps[0]
    # exposure with the tracking loss is refused
    with pytest.raises(gs.GsError):
        gs.gs_register(ctx, g, g, [], [(cam, dev(t_rgb), dev(t_dep))], 2,
                       gs.default_options(exposure=1, tracking_loss=1))
