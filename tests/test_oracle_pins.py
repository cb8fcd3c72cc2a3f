"""Pins of the FP64 oracle against what the mathematics and the paper fix.

None of these checks re-types the oracle's own formula: each compares it with
a closed form, an invariant, brute force on a tiny input, a library routine
(scipy rotations, numpy SVD / eigendecomposition, Python's stable sort) or a
finite difference.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2408_10154_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_gaussian(mu, log_scale, quat, logit, rgb):
    return O.Gaussians(np.array([[*mu, 0]], np.float32), np.array([[*log_scale, 0]], np.float32),
                       np.array([quat], np.float32), np.array([logit], np.float32),
                       np.array([[*rgb, 0]], np.float32))


def cam_identity(W, H, f, cx, cy):
    return synth.camera(f, f, cx, cy, W, H, np.eye(3, 4))


def logit_of(o):
    return math.log(o / (1 - o))


# --------------------------------------------------------------------------
# FP32 mirror exponential
# --------------------------------------------------------------------------

def test_exp32_against_libm():
    xs = np.concatenate([np.linspace(-80, 80, 4001), np.linspace(-6, 0, 3001), [0.0, -1e-8, 1e-8]])
    worst = 0.0
    for x in xs:
        x32 = float(np.float32(x))
        ref = math.exp(x32)
        got = O.exp32(x32)
        worst = max(worst, abs(got - ref) / ref)
    assert worst < 3e-7, worst
    assert O.exp32(0.0) == 1.0


def test_exp32_at_most_one_for_every_nonpositive_float():
    # exhaustive over the 1.1e9 floats from -0 (0x80000000) to -80
    # (0xC2A00000), plus +0: e^x <= 1 for x <= 0, so x o <= o and a Gaussian
    # whose opacity is at most alpha_max never reaches the alpha clamp
    # (below -80 the argument is clamped to -80)
    prev = O.set_threads(os.cpu_count() or 1)
    try:
        assert O.exp32_count_above_one(0x80000000, 0xC2A00000) == 0
    finally:
        O.set_threads(prev)
    assert O.exp32(0.0) == 1.0
    assert O.exp32_count_above_one(0x00000000, 0x00000000) == 0
    assert O.exp32_count_above_one(0x3F000000, 0x3F000001) == 2  # the scan sees e^0.5 > 1


def test_well_conditioned_conic_exponent_is_never_positive():
    # The compositing walks drop the positive-exponent test for batches whose
    # conics all satisfy ca, cc < -1e-12 and ca cc - cb^2 / 4 >= 1e-6 S^2
    # (S = |ca| + |cb| + |cc|): a negative-definite quadratic form whose FP32
    # evaluation cannot round above 0.  Adversarial sample: conics of every
    # scale and axis ratio, down to and past the criterion's edge, with pixel
    # samples along an eigen-axis (mostly the weak one) from 2^-26 px to
    # 8000 px away.  No conic that passes may give a positive mirror
    # exponent; near-singular and indefinite ones that fail must give some,
    # which shows that the sample reaches the regime.
    rng = np.random.default_rng(7)
    n = 8_000_000
    l1 = np.exp(rng.uniform(-30.0, 5.0, n))
    ratio = np.exp(rng.uniform(-30.0, 0.0, n))
    indef = rng.random(n) < 0.3
    ratio[indef] *= -1e-3
    l2 = l1 * ratio
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    c, s_ = np.cos(th), np.sin(th)
    ca = (-(l1 * c * c + l2 * s_ * s_)).astype(np.float32)
    cc = (-(l1 * s_ * s_ + l2 * c * c)).astype(np.float32)
    cb = (-2.0 * (l1 - l2) * c * s_).astype(np.float32)
    mag = np.exp(rng.uniform(-18.0, 9.0, n))
    d = th + np.where(rng.random(n) < 0.8, 0.5 * np.pi, 0.0) + (rng.random(n) - 0.5) * 1e-3 * rng.random(n)
    ox, oy = mag * np.cos(d), mag * np.sin(d)
    u = 1000.0 * rng.random(n)
    v = 1000.0 * rng.random(n)
    pxf = np.floor(u - ox) + 0.5
    pyf = np.floor(v - oy) + 0.5
    near = rng.random(n) < 0.5  # the mean placed at the exact offset from a pixel centre
    u = np.where(near, pxf + ox, u)
    v = np.where(near, pyf + oy, v)
    f32 = np.float32
    S = np.abs(ca) + np.abs(cb) + np.abs(cc)
    det = ca * cc - f32(0.25) * cb * cb
    ok = (ca < f32(-1e-12)) & (cc < f32(-1e-12)) & (det >= f32(1e-6) * (S * S))
    args = [a.astype(np.float32) for a in (ca, cb, cc, u, v, pxf, pyf)]
    assert ok.sum() > n // 4 and (~ok).sum() > n // 4
    prev = O.set_threads(os.cpu_count() or 1)
    try:
        assert O.count_positive_power(*[a[ok] for a in args]) == 0
        assert O.count_positive_power(*[a[~ok] for a in args]) > 1000
    finally:
        O.set_threads(prev)


def test_exp32_monotone_on_alpha_range():
    xs = np.float32(-6.0) + np.arange(60000, dtype=np.float32) * np.float32(1e-4)
    vals = [O.exp32(float(x)) for x in xs]
    assert all(b >= a for a, b in zip(vals, vals[1:]))


# --------------------------------------------------------------------------
# projection
# --------------------------------------------------------------------------

def test_isotropic_gaussian_on_axis_closed_form():
    # sigma = 0.05 m at z = 2 m, f = 100: 2D variance (f sigma / z)^2 + 0.3
    g = one_gaussian((0, 0, 2.0), [math.log(0.05)] * 3, (1, 0, 0, 0), logit_of(0.6), (0.2, 0.5, 0.9))
    cam = cam_identity(64, 48, 100.0, 32.5, 24.5)
    p = O.project64(g, np.eye(3, 4), cam)[0]
    var = (100 * 0.05 / 2) ** 2 + 0.3
    assert p[0] == pytest.approx(32.5, abs=1e-12) and p[1] == pytest.approx(24.5, abs=1e-12)
    assert p[2] == pytest.approx(2.0, rel=1e-12)
    assert p[3] == pytest.approx(1 / var, rel=1e-6) and p[5] == pytest.approx(1 / var, rel=1e-6)
    assert abs(p[4]) < 1e-12
    assert p[6] == pytest.approx(0.6, rel=1e-6)
    f, i = O.project32(g, np.eye(3, 4), cam)
    r = math.ceil(3 * math.sqrt(var))  # 3 sigma of the larger eigenvalue
    assert i[0, 0] == 1 and i[0, 1] == r
    # tile rect [floor((u-r)/16), floor((u+r)/16)+1) clamped to the 4x3 tile grid
    assert list(i[0, 2:]) == [math.floor((32.5 - r) / 16), math.floor((32.5 + r) / 16) + 1,
                              math.floor((24.5 - r) / 16), min(3, math.floor((24.5 + r) / 16) + 1)]


def test_projection_culls_behind_near_plane():
    g = one_gaussian((0, 0, 0.1), [-3] * 3, (1, 0, 0, 0), 0.0, (1, 1, 1))
    _, i = O.project32(g, np.eye(3, 4), cam_identity(32, 32, 30, 16, 16))
    assert i[0, 0] == 0


def test_covariance_is_rigidly_invariant():
    # eigenvalues of the camera-space covariance = e^{2s} for any pose / view
    rng = np.random.default_rng(3)
    c = synth.small_case(20, 64, 48, 50.0, seed=3)
    g = O.Gaussians.from_dict(c["gaussians"])
    pose = synth.random_rigid(rng, 20.0, 0.1)
    cam = synth.camera(50, 50, 32, 24, 64, 48, synth.random_rigid(rng, 10.0, 0.05))
    p = O.project64(g, pose, cam)
    for k in range(g.n):
        S = np.array([[p[k, 9], p[k, 10], p[k, 11]], [p[k, 10], p[k, 12], p[k, 13]], [p[k, 11], p[k, 13], p[k, 14]]])
        ev = np.sort(np.linalg.eigvalsh(S))
        want = np.sort(np.exp(2 * g.log_scales4[k, :3].astype(np.float64)))
        # the camera rotation is stored in FP32, orthonormal to ~1e-7
        np.testing.assert_allclose(ev, want, rtol=1e-6)


def test_pose_and_view_compose():
    # transforming the Gaussians by P and viewing with the identity camera
    # equals the identity pose seen through world_to_cam = P (FP64 values)
    rng = np.random.default_rng(4)
    c = synth.small_case(30, 64, 48, 50.0, seed=4)
    g = O.Gaussians.from_dict(c["gaussians"])
    P = synth.random_rigid(rng, 7.0, 0.05)
    a = O.project64(g, P, synth.camera(50, 50, 32, 24, 64, 48, np.eye(3, 4)))
    b = O.project64(g, np.eye(3, 4), synth.camera(50, 50, 32, 24, 64, 48, P.astype(np.float32)))
    P32 = P.astype(np.float32).astype(np.float64)
    a2 = O.project64(g, P32, synth.camera(50, 50, 32, 24, 64, 48, np.eye(3, 4)))
    np.testing.assert_allclose(a2[:, :15], b[:, :15], rtol=1e-10, atol=1e-12)
    assert np.abs(a[:, 0] - b[:, 0]).max() < 1e-3  # P vs its FP32 rounding


# --------------------------------------------------------------------------
# compositing
# --------------------------------------------------------------------------

def test_single_gaussian_at_sample_point():
    o, col, z = 0.6, (0.2, 0.5, 0.9), 2.0
    g = one_gaussian((0, 0, z), [math.log(0.05)] * 3, (1, 0, 0, 0), logit_of(o), col)
    cam = cam_identity(64, 48, 100.0, 32.5, 24.5)  # u = 32.5 = sample of pixel (32, 24)
    r = O.render(g, np.eye(3, 4), cam)
    np.testing.assert_allclose(r["rgb"][:, 24, 32], np.array(col) * o, rtol=1e-6)
    assert r["depth"][24, 32] == pytest.approx(o * z, rel=1e-6)
    assert r["alpha"][24, 32] == pytest.approx(o, rel=1e-6)
    assert r["t_final"][24, 32] == pytest.approx(1 - o, rel=1e-6)
    assert r["last"][24, 32] == 1
    # neighbours: alpha = o exp(-d^2 / (2 var)) (isotropic), when >= 1/255
    var = (100 * 0.05 / 2) ** 2 + 0.3
    for (px, py) in [(33, 24), (30, 24), (32, 27), (35, 21)]:
        d2 = (px - 32) ** 2 + (py - 24) ** 2
        a = o * math.exp(-0.5 * d2 / var)
        assert r["alpha"][py, px] == pytest.approx(a, rel=1e-6)


def test_two_gaussians_front_to_back():
    # same screen position, depths 2 and 3; the back one is listed first
    of, ob, cf, cb = 0.7, 0.5, (1.0, 0.2, 0.1), (0.1, 0.3, 0.9)
    g = O.Gaussians(np.array([[0, 0, 3.0, 0], [0, 0, 2.0, 0]], np.float32),
                    np.full((2, 4), math.log(0.05), np.float32), np.array([[1, 0, 0, 0]] * 2, np.float32),
                    np.array([logit_of(ob), logit_of(of)], np.float32),
                    np.array([[*cb, 0], [*cf, 0]], np.float32))
    r = O.render(g, np.eye(3, 4), cam_identity(64, 48, 100.0, 32.5, 24.5))
    want = np.array(cf) * of + np.array(cb) * ob * (1 - of)
    np.testing.assert_allclose(r["rgb"][:, 24, 32], want, rtol=1e-6)
    assert r["depth"][24, 32] == pytest.approx(2.0 * of + 3.0 * ob * (1 - of), rel=1e-6)
    assert r["t_final"][24, 32] == pytest.approx((1 - of) * (1 - ob), rel=1e-6)


def test_early_stop_and_clamp():
    # 8 stacked opaque splats (o = 0.8): T = 0.2^k; the 6th would bring T to
    # 6.4e-5 < 1e-4, so exactly 5 contribute.  Colours differ per layer.
    n = 8
    means = np.array([[0, 0, 2.0 + 0.1 * k, 0] for k in range(n)], np.float32)
    cols = np.array([[k / n, 1 - k / n, 0.5, 0] for k in range(n)], np.float32)
    g = O.Gaussians(means, np.full((n, 4), math.log(0.05), np.float32), np.array([[1, 0, 0, 0]] * n, np.float32),
                    np.full(n, logit_of(0.8), np.float32), cols)
    r = O.render(g, np.eye(3, 4), cam_identity(64, 48, 100.0, 32.5, 24.5))
    assert r["last"][24, 32] == 5
    want = sum(cols[k, :3] * 0.8 * 0.2 ** k for k in range(5))
    np.testing.assert_allclose(r["rgb"][:, 24, 32], want, rtol=1e-6)
    assert r["t_final"][24, 32] == pytest.approx(0.2 ** 5, rel=1e-6)
    # opacity above 0.99 is clamped: alpha = 0.99 exactly at the sample point
    g1 = one_gaussian((0, 0, 2.0), [math.log(0.05)] * 3, (1, 0, 0, 0), 8.0, (1, 1, 1))
    r1 = O.render(g1, np.eye(3, 4), cam_identity(64, 48, 100.0, 32.5, 24.5))
    assert r1["alpha"][24, 32] == pytest.approx(0.99, abs=1e-7)


def smooth_bruteforce(g, pose, cam):
    """Front-to-back compositing over ALL visible Gaussians sorted by
    (FP32 depth, index), with no tiles and no thresholds (smooth mode)."""
    p64 = O.project64(g, pose, cam, O.SMOOTH_OPT)
    f32, i32 = O.project32(g, pose, cam, O.SMOOTH_OPT)
    vis = np.nonzero(i32[:, 0])[0]
    order = vis[np.lexsort((vis, f32[vis, 2].view(np.uint32)))]
    W, H = int(cam[4]), int(cam[5])
    ys, xs = np.mgrid[0:H, 0:W]
    T = np.ones((H, W))
    C = np.zeros((3, H, W))
    D = np.zeros((H, W))
    for k in order:
        U, V, z, A, B, Cc, o = p64[k, :7]
        dx, dy = U - (xs + 0.5), V - (ys + 0.5)
        a = o * np.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
        C += g.rgb4[k, :3, None, None] * (a * T)
        D += z * a * T
        T = T * (1 - a)
    return C, D, T


def test_smooth_render_equals_bruteforce():
    c = synth.small_case(40, 48, 32, 40.0, seed=11, ls_mean=-2.5)
    g = O.Gaussians.from_dict(c["gaussians"])
    pose = synth.random_rigid(np.random.default_rng(1), 4.0, 0.03)
    r = O.render(g, pose, c["cams"][0], O.SMOOTH_OPT)
    C, D, T = smooth_bruteforce(g, pose, c["cams"][0])
    np.testing.assert_allclose(r["rgb"], C, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r["depth"], D, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(r["t_final"], T, rtol=1e-10, atol=1e-12)


def test_smooth_render_is_independent_of_tile_size():
    c = synth.small_case(40, 48, 32, 40.0, seed=12, ls_mean=-2.5)
    g = O.Gaussians.from_dict(c["gaussians"])
    big = O.SMOOTH_OPT.copy()
    big[0] = 64
    a = O.render(g, np.eye(3, 4), c["cams"][0], O.SMOOTH_OPT)
    b = O.render(g, np.eye(3, 4), c["cams"][0], big)
    for k in ("rgb", "depth", "t_final"):
        np.testing.assert_array_equal(a[k], b[k])


def test_transmittance_monotone_and_product():
    # along any pixel, adding Gaussians behind can only lower T; alpha = 1 - T
    c = synth.small_case(200, 64, 48, 50.0, seed=13)
    g = O.Gaussians.from_dict(c["gaussians"])
    r = O.render(g, np.eye(3, 4), c["cams"][0])
    assert np.all(r["t_final"] <= 1.0) and np.all(r["t_final"] > 0)
    np.testing.assert_allclose(r["alpha"], 1 - r["t_final"], atol=1e-15)
    half = O.Gaussians(g.means4[:100], g.log_scales4[:100], g.quats4[:100], g.logits[:100], g.rgb4[:100])
    r2 = O.render(half, np.eye(3, 4), c["cams"][0], O.SMOOTH_OPT)
    r3 = O.render(g, np.eye(3, 4), c["cams"][0], O.SMOOTH_OPT)
    assert np.all(r3["t_final"] <= r2["t_final"] + 1e-15)


# --------------------------------------------------------------------------
# binning: brute force over (tile, Gaussian) pairs, Python's stable sort
# --------------------------------------------------------------------------

def test_binning_matches_bruteforce():
    c = synth.small_case(300, 80, 56, 60.0, n_views=3, seed=21)
    g = O.Gaussians.from_dict(c["gaussians"])
    rng = np.random.default_rng(2)
    poses = np.stack([synth.random_rigid(rng, 3.0, 0.02) for _ in range(3)])
    keys, vals, ranges = O.bin_tiles(g, poses, c["cams"])
    bk, bv = [], []
    tile_base = 0
    for cam_i, cam in enumerate(c["cams"]):
        f, i = O.project32(g, poses[cam_i], cam)
        TX = (int(cam[4]) + 15) // 16
        pairs = []
        for k in range(g.n):
            if not i[k, 0]:
                continue
            zb = int(np.float32(f[k, 2]).view(np.uint32))
            for ty in range(i[k, 4], i[k, 5]):
                for tx in range(i[k, 2], i[k, 3]):
                    pairs.append((((tile_base + ty * TX + tx) << 32) | zb, cam_i * g.n + k))
        pairs = sorted(pairs, key=lambda kv: kv[0])  # stable: ties keep emission order
        bk += [p[0] for p in pairs]
        bv += [p[1] for p in pairs]
        tile_base += O.n_tiles(cam)
    np.testing.assert_array_equal(keys, np.array(bk, np.uint64))
    np.testing.assert_array_equal(vals, np.array(bv, np.uint32))
    tiles = np.array(bk, np.uint64) >> np.uint64(32)
    for t in range(len(ranges)):
        idx = np.nonzero(tiles == t)[0]
        want = (idx[0], idx[-1] + 1) if len(idx) else (0, 0)
        assert tuple(ranges[t]) == want
    # second opinion: numpy's stable argsort of the emitted keys
    order = np.argsort(np.array([p for p in bk], np.uint64), kind="stable")
    np.testing.assert_array_equal(order, np.arange(len(bk)))


@pytest.mark.parametrize("opt", ["tight", "loose"])
def test_binning_matches_bruteforce_both_rectangles(opt):
    # the brute force above reads the rectangles of project32; here the two
    # rectangle rules side by side: the tight lists are the 3-sigma lists
    # with the dropped (tile, record) pairs removed, order kept
    c = synth.small_case(300, 80, 56, 60.0, n_views=2, seed=22)
    g = O.Gaussians.from_dict(c["gaussians"])
    rng = np.random.default_rng(3)
    poses = np.stack([synth.random_rigid(rng, 3.0, 0.02) for _ in range(2)])
    o = O.DEFAULT_OPT if opt == "tight" else O.LOOSE_OPT
    keys, vals, ranges = O.bin_tiles(g, poses, c["cams"], o)
    lk, lv, _ = O.bin_tiles(g, poses, c["cams"], O.LOOSE_OPT)
    loose = list(zip(lk.tolist(), lv.tolist()))
    tight = list(zip(keys.tolist(), vals.tolist()))
    keep = set(tight)
    assert [kv for kv in loose if kv in keep] == tight  # a subsequence of the 3-sigma lists
    if opt == "tight":
        assert len(tight) < len(loose)


# --------------------------------------------------------------------------
# tight tile rectangles: the FP32 logarithm, and what the rectangles drop
# --------------------------------------------------------------------------

def test_log32_against_libm():
    xs = np.concatenate([np.logspace(-37, 0, 4001), np.linspace(0.5, 2.0, 3001), [1.0 / 255.0, 1.0]])
    worst = 0.0
    for x in xs:
        x32 = float(np.float32(x))
        ref = math.log(x32)
        worst = max(worst, abs(O.log32(x32) - ref) / max(1.0, abs(ref)))
    assert worst < 3e-7, worst
    assert O.log32(1.0) == 0.0


def _needle_scene(n, W, H, f, seed):
    # needle-shaped splats (one axis x4.5, one x0.08) in all orientations,
    # half of them with opacities near alpha_min: where a threshold box is
    # closest to the pixels it must keep
    c = synth.small_case(n, W, H, f, n_views=2, seed=seed, ls_mean=-3.2, ls_std=0.3)
    g = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    rng = np.random.default_rng(seed)
    g["log_scales4"][:, 0] += 1.5
    g["log_scales4"][:, 1] -= 2.5
    near = rng.random(n) < 0.5
    g["logits"][near] = rng.normal(-5.55, 0.15, int(near.sum()))
    return O.Gaussians.from_dict(g), c["cams"]


def _scenes():
    yield _needle_scene(1200, 240, 160, 160.0, 21)
    c = synth.small_case(900, 120, 90, 100.0, n_views=2, seed=23, ls_mean=-3.0)
    yield O.Gaussians.from_dict(c["gaussians"]), c["cams"]


def test_tight_rectangles_drop_only_tiles_below_alpha_min():
    # FP64 check of every dropped (record, tile) pair: at each pixel centre
    # of the tile the exact alpha o e^power of the FP64 projection stays
    # below alpha_min e^-0.05 (the rectangle's margin is 0.06 in the
    # exponent); the tight rectangle lies inside the 3-sigma one
    amin = float(O.DEFAULT_OPT[3])
    dropped = 0
    for g, cams in _scenes():
        rng = np.random.default_rng(7)
        for cam in cams:
            pose = synth.random_rigid(rng, 3.0, 0.03)
            _, it = O.project32(g, pose, cam, O.DEFAULT_OPT)
            _, il = O.project32(g, pose, cam, O.LOOSE_OPT)
            p64 = O.project64(g, pose, cam)
            W, H = int(cam[4]), int(cam[5])
            assert np.all(il[it[:, 0] == 1, 0] == 1)
            for k in np.nonzero(il[:, 0] == 1)[0]:
                x0, x1, y0, y1 = il[k, 2:6]
                if it[k, 0]:
                    a0, a1, b0, b1 = it[k, 2:6]
                    assert x0 <= a0 < a1 <= x1 and y0 <= b0 < b1 <= y1
                else:
                    a0 = a1 = b0 = b1 = 0
                px = np.arange(16 * x0, min(16 * x1, W))
                py = np.arange(16 * y0, min(16 * y1, H))
                X, Y = np.meshgrid(px, py)
                tx, ty = X // 16, Y // 16
                out = ~((tx >= a0) & (tx < a1) & (ty >= b0) & (ty < b1))
                if not out.any():
                    continue
                U, V, _, A, B, C, o = p64[k, :7]
                dx, dy = U - (X + 0.5), V - (Y + 0.5)
                alpha = o * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
                assert alpha[out].max() < amin * math.exp(-0.05), (k, alpha[out].max())
                dropped += int(len(set(zip(tx[out].ravel(), ty[out].ravel()))))
    assert dropped > 500, dropped


def test_tight_lists_render_identically_to_3sigma_lists():
    # every pair the tight lists drop fails the FP32 alpha test at every
    # pixel: the same contributors in the same order, so the FP32 final
    # transmittance and the FP64 colour and depth are bit-equal; only list
    # positions (last) move forward
    for g, cams in _scenes():
        rng = np.random.default_rng(8)
        for cam in cams:
            pose = synth.random_rigid(rng, 3.0, 0.03)
            rt = O.render(g, pose, cam, O.DEFAULT_OPT)
            rl = O.render(g, pose, cam, O.LOOSE_OPT)
            np.testing.assert_array_equal(rt["t_final32"].view(np.uint32), rl["t_final32"].view(np.uint32))
            np.testing.assert_array_equal(rt["rgb"], rl["rgb"])
            np.testing.assert_array_equal(rt["depth"], rl["depth"])
            assert np.all(rt["last"] <= rl["last"]) and np.any(rt["last"] < rl["last"])


def test_tight_lists_shrink_the_room_lists():
    c = synth.room_150k()
    g = O.Gaussians.from_dict(c["gaussians"])
    cams = c["src_cams"][:2]
    poses = np.stack([np.eye(3, 4)] * 2)
    kt, _, _ = O.bin_tiles(g, poses, cams, O.DEFAULT_OPT)
    kl, _, _ = O.bin_tiles(g, poses, cams, O.LOOSE_OPT)
    assert len(kt) < 0.8 * len(kl), (len(kt), len(kl))


# --------------------------------------------------------------------------
# loss
# --------------------------------------------------------------------------

def test_l1_loss_closed_form():
    rng = np.random.default_rng(5)
    H, W = 3, 4
    rgb = rng.uniform(size=(3, H, W))
    dep = rng.uniform(1, 3, size=(H, W))
    t_rgb = rgb.copy()
    t_rgb[0, 0, 0] += 0.5
    t_rgb[1, 2, 3] -= 0.25
    t_dep = dep + 0.1
    t_dep[1, 1] = dep[1, 1]  # equal pixel: zero subgradient
    L, gr, gd = O.loss(rgb, dep, t_rgb, t_dep)
    assert L == pytest.approx((0.5 + 0.25) / (3 * H * W) + 0.1 * (H * W - 1) / (H * W), rel=1e-9)
    assert gr[0, 0, 0] == pytest.approx(-1 / (3 * H * W)) and gr[1, 2, 3] == pytest.approx(1 / (3 * H * W))
    assert np.count_nonzero(gr) == 2
    assert gd[1, 1] == 0 and gd[0, 0] == pytest.approx(-1 / (H * W))


def test_self_rendered_target_gives_zero_loss_and_gradient():
    c = synth.small_case(150, 64, 48, 50.0, seed=31)
    g = O.Gaussians.from_dict(c["gaussians"])
    pose = synth.random_rigid(np.random.default_rng(6), 2.0, 0.01)
    r = O.render(g, pose, c["cams"][0])
    L, gr, gd = O.loss(r["rgb"], r["depth"], r["rgb"], r["depth"])
    assert L == 0.0
    b = O.backward(g, pose, c["cams"][0], gr, gd, pivot=O.centroid(g))
    assert np.all(b["twist"] == 0.0)
    for k in ("means", "log_scales", "quats", "logits", "rgb"):
        assert np.all(b[k] == 0.0)


# --------------------------------------------------------------------------
# adjoint: central finite differences in FP64 (smooth mode)
# --------------------------------------------------------------------------

def _fd_setup(n, W, H, f, seed):
    c = synth.small_case(n, W, H, f, seed=seed, ls_mean=-2.5)
    g = O.Gaussians.from_dict(c["gaussians"])
    rng = np.random.default_rng(seed + 100)
    cot = (rng.standard_normal((3, H, W)), rng.standard_normal((H, W)), rng.standard_normal((H, W)))
    pose = synth.random_rigid(rng, 2.0, 0.02)
    return g, c["cams"][0], cot, pose


def _objective(g, pose, cam, cot, opt):
    r = O.render(g, pose, cam, opt)
    return float((cot[0] * r["rgb"]).sum() + (cot[1] * r["depth"]).sum() + (cot[2] * r["alpha"]).sum())


FIELDS = (("means", "means4", 3), ("log_scales", "log_scales4", 3), ("quats", "quats4", 4),
          ("logits", "logits", 1), ("rgb", "rgb4", 3))


def _fd_param(g, pose, cam, cot, opt, field, i, k, h):
    arrs = {a: getattr(g, a) for _, a, _ in FIELDS}
    vals, xs = [], []
    for s in (1, -1):
        d = {a: v.copy() for a, v in arrs.items()}
        if field == "logits":
            d[field][i] = np.float32(float(d[field][i]) + s * h)
            xs.append(float(d[field][i]))
        else:
            d[field][i, k] = np.float32(float(d[field][i, k]) + s * h)
            xs.append(float(d[field][i, k]))
        vals.append(_objective(O.Gaussians(d["means4"], d["log_scales4"], d["quats4"], d["logits"], d["rgb4"]),
                               pose, cam, cot, opt))
    return (vals[0] - vals[1]) / (xs[0] - xs[1])


def test_adjoint_matches_finite_differences_exhaustive_small():
    g, cam, cot, pose = _fd_setup(24, 24, 16, 20.0, seed=41)
    b = O.backward(g, pose, cam, *cot, pivot=O.centroid(g), opt=O.SMOOTH_OPT)
    for name, field, K in FIELDS:
        an = b[name].reshape(g.n, -1)
        scale = np.abs(an).max()
        for i in range(g.n):
            for k in range(K):
                fd = _fd_param(g, pose, cam, cot, O.SMOOTH_OPT, field, i, k, 1e-3 if name != "means" else 2e-4)
                assert abs(fd - an[i, k]) <= 2e-3 * max(abs(an[i, k]), 0.02 * scale), (name, i, k, fd, an[i, k])


def test_adjoint_matches_finite_differences_500_subset():
    g, cam, cot, pose = _fd_setup(500, 64, 48, 56.0, seed=42)
    b = O.backward(g, pose, cam, *cot, pivot=O.centroid(g), opt=O.SMOOTH_OPT)
    rng = np.random.default_rng(1003)
    bad = []
    for name, field, K in FIELDS:
        an = b[name].reshape(g.n, -1)
        scale = np.abs(an).max()
        for i in rng.choice(g.n, 6, replace=False):
            for k in range(K):
                fd = _fd_param(g, pose, cam, cot, O.SMOOTH_OPT, field, i, k, 1e-3 if name != "means" else 2e-4)
                if abs(fd - an[i, k]) > 2e-3 * max(abs(an[i, k]), 0.02 * scale):
                    bad.append((name, i, k, fd, an[i, k]))
    assert not bad, bad


def _threshold_scene():
    # 40 Gaussians of ~2.5 px in front of a 40 x 30 image (2 x 3 tiles,
    # ragged): a third nearly opaque (o ~ 0.996: clamped at alpha_max near
    # their centres, and stacks of them stop early on t_min), a third with
    # opacities near alpha_min, a third ordinary; grey background
    c = synth.small_case(40, 40, 30, 60.0, seed=44, ls_mean=-2.5, ls_std=0.2, half=0.25)
    d = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    rng = np.random.default_rng(44)
    kind = np.arange(40) % 3
    d["logits"][kind == 0] = rng.normal(5.5, 0.3, int((kind == 0).sum()))
    d["logits"][kind == 1] = rng.normal(-5.4, 0.2, int((kind == 1).sum()))
    opt = O.DEFAULT_OPT.copy()
    opt[6:9] = (0.3, 0.5, 0.7)
    cam = c["cams"][0]
    H, W = int(cam[5]), int(cam[4])
    cot = (rng.standard_normal((3, H, W)), rng.standard_normal((H, W)), rng.standard_normal((H, W)))
    return O.Gaussians.from_dict(d), cam, cot, np.eye(3, 4), opt


def test_adjoint_matches_finite_differences_with_thresholds_on():
    # alpha_min, alpha_max and t_min active, a non-zero background: central
    # differences on every parameter whose +h and -h renders keep the same
    # contributor sequence (alpha test, clamp and early stop) at every pixel
    g, cam, cot, pose, opt = _threshold_scene()
    # the scene exercises what the thresholds change: early stops (the
    # final transmittance differs without t_min), clamps (it differs with
    # alpha_max = 1) and the alpha test (with alpha_min = 0)
    base = O.render(g, pose, cam, opt)
    for k, v in ((5, 0.0), (4, 1.0), (3, 0.0)):
        o2 = opt.copy()
        o2[k] = v
        if k == 3:
            o2[10] = 0.0  # no alpha threshold: 3-sigma rectangles
        assert np.any(O.render(g, pose, cam, o2)["t_final32"] != base["t_final32"]), k
    sig0 = O.contrib_sig(g, pose, cam, opt)
    b = O.backward(g, pose, cam, *cot, pivot=O.centroid(g), opt=opt)
    arrs = {a: getattr(g, a) for _, a, _ in FIELDS}
    tested, bad = 0, []
    for name, field, K in FIELDS:
        an = b[name].reshape(g.n, -1)
        scale = np.abs(an).max()
        h = 2e-4 if name == "means" else 1e-3
        for i in range(g.n):
            for k in range(K):
                same = True
                for sgn in (1, -1):
                    d = {a: v.copy() for a, v in arrs.items()}
                    if field == "logits":
                        d[field][i] = np.float32(float(d[field][i]) + sgn * h)
                    else:
                        d[field][i, k] = np.float32(float(d[field][i, k]) + sgn * h)
                    gp = O.Gaussians(d["means4"], d["log_scales4"], d["quats4"], d["logits"], d["rgb4"])
                    same = same and np.array_equal(O.contrib_sig(gp, pose, cam, opt), sig0)
                if not same:
                    continue
                fd = _fd_param(g, pose, cam, cot, opt, field, i, k, h)
                tested += 1
                if abs(fd - an[i, k]) > 2e-3 * max(abs(an[i, k]), 0.02 * scale):
                    bad.append((name, i, k, fd, an[i, k]))
    assert not bad, bad
    assert tested >= 300, tested


def _twist_pose(pose, xi, pivot):
    """Left perturbation about ``pivot``: x -> exp(w)(x - c) + c + v, with
    exp from scipy's rotation-vector map."""
    Rd = Rotation.from_rotvec(xi[:3]).as_matrix()
    R, t = pose[:, :3], pose[:, 3]
    return np.concatenate([Rd @ R, (Rd @ (t - pivot) + pivot + xi[3:])[:, None]], axis=1)


def test_twist_gradient_matches_finite_differences():
    # smooth mode only: with the alpha / transmittance thresholds on, any pose
    # perturbation moves some pixel across a threshold and the loss jumps
    opt = O.SMOOTH_OPT
    g, cam, cot, pose = _fd_setup(80, 48, 32, 40.0, seed=43)
    pivot = O.centroid(g) + np.array([0.05, -0.02, 0.1])
    b = O.backward(g, pose, cam, *cot, pivot=pivot, opt=opt)
    h = 1e-4
    fd = np.zeros(6)
    for k in range(6):
        xp = np.zeros(6)
        xp[k] = h
        fd[k] = (_objective(g, _twist_pose(pose, xp, pivot), cam, cot, opt)
                 - _objective(g, _twist_pose(pose, -xp, pivot), cam, cot, opt)) / (2 * h)
    err = np.linalg.norm(fd - b["twist"]) / np.linalg.norm(b["twist"])
    assert err < 2e-3, (fd, b["twist"])


def test_clamped_alpha_has_zero_opacity_gradient():
    # o = sigmoid(8) > 0.99: alpha is clamped at the centre pixel only
    g = one_gaussian((0, 0, 2.0), [math.log(0.02)] * 3, (1, 0, 0, 0), 8.0, (0.4, 0.6, 0.8))
    cam = cam_identity(16, 16, 100.0, 8.5, 8.5)
    cot = np.zeros((3, 16, 16))
    cot[0, 8, 8] = 1.0
    b = O.backward(g, np.eye(3, 4), cam, cot_rgb=cot, pivot=np.zeros(3))
    assert b["logits"][0] == 0.0 and np.all(b["means"] == 0.0)
    assert b["rgb"][0, 0] == pytest.approx(0.99, abs=1e-7)


# --------------------------------------------------------------------------
# pose update, registration, fusion, rigid transform
# --------------------------------------------------------------------------

def test_first_adam_step_closed_form():
    grad = np.array([0.3, -2.0, 0.5, 1e-3, -4.0, 0.7])
    pivot = np.array([0.2, -0.1, 2.5])
    hyper = O.DEFAULT_HYPER
    pose, state = O.pose_step(np.eye(3, 4), np.zeros(13), grad, pivot, 0, 50)
    # first step: bias-corrected m/sqrt(v) = sign(g) |g|/(|g|+eps); schedule(0) = 1
    step = np.concatenate([np.full(3, hyper[0]), np.full(3, hyper[1])]) * grad / (np.abs(grad) + hyper[4])
    Rd = Rotation.from_rotvec(-step[:3]).as_matrix()
    want_t = Rd @ (-pivot) + pivot - step[3:]
    np.testing.assert_allclose(pose[:, :3], Rd, atol=1e-14)
    np.testing.assert_allclose(pose[:, 3], want_t, atol=1e-14)
    assert state[12] == 1.0


def test_cosine_schedule_reaches_final_fraction():
    # a constant gradient keeps m/sqrt(v) = 1 after bias correction, so the
    # k-th step length is lr * (f + (1-f) (1 + cos(pi k / K)) / 2)
    K, hyper = 10, O.DEFAULT_HYPER
    grad = np.array([0, 0, 0, 1.0, 0, 0])
    pose, state = np.eye(3, 4), np.zeros(13)
    for k in range(K):
        prev = pose[0, 3]
        pose, state = O.pose_step(pose, state, grad, np.zeros(3), k, K)
        sched = hyper[5] + (1 - hyper[5]) * 0.5 * (1 + math.cos(math.pi * k / K))
        assert prev - pose[0, 3] == pytest.approx(hyper[1] * sched, rel=1e-6)


def _rot_err(P, T):
    R = P[:, :3].T @ T[:, :3]
    ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2))))
    return ang, float(np.linalg.norm(P[:, 3] - T[:, 3]))


def test_registration_recovers_known_transform():
    # plain 2k workload, two of its four keyframes, 50 iterations each
    c = synth.plain_2k()
    g = O.Gaussians.from_dict(c["gaussians"])
    T = c["T_gt"]
    for k in (0, 3):
        tr = O.render(g, T, c["cams"][k])
        P, eps, hist = O.register_view(g, c["cams"][k], tr["rgb"], tr["depth"], 50, history=True)
        ang, dt = _rot_err(P, T)
        assert ang < 0.005 and dt < 2e-4, (k, ang, dt)
        assert eps < 0.01 * hist[0]


def test_fused_registration_meets_the_convergence_precheck():
    # the plain 2k workload with its four keyframes, 50 iterations each,
    # fused by Eq. 7: the fused estimate recovers the known transform within
    # 0.1 mm / 0.002 deg, the pre-check the registration parity bar rests on
    # (each keyframe alone is within 0.005 deg / 0.2 mm, three of the four
    # within the pre-check too)
    O.set_threads(os.cpu_count() or 1)  # results do not depend on the thread count
    c = synth.plain_2k()
    g = O.Gaussians.from_dict(c["gaussians"])
    T = c["T_gt"]
    ests, epss, tight = [], [], 0
    for cam in c["cams"]:
        tr = O.render(g, T, cam)
        P, eps, _ = O.register_view(g, cam, tr["rgb"], tr["depth"], 50)
        ang, dt = _rot_err(P, T)
        assert ang < 0.005 and dt < 2e-4, (ang, dt)
        tight += ang < 0.002 and dt < 1e-4
        ests.append(P)
        epss.append(eps)
    assert tight >= 3
    Tf, _ = O.fuse(np.stack(ests), epss, [False] * 4)
    ang, dt = _rot_err(Tf, T)
    assert ang < 0.002 and dt < 1e-4, (ang, dt)


def test_fuse_closed_forms():
    rng = np.random.default_rng(7)
    T = synth.random_rigid(rng, 20.0, 0.3)
    # identical estimates -> the same transform; confidence = mean weight
    Tf, conf = O.fuse(np.stack([T, T, T]), [0.1, 0.2, 0.4], [False] * 3)
    np.testing.assert_allclose(Tf, T, atol=1e-12)
    assert conf == pytest.approx(np.mean([10, 5, 2.5]))
    # a reverse estimate is inverted before averaging
    Tf, _ = O.fuse(np.stack([T, synth.inverse(T)]), [0.1, 0.1], [False, True])
    np.testing.assert_allclose(Tf, T, atol=1e-12)
    # two rotations about one axis, equal weights -> the geodesic midpoint
    ax = np.array([0.3, -0.5, 0.8])
    ax /= np.linalg.norm(ax)
    A = np.concatenate([Rotation.from_rotvec(ax * 0.2).as_matrix(), [[0.0], [0.0], [0.0]]], axis=1)
    B = np.concatenate([Rotation.from_rotvec(ax * 0.6).as_matrix(), [[1.0], [0.0], [0.0]]], axis=1)
    Tf, _ = O.fuse(np.stack([A, B]), [0.5, 0.5], [False, False])
    np.testing.assert_allclose(Tf[:, :3], Rotation.from_rotvec(ax * 0.4).as_matrix(), atol=1e-12)
    np.testing.assert_allclose(Tf[:, 3], [0.5, 0, 0], atol=1e-12)
    # a near-zero residual dominates; the result is a proper rotation
    Tf, _ = O.fuse(np.stack([A, B]), [1e-9, 1.0], [False, False])
    assert np.linalg.det(Tf[:, :3]) == pytest.approx(1.0)
    np.testing.assert_allclose(Tf[:, :3], A[:, :3], atol=1e-7)


def test_rigid_transform_preserves_renders():
    # Eq. 8/9: render(T G, camera moved by T) = render(G, camera)
    c = synth.small_case(120, 64, 48, 50.0, seed=51)
    g = O.Gaussians.from_dict(c["gaussians"])
    T = synth.random_rigid(np.random.default_rng(8), 25.0, 0.2)
    gt = O.transform(g, T)
    cam2 = synth.moved_cameras(c["cams"], T)[0]
    a = O.render(g, np.eye(3, 4), c["cams"][0], O.SMOOTH_OPT)
    b = O.render(gt, np.eye(3, 4), cam2, O.SMOOTH_OPT)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=2e-4)
    np.testing.assert_allclose(a["depth"], b["depth"], atol=2e-4)
    # the quaternion of each transformed Gaussian is R q (scipy composition)
    want = (Rotation.from_matrix(T[:, :3]) * Rotation.from_quat(g.quats4[:, [1, 2, 3, 0]].astype(np.float64)))
    got = Rotation.from_quat(gt.quats4[:, [1, 2, 3, 0]].astype(np.float64))
    assert np.max((want.inv() * got).magnitude()) < 1e-6


def test_default_learning_rates_follow_the_paper():
    hp = json.load(open(os.path.join(GOLDEN, "loop_closure_hyperparams.json")))
    # real-data column (TUM-RGBD / ScanNet / ScanNet++) is the default
    assert O.DEFAULT_HYPER[0] == hp["lr_rotation"]["ScanNet"]
    assert O.DEFAULT_HYPER[1] == hp["lr_translation"]["ScanNet"]


# ----------------------------------------------------------------- tracking loss (Eq. 2, Supp. A)
def _fake_render(depth, tf, rgb=None):
    depth = np.asarray(depth, np.float64)
    H, W = depth.shape
    return dict(rgb=np.zeros((3, H, W)) if rgb is None else np.asarray(rgb, np.float64), depth=depth,
                t_final=np.asarray(tf, np.float64), depth32=depth.astype(np.float32))


def test_track_loss_median_inliers_and_depth_weight():
    # 2x3 image, alpha = 1 everywhere (T_final = 0), colours exact; depth
    # errors 0.25, 0.5, 0.75, 1.0, 50 and one pixel without input depth.
    # Valid errors sorted: 0.25 0.5 0.75 1 50 -> lower median 0.75, threshold
    # 37.5: the 50 error is an outlier.  Loss = (1 - 0.6) * (0.25 + 0.5 + 0.75 + 1) = 1.
    t_depth = np.array([[2.0, 2.0, 2.0], [2.0, 2.0, 0.0]], np.float32)
    depth = np.array([[2.25, 1.5, 2.75], [3.0, 52.0, 7.0]])
    r = _fake_render(depth, np.zeros((2, 3)))
    out = O.track_loss(r, np.zeros((3, 2, 3), np.float32), t_depth, 0.6)
    assert out["median"] == 0.75
    np.testing.assert_array_equal(out["inlier"], [[True, True, True], [True, False, False]])
    assert abs(out["loss"] - 1.0) < 1e-12
    np.testing.assert_allclose(out["g_depth"], [[0.4, -0.4, 0.4], [0.4, 0.0, 0.0]], atol=1e-12)
    assert not out["g_rgb"].any()  # colour errors are zero: sign(0) = 0


def test_track_loss_alpha_cube_and_colour_weight():
    # one pixel, alpha = 0.5 (weight 1/8), colour errors (0.5, -1, 0), depth exact:
    # loss = 1/8 * 0.6 * 1.5 = 0.1125; dL/dI = 1/8 * 0.6 * sign = (0.075, -0.075, 0)
    r = _fake_render([[2.0]], [[0.5]], rgb=np.array([0.5, 0.0, 0.25]).reshape(3, 1, 1))
    t_rgb = np.array([0.0, 1.0, 0.25], np.float32).reshape(3, 1, 1)
    out = O.track_loss(r, t_rgb, np.array([[2.0]], np.float32), 0.6)
    assert out["median"] == 0.0 and out["inlier"][0, 0]
    assert abs(out["loss"] - 0.1125) < 1e-12
    np.testing.assert_allclose(out["g_rgb"].reshape(3), [0.075, -0.075, 0.0], atol=1e-15)
    assert out["g_depth"][0, 0] == 0.0


def test_track_loss_even_count_zero_median_and_no_valid_depth():
    # even count: errors 1 2 3 4 -> lower median 2 (rank 1), all inliers
    t = np.full((1, 4), 1.0, np.float32)
    r = _fake_render([[2.0, 3.0, 4.0, 5.0]], np.zeros((1, 4)))
    out = O.track_loss(r, np.zeros((3, 1, 4), np.float32), t, 0.5)
    assert out["median"] == 2.0 and out["inlier"].all() and abs(out["loss"] - 0.5 * 10) < 1e-12
    # zero median: only exact pixels are inliers (threshold 50 * 0 = 0)
    r = _fake_render([[1.0, 1.0, 1.0, 6.0]], np.zeros((1, 4)))
    out = O.track_loss(r, np.zeros((3, 1, 4), np.float32), t, 0.5)
    np.testing.assert_array_equal(out["inlier"], [[True, True, True, False]])
    assert out["loss"] == 0.0
    # no valid input depth: nothing is an inlier
    out = O.track_loss(r, np.ones((3, 1, 4), np.float32), np.zeros((1, 4), np.float32), 0.5)
    assert not out["inlier"].any() and out["loss"] == 0.0 and not out["g_rgb"].any()


def test_depth_mirror_tracks_fp64_depth():
    c = synth.small_case(600, 64, 48, 56.0, seed=5)
    g = O.Gaussians.from_dict(c["gaussians"])
    r = O.render(g, np.eye(3, 4), c["cams"][0])
    assert r["depth"].max() > 0.5
    np.testing.assert_allclose(r["depth32"], r["depth"], rtol=2e-5, atol=2e-6)


def test_tracking_hyperparameters_follow_the_paper():
    hp = json.load(open(os.path.join(GOLDEN, "tracking_hyperparams.json")))
    assert O.TRACK_LAMBDA_C == hp["lambda_c"]["ScanNet"]
    assert hp["inlier_factor"] == 50 and hp["alpha_mask_power"] == 3


def test_tracking_recovers_a_small_camera_motion():
    # one plain-2k keyframe seen from a camera moved by 0.69 deg / 1.34 cm
    # (the mean ScanNet frame motion): 40 iterations of the tracking loss at
    # the paper's tracking learning rates recover it
    hp = json.load(open(os.path.join(GOLDEN, "tracking_hyperparams.json")))
    c = synth.plain_2k()
    g = O.Gaussians.from_dict(c["gaussians"])
    T = synth.about_point(synth.random_rigid(np.random.default_rng(77), 0.69, 0.0134),
                          synth.centroid(c["gaussians"]))
    cam = c["cams"][1]
    tr = O.render(g, T, cam)
    hyper = [hp["lr_rotation"]["ScanNet"], hp["lr_translation"]["ScanNet"]] + list(O.DEFAULT_HYPER[2:])
    ang0, dt0 = _rot_err(np.eye(3, 4), T)
    P, eps, hist = O.register_view(g, cam, tr["rgb"].astype(np.float32), tr["depth32"], 40, hyper=hyper,
                                   history=True, track_lambda_c=O.TRACK_LAMBDA_C)
    ang, dt = _rot_err(P, T)
    assert ang < 0.2 * ang0 and dt < 0.2 * dt0, (ang, dt, ang0, dt0)
    assert eps < 0.1 * hist[0]


# ----------------------------------------------------------------- exposure compensation (Supp. B)
def test_exposure_loss_reduces_to_l1_and_matches_finite_differences():
    rng = np.random.default_rng(12)
    rgb, depth = rng.uniform(0, 1, (3, 6, 5)), rng.uniform(1, 3, (6, 5))
    t_rgb, t_depth = rng.uniform(0, 1, (3, 6, 5)), rng.uniform(1, 3, (6, 5))
    # zero exposure: exactly the registration loss
    L0, g0, gd0, _ = O.exposure_loss(rgb, depth, t_rgb, t_depth, [0.0, 0.0])
    L1, g1, gd1 = O.loss(rgb, depth, t_rgb, t_depth)
    assert L0 == L1
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(gd0, gd1)
    # gain / offset gradient and the raw render's cotangent by central differences
    ab = np.array([0.2, -0.05])
    L, g, gd, gab = O.exposure_loss(rgb, depth, t_rgb, t_depth, ab)
    h = 1e-7
    for i in range(2):
        e = np.zeros(2)
        e[i] = h
        fd = (O.exposure_loss(rgb, depth, t_rgb, t_depth, ab + e)[0] -
              O.exposure_loss(rgb, depth, t_rgb, t_depth, ab - e)[0]) / (2 * h)
        assert abs(fd - gab[i]) <= 1e-6 * max(1.0, abs(gab[i])), (i, fd, gab[i])
    for idx in [(0, 1, 2), (2, 5, 4)]:
        r2 = rgb.copy()
        r2[idx] += h
        r3 = rgb.copy()
        r3[idx] -= h
        fd = (O.exposure_loss(r2, depth, t_rgb, t_depth, ab)[0] - O.exposure_loss(r3, depth, t_rgb, t_depth, ab)[0]) / (
            2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * abs(g[idx]), (idx, fd, g[idx])


def test_exposure_compensation_recovers_gain_offset_and_pose():
    # a keyframe of the 2k workload whose colours were taken with another
    # exposure (gain e^0.15, offset -0.03): registering pose and exposure
    # together (Supp. B rate 0.1) recovers both; pose alone cannot fit it
    hp = json.load(open(os.path.join(GOLDEN, "loop_closure_hyperparams.json")))
    c = synth.plain_2k()
    g = O.Gaussians.from_dict(c["gaussians"])
    T = c["T_gt"]
    cam = c["cams"][0]
    tr = O.render(g, T, cam)
    t_rgb = (math.exp(0.15) * tr["rgb"] - 0.03).astype(np.float32)
    P, eps, _, ab = O.register_view(g, cam, t_rgb, tr["depth"], 50, lr_exposure=hp["lr_exposure"]["ScanNet"])
    ang, dt = _rot_err(P, T)
    assert ang < 0.05 and dt < 2e-3, (ang, dt)
    assert abs(ab[0] - 0.15) < 0.01 and abs(ab[1] + 0.03) < 0.005, ab
    P2, eps2, _ = O.register_view(g, cam, t_rgb, tr["depth"], 50)
    assert eps2 > 5 * eps


# ----------------------------------------------------------------- overlap ratio (loop filter, Supp.)
def _pts(x):
    x = np.asarray(x, np.float32)
    return O.Gaussians(np.concatenate([x, np.zeros((len(x), 1), np.float32)], 1), np.zeros((len(x), 4)),
                       np.tile([1.0, 0, 0, 0], (len(x), 1)), np.zeros(len(x)), np.zeros((len(x), 4)))


def test_overlap_identical_and_disjoint_sets():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (500, 3))
    r, k, nn, _ = O.overlap_ratio(_pts(x), _pts(x), np.eye(3, 4))
    assert (r, k) == (1.0, 500) and (nn == np.arange(500)).all()
    # far-away outliers added to Q match nothing of P reciprocally
    y = np.concatenate([x, rng.uniform(99, 101, (50, 3))])
    r, k, _, _ = O.overlap_ratio(_pts(x), _pts(y), np.eye(3, 4))
    assert (r, k) == (1.0, 500)
    # Q 10 m away: reciprocal pairs exist (the closest pair always is one) but none is within tau
    r, k, _, _ = O.overlap_ratio(_pts(x), _pts(x + [10.0, 0, 0]), np.eye(3, 4))
    assert r == 0.0 and k >= 1


def test_overlap_nearest_neighbours_match_a_kd_tree():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(4)
    a, b = rng.uniform(-2, 2, (1500, 3)), rng.uniform(-2, 2, (1200, 3))
    T = synth.random_rigid(rng, 20.0, 0.3)
    _, _, nn_pq, nn_qp = O.overlap_ratio(_pts(a), _pts(b), T)
    at = (np.asarray(T, np.float32)[:, :3].astype(np.float64) @ np.float32(a).T).T + np.float32(T)[:, 3]
    np.testing.assert_array_equal(nn_pq, cKDTree(np.float32(b)).query(at)[1])
    np.testing.assert_array_equal(nn_qp, cKDTree(at).query(np.float32(b))[1])
    np.testing.assert_array_equal(O.nearest_subset(_pts(a), _pts(b), T, [0, 7, 1499]), nn_pq[[0, 7, 1499]])


def test_overlap_of_a_rigidly_moved_submap_is_one():
    # Q = T P (Eq. 8 on the means): under T_{P->Q} = T every mean meets its image
    c = synth.plain_2k()
    g = O.Gaussians.from_dict(c["gaussians"])
    q = O.transform(g, c["T_gt"])
    r, k, nn, _ = O.overlap_ratio(g, q, c["T_gt"], tau=0.01)
    assert r == 1.0 and k == g.n and (nn == np.arange(g.n)).all()
    # under the identity the 5 cm / 5 deg offset pushes many pairs past 1 cm
    r0, _, _, _ = O.overlap_ratio(g, q, np.eye(3, 4), tau=0.01)
    assert r0 < 0.5


def test_overlap_threshold_follows_the_paper():
    hp = json.load(open(os.path.join(GOLDEN, "loop_closure_hyperparams.json")))
    assert O.OVERLAP_TAU == hp["overlap_tau"]["ScanNet"]
