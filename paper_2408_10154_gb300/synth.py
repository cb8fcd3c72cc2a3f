"""Seeded synthetic workloads for 3D-Gaussian submap registration.

This module only draws inputs: Gaussian submaps, keyframe cameras and
ground-truth rigid transforms.  It holds none of the method's arithmetic
(no projection, rendering, loss or pose update) and serves the CUDA path,
the tests and the benchmark alike.  Target images are rendered by whichever
side consumes the inputs.

The shapes follow the paper's workloads (LoopSplat, arXiv 2408.10154):
room-sized submaps of 10^5 Gaussians (Supp. E, Gaussians-per-scene table:
219K-331K per scene), Replica-like 1200x680 keyframes, rigid offsets of a
few degrees and centimetres between overlapping submaps.  The datasets the
paper evaluates on (Replica, TUM-RGBD, ScanNet, ScanNet++) are not used;
these seeded inputs stand in for them.

Layouts (all float32, C-contiguous):
  means4 [n,4] (x, y, z, 0); log_scales4 [n,4] (sx, sy, sz, 0);
  quats4 [n,4] (w, x, y, z), unit; logits [n]; rgb4 [n,4] (r, g, b, 0);
  camera cam18 = [fx, fy, cx, cy, W, H, world_to_cam 3x4 row-major]
  (OpenCV convention: x right, y down, z forward).
Rigid transforms are float64 [3,4] row-major [R | t].
"""
from __future__ import annotations

import math

import numpy as np

ROOM_HALF = np.array([3.0, 2.5, 1.5])  # 6 x 5 x 3 m room, z vertical


def _finish(means, log_scales, rng):
    n = means.shape[0]
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    out = dict(
        means4=np.zeros((n, 4), np.float32),
        log_scales4=np.zeros((n, 4), np.float32),
        quats4=q.astype(np.float32),
        logits=rng.standard_normal(n).astype(np.float32),
        rgb4=np.zeros((n, 4), np.float32),
    )
    out["means4"][:, :3] = means
    out["log_scales4"][:, :3] = log_scales
    out["rgb4"][:, :3] = rng.uniform(0.0, 1.0, (n, 3))
    return out


def gaussians_box(n, rng, center=(0.0, 0.0, 2.5), half=1.0, ls_mean=-4.0, ls_std=0.5):
    """n anisotropic Gaussians with means uniform in a cube of side 2*half
    around ``center``; log-scales N(ls_mean, ls_std) per axis; uniformly
    random unit quaternions; opacity logit N(0,1); RGB uniform in [0,1]."""
    means = rng.uniform(-half, half, (n, 3)) + np.asarray(center, dtype=np.float64)
    ls = rng.normal(ls_mean, ls_std, (n, 3))
    return _finish(means, ls, rng)


def gaussians_room(n, rng, scale=1.0, wall_frac=0.8, wall_offset=0.02, ls_mean=-4.5, ls_std=0.6):
    """n Gaussians in a room-shaped shell of half extents ROOM_HALF*scale:
    ``wall_frac`` of the means lie on the six walls (a wall drawn with
    probability proportional to its area, a point uniform on it, offset
    U(-wall_offset, wall_offset) along its normal), the rest uniform in the
    interior."""
    h = ROOM_HALF * scale
    n_wall = int(round(wall_frac * n))
    areas = np.array([h[1] * h[2], h[1] * h[2], h[0] * h[2], h[0] * h[2], h[0] * h[1], h[0] * h[1]])
    wall = rng.choice(6, size=n_wall, p=areas / areas.sum())
    pts = rng.uniform(-1.0, 1.0, (n_wall, 3)) * h
    axis = wall // 2
    sign = np.where(wall % 2 == 0, -1.0, 1.0)
    pts[np.arange(n_wall), axis] = sign * h[axis] + rng.uniform(-wall_offset, wall_offset, n_wall)
    interior = rng.uniform(-1.0, 1.0, (n - n_wall, 3)) * h
    means = np.concatenate([pts, interior], axis=0)
    means = means[rng.permutation(n)]
    ls = rng.normal(ls_mean, ls_std, (n, 3))
    return _finish(means, ls, rng)


def look_at(eye, target, down):
    """world -> camera [R|t] of a camera at ``eye`` looking at ``target``
    with image y along ``down``."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(down, np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return np.concatenate([R, (-R @ eye)[:, None]], axis=1)


def camera(fx, fy, cx, cy, W, H, w2c):
    c = np.zeros(18, np.float32)
    c[:6] = [fx, fy, cx, cy, W, H]
    c[6:] = np.asarray(w2c, np.float64).reshape(12)
    return c


def axis_angle_matrix(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def random_rigid(rng, angle_deg, trans_m):
    """[R|t]: rotation by ``angle_deg`` about a uniform random axis,
    translation of length ``trans_m`` in a uniform random direction."""
    ax = rng.standard_normal(3)
    d = rng.standard_normal(3)
    R = axis_angle_matrix(ax, math.radians(angle_deg))
    t = d / np.linalg.norm(d) * trans_m
    return np.concatenate([R, t[:, None]], axis=1)


def about_point(T, c):
    """The rigid map x -> R (x - c) + c + t of T = [R|t], i.e. the rotation
    of T taken about the point c instead of the origin."""
    T = np.asarray(T, np.float64).reshape(3, 4)
    c = np.asarray(c, np.float64)
    return np.concatenate([T[:, :3], (T[:, 3] + c - T[:, :3] @ c)[:, None]], axis=1)


def centroid(g):
    return g["means4"][:, :3].astype(np.float64).mean(axis=0)


def compose(A, B):
    """[R|t] of x -> A(B(x))."""
    A = np.asarray(A, np.float64).reshape(3, 4)
    B = np.asarray(B, np.float64).reshape(3, 4)
    return np.concatenate([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]], axis=1)


def inverse(T):
    T = np.asarray(T, np.float64).reshape(3, 4)
    R = T[:, :3]
    return np.concatenate([R.T, (-R.T @ T[:, 3])[:, None]], axis=1)


def moved_cameras(cams, T):
    """Cameras of a submap moved by the rigid map T (camera-to-world C ->
    T C, i.e. world_to_cam -> world_to_cam o T^-1)."""
    out = []
    Ti = inverse(T)
    for c in cams:
        c2 = np.array(c, np.float32).copy()
        c2[6:] = compose(np.asarray(c[6:], np.float64).reshape(3, 4), Ti).reshape(12)
        out.append(c2)
    return np.stack(out)


def circle_cameras(n_views, radius, target, W, H, f, down=(0.0, 1.0, 0.0)):
    """Cameras on a circle of ``radius`` in the plane z = 0 about the origin
    (angles 0, 360/n, ...), each looking at ``target``."""
    cams = []
    for k in range(n_views):
        a = 2 * math.pi * k / n_views
        eye = (radius * math.cos(a), radius * math.sin(a), 0.0)
        cams.append(camera(f, f, W / 2, H / 2, W, H, look_at(eye, target, down)))
    return np.stack(cams)


def room_cameras(n_views, rng, W, H, f, scale=1.0, shrink=0.75, pitch_deg=15.0):
    """Cameras uniform in the room interior shrunk by ``shrink`` metres,
    yaw U(0, 2pi), pitch U(-pitch_deg, pitch_deg), image y pointing down."""
    h = ROOM_HALF * scale - shrink
    cams = []
    for _ in range(n_views):
        eye = rng.uniform(-1.0, 1.0, 3) * h
        yaw = rng.uniform(0, 2 * math.pi)
        pitch = math.radians(rng.uniform(-pitch_deg, pitch_deg))
        fwd = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch)])
        cams.append(camera(f, f, W / 2, H / 2, W, H, look_at(eye, eye + fwd, (0.0, 0.0, -1.0))))
    return np.stack(cams)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def plain_2k(seed=1000):
    """Plain single registration: 2,000 Gaussians in a 2 m cube centred
    2.5 m in front of the origin (log-scales N(-4, 0.5)), 4 keyframes of
    160x120 (f = 140) on a 0.3 m circle looking at the cube centre, ground
    truth 5 deg about the submap centroid / 5 cm, 50 iterations, one
    direction."""
    rng = np.random.default_rng(seed)
    g = gaussians_box(2000, rng)
    cams = circle_cameras(4, 0.3, (0.0, 0.0, 2.5), 160, 120, 140.0)
    T = about_point(random_rigid(rng, 5.0, 0.05), centroid(g))
    return dict(name="plain_2k", gaussians=g, cams=cams, T_gt=T, iters=50)


def room_150k(seed=1001, n=150_000, n_views=8, W=1200, H=680, f=600.0):
    """Room-scale registration: 150,000 Gaussians on a 6x5x3 m room shell
    (80 % within 2 cm of the walls, log-scales N(-4.5, 0.6)), 8 keyframes of
    1200x680 (f = 600) per submap, ground truth 10 deg (about the submap
    centroid) / 15 cm, 100
    iterations in both directions.  The target submap is the source moved by
    T_gt; its keyframes are the source keyframes moved by T_gt."""
    rng = np.random.default_rng(seed)
    g = gaussians_room(n, rng)
    cams = room_cameras(n_views, rng, W, H, f)
    T = about_point(random_rigid(rng, 10.0, 0.15), centroid(g))
    return dict(name="room_150k", gaussians=g, src_cams=cams, tgt_cams=moved_cameras(cams, T), T_gt=T,
                iters=100)


def batched_pairs(seed=1002, n_pairs=32, n_min=20_000, n_max=400_000):
    """Batched uneven registration: ``n_pairs`` submap pairs with sizes
    log-uniform in [n_min, n_max] (room distributions, room scaled by
    (n/150k)^(1/3)), U{4..12} keyframes per submap at 640x480 (f = 320) or
    1200x680 (f = 600), ground truth angle U(0, 15 deg), translation
    U(0, 25 cm), 100 iterations, both directions."""
    rng = np.random.default_rng(seed)
    pairs = []
    for _ in range(n_pairs):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        scale = (n / 150_000) ** (1.0 / 3.0)
        g = gaussians_room(n, rng, scale=scale)
        nv = int(rng.integers(4, 13))
        if rng.uniform() < 0.5:
            W, H, f = 640, 480, 320.0
        else:
            W, H, f = 1200, 680, 600.0
        cams = room_cameras(nv, rng, W, H, f, scale=scale, shrink=0.75 * scale)
        T = about_point(random_rigid(rng, rng.uniform(0, 15.0), rng.uniform(0, 0.25)), centroid(g))
        pairs.append(dict(gaussians=g, src_cams=cams, tgt_cams=moved_cameras(cams, T), T_gt=T))
    return dict(name="batched_32", pairs=pairs, iters=100)


def serving_stream(seed=1004, rate=200.0, seconds=60.0, n_submaps=64, frames=4, n_edges=32, track_frac=0.7):
    """Serving stream: Poisson arrivals at ``rate`` per second for
    ``seconds``; a fraction ``track_frac`` are frame-to-model tracking
    requests (one 640x480 RGB-D frame of a resident submap of U[50k, 300k]
    room Gaussians, the request's camera the frame's true camera perturbed by
    0.69 deg and 1.34 cm, 40 iterations), the rest loop edges drawn from a
    pool of ``n_edges`` batched-workload pairs (100 iterations, both
    directions).  Returns dict(submaps=[dict(gaussians, cams, guesses)],
    arrivals=[(t, kind, index, frame)]) with kind "track" or "edge"."""
    rng = np.random.default_rng(seed)
    submaps = []
    for _ in range(n_submaps):
        n = int(rng.integers(50_000, 300_001))
        scale = (n / 150_000) ** (1.0 / 3.0)
        g = gaussians_room(n, rng, scale=scale)
        cams = room_cameras(frames, rng, 640, 480, 320.0, scale=scale, shrink=0.75 * scale)
        guesses = []
        for c in cams:
            c2 = np.array(c, np.float32).copy()
            # the camera moved by a small rigid motion in its own frame
            c2[6:] = compose(random_rigid(rng, 0.69, 0.0134), np.asarray(c[6:], np.float64).reshape(3, 4)).reshape(12)
            guesses.append(c2)
        submaps.append(dict(gaussians=g, cams=cams, guesses=np.stack(guesses)))
    arrivals, t = [], 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= seconds:
            break
        if rng.uniform() < track_frac:
            arrivals.append((t, "track", int(rng.integers(n_submaps)), int(rng.integers(frames))))
        else:
            arrivals.append((t, "edge", int(rng.integers(n_edges)), 0))
    return dict(name="serving", submaps=submaps, arrivals=arrivals, track_iters=40, edge_iters=100)


def diff_check_300k(seed=1003):
    """Differentiation check: 300,000 room Gaussians, 4 keyframes of
    1200x680; plus the exhaustive small case (500 Gaussians, 64x48,
    f = 56)."""
    rng = np.random.default_rng(seed)
    g = gaussians_room(300_000, rng)
    cams = room_cameras(4, rng, 1200, 680, 600.0)
    small = small_case(500, 64, 48, 56.0, n_views=1, seed=seed)
    return dict(name="diff_check_300k", gaussians=g, cams=cams, small=small)


def small_case(n, W, H, f, n_views=1, seed=0, ls_mean=-3.0, ls_std=0.4, half=0.8, depth=2.0,
               angle_deg=3.0, trans_m=0.03):
    """A small scene for parity tests: ``n`` Gaussians in a cube of side
    2*half at ``depth`` in front of the origin, ``n_views`` cameras on a
    0.25 m circle looking at it (one camera at the origin when n_views=1),
    and a ground-truth rigid offset."""
    rng = np.random.default_rng(seed)
    g = gaussians_box(n, rng, center=(0.0, 0.0, depth), half=half, ls_mean=ls_mean, ls_std=ls_std)
    if n_views == 1:
        cams = np.stack([camera(f, f, W / 2, H / 2, W, H, np.eye(3, 4))])
    else:
        cams = circle_cameras(n_views, 0.25, (0.0, 0.0, depth), W, H, f)
    T = about_point(random_rigid(rng, angle_deg, trans_m), centroid(g))
    return dict(name=f"small_{n}_{W}x{H}", gaussians=g, cams=cams, T_gt=T)


def saturated_case(seed=41):
    """A small scene whose left half holds near-opaque Gaussians (opacity
    logits N(6, 1): most opacities above the 0.99 alpha clamp) and whose
    right half the usual N(0, 1) logits, so that some screen tiles see
    clamped alphas and others none, 2 views of 160x120."""
    c = small_case(1500, 160, 120, 150.0, n_views=2, seed=seed, ls_mean=-3.2, ls_std=0.3)
    g = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    rng = np.random.default_rng(seed + 1)
    left = g["means4"][:, 0] < 0.0
    g["logits"][left] = rng.normal(6.0, 1.0, int(left.sum()))
    c["gaussians"] = g
    return c


def giant_needles_case(seed=51):
    """A small scene with a few giant needles (3 % of the Gaussians: one
    axis e^1.8 = 6 m, the others e^-6 = 2.5 mm) among ordinary splats: their
    projections cross the whole 120x90 image with 2D covariances so
    elongated that their conics' condition numbers pass 10^6, 2 views."""
    c = small_case(600, 120, 90, 100.0, n_views=2, seed=seed, ls_mean=-3.0, ls_std=0.3)
    g = {k: np.array(v, copy=True) for k, v in c["gaussians"].items()}
    rng = np.random.default_rng(seed + 1)
    giant = rng.random(len(g["logits"])) < 0.03
    g["log_scales4"][giant, 0] = 1.8
    g["log_scales4"][giant, 1] = -6.0
    g["log_scales4"][giant, 2] = -6.0
    c["gaussians"] = g
    return c

