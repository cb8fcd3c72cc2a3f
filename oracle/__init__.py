"""FP64 CPU oracle of the 3D-Gaussian registration hot path (LoopSplat,
arXiv 2408.10154).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this
package.  The product path never does; it shares no code with the CUDA
library.

The arithmetic lives in ``gs_oracle.c`` (plain C, FP64 values, FP32 decision
mirror; see its header).  This module builds and loads it through ctypes and
adds the one step written in numpy: the residual-weighted rotation averaging
of Eq. 7 (Sec. 3.2, "Multi-view Pose Refinement").

Every function takes numpy arrays in the layout of the C-ABI inputs:
Gaussians as float32 ``means4 [n,4]``, ``log_scales4 [n,4]``, ``quats4 [n,4]``
(w, x, y, z), ``logits [n]``, ``rgb4 [n,4]``; a camera as float32
``cam18 = [fx, fy, cx, cy, W, H, world_to_cam (3x4 row-major)]``; options
as float32 ``opt11 = [tile, z_near, dilation, alpha_min, alpha_max, t_min,
bg_r, bg_g, bg_b, smooth, tight]``; poses as float64 ``[3,4]`` (object -> world).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# default options: 16-pixel tiles, near plane 0.2 m, dilation 0.3 px^2,
# alpha in [1/255, 0.99], early stop below transmittance 1e-4, black
# background, tight tile rectangles (the alpha-threshold box of each record)
DEFAULT_OPT = np.array([16, 0.2, 0.3, 1.0 / 255.0, 0.99, 1e-4, 0, 0, 0, 0, 1], dtype=np.float32)
# the same with the plain 3-sigma tile rectangles
LOOSE_OPT = np.array([16, 0.2, 0.3, 1.0 / 255.0, 0.99, 1e-4, 0, 0, 0, 0, 0], dtype=np.float32)
# smooth options (finite-difference checks): no thresholds, no radius cull
SMOOTH_OPT = np.array([16, 0.2, 0.3, 0.0, 1.0, 0.0, 0, 0, 0, 1, 0], dtype=np.float32)
N_OPT = 11
# registration hyper-parameters {lr_rot, lr_trans, beta1, beta2, eps, final lr fraction}:
# learning rates of the paper's real-data column (Supp. B, loop-closure table);
# Adam constants and the cosine decay to 0.1 % are this implementation's reading
DEFAULT_HYPER = np.array([0.015, 0.005, 0.8, 0.99, 1e-8, 0.001], dtype=np.float64)


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into oracle/_build/liboracle.so (gcc, C11,
    -ffp-contract=off so that the FP32 mirror is evaluated exactly as
    written; OpenMP for the optional multi-threaded loops, one thread unless
    set_threads asks for more)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        L = ctypes.c_long
        lib.or_exp32.argtypes = [ctypes.c_float]
        lib.or_exp32_count_above_one.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.or_exp32_count_above_one.restype = ctypes.c_int64
        lib.or_count_positive_power.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 7
        lib.or_count_positive_power.restype = ctypes.c_int64
        lib.or_exp32.restype = ctypes.c_float
        lib.or_log32.argtypes = [ctypes.c_float]
        lib.or_log32.restype = ctypes.c_float
        lib.or_project32.argtypes = [I, P, P, P, P, P, P, P, P, P]
        lib.or_project64.argtypes = [I, P, P, P, P, P, P, P, P]
        lib.or_bin.argtypes = [I, P, P, P, P, I, P, P, P, P, P, L, P, P]
        lib.or_render.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.or_loss.argtypes = [I, I, P, P, P, P, P, P]
        lib.or_loss.restype = ctypes.c_double
        lib.or_backward.argtypes = [I, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.or_pose_step.argtypes = [P, P, P, P, P, I, I]
        lib.or_register_view.argtypes = [I, P, P, P, P, P, P, P, P, P, P, I, P, P, P, P, P, P]
        lib.or_exposure_loss.argtypes = [I, I, P, P, P, P, P, P, P, P]
        lib.or_overlap_ratio.argtypes = [I, P, I, P, P, ctypes.c_float, P, P, P]
        lib.or_overlap_ratio.restype = ctypes.c_double
        lib.or_nearest_subset.argtypes = [I, P, I, P, P, I, P, P]
        lib.or_nearest_subset.restype = I
        lib.or_moved_means.argtypes = [I, P, P, P]
        lib.or_moved_means.restype = I
        lib.or_exposure_loss.restype = ctypes.c_double
        lib.or_track_loss.argtypes = [I, I, P, P, P, P, P, P, ctypes.c_double, P, P, P, P]
        lib.or_track_loss.restype = ctypes.c_double
        lib.or_transform.argtypes = [I, P, P, P, P, P]
        for f in ("or_project32", "or_project64", "or_bin", "or_render", "or_backward",
                  "or_pose_step", "or_register_view", "or_transform"):
            getattr(lib, f).restype = ctypes.c_int
        lib.or_contrib_sig.argtypes = [I, P, P, P, P, P, P, P, P, P]
        lib.or_contrib_sig.restype = I
        lib.or_set_threads.argtypes = [I]
        lib.or_set_threads.restype = I
        lib.or_set_threads(1)
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (compositing rows, adjoint
    bands); results do not depend on it.  Returns the number in effect."""
    return int(_load().or_set_threads(int(n)))


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _opt(opt):
    o = _f32(opt)
    if o.shape != (N_OPT,):
        raise ValueError(f"oracle options must be {N_OPT} floats, got shape {o.shape}")
    return o


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


class Gaussians:
    """Host-side FP32 submap in the C-ABI layout (float4-padded SoA)."""

    def __init__(self, means4, log_scales4, quats4, logits, rgb4):
        self.means4 = _f32(means4)
        self.log_scales4 = _f32(log_scales4)
        self.quats4 = _f32(quats4)
        self.logits = _f32(logits)
        self.rgb4 = _f32(rgb4)
        self.n = int(self.means4.shape[0])

    @classmethod
    def from_dict(cls, d):
        return cls(d["means4"], d["log_scales4"], d["quats4"], d["logits"], d["rgb4"])

    def args(self):
        return (self.n, _p(self.means4), _p(self.log_scales4), _p(self.quats4), _p(self.logits))


def exp32(x: float) -> float:
    """The FP32 mirror's exponential (Cody-Waite + degree-6 Taylor)."""
    return float(_load().or_exp32(float(x)))


def exp32_count_above_one(lo_bits: int, hi_bits: int) -> int:
    """How many floats with bit patterns in [lo_bits, hi_bits] the mirror's
    exponential maps above 1."""
    return int(_load().or_exp32_count_above_one(lo_bits, hi_bits))


def count_positive_power(ca, cb, cc, u, v, pxf, pyf) -> int:
    """How many of the given (conic, mean, pixel sample) cases the mirror's
    FP32 exponent puts above 0 (float32 arrays of one length)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (ca, cb, cc, u, v, pxf, pyf)]
    n = len(arrs[0])
    assert all(len(a) == n for a in arrs)
    return int(_load().or_count_positive_power(n, *[a.ctypes.data for a in arrs]))


def log32(x: float) -> float:
    """The FP32 mirror's logarithm of the tight tile rectangles."""
    return float(_load().or_log32(float(x)))


def project32(g: Gaussians, pose, cam, opt=DEFAULT_OPT):
    """FP32 mirror projection.  Returns (f [n,8] = u, v, z, ca, cb, cc, o, 0;
    i [n,6] = visible, radius, x0, x1, y0, y1)."""
    lib = _load()
    f = np.zeros((g.n, 8), np.float32)
    i = np.zeros((g.n, 6), np.int32)
    _check(lib.or_project32(*g.args(), _p(_f64(pose, (12,))), _p(_f32(cam)), _p(_opt(opt)), _p(f), _p(i)),
           "project32")
    return f, i


def project64(g: Gaussians, pose, cam, opt=DEFAULT_OPT):
    """FP64 projection: [n,16] = U, V, z, A, B, C, o, x, y, Sc(6), 0."""
    lib = _load()
    out = np.zeros((g.n, 16), np.float64)
    _check(lib.or_project64(*g.args(), _p(_f64(pose, (12,))), _p(_f32(cam)), _p(_opt(opt)), _p(out)),
           "project64")
    return out


def n_tiles(cam, opt=DEFAULT_OPT):
    B = int(opt[0])
    return ((int(cam[4]) + B - 1) // B) * ((int(cam[5]) + B - 1) // B)


def bin_tiles(g: Gaussians, poses, cams, opt=DEFAULT_OPT):
    """Tile binning over several cameras (pose k for camera k).  Returns
    (keys uint64 [d], values uint32 [d], ranges int64 [tiles, 2]); record
    index = camera * n + Gaussian, global tile = camera tile base + local."""
    lib = _load()
    cams = _f32(cams, (-1, 18))
    poses = _f64(poses, (-1, 12))
    tiles = sum(n_tiles(c, opt) for c in cams)
    ranges = np.zeros((tiles, 2), np.int64)
    nd = ctypes.c_long(0)
    # first pass: count
    _check(lib.or_bin(*g.args(), len(cams), _p(poses), _p(cams), _p(_opt(opt)), None, None, 0, _p(ranges),
                      ctypes.byref(nd)), "bin")
    keys = np.zeros(max(nd.value, 1), np.uint64)
    vals = np.zeros(max(nd.value, 1), np.uint32)
    _check(lib.or_bin(*g.args(), len(cams), _p(poses), _p(cams), _p(_opt(opt)), _p(keys), _p(vals), nd.value,
                      _p(ranges), ctypes.byref(nd)), "bin")
    return keys[: nd.value], vals[: nd.value], ranges


def render(g: Gaussians, pose, cam, opt=DEFAULT_OPT):
    """FP64 render at one camera.  Returns dict(rgb [3,H,W], depth, alpha,
    t_final (FP64), t_final32 and depth32 (the FP32 mirror), last (int32))."""
    lib = _load()
    W, H = int(cam[4]), int(cam[5])
    rgb = np.zeros((3, H, W), np.float64)
    depth = np.zeros((H, W), np.float64)
    alpha = np.zeros((H, W), np.float64)
    tf = np.zeros((H, W), np.float64)
    tf32 = np.zeros((H, W), np.float32)
    last = np.zeros((H, W), np.int32)
    d32 = np.zeros((H, W), np.float32)
    _check(lib.or_render(*g.args(), _p(g.rgb4), _p(_f64(pose, (12,))), _p(_f32(cam)), _p(_opt(opt)), _p(rgb),
                         _p(depth), _p(alpha), _p(tf), _p(tf32), _p(last), _p(d32)), "render")
    return dict(rgb=rgb, depth=depth, alpha=alpha, t_final=tf, t_final32=tf32, last=last, depth32=d32)


def contrib_sig(g: Gaussians, pose, cam, opt=DEFAULT_OPT):
    """Per-pixel signature [H, W] (uint64) of the contributor sequence of
    ``render``: equal signatures mean the same alpha-test, clamp and
    early-stop decisions at that pixel."""
    lib = _load()
    W, H = int(cam[4]), int(cam[5])
    sig = np.zeros((H, W), np.uint64)
    _check(lib.or_contrib_sig(*g.args(), _p(g.rgb4), _p(_f64(pose, (12,))), _p(_f32(cam)), _p(_opt(opt)), _p(sig)),
           "contrib_sig")
    return sig


# lambda_c of the tracking loss (Supp. A, per-dataset hyperparameters: 0.6 on
# TUM-RGBD and ScanNet)
TRACK_LAMBDA_C = 0.6


def track_loss(r, t_rgb, t_depth, lambda_c=TRACK_LAMBDA_C):
    """Frame-to-model tracking loss (Eq. 2 with the alpha^3 and inlier masks
    of Supp. A) of a render ``r`` (a dict of ``render``) against FP32 targets.
    Returns dict(loss, g_rgb, g_depth, inlier (bool [H,W]), median)."""
    lib = _load()
    H, W = r["depth"].shape
    g_rgb = np.zeros((3, H, W), np.float64)
    g_depth = np.zeros((H, W), np.float64)
    inl = np.zeros((H, W), np.int8)
    med = ctypes.c_float(0.0)
    L = lib.or_track_loss(H, W, _p(_f64(r["rgb"])), _p(_f64(r["depth"])), _p(_f64(r["t_final"])),
                          _p(_f32(r["depth32"])), _p(_f32(t_rgb)), _p(_f32(t_depth)), float(lambda_c), _p(g_rgb),
                          _p(g_depth), _p(inl), ctypes.byref(med))
    if L != L:
        raise RuntimeError("oracle track_loss: out of memory")
    return dict(loss=float(L), g_rgb=g_rgb, g_depth=g_depth, inlier=inl.astype(bool), median=float(med.value))


def loss(rgb, depth, t_rgb, t_depth):
    """L1 colour + L1 depth loss (Sec. 3.2) and its image gradients
    (targets may be FP32 or FP64; they are compared in FP64)."""
    lib = _load()
    rgb = _f64(rgb)
    depth = _f64(depth)
    H, W = depth.shape
    g_rgb = np.zeros_like(rgb)
    g_depth = np.zeros_like(depth)
    L = lib.or_loss(H, W, _p(rgb), _p(depth), _p(_f64(t_rgb)), _p(_f64(t_depth)), _p(g_rgb), _p(g_depth))
    return float(L), g_rgb, g_depth


def backward(g: Gaussians, pose, cam, cot_rgb=None, cot_depth=None, cot_alpha=None, pivot=None,
             opt=DEFAULT_OPT, params=True):
    """Adjoint of ``render``.  Returns dict(twist [6] about ``pivot``, and when
    ``params``: means [n,3], log_scales [n,3], quats [n,4], logits [n],
    rgb [n,3])."""
    lib = _load()
    n = g.n
    tw = np.zeros(6, np.float64)
    out = dict(twist=tw)
    if params:
        out.update(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                   logits=np.zeros(n), rgb=np.zeros((n, 3)))
    cr = None if cot_rgb is None else _f64(cot_rgb)
    cd = None if cot_depth is None else _f64(cot_depth)
    ca = None if cot_alpha is None else _f64(cot_alpha)
    pv = None if pivot is None else _f64(pivot, (3,))
    _check(lib.or_backward(*g.args(), _p(g.rgb4), _p(_f64(pose, (12,))), _p(_f32(cam)), _p(_opt(opt)), _p(cr),
                           _p(cd), _p(ca), _p(pv), _p(tw), _p(out.get("means")), _p(out.get("log_scales")),
                           _p(out.get("quats")), _p(out.get("logits")), _p(out.get("rgb"))), "backward")
    return out


def centroid(g: Gaussians):
    return g.means4[:, :3].astype(np.float64).mean(axis=0) if g.n else np.zeros(3)


def pose_step(pose, state, grad, pivot, k, iters, hyper=DEFAULT_HYPER):
    """One Adam step + pose update about ``pivot`` (in place on copies).
    Returns (pose [3,4], state [13])."""
    lib = _load()
    pose = _f64(pose, (12,)).copy()
    state = _f64(state, (13,)).copy()
    _check(lib.or_pose_step(_p(pose), _p(state), _p(_f64(grad, (6,))), _p(_f64(pivot, (3,))),
                            _p(_f64(hyper, (6,))), int(k), int(iters)), "pose_step")
    return pose.reshape(3, 4), state


def register_view(g: Gaussians, cam, t_rgb, t_depth, iters, pose0=None, opt=DEFAULT_OPT,
                  hyper=DEFAULT_HYPER, history=False, track_lambda_c=None, lr_exposure=None):
    """Keyframe localisation of one view (Sec. 3.2).  Returns (pose [3,4],
    eps, loss history or None), plus the exposure (a, b) when
    ``lr_exposure`` is given.  track_lambda_c: None = the registration loss,
    else the tracking loss of Eq. 2 with that lambda_c."""
    lib = _load()
    pose = np.eye(3, 4, dtype=np.float64).reshape(12).copy() if pose0 is None else _f64(pose0, (12,)).copy()
    eps = ctypes.c_double(0.0)
    hist = np.zeros(max(iters, 1), np.float64) if history else None
    trk = None if track_lambda_c is None else np.array([track_lambda_c], np.float64)
    ex = None if lr_exposure is None else np.array([lr_exposure], np.float64)
    ab = np.zeros(2, np.float64)
    _check(lib.or_register_view(*g.args(), _p(g.rgb4), _p(_f32(cam)), _p(_opt(opt)), _p(_f32(t_rgb)),
                                _p(_f32(t_depth)), _p(_f64(hyper, (6,))), int(iters), _p(pose),
                                ctypes.byref(eps), _p(hist), _p(trk), _p(ex), _p(ab)), "register_view")
    out = (pose.reshape(3, 4), eps.value, (hist[:iters] if history else None))
    return out + (ab,) if lr_exposure is not None else out


def exposure_loss(rgb, depth, t_rgb, t_depth, ab):
    """Registration loss of the exposure-compensated colour e^a I^ + b
    (Supp. B).  Returns (L, dL/dI^ of the raw render, dL/dD^, (dL/da, dL/db))."""
    lib = _load()
    rgb = _f64(rgb)
    depth = _f64(depth)
    H, W = depth.shape
    g_rgb = np.zeros_like(rgb)
    g_depth = np.zeros_like(depth)
    g_ab = np.zeros(2, np.float64)
    L = lib.or_exposure_loss(H, W, _p(rgb), _p(depth), _p(_f64(t_rgb)), _p(_f64(t_depth)), _p(_f64(ab, (2,))),
                             _p(g_rgb), _p(g_depth), _p(g_ab))
    if L != L:
        raise RuntimeError("oracle exposure_loss: out of memory")
    return float(L), g_rgb, g_depth, g_ab


def transform(g: Gaussians, T):
    """Rigid transform of a submap (Eq. 8 / Eq. 9); returns a new Gaussians."""
    lib = _load()
    m = np.zeros_like(g.means4)
    q = np.zeros_like(g.quats4)
    _check(lib.or_transform(g.n, _p(g.means4), _p(g.quats4), _p(_f64(T, (12,))), _p(m), _p(q)), "transform")
    return Gaussians(m, g.log_scales4.copy(), q, g.logits.copy(), g.rgb4.copy())


def invert(T):
    T = _f64(T, (3, 4))
    R, t = T[:, :3], T[:, 3]
    return np.concatenate([R.T, (-R.T @ t)[:, None]], axis=1)


def fuse(estimates, eps, reverse):
    """Multi-view pose refinement (Eq. 7).  ``estimates`` [k,3,4]: the
    optimised transforms; ``reverse[i]`` marks an estimate of the opposite
    direction, which is inverted first.  Weights are 1/max(eps, 1e-12);
    the rotation is the weighted chordal L2 mean (projection of sum w_i R_i
    onto SO(3) by SVD), the translation the weighted mean of the (inverted)
    estimates' translations.  Returns (T [3,4], confidence = mean weight)."""
    est = _f64(estimates, (-1, 3, 4))
    eps = _f64(eps, (-1,))
    rev = np.asarray(reverse, dtype=bool).reshape(-1)
    Ts = np.stack([invert(T) if r else T for T, r in zip(est, rev)])
    w = 1.0 / np.maximum(eps, 1e-12)
    M = np.einsum("i,ijk->jk", w, Ts[:, :, :3])
    U, _, Vt = np.linalg.svd(M)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    R = U @ D @ Vt
    t = (w[:, None] * Ts[:, :, 3]).sum(0) / w.sum()
    return np.concatenate([R, t[:, None]], axis=1), float(w.mean())


# overlap threshold tau_1 of the loop filter (Supp.: 0.2 m on TUM-RGBD,
# ScanNet, ScanNet++; 0.1 m on Replica)
OVERLAP_TAU = 0.2


def overlap_ratio(p: Gaussians, q: Gaussians, T, tau=OVERLAP_TAU):
    """Overlap ratio of P and Q under T_{P->Q} (reciprocal closest points,
    FP32 distances).  Returns (OR, |K|, nn_pq [np], nn_qp [nq])."""
    lib = _load()
    nn_pq = np.zeros(max(p.n, 1), np.int32)
    nn_qp = np.zeros(max(q.n, 1), np.int32)
    k = ctypes.c_long(0)
    r = lib.or_overlap_ratio(p.n, _p(p.means4), q.n, _p(q.means4), _p(_f64(T, (12,))), float(tau), _p(nn_pq),
                             _p(nn_qp), ctypes.byref(k))
    if r < 0:
        raise RuntimeError("oracle overlap_ratio: out of memory")
    return float(r), int(k.value), nn_pq[:p.n], nn_qp[:q.n]


def nearest_subset(p: Gaussians, q: Gaussians, T, idx):
    """Nearest neighbours in Q of the moved means of P[idx]."""
    lib = _load()
    idx = np.ascontiguousarray(idx, np.int32)
    nn = np.zeros(max(len(idx), 1), np.int32)
    _check(lib.or_nearest_subset(p.n, _p(p.means4), q.n, _p(q.means4), _p(_f64(T, (12,))), len(idx), _p(idx), _p(nn)),
           "nearest_subset")
    return nn[:len(idx)]


def moved_means(g: Gaussians, T):
    """The overlap ratio's FP32 moved means T mu, [n, 4] (w = 0)."""
    lib = _load()
    out = np.zeros((max(g.n, 1), 4), np.float32)
    _check(lib.or_moved_means(g.n, _p(g.means4), _p(_f64(T, (12,))), _p(out)), "moved_means")
    return out[:g.n]
