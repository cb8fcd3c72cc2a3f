"""Python binding of libgsreg.so (include/gsreg.h): ctypes argument
marshalling only.  Every step of the path runs in the CUDA library; PyTorch
supplies device memory (CUDA tensors) and the current stream.  There is no
CPU fallback: if the compiled library cannot be loaded, every call raises.

The functions carry the C names (gs_project, gs_bin, gs_render,
gs_render_backward, gs_loss, gs_pose_step, gs_fuse, gs_register,
gs_transform) and take tensors in the C-ABI layouts.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

GS_TILE = 16
GS_RECORD_FLOATS = 12
GS_AUX_FLOATS = 8

STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_OOM", 3: "GS_ERR_CUDA", 4: "GS_ERR_NONFINITE",
          5: "GS_ERR_TIMEOUT", 6: "GS_ERR_DIVERGED", 7: "GS_ERR_CAPACITY"}


class GsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class gs_gaussians_t(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("rgb", ctypes.c_void_p), ("n", ctypes.c_int64)]


class gs_camera_t(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("world_to_cam", ctypes.c_float * 12)]


class gs_view_t(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("cam", gs_camera_t)]


class gs_options_t(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("z_near", ctypes.c_float), ("dilation", ctypes.c_float),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("smooth", ctypes.c_int32), ("lr_rot", ctypes.c_float),
                ("lr_trans", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("lr_final", ctypes.c_float), ("profile", ctypes.c_int32),
                ("tracking_loss", ctypes.c_int32), ("lambda_c", ctypes.c_float), ("exposure", ctypes.c_int32),
                ("lr_exposure", ctypes.c_float), ("tile_schedule", ctypes.c_int32),
                ("tight_lists", ctypes.c_int32), ("list_headroom", ctypes.c_float),
                ("fuse_compositing", ctypes.c_int32)]


class gs_stats_t(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("n_dups", ctypes.c_int64), ("n_pixels", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("iterations", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("phase_ms", ctypes.c_double * 5), ("contributing", ctypes.c_int64)]


class gs_gaussian_grads_t(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("rgb", ctypes.c_void_p)]


EXPORTS = ["gs_default_options", "gs_ctx_create", "gs_ctx_destroy", "gs_last_error", "gs_ctx_bytes", "gs_ctx_stats",
           "gs_abi_sizes", "gs_project", "gs_bin", "gs_render", "gs_render_backward", "gs_render_saved",
           "gs_saved_outputs", "gs_render_backward_saved", "gs_saved_destroy", "gs_loss", "gs_pose_step",
           "gs_fuse", "gs_register", "gs_register_batch", "gs_register_async", "gs_register_batch_async", "gs_register_gradient", "gs_transform", "gs_render_noalloc", "gs_track_loss",
           "gs_overlap_ratio", "gs_transform_batch", "gs_sort_u32", "gs_selftest_bounded_wait", "gs_probe_fp32",
           "gs_server_create",
           "gs_server_destroy", "gs_server_last_error", "gs_server_submit", "gs_server_step", "gs_server_poll",
           "gs_server_counts", "gs_server_admission", "gs_server_footprint"]

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads the compiled library (building it first if asked and absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libgsreg.so not built ({path}); run __graft_entry__.build()")
            _build.build()
        L = ctypes.CDLL(path)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "gs_default_options": ([P], None),
            "gs_ctx_create": ([I, ctypes.c_size_t, P], I),
            "gs_ctx_destroy": ([P], I),
            "gs_last_error": ([P], ctypes.c_char_p),
            "gs_ctx_bytes": ([P], ctypes.c_size_t),
            "gs_ctx_stats": ([P, P], I),
            "gs_abi_sizes": ([P, I], I),
            "gs_project": ([P, P, P, P, I, P, P, P, P, P], I),
            "gs_bin": ([P, P, P, P, I, I64, P, P, I64, P, P, P], I),
            "gs_render": ([P, P, P, P, I, P, P, P, P, P, P, P], I),
            "gs_render_backward": ([P, P, P, P, I, P, P, P, P, P, P, P, P, P, P], I),
            "gs_render_saved": ([P, P, P, P, I, P, P, P, P, P, P], I),
            "gs_saved_outputs": ([P, P, P], I),
            "gs_render_backward_saved": ([P, P, P, P, P, P, P, P, P], I),
            "gs_saved_destroy": ([P, P], I),
            "gs_loss": ([P, P, I, P, P, P, P, P, P, P, P], I),
            "gs_track_loss": ([P, P, I, P, P, P, P, P, ctypes.c_float, P, P, P, P, P, P], I),
            "gs_overlap_ratio": ([P, P, P, P, ctypes.c_float, P, P, P, P, P], I),
            "gs_transform_batch": ([P, P, I, P, P, P, P], I),
            "gs_sort_u32": ([P, P, P, I64, I, P], I),
            "gs_selftest_bounded_wait": ([P, P, P, I64, P], I),
            "gs_probe_fp32": ([P, P, P, P], I),
            "gs_pose_step": ([P, I, P, P, P, P, I, I, P, P], I),
            "gs_fuse": ([P, I, P, P, P, P, P, P], I),
            "gs_register": ([P, P, P, P, I, P, I, P, I, P, P, P, P, P], I),
            "gs_transform": ([P, P, P, P, P, P], I),
            "gs_render_noalloc": ([P, P, P, I, P, P, P, P, P, P, P], I),
            "gs_register_batch": ([P, P, I, P, I, P, P, P, P], I),
            "gs_register_async": ([P, P, P, P, I, P, I, P, I, P, P, P, P, P, P], I),
            "gs_register_batch_async": ([P, P, I, P, I, P, P, P, P, P], I),
            "gs_register_gradient": ([P, P, P, P, I, P, I, P, P, P, P], I),
            "gs_server_create": ([I, ctypes.c_size_t, I, I, P, P], I),
            "gs_server_destroy": ([P], I),
            "gs_server_last_error": ([P], ctypes.c_char_p),
            "gs_server_submit": ([P, P, I, P], I),
            "gs_server_step": ([P, P, P, I, P], I),
            "gs_server_poll": ([P, I64, P, P, P, P, P, P], I),
            "gs_server_counts": ([P, P], I),
            "gs_server_admission": ([P, P], I),
            "gs_server_footprint": ([P, I64, P, P], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        # the binding's struct layouts must be the library's
        ABI_STRUCTS = abi_structs()
        sizes = (ctypes.c_size_t * len(ABI_STRUCTS))()
        L.gs_abi_sizes(sizes, len(ABI_STRUCTS))
        for st, sz in zip(ABI_STRUCTS, sizes):
            if ctypes.sizeof(st) != sz:
                raise RuntimeError(f"{st.__name__}: binding has {ctypes.sizeof(st)} bytes, library {sz}")
        _lib = L
        return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("device tensor expected")
        if not t.is_contiguous():
            raise ValueError("contiguous tensor expected")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_options(**kw) -> gs_options_t:
    o = gs_options_t()
    load().gs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "bg":
            o.bg = (ctypes.c_float * 3)(*v)
        else:
            setattr(o, k, v)
    return o


def camera(cam18) -> gs_camera_t:
    c = np.asarray(cam18, np.float32).reshape(18)
    out = gs_camera_t(float(c[0]), float(c[1]), float(c[2]), float(c[3]), int(c[4]), int(c[5]))
    out.world_to_cam = (ctypes.c_float * 12)(*[float(v) for v in c[6:]])
    return out


def cameras(cams):
    cams = np.asarray(cams, np.float32).reshape(-1, 18)
    arr = (gs_camera_t * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = camera(c)
    return arr, len(cams)


@dataclass
class Gaussians:
    """Device submap in the C-ABI layout (float32, float4-padded SoA)."""
    means4: torch.Tensor
    log_scales4: torch.Tensor
    quats4: torch.Tensor
    logits: torch.Tensor
    rgb4: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.means4.shape[0])

    @classmethod
    def from_numpy(cls, d, device="cuda"):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
        return cls(f(d["means4"]), f(d["log_scales4"]), f(d["quats4"]), f(d["logits"]), f(d["rgb4"]))

    def c_struct(self) -> gs_gaussians_t:
        return gs_gaussians_t(self.means4.data_ptr(), self.log_scales4.data_ptr(), self.quats4.data_ptr(),
                              self.logits.data_ptr(), self.rgb4.data_ptr(), self.n)


class Context:
    """A gs_ctx_t: scratch arena of at most ``budget_bytes`` on ``device``."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        st = self._lib.gs_ctx_create(int(device), int(budget_bytes), ctypes.byref(self._h))
        if st != 0:
            raise GsError(st, "gs_ctx_create failed")
        self.device = device

    def check(self, st):
        if st != 0:
            raise GsError(st, self._lib.gs_last_error(self._h).decode())

    @property
    def handle(self):
        return self._h

    def bytes(self) -> int:
        return int(self._lib.gs_ctx_bytes(self._h))

    def close(self):
        if self._h:
            self._lib.gs_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _npix(cams):
    c = np.asarray(cams, np.float32).reshape(-1, 18)
    return int(sum(int(x[4]) * int(x[5]) for x in c))


def gs_project(ctx: Context, g: Gaussians, poses: torch.Tensor, cams, opt=None, with_aux=True):
    cam_arr, nc = cameras(cams)
    opt = opt or default_options()
    dev = g.means4.device
    records = torch.empty((nc * g.n, GS_RECORD_FLOATS), dtype=torch.float32, device=dev)
    aux = torch.empty((nc * g.n, GS_AUX_FLOATS), dtype=torch.float32, device=dev) if with_aux else None
    counts = torch.empty(nc * g.n, dtype=torch.int32, device=dev)
    gst = g.c_struct()
    ctx.check(ctx._lib.gs_project(ctx.handle, ctypes.byref(gst), _ptr(poses.contiguous()), cam_arr, nc,
                                  ctypes.byref(opt), _ptr(records), _ptr(aux), _ptr(counts), _stream()))
    return records, aux, counts


def gs_bin(ctx: Context, records, counts, cams, n, capacity=None):
    cam_arr, nc = cameras(cams)
    tiles = sum(((int(c[4]) + 15) // 16) * ((int(c[5]) + 15) // 16) for c in np.asarray(cams).reshape(-1, 18))
    dev = records.device
    ranges = torch.zeros((max(tiles, 1), 2), dtype=torch.int32, device=dev)
    nd = ctypes.c_int64(0)
    if capacity is None:
        capacity = int(counts.to(torch.int64).sum().item())
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    vals = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    ctx.check(ctx._lib.gs_bin(ctx.handle, _ptr(records), _ptr(counts), cam_arr, nc, int(n), _ptr(keys), _ptr(vals),
                              int(capacity), _ptr(ranges), ctypes.byref(nd), _stream()))
    return keys[: nd.value], vals[: nd.value], ranges[:tiles]


def gs_render(ctx: Context, g: Gaussians, poses: torch.Tensor, cams, opt=None):
    cam_arr, nc = cameras(cams)
    opt = opt or default_options()
    npx = _npix(cams)
    dev = g.means4.device
    out = dict(rgb=torch.empty(3 * npx, device=dev), depth=torch.empty(npx, device=dev),
               alpha=torch.empty(npx, device=dev), t_final=torch.empty(npx, device=dev),
               last=torch.empty(npx, dtype=torch.int32, device=dev))
    gst = g.c_struct()
    ctx.check(ctx._lib.gs_render(ctx.handle, ctypes.byref(gst), _ptr(poses.contiguous()), cam_arr, nc,
                                 ctypes.byref(opt), _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["alpha"]),
                                 _ptr(out["t_final"]), _ptr(out["last"]), _stream()))
    return out


def split_views(flat, cams, channels):
    """Splits a concatenated per-camera buffer into [channels, H, W] views."""
    out, o = [], 0
    for c in np.asarray(cams).reshape(-1, 18):
        W, H = int(c[4]), int(c[5])
        out.append(flat[o: o + channels * H * W].view(channels, H, W) if channels > 1
                   else flat[o: o + H * W].view(H, W))
        o += channels * H * W
    return out


def gs_render_backward(ctx: Context, g: Gaussians, poses, cams, t_final, last, d_rgb=None, d_depth=None,
                       d_alpha=None, pivots=None, opt=None, params=False):
    """Pose twist gradient [n_cams, 6]; with ``params`` also the per-Gaussian
    gradients as a dict in the submap layout (means4, log_scales4, quats4,
    logits, rgb4)."""
    cam_arr, nc = cameras(cams)
    opt = opt or default_options()
    dev = g.means4.device
    pose_grad = torch.empty((nc, 6), dtype=torch.float32, device=dev)
    gst = g.c_struct()
    out, grads = None, None
    if params:
        out = dict(means4=torch.empty_like(g.means4), log_scales4=torch.empty_like(g.log_scales4),
                   quats4=torch.empty_like(g.quats4), logits=torch.empty_like(g.logits), rgb4=torch.empty_like(g.rgb4))
        grads = ctypes.byref(gs_gaussian_grads_t(out["means4"].data_ptr(), out["log_scales4"].data_ptr(),
                                                 out["quats4"].data_ptr(), out["logits"].data_ptr(),
                                                 out["rgb4"].data_ptr()))
    ctx.check(ctx._lib.gs_render_backward(ctx.handle, ctypes.byref(gst), _ptr(poses.contiguous()), cam_arr, nc,
                                          ctypes.byref(opt), _ptr(t_final), _ptr(last), _ptr(d_rgb),
                                          _ptr(d_depth), _ptr(d_alpha), _ptr(pivots), _ptr(pose_grad), grads,
                                          _stream()))
    return (pose_grad, out) if params else pose_grad


class Saved:
    """A forward pass kept for its adjoint (gs_render_saved); freed on
    close() or when collected.  Keeps the submap, poses and options alive."""

    def __init__(self, ctx: Context, handle, g: Gaussians, poses, cams, npx):
        self.ctx, self.handle, self.g, self.poses, self.cams = ctx, handle, g, poses, cams
        tf, last = ctypes.c_void_p(), ctypes.c_void_p()
        ctx.check(ctx._lib.gs_saved_outputs(handle, ctypes.byref(tf), ctypes.byref(last)))
        self._tf, self._last, self.npx = tf.value, last.value, npx

    def close(self, stream=None):
        if self.handle:
            self.ctx._lib.gs_saved_destroy(self.handle, stream if stream is not None else _stream())
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_render_saved(ctx: Context, g: Gaussians, poses: torch.Tensor, cams, opt=None):
    """gs_render that keeps its projection, tile lists and per-pixel state
    for gs_render_backward_saved.  Returns (dict(rgb, depth, alpha), Saved)."""
    cam_arr, nc = cameras(cams)
    opt = opt or default_options()
    npx = _npix(cams)
    dev = g.means4.device
    out = dict(rgb=torch.empty(3 * npx, device=dev), depth=torch.empty(npx, device=dev),
               alpha=torch.empty(npx, device=dev))
    gst = g.c_struct()
    h = ctypes.c_void_p()
    poses = poses.contiguous()
    ctx.check(ctx._lib.gs_render_saved(ctx.handle, ctypes.byref(gst), _ptr(poses), cam_arr, nc, ctypes.byref(opt),
                                       _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["alpha"]), ctypes.byref(h),
                                       _stream()))
    sv = Saved(ctx, h, g, poses, cams, npx)
    sv.opt = opt
    return out, sv


def gs_render_backward_saved(ctx: Context, saved: Saved, d_rgb=None, d_depth=None, d_alpha=None, pivots=None,
                             params=False):
    """gs_render_backward from a saved forward: pose twist gradient
    [n_cams, 6], and with ``params`` the per-Gaussian gradients."""
    nc = len(np.asarray(saved.cams).reshape(-1, 18))
    g = saved.g
    dev = g.means4.device
    pose_grad = torch.empty((nc, 6), dtype=torch.float32, device=dev)
    out, grads = None, None
    if params:
        out = dict(means4=torch.empty_like(g.means4), log_scales4=torch.empty_like(g.log_scales4),
                   quats4=torch.empty_like(g.quats4), logits=torch.empty_like(g.logits), rgb4=torch.empty_like(g.rgb4))
        grads = ctypes.byref(gs_gaussian_grads_t(out["means4"].data_ptr(), out["log_scales4"].data_ptr(),
                                                 out["quats4"].data_ptr(), out["logits"].data_ptr(),
                                                 out["rgb4"].data_ptr()))
    ctx.check(ctx._lib.gs_render_backward_saved(ctx.handle, saved.handle, _ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha),
                                                _ptr(pivots), _ptr(pose_grad), grads, _stream()))
    return (pose_grad, out) if params else pose_grad


def gs_loss(ctx: Context, cams, rgb, depth, t_rgb, t_depth):
    cam_arr, nc = cameras(cams)
    dev = rgb.device
    loss = torch.empty(nc, dtype=torch.float64, device=dev)
    d_rgb = torch.empty_like(rgb)
    d_depth = torch.empty_like(depth)
    ctx.check(ctx._lib.gs_loss(ctx.handle, cam_arr, nc, _ptr(rgb), _ptr(depth), _ptr(t_rgb), _ptr(t_depth),
                               _ptr(loss), _ptr(d_rgb), _ptr(d_depth), _stream()))
    return loss, d_rgb, d_depth


def gs_track_loss(ctx: Context, cams, rgb, depth, t_final, t_rgb, t_depth, lambda_c=0.6):
    """Tracking loss (Eq. 2 with the masks of Supp. A) of rendered images.
    Returns (loss [n] float64, d_rgb, d_depth, inlier (uint8 per pixel),
    median [n] float32)."""
    cam_arr, nc = cameras(cams)
    dev = rgb.device
    loss = torch.empty(nc, dtype=torch.float64, device=dev)
    d_rgb = torch.empty_like(rgb)
    d_depth = torch.empty_like(depth)
    inl = torch.empty(depth.shape, dtype=torch.uint8, device=dev)
    med = torch.empty(nc, dtype=torch.float32, device=dev)
    ctx.check(ctx._lib.gs_track_loss(ctx.handle, cam_arr, nc, _ptr(rgb), _ptr(depth), _ptr(t_final), _ptr(t_rgb),
                                     _ptr(t_depth), float(lambda_c), _ptr(loss), _ptr(d_rgb), _ptr(d_depth),
                                     _ptr(inl), _ptr(med), _stream()))
    return loss, d_rgb, d_depth, inl, med


def gs_overlap_ratio(ctx: Context, p: Gaussians, q: Gaussians, T, tau=0.2, with_nn=False):
    """Overlap ratio of P and Q under T_{P->Q} (loop filter).  Returns
    (OR, |K|) or, with ``with_nn``, (OR, |K|, nn_pq, nn_qp) device int32."""
    Th = np.ascontiguousarray(np.asarray(T, np.float64).reshape(12))
    ratio, k = ctypes.c_double(), ctypes.c_int64()
    nn_pq = torch.empty(max(p.n, 1), dtype=torch.int32, device=p.means4.device) if with_nn else None
    nn_qp = torch.empty(max(q.n, 1), dtype=torch.int32, device=p.means4.device) if with_nn else None
    pst, qst = p.c_struct(), q.c_struct()
    ctx.check(ctx._lib.gs_overlap_ratio(ctx.handle, ctypes.byref(pst), ctypes.byref(qst),
                                        Th.ctypes.data_as(ctypes.c_void_p), float(tau), ctypes.byref(ratio),
                                        ctypes.byref(k), _ptr(nn_pq), _ptr(nn_qp), _stream()))
    if with_nn:
        return ratio.value, k.value, nn_pq[:p.n], nn_qp[:q.n]
    return ratio.value, k.value


def gs_pose_step(ctx: Context, pose, state, grad, pivot, k, iters, opt=None):
    """In place on ``pose`` [n,12] and ``state`` [n,13] (float64 CUDA)."""
    opt = opt or default_options()
    ctx.check(ctx._lib.gs_pose_step(ctx.handle, int(pose.shape[0]), _ptr(pose), _ptr(state), _ptr(grad),
                                    _ptr(pivot), int(k), int(iters), ctypes.byref(opt), _stream()))


def gs_fuse(ctx: Context, est, reverse, eps):
    dev = est.device
    T = torch.empty(12, dtype=torch.float64, device=dev)
    conf = torch.empty(1, dtype=torch.float64, device=dev)
    ctx.check(ctx._lib.gs_fuse(ctx.handle, int(est.shape[0]), _ptr(est.contiguous()), _ptr(reverse.contiguous()),
                               _ptr(eps.contiguous()), _ptr(T), _ptr(conf), _stream()))
    return T, conf


def _views(views):
    arr = (gs_view_t * max(len(views), 1))()
    for k, (cam18, rgb, depth) in enumerate(views):
        arr[k] = gs_view_t(rgb.data_ptr(), depth.data_ptr(), camera(cam18))
    return arr


def gs_register(ctx: Context, src: Gaussians, tgt: Gaussians, src_views, tgt_views, iters, opt=None):
    """3DGS registration of src (P) and tgt (Q).  ``*_views`` are lists of
    (cam18, rgb [3,H,W] CUDA, depth [H,W] CUDA).  Returns (T_{P->Q} [3,4]
    float64 numpy, confidence, eps [n], per-keyframe estimates [n,3,4])."""
    opt = opt or default_options()
    for _, rgb, depth in list(src_views) + list(tgt_views):
        if not (rgb.is_cuda and depth.is_cuda and rgb.is_contiguous() and depth.is_contiguous()):
            raise ValueError("keyframe images must be contiguous CUDA tensors")
    sv, tv = _views(src_views), _views(tgt_views)
    n = len(src_views) + len(tgt_views)
    T = np.zeros(12, np.float64)
    conf = ctypes.c_double(0)
    eps = np.zeros(max(n, 1), np.float64)
    est = np.zeros((max(n, 1), 12), np.float64)
    s, t = src.c_struct(), tgt.c_struct()
    d = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ctx.check(ctx._lib.gs_register(ctx.handle, ctypes.byref(s), ctypes.byref(t), sv, len(src_views), tv,
                                   len(tgt_views), ctypes.byref(opt), int(iters), d(T), ctypes.byref(conf), d(eps),
                                   d(est), _stream()))
    return T.reshape(3, 4), conf.value, eps[:n], est[:n].reshape(n, 3, 4)


def gs_register_gradient(ctx: Context, src: Gaussians, tgt: Gaussians, src_views, tgt_views, opt=None):
    """The registration loss and its pose gradient at the starting poses of
    the keyframe problems gs_register would set up.  Returns (loss [n],
    grad [n,6] world-frame twists about the moving submap's centroid)."""
    opt = opt or default_options()
    for _, rgb, depth in list(src_views) + list(tgt_views):
        if not (rgb.is_cuda and depth.is_cuda and rgb.is_contiguous() and depth.is_contiguous()):
            raise ValueError("keyframe images must be contiguous CUDA tensors")
    sv, tv = _views(src_views), _views(tgt_views)
    n = len(src_views) + len(tgt_views)
    loss = np.zeros(max(n, 1), np.float64)
    grad = np.zeros((max(n, 1), 6), np.float64)
    s, t = src.c_struct(), tgt.c_struct()
    d = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ctx.check(ctx._lib.gs_register_gradient(ctx.handle, ctypes.byref(s), ctypes.byref(t), sv, len(src_views), tv,
                                            len(tgt_views), ctypes.byref(opt), d(loss), d(grad), _stream()))
    return loss[:n], grad[:n]


def gs_transform(ctx: Context, g: Gaussians, T) -> Gaussians:
    """Rigid transform of a submap (Eq. 8/9) on the device."""
    Th = np.ascontiguousarray(np.asarray(T, np.float64).reshape(12))
    m = torch.empty_like(g.means4)
    q = torch.empty_like(g.quats4)
    gst = g.c_struct()
    ctx.check(ctx._lib.gs_transform(ctx.handle, ctypes.byref(gst), Th.ctypes.data_as(ctypes.c_void_p), _ptr(m),
                                    _ptr(q), _stream()))
    return Gaussians(m, g.log_scales4.clone(), q, g.logits.clone(), g.rgb4.clone())


def gs_sort_u32(ctx: Context, keys, vals, bits=32):
    """Stable device sort of (keys, vals) (32-bit CUDA tensors, in place) by
    the low ``bits`` key bits."""
    ctx.check(ctx._lib.gs_sort_u32(ctx.handle, _ptr(keys), _ptr(vals), int(keys.numel()), int(bits), _stream()))
    return keys, vals


def gs_probe_fp32(ctx: Context):
    """Measured FP32 FMA throughput of the device: (TFLOP/s, SM count)."""
    tf, sms = ctypes.c_double(), ctypes.c_int()
    ctx.check(ctx._lib.gs_probe_fp32(ctx.handle, ctypes.byref(tf), ctypes.byref(sms), _stream()))
    return tf.value, sms.value


def gs_transform_batch(ctx: Context, maps, Ts):
    """Map adjustment: every submap of ``maps`` moved by its own T (Eq. 8/9)
    in one launch.  Returns new Gaussians per map."""
    n = len(maps)
    arr = (gs_gaussians_t * max(n, 1))(*[g.c_struct() for g in maps])
    Th = np.ascontiguousarray(np.asarray(Ts, np.float64).reshape(n, 12))
    outs = [(torch.empty_like(g.means4), torch.empty_like(g.quats4)) for g in maps]
    om = (ctypes.c_void_p * max(n, 1))(*[m.data_ptr() for m, _ in outs])
    oq = (ctypes.c_void_p * max(n, 1))(*[q.data_ptr() for _, q in outs])
    ctx.check(ctx._lib.gs_transform_batch(ctx.handle, arr, n, Th.ctypes.data_as(ctypes.c_void_p), om, oq, _stream()))
    return [Gaussians(m, g.log_scales4, q, g.logits, g.rgb4) for g, (m, q) in zip(maps, outs)]


def gs_render_noalloc(g: Gaussians, poses: torch.Tensor, cams, opt=None, out=None):
    """gs_render without a context and without any device allocation by the
    library: its scratch is a fixed device array (see include/gsreg.h), for
    callers whose host program forbids cudaMalloc / cudaFree at run time.
    ``out`` may hold caller-allocated output tensors (rgb, depth, alpha,
    t_final, last); missing ones are created here with torch.  Returns the
    status code (0 = GS_OK) and the outputs."""
    cam_arr, nc = cameras(cams)
    opt = opt or default_options()
    npx = _npix(cams)
    dev = g.means4.device
    if poses.dtype != torch.float32 or tuple(poses.shape) != (nc, 12) or poses.device != dev:
        raise ValueError(f"poses must be float32 [{nc}, 12] on {dev}")
    # the C call runs on the current device: make it the submap's
    with torch.cuda.device(dev):
        out = dict(out or {})
        out.setdefault("rgb", torch.empty(3 * npx, device=dev))
        out.setdefault("depth", torch.empty(npx, device=dev))
        out.setdefault("alpha", torch.empty(npx, device=dev))
        out.setdefault("t_final", torch.empty(npx, device=dev))
        out.setdefault("last", torch.empty(npx, dtype=torch.int32, device=dev))
        gst = g.c_struct()
        st = load().gs_render_noalloc(ctypes.byref(gst), _ptr(poses.contiguous()), cam_arr, nc, ctypes.byref(opt),
                                      _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["alpha"]),
                                      _ptr(out["t_final"]), _ptr(out["last"]), _stream())
    return st, out


class gs_problem_t(ctypes.Structure):
    _fields_ = [("src", gs_gaussians_t), ("tgt", gs_gaussians_t), ("src_views", ctypes.c_void_p),
                ("n_src_views", ctypes.c_int32), ("tgt_views", ctypes.c_void_p), ("n_tgt_views", ctypes.c_int32),
                ("opt", ctypes.c_void_p)]


def _problem(p, keep):
    """gs_problem_t of (src, tgt, src_views, tgt_views[, options]); the ctypes
    arrays it points to are appended to ``keep``."""
    s, t, sv, tv = p[:4]
    o = p[4] if len(p) > 4 else None
    sva, tva = _views(sv), _views(tv)
    keep += [sva, tva, o]
    return gs_problem_t(s.c_struct(), t.c_struct(), ctypes.cast(sva, ctypes.c_void_p), len(sv),
                        ctypes.cast(tva, ctypes.c_void_p), len(tv),
                        ctypes.cast(ctypes.pointer(o), ctypes.c_void_p) if o is not None else None)


def gs_register_batch(ctx: Context, problems, iters, opt=None):
    """Batched registration.  ``problems``: list of (src Gaussians, tgt
    Gaussians, src_views, tgt_views[, gs_options_t of this problem]) with
    views as in gs_register.  Returns (T [n,3,4] float64, confidence [n],
    eps [sum of keyframes])."""
    opt = opt or default_options()
    n = len(problems)
    arr = (gs_problem_t * n)()
    keep = []
    total = 0
    for i, p in enumerate(problems):
        arr[i] = _problem(p, keep)
        total += len(p[2]) + len(p[3])
    T = np.zeros((n, 12), np.float64)
    conf = np.zeros(n, np.float64)
    eps = np.zeros(max(total, 1), np.float64)
    d = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ctx.check(ctx._lib.gs_register_batch(ctx.handle, arr, n, ctypes.byref(opt), int(iters), d(T), d(conf), d(eps),
                                         _stream()))
    return T.reshape(n, 3, 4), conf, eps[:total]


def gs_register_async(ctx: Context, src: Gaussians, tgt: Gaussians, src_views, tgt_views, iters, opt=None,
                      out=None):
    """gs_register enqueued on the current stream with device outputs (no
    host synchronisation once the plan shape's list size is known).  Returns
    dict(T [3,4], conf [1], eps [n], est [n,3,4] float64, status [1] int32),
    all CUDA tensors, valid once the stream reaches them; ``out`` may supply
    them.  The returned dict also keeps the keyframe arrays the call reads."""
    opt = opt or default_options()
    n = len(src_views) + len(tgt_views)
    dev = src.means4.device
    o = dict(out or {})
    o.setdefault("T", torch.empty((3, 4), dtype=torch.float64, device=dev))
    o.setdefault("conf", torch.empty(1, dtype=torch.float64, device=dev))
    o.setdefault("eps", torch.empty(max(n, 1), dtype=torch.float64, device=dev))
    o.setdefault("est", torch.empty((max(n, 1), 3, 4), dtype=torch.float64, device=dev))
    o.setdefault("status", torch.full((1,), -1, dtype=torch.int32, device=dev))
    sv, tv = _views(src_views), _views(tgt_views)
    s, t = src.c_struct(), tgt.c_struct()
    ctx.check(ctx._lib.gs_register_async(ctx.handle, ctypes.byref(s), ctypes.byref(t), sv, len(src_views), tv,
                                         len(tgt_views), ctypes.byref(opt), int(iters), _ptr(o["T"]), _ptr(o["conf"]),
                                         _ptr(o["eps"]), _ptr(o["est"]), _ptr(o["status"]), _stream()))
    o["_keep"] = (src, tgt, src_views, tgt_views)
    return o


def gs_register_batch_async(ctx: Context, problems, iters, opt=None):
    """gs_register_batch enqueued on the current stream with device outputs:
    dict(T [n,3,4], conf [n], eps [keyframes] float64, status [1] int32)."""
    opt = opt or default_options()
    n = len(problems)
    arr = (gs_problem_t * n)()
    keep = []
    total = 0
    for i, p in enumerate(problems):
        arr[i] = _problem(p, keep)
        total += len(p[2]) + len(p[3])
    dev = problems[0][0].means4.device
    o = dict(T=torch.empty((n, 3, 4), dtype=torch.float64, device=dev),
             conf=torch.empty(n, dtype=torch.float64, device=dev),
             eps=torch.empty(max(total, 1), dtype=torch.float64, device=dev),
             status=torch.full((1,), -1, dtype=torch.int32, device=dev))
    ctx.check(ctx._lib.gs_register_batch_async(ctx.handle, arr, n, ctypes.byref(opt), int(iters), _ptr(o["T"]),
                                               _ptr(o["conf"]), _ptr(o["eps"]), _ptr(o["status"]), _stream()))
    o["_keep"] = (problems, keep)
    return o


class Server:
    """Continuous-batching registration server (gs_server_*).  Requests are
    registration problems as in gs_register_batch -- (src, tgt, src_views,
    tgt_views) -- with their own iteration count; a tracking request is
    (submap, submap, [], [frame view]).  The caller keeps every array of a
    request alive until it is done (this object keeps references)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, max_keyframes: int = 256, max_round_iters: int = 10,
                 opt=None):
        self._lib = load()
        self.opt = opt or default_options()
        h = ctypes.c_void_p()
        st = self._lib.gs_server_create(int(device), int(budget_bytes), int(max_keyframes), int(max_round_iters),
                                        ctypes.byref(self.opt), ctypes.byref(h))
        if st != 0:
            raise GsError(st, "gs_server_create failed")
        self.handle = h
        self._keep = {}
        self._nvps = {}

    def check(self, st):
        if st != 0:
            raise GsError(st, self._lib.gs_server_last_error(self.handle).decode())

    def submit(self, src: Gaussians, tgt: Gaussians, src_views, tgt_views, iters: int, opt=None) -> int:
        """Queues a request; ``opt`` (gs_options_t or None = the server's)
        sets its learning rates and loss."""
        keep = []
        q = _problem((src, tgt, src_views, tgt_views, opt), keep)
        rid = ctypes.c_int64()
        self.check(self._lib.gs_server_submit(self.handle, ctypes.byref(q), int(iters), ctypes.byref(rid)))
        self._keep[rid.value] = (src, tgt, src_views, tgt_views, keep)
        self._nvps[rid.value] = len(src_views) + len(tgt_views)
        return rid.value

    def step(self, max_done: int = 4096):
        """One round; returns the ids retired in it."""
        ids = (ctypes.c_int64 * max_done)()
        n = ctypes.c_int()
        self.check(self._lib.gs_server_step(self.handle, _stream(), ids, max_done, ctypes.byref(n)))
        done = [ids[k] for k in range(min(n.value, max_done))]
        for i in done:
            self._keep.pop(i, None)
        return done

    def poll(self, rid: int):
        """dict(state, T [3,4], confidence, eps, t_submit, t_done)."""
        state = ctypes.c_int()
        T = np.zeros(12, np.float64)
        conf = ctypes.c_double()
        eps = np.zeros(max(self._nvps.get(rid, 1), 1), np.float64)
        ts, td = ctypes.c_double(), ctypes.c_double()
        self.check(self._lib.gs_server_poll(self.handle, int(rid), ctypes.byref(state), T.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(conf), eps.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(ts), ctypes.byref(td)))
        return dict(state=state.value, T=T.reshape(3, 4), confidence=conf.value, eps=eps, t_submit=ts.value,
                    t_done=td.value)

    def counts(self):
        """(waiting, in flight, done, rounds, re-plans)."""
        out = (ctypes.c_int64 * 5)()
        self.check(self._lib.gs_server_counts(self.handle, out))
        return tuple(out)

    def admission(self):
        """(requests measured, requests held back by the memory budget,
        bytes in flight)."""
        out = (ctypes.c_int64 * 3)()
        self.check(self._lib.gs_server_admission(self.handle, out))
        return tuple(out)

    def footprint(self, rid: int):
        """(tile duplicates at the starting poses, scratch bytes) of a request."""
        d, b = ctypes.c_int64(), ctypes.c_int64()
        self.check(self._lib.gs_server_footprint(self.handle, int(rid), ctypes.byref(d), ctypes.byref(b)))
        return d.value, b.value

    def close(self):
        if self.handle:
            self._lib.gs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def abi_structs():
    """The ABI structs in the order gs_abi_sizes reports them."""
    return [gs_gaussians_t, gs_camera_t, gs_view_t, gs_options_t, gs_stats_t, gs_gaussian_grads_t, gs_problem_t]
