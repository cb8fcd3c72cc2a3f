"""gs_render_noalloc, the context-free render for callers that may not
allocate device memory (host programs that own all device memory, or loops
where an allocation would synchronise the device), must give what
gs_render gives.  Collected last on purpose: if it fails, a run that stops
at the first failure has already run every other test."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2408_10154_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GS_ERR_CAPACITY = 7
SCRATCH = 32 << 20  # GS_NOALLOC_SCRATCH_BYTES
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_10154_gb300 as gsmod
    from paper_2408_10154_gb300 import build
    build.build()
    return gsmod


def poses_for(k, seed):
    rng = np.random.default_rng(seed)
    P = np.stack([synth.random_rigid(rng, 4.0, 0.04) for _ in range(k)]).reshape(k, 12)
    return torch.tensor(P, dtype=torch.float32, device="cuda")


def compare(a, b):
    # the same kernels on the same inputs: the render tolerance of the other
    # tests (1e-4 max-abs) and bit-equal integer / transmittance outputs
    for k in ("rgb", "depth", "alpha"):
        assert float((a[k] - b[k]).abs().max()) <= 1e-4, k
    assert torch.equal(a["t_final"], b["t_final"])
    assert torch.equal(a["last"], b["last"])


def sentinel_outputs(cams):
    npx = sum(int(c[4]) * int(c[5]) for c in np.asarray(cams).reshape(-1, 18))
    return dict(rgb=torch.full((3 * npx,), -7.0, device="cuda"), depth=torch.full((npx,), -7.0, device="cuda"),
                alpha=torch.full((npx,), -7.0, device="cuda"), t_final=torch.full((npx,), -7.0, device="cuda"),
                last=torch.full((npx,), 12345, dtype=torch.int32, device="cuda"))


def untouched(out):
    return all(bool((v == (12345 if k == "last" else -7.0)).all()) for k, v in out.items())


def test_noalloc_render_matches_render_on_two_calls_in_a_row(gs):
    ctx = gs.Context(0)
    c1 = synth.plain_2k()
    c2 = synth.small_case(700, 100, 70, 70.0, n_views=3, seed=9, ls_mean=-3.5)
    for case, seed in ((c1, 21), (c2, 22)):
        g = gs.Gaussians.from_numpy(case["gaussians"])
        P = poses_for(len(case["cams"]), seed)
        ref = gs.gs_render(ctx, g, P, case["cams"])
        st, out = gs.gs_render_noalloc(g, P, case["cams"])
        assert st == 0
        compare(out, ref)
    ctx.close()


def test_noalloc_render_rejects_records_beyond_its_scratch(gs):
    # 8 x 150k records need more than the 32 MiB before any duplicate is
    # counted: rejected before any GPU work, outputs untouched
    c = synth.room_150k()
    g = gs.Gaussians.from_numpy(c["gaussians"])
    P = poses_for(8, 23)
    out = sentinel_outputs(c["src_cams"])
    st, out = gs.gs_render_noalloc(g, P, c["src_cams"], out=out)
    assert st == GS_ERR_CAPACITY
    assert untouched(out)


def test_noalloc_render_rejects_duplicates_beyond_its_scratch(gs):
    # few records (5k, 0.3 MB) with large screen footprints (about 60 px
    # standard deviation): the records fit, their ~1.7 M tile duplicates do
    # not; rejected after counting them, outputs untouched
    c = synth.small_case(5000, 640, 480, 320.0, n_views=1, seed=24, ls_mean=-1.0, ls_std=0.1, half=0.25)
    g = gs.Gaussians.from_numpy(c["gaussians"])
    P = torch.tensor(np.eye(3, 4).reshape(1, 12), dtype=torch.float32, device="cuda")
    ctx = gs.Context(0)
    _, _, counts = gs.gs_project(ctx, g, P, c["cams"], with_aux=False)
    dups = int(counts.to(torch.int64).sum())
    ctx.close()
    assert 52 * g.n < SCRATCH < 24 * dups, (g.n, dups)
    out = sentinel_outputs(c["cams"])
    st, out = gs.gs_render_noalloc(g, P, c["cams"], out=out)
    assert st == GS_ERR_CAPACITY
    assert untouched(out)


def test_noalloc_render_accepts_work_close_to_its_scratch(gs):
    # about 52 B per record and 24.5 B per tile duplicate: a scene sized to
    # fill 75-95 % of the scratch is accepted and equals gs_render
    c = synth.small_case(200_000, 800, 600, 400.0, n_views=1, seed=25, ls_mean=-3.8, ls_std=0.3, half=0.6)
    full = c["gaussians"]
    P = torch.tensor(np.eye(3, 4).reshape(1, 12), dtype=torch.float32, device="cuda")
    ctx = gs.Context(0)
    _, _, counts = gs.gs_project(ctx, gs.Gaussians.from_numpy(full), P, c["cams"], with_aux=False)
    per = counts.to(torch.float64).mean().item()
    n = int(0.85 * SCRATCH / (52.0 + 24.5 * per))
    assert n < len(full["logits"]), n
    sub = {k: v[:n] for k, v in full.items()}
    g = gs.Gaussians.from_numpy(sub)
    _, _, counts = gs.gs_project(ctx, g, P, c["cams"], with_aux=False)
    use = 52.0 * n + 24.5 * int(counts.to(torch.int64).sum())
    assert 0.75 * SCRATCH < use < 0.95 * SCRATCH, use / SCRATCH
    ref = gs.gs_render(ctx, g, P, c["cams"])
    for _ in range(2):
        st, out = gs.gs_render_noalloc(g, P, c["cams"])
        assert st == 0
        compare(out, ref)
    ctx.close()


# Runs in a fresh process: the render in the primary context, then in a
# context made with the driver API (inputs and outputs allocated there), then
# in the primary context again.  The scratch has a different device address
# in each context, so each must look up its own.
CHILD = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2408_10154_gb300 as gs
from paper_2408_10154_gb300 import synth
torch.cuda.set_device(0)
case = synth.plain_2k()
gd, cams = case["gaussians"], case["cams"]
rng = np.random.default_rng(31)
P = np.stack([synth.random_rigid(rng, 4.0, 0.04) for _ in range(len(cams))]).reshape(-1, 12).astype(np.float32)
ctx = gs.Context(0)
g = gs.Gaussians.from_numpy(gd)
Pd = torch.tensor(P, device="cuda")
ref = {k: v.cpu().numpy() for k, v in gs.gs_render(ctx, g, Pd, cams).items()}

def check(out, what):
    for k in ("rgb", "depth", "alpha"):
        assert np.abs(out[k] - ref[k]).max() <= 1e-4, (what, k)
    assert np.array_equal(out["t_final"].view(np.uint32), ref["t_final"].view(np.uint32)), what
    assert np.array_equal(out["last"], ref["last"]), what

st, out = gs.gs_render_noalloc(g, Pd, cams)
assert st == 0, st
check({k: v.cpu().numpy() for k, v in out.items()}, "primary")
torch.cuda.synchronize()

cu = ctypes.CDLL("libcuda.so.1")
U64, VP, SZ = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
cu.cuMemAlloc_v2.argtypes = [ctypes.POINTER(U64), SZ]
cu.cuMemcpyHtoD_v2.argtypes = [U64, VP, SZ]
cu.cuMemcpyDtoH_v2.argtypes = [VP, U64, SZ]
cu.cuMemFree_v2.argtypes = [U64]
cu.cuCtxCreate_v2.argtypes = [ctypes.POINTER(VP), ctypes.c_uint, ctypes.c_int]
cu.cuCtxDestroy_v2.argtypes = [VP]
dev = ctypes.c_int()
assert cu.cuInit(0) == 0
assert cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
c2 = VP()
assert cu.cuCtxCreate_v2(ctypes.byref(c2), 0, dev) == 0   # current on this thread from here
bufs = []

def upload(a):
    a = np.ascontiguousarray(a)
    p = U64()
    assert cu.cuMemAlloc_v2(ctypes.byref(p), max(a.nbytes, 4)) == 0
    assert cu.cuMemcpyHtoD_v2(p, a.ctypes.data_as(VP), a.nbytes) == 0
    bufs.append(p)
    return p.value

def alloc(nbytes):
    p = U64()
    assert cu.cuMemAlloc_v2(ctypes.byref(p), nbytes) == 0
    bufs.append(p)
    return p.value

f32 = lambda a: np.asarray(a, np.float32)
gst = gs.gsreg.gs_gaussians_t(upload(f32(gd["means4"])), upload(f32(gd["log_scales4"])), upload(f32(gd["quats4"])),
                              upload(f32(gd["logits"])), upload(f32(gd["rgb4"])), len(gd["logits"]))
pose_d = upload(P)
npx = sum(int(c[4]) * int(c[5]) for c in cams)
outs = dict(rgb=(alloc(12 * npx), 3 * npx, np.float32), depth=(alloc(4 * npx), npx, np.float32),
            alpha=(alloc(4 * npx), npx, np.float32), t_final=(alloc(4 * npx), npx, np.float32),
            last=(alloc(4 * npx), npx, np.int32))
cam_arr, nc = gs.gsreg.cameras(cams)
opt = gs.default_options()
lib = gs.gsreg.load()
for rep in range(2):
    st = lib.gs_render_noalloc(ctypes.byref(gst), VP(pose_d), cam_arr, nc, ctypes.byref(opt),
                               *[VP(outs[k][0]) for k in ("rgb", "depth", "alpha", "t_final", "last")], None)
    assert st == 0, st
    assert cu.cuCtxSynchronize() == 0
    host = {}
    for k, (p, n, dt) in outs.items():
        h = np.empty(n, dt)
        assert cu.cuMemcpyDtoH_v2(h.ctypes.data_as(VP), p, h.nbytes) == 0
        host[k] = h
    check(host, "second context")
for p in bufs:
    cu.cuMemFree_v2(p)
assert cu.cuCtxDestroy_v2(c2) == 0
torch.cuda.set_device(0)
st, out = gs.gs_render_noalloc(g, Pd, cams)
assert st == 0, st
check({k: v.cpu().numpy() for k, v in out.items()}, "primary again")
ctx.close()
print("ok")
"""


def test_noalloc_render_in_a_driver_api_context(gs):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-4000:]
