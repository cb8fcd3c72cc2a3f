"""gs_render_noalloc, the context-free render for callers that may not
allocate device memory (host programs that own all device memory, or loops
where an allocation would synchronise the device), must give what
gs_render gives.  Collected last on purpose: if it fails, a run that stops
at the first failure has already run every other test."""
import numpy as np
import pytest

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


def test_noalloc_render_rejects_work_beyond_its_scratch(gs):
    c = synth.room_150k()
    g = gs.Gaussians.from_numpy(c["gaussians"])
    P = poses_for(8, 23)
    st, _ = gs.gs_render_noalloc(g, P, c["src_cams"])  # 1.2 M records > 32 MiB of scratch
    assert st == GS_ERR_CAPACITY
