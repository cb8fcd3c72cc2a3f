"""Overlap ratio (loop filter) on the GPU vs the oracle: nearest-neighbour
indices, |K| and OR bit-exact (FP32 distances on both sides, ties to the
smaller index); at room size on a sample of queries."""
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


def dev_g(gs, og):
    d = dict(means4=og.means4, log_scales4=og.log_scales4, quats4=og.quats4, logits=og.logits, rgb4=og.rgb4)
    return gs.Gaussians.from_numpy(d)


def check(gs, ctx, op, oq, T, tau=0.2):
    r, k, nn_pq, nn_qp = O.overlap_ratio(op, oq, T, tau)
    rg, kg, gpq, gqp = gs.gs_overlap_ratio(ctx, dev_g(gs, op), dev_g(gs, oq), T, tau, with_nn=True)
    np.testing.assert_array_equal(gpq.cpu().numpy(), nn_pq)
    np.testing.assert_array_equal(gqp.cpu().numpy(), nn_qp)
    assert (kg, rg) == (k, r)
    return r, k


def test_overlap_plain_2k(gs, ctx):
    c = synth.plain_2k()
    g = O.Gaussians.from_dict(c["gaussians"])
    q = O.transform(g, c["T_gt"])
    est = synth.compose(synth.about_point(synth.random_rigid(np.random.default_rng(5), 1.0, 0.01),
                                          synth.centroid(c["gaussians"])), c["T_gt"])
    r, k = check(gs, ctx, g, q, est, tau=0.02)
    assert 0.0 < r < 1.0 and k > 100
    check(gs, ctx, g, q, c["T_gt"], tau=0.01)


def test_overlap_ragged_ties_and_empty(gs, ctx):
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, (1037, 3))
    # Q holds every point of a grid twice (exact ties) plus P's first points
    grid = np.stack(np.meshgrid(*[np.linspace(-1, 1, 7)] * 3), -1).reshape(-1, 3)
    y = np.concatenate([grid, grid, x[:100]])

    def pts(a):
        a = np.asarray(a, np.float32)
        return O.Gaussians(np.concatenate([a, np.zeros((len(a), 1), np.float32)], 1), np.zeros((len(a), 4)),
                           np.tile([1.0, 0, 0, 0], (len(a), 1)), np.zeros(len(a)), np.zeros((len(a), 4)))

    check(gs, ctx, pts(x), pts(y), np.eye(3, 4))
    check(gs, ctx, pts(grid), pts(y), synth.random_rigid(rng, 3.0, 0.05))
    assert gs.gs_overlap_ratio(ctx, dev_g(gs, pts(x)), dev_g(gs, pts(np.zeros((0, 3)))), np.eye(3, 4)) == (0.0, 0)
    assert gs.gs_overlap_ratio(ctx, dev_g(gs, pts(np.zeros((0, 3)))), dev_g(gs, pts(x)), np.eye(3, 4)) == (0.0, 0)


def test_overlap_room_full_size_sampled(gs, ctx):
    # the room submap pair (150k means each) under a perturbed estimate:
    # nearest neighbours of 2000 sampled queries each way vs the oracle
    c = synth.room_150k()
    g = O.Gaussians.from_dict(c["gaussians"])
    q = O.transform(g, c["T_gt"])
    rng = np.random.default_rng(9)
    est = synth.compose(synth.about_point(synth.random_rigid(rng, 2.0, 0.05), synth.centroid(c["gaussians"])),
                        c["T_gt"])
    r, k, gpq, gqp = gs.gs_overlap_ratio(ctx, dev_g(gs, g), dev_g(gs, q), est, 0.2, with_nn=True)
    gpq, gqp = gpq.cpu().numpy(), gqp.cpu().numpy()
    ip = np.sort(rng.choice(g.n, 2000, replace=False)).astype(np.int32)
    np.testing.assert_array_equal(gpq[ip], O.nearest_subset(g, q, est, ip))
    moved = O.moved_means(g, est)
    pm = O.Gaussians(moved, g.log_scales4, g.quats4, g.logits, g.rgb4)
    iq = np.sort(rng.choice(q.n, 2000, replace=False)).astype(np.int32)
    np.testing.assert_array_equal(gqp[iq], O.nearest_subset(q, pm, np.eye(3, 4), iq))
    # |K| and OR from the device nearest neighbours, recounted on the host
    recip = gqp[gpq] == np.arange(g.n)
    assert k == int(recip.sum())
    assert 0.5 < r <= 1.0


def test_overlap_grid_with_far_outliers(gs, ctx):
    # a dense cluster plus a few points tens of metres away: the grid's cells
    # grow with the box, the cluster's queries stop after a shell or two and
    # the far ones run past the shell limit into the brute-force sweep
    rng = np.random.default_rng(12)

    def pts(a):
        a = np.asarray(a, np.float32)
        return O.Gaussians(np.concatenate([a, np.zeros((len(a), 1), np.float32)], 1), np.zeros((len(a), 4)),
                           np.tile([1.0, 0, 0, 0], (len(a), 1)), np.zeros(len(a)), np.zeros((len(a), 4)))

    x = np.concatenate([rng.uniform(-0.5, 0.5, (3000, 3)), rng.uniform(40, 80, (20, 3))])
    y = np.concatenate([rng.uniform(-0.5, 0.5, (2500, 3)), rng.uniform(-80, -40, (10, 3))])
    r, k = check(gs, ctx, pts(x), pts(y), synth.random_rigid(rng, 5.0, 0.05), tau=0.05)
    assert 0.0 < r < 1.0 and k > 100
