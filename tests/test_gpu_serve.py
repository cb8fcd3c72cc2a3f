"""The continuous-batching server (gs_server_*): every request's result is
the same alone and in a changing mix of in-flight requests, and equals
gs_register's for the same problem and iteration count (bit for bit: each
iteration of a request depends only on its own problem); admission respects
the keyframe and memory limits."""
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
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda().contiguous()


def view(og, cam):
    r = O.render(og, np.eye(3, 4), cam)
    return cam, dev(r["rgb"]), dev(r["depth"])


def edge(gs, n, W, H, f, n_src, n_tgt, seed):
    """A loop edge: P, Q = T_gt P, keyframes of each rendered by the oracle."""
    c = synth.small_case(n, W, H, f, n_views=max(n_src + n_tgt, 2), seed=seed, ls_mean=-3.3)
    og = O.Gaussians.from_dict(c["gaussians"])
    oq = O.transform(og, c["T_gt"])
    sv = [view(og, cam) for cam in c["cams"][:n_src]]
    tv = [view(oq, cam) for cam in synth.moved_cameras(c["cams"][n_src:n_src + n_tgt], c["T_gt"])] if n_tgt else []
    src = gs.Gaussians.from_numpy(c["gaussians"])
    tgt = gs.Gaussians(*[dev(a) for a in (oq.means4, oq.log_scales4, oq.quats4, oq.logits, oq.rgb4)])
    return src, tgt, sv, tv


def tracking(gs, n, W, H, f, seed, ls_mean=-3.3):
    """Frame-to-model tracking: one frame rendered at the true camera, the
    request's camera a small perturbation of it (0.7 deg, 1.3 cm)."""
    c = synth.small_case(n, W, H, f, n_views=1, seed=seed, ls_mean=ls_mean)
    og = O.Gaussians.from_dict(c["gaussians"])
    cam = c["cams"][0]
    _, rgb, depth = view(og, cam)
    guess = synth.moved_cameras([cam], synth.about_point(synth.random_rigid(np.random.default_rng(seed), 0.69, 0.0134),
                                                          synth.centroid(c["gaussians"])))[0]
    g = gs.Gaussians.from_numpy(c["gaussians"])
    return g, g, [], [(guess, rgb, depth)]


@pytest.fixture(scope="module")
def requests(gs):
    return [(tracking(gs, 700, 96, 64, 80.0, 41), 12), (edge(gs, 900, 96, 64, 80.0, 1, 2, 42), 25),
            (tracking(gs, 1200, 80, 72, 70.0, 43), 9), (edge(gs, 400, 64, 40, 50.0, 2, 0, 44), 17),
            (tracking(gs, 500, 100, 60, 90.0, 45), 30), (edge(gs, 1500, 120, 90, 100.0, 2, 1, 46), 11)]


def drain(srv, limit=10_000):
    done = []
    for _ in range(limit):
        if srv.counts()[0] == 0 and srv.counts()[1] == 0:
            break
        done += srv.step()
    return done


def same(res, ref):
    T, conf, eps, _ = ref
    np.testing.assert_array_equal(res["T"], T)
    assert res["confidence"] == conf
    np.testing.assert_array_equal(res["eps"][:len(eps)], eps)


def test_alone_equals_gs_register(gs, ctx, requests):
    for (prob, iters) in requests[:2]:
        srv = gs.Server(0, max_round_iters=5)
        rid = srv.submit(*prob, iters)
        assert drain(srv) == [rid]
        same(srv.poll(rid), gs.gs_register(ctx, *prob, iters))
        assert srv.counts()[3] == -(-(iters + 1) // 5)  # rounds of at most 5 iterations
        srv.close()


def test_mix_equals_alone(gs, ctx, requests):
    refs = [gs.gs_register(ctx, *prob, iters) for prob, iters in requests]
    srv = gs.Server(0, max_round_iters=7)
    ids, peak = [], 0
    # arrivals while others are in flight: 2, then 1 per round, then the rest
    schedule = [2, 1, 0, 1, 0, 2]
    pending = list(range(len(requests)))
    for k in schedule:
        for _ in range(k):
            i = pending.pop(0)
            ids.append((srv.submit(*requests[i][0], requests[i][1]), i))
        srv.step()
        peak = max(peak, srv.counts()[1])
    drain(srv)
    waiting, inflight, done, rounds, replans = srv.counts()
    assert waiting == 0 and inflight == 0 and done == len(requests)
    assert peak >= 2 and replans >= 4
    for rid, i in ids:
        res = srv.poll(rid)
        assert res["state"] == 2 and res["t_done"] >= res["t_submit"]
        same(res, refs[i])
    srv.close()


def test_admission_limits(gs, ctx, requests):
    # at most 3 keyframe problems in flight: the 3-keyframe edge waits for an empty server
    srv = gs.Server(0, max_keyframes=3, max_round_iters=4)
    for prob, iters in requests[:4]:
        srv.submit(*prob, iters)
    kf = {0: 1, 1: 3, 2: 1, 3: 2}
    while srv.counts()[0] or srv.counts()[1]:
        srv.step()
        inflight_ids = [i for i in range(4) if srv.poll(i)["state"] == 1]
        assert sum(kf[i] for i in inflight_ids) <= 3
    srv.close()
    # a 300 kB budget holds one of the tracking requests at a time (their
    # footprints are about 200-290 kB); the 3-keyframe edge is refused
    srv = gs.Server(0, budget_bytes=300_000, max_round_iters=4)
    track = [requests[i] for i in (0, 2, 4)]
    for prob, iters in track:
        srv.submit(*prob, iters)
    with pytest.raises(gs.GsError):
        srv.submit(*requests[1][0], 5)
    while srv.counts()[0] or srv.counts()[1]:
        srv.step()
        assert srv.counts()[1] <= 1
    assert srv.counts()[2] == 3
    for i, (prob, iters) in enumerate(track):
        same(srv.poll(i), gs.gs_register(ctx, *prob, iters))
    srv.close()


def test_rejects_bad_requests(gs, requests):
    srv = gs.Server(0, max_keyframes=2)
    prob, _ = requests[1]  # 3 keyframes
    with pytest.raises(gs.GsError):
        srv.submit(*prob, 10)
    with pytest.raises(gs.GsError):
        srv.submit(*requests[0][0], -1)
    assert srv.counts()[0] == 0
    srv.close()


def fixed_estimate(prob):
    # the footprint rule this admission replaces: three tile duplicates per
    # record whatever the splats' screen sizes, 16 B each with headroom 1.5
    src, tgt, sv, tv = prob
    b = 0.0
    for g, views in ((tgt, sv), (src, tv)):
        for cam, _, _ in views:
            px = int(cam[4]) * int(cam[5])
            tiles = ((int(cam[4]) + 15) // 16) * ((int(cam[5]) + 15) // 16)
            b += g.n * 100 + 3.0 * g.n * 16 * 1.5 + px * 9 + tiles * 92
    return b


@pytest.mark.parametrize("splats", ["large", "small"])
def test_admission_by_measured_footprint(gs, ctx, splats):
    # two tracking requests whose splats cover many tiles each (large) or
    # about one (small): their measured footprints lie on the other side of
    # the budget from the fixed three-duplicates-per-record rule, and
    # admission follows the measurement -- one at a time for the large
    # splats, both together for the small ones; results are gs_register's
    if splats == "large":
        probs = [tracking(gs, 2000, 128, 96, 120.0, 51, ls_mean=-1.8), tracking(gs, 2000, 128, 96, 120.0, 52, -1.8)]
    else:
        probs = [tracking(gs, 3000, 64, 48, 40.0, 53, ls_mean=-4.5), tracking(gs, 3000, 64, 48, 40.0, 54, -4.5)]
    probe = gs.Server(0)
    fp = [probe.footprint(probe.submit(*p, 8)) for p in probs]
    probe.close()
    measured = sum(b for _, b in fp)
    fixed = sum(fixed_estimate(p) for p in probs)
    budget = int((measured + fixed) / 2)
    srv = gs.Server(0, budget_bytes=budget, max_round_iters=4)
    ids = [srv.submit(*p, 8) for p in probs]
    assert [srv.footprint(i) for i in ids] == fp
    srv.step()
    together = srv.counts()[1] == 2  # 8 iterations take more than one round of 4
    if splats == "large":
        assert fp[0][0] > 10 * 2000 and measured > budget > fixed
        assert srv.admission()[1] == 1 and not together
    else:
        assert fp[0][0] < 2 * 3000 and fixed > budget > measured
        assert srv.admission()[1] == 0 and together
    drain(srv)
    assert srv.admission()[0] == 2
    for i, p in zip(ids, probs):
        same(srv.poll(i), gs.gs_register(ctx, *p, 8))
    srv.close()
