"""Several views at once: the asynchronous submit/finish pair, the batch
call and the continuous-batching server must give each view exactly the
frames it gets alone (views are independent; same kernels, same buffers
layout), and the first frames match the oracle."""
import numpy as np
import pytest

import oracle
import scenegen
from parity import check_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402


def _cams(client, n, size):
    """A short walk per client through the 30 x 30 x 8 m box."""
    W, H = size
    f = 260.0 * W / 328.0
    return [scenegen.camera((2.0 + 0.9 * client + 0.04 * k, 6.0 + 3.0 * client, 3.0), 0.2 + 0.15 * client + 0.01 * k,
                            W, H, f) for k in range(n)]


SIZES = [(328, 250), (200, 120), (64, 48), (257, 131)]


@pytest.fixture(scope="module")
def h_small(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    yield h
    h.close()


def test_submit_finish_equals_render(h_small):
    va, vb = vgr.View(h_small), vgr.View(h_small)
    for cam in _cams(0, 4, SIZES[0]):
        va.submit(cam, 3.0)
        while not va.done():
            pass
        a = va.finish()
        b = vb.render(cam, 3.0)
        np.testing.assert_array_equal(a.cut().cpu().numpy(), b.cut().cpu().numpy())
        assert np.array_equal(a.image().cpu().numpy(), b.image().cpu().numpy())
    with pytest.raises(vgr.VgrError):
        va.finish()  # nothing in flight
    va.submit(_cams(0, 1, SIZES[0])[0], 3.0)
    with pytest.raises(vgr.VgrError):
        va.submit(_cams(0, 1, SIZES[0])[0], 3.0)  # one frame in flight per view
    with pytest.raises(vgr.VgrError):
        va.reset()
    va.finish()
    va.close(); vb.close()


def test_batch_equals_individual(small_sh3_scene, h_small):
    n = len(SIZES)
    batch = [vgr.View(h_small, use_graph=(i % 2 == 0)) for i in range(n)]
    solo = [vgr.View(h_small) for _ in range(n)]
    walks = [_cams(i, 3, SIZES[i]) for i in range(n)]
    for k in range(3):
        cams = [walks[i][k] for i in range(n)]
        hosts = [np.empty((c["height"], c["width"], 3), np.float32) if i % 2 else None for i, c in enumerate(cams)]
        res = vgr.render_batch(batch, cams, [3.0] * n, hosts)
        for i in range(n):
            r = solo[i].render(cams[i], 3.0)
            np.testing.assert_array_equal(res[i].cut().cpu().numpy(), r.cut().cpu().numpy())
            img = res[i].image().cpu().numpy()
            assert np.array_equal(img, r.image().cpu().numpy())
            if hosts[i] is not None:
                assert np.array_equal(hosts[i], img)
            assert res[i].stats["lod_from_scratch"] == (1 if k == 0 else 0)
        if k == 0:
            ref = oracle.render(small_sh3_scene, cams[1], 3.0)
            np.testing.assert_array_equal(res[1].cut().cpu().numpy().view(np.uint32), ref["cut"])
            check_image(res[1].image().cpu().numpy(), ref)
    with pytest.raises(vgr.VgrError):
        vgr.render_batch([batch[0], batch[0]], walks[0][:2], [3.0, 3.0])  # repeated view
    r = vgr.render_batch(batch[:1], walks[0][:1], [3.0])  # still usable
    assert r[0].cut_count > 0
    for v in batch + solo:
        v.close()


def _trace(n_clients, per_client, rate, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for c in range(n_clients):
        t = np.cumsum(rng.exponential(1.0 / rate, per_client))
        for k, cam in enumerate(_cams(c, per_client, SIZES[c % len(SIZES)])):
            reqs.append(dict(client=c, arrival_s=float(t[k]), cam=cam, tau=3.0, k=k))
    reqs.sort(key=lambda r: r["arrival_s"])
    return reqs


@pytest.mark.parametrize("max_inflight", [0, 1])
def test_server_trace_equals_solo(h_small, max_inflight):
    C, K = 4, 6
    reqs = _trace(C, K, 200.0, 5)
    sv = vgr.Server(h_small, C, max_inflight=max_inflight, host_images=True)
    res = sv.serve(reqs)
    assert (res["status"] == 0).all()
    assert (res["finish_s"] >= res["start_s"]).all() and (res["start_s"] >= res["arrival_s"] - 1e-9).all()
    # per client: requests started in arrival order and never overlapped
    for c in range(C):
        rc = res[res["client"] == c]
        assert (np.diff(rc["start_s"]) >= 0).all()
        assert (rc["start_s"][1:] >= rc["finish_s"][:-1]).all()
        assert rc["lod_from_scratch"][0] == 1 and (rc["lod_from_scratch"][1:] == 0).all()
    if max_inflight == 1:
        order = np.argsort(res["start_s"])
        assert (res["start_s"][order][1:] >= res["finish_s"][order][:-1]).all()
    # each client's last image equals the same walk rendered alone
    for c in range(C):
        v = vgr.View(h_small)
        for cam in _cams(c, K, SIZES[c % len(SIZES)]):
            r = v.render(cam, 3.0)
        W, H = SIZES[c % len(SIZES)]
        assert np.array_equal(sv.client_host_image(c, H, W), r.image().cpu().numpy())
        rc = res[res["client"] == c]
        assert rc["cut_count"][-1] == r.cut_count and rc["pair_count"][-1] == r.stats["pair_count"]
        v.close()
    sv.close()


def test_server_admission_refusal(h_small):
    sv = vgr.Server(h_small, 2, hbm_reserve=1 << 62)
    res = sv.serve(_trace(2, 2, 500.0, 6))
    assert (res["status"] == 2).all()  # VGR_E_NOMEM: not admitted, nothing rendered
    sv.close()


def test_whole_batch_graph_equals_individual(small_sh3_scene, h_small):
    """Every view replays captured frames on its own stream: the batch runs
    as one captured graph (re-captured when a view's buffers grow, reused
    when the combination repeats) and each frame equals the view rendered
    alone, over several frames and both buffer parities."""
    n = len(SIZES)
    batch = [vgr.View(h_small, use_graph=True, pair_capacity=(16 if i == 1 else 0)) for i in range(n)]
    solo = [vgr.View(h_small) for _ in range(n)]
    walks = [_cams(i, 5, SIZES[i]) for i in range(n)]
    for k in range(5):
        cams = [walks[i][k] for i in range(n)]
        pinned = [torch.empty((c["height"], c["width"], 3), dtype=torch.float32, pin_memory=True) for c in cams]
        hosts = [pinned[0].numpy(), None, np.empty((cams[2]["height"], cams[2]["width"], 3), np.float32), None]
        res = vgr.render_batch(batch, cams, [3.0] * n, hosts)
        for i in range(n):
            r = solo[i].render(cams[i], 3.0)
            np.testing.assert_array_equal(res[i].cut().cpu().numpy(), r.cut().cpu().numpy())
            img = res[i].image().cpu().numpy()
            assert np.array_equal(img, r.image().cpu().numpy())
            if hosts[i] is not None:
                assert np.array_equal(hosts[i], img)
        if k == 0:
            assert res[1].stats["replays"] >= 1  # the small pair buffer grew
    for v in batch + solo:
        v.close()


def test_batch_with_variant_views(small_sh3_scene, h_small):
    """Views with the frustum-aware test, weight interpolation or both, in
    one captured batch graph: each frame equals the view rendered alone, and
    the combined variant matches the oracle."""
    n = len(SIZES)
    kinds = [dict(lod_frustum=True), dict(lod_interp=True), dict(lod_frustum=True, lod_interp=True), dict()]
    batch = [vgr.View(h_small, use_graph=True, **kinds[i]) for i in range(n)]
    solo = [vgr.View(h_small, **kinds[i]) for i in range(n)]
    walks = [_cams(i, 3, SIZES[i]) for i in range(n)]
    for k in range(3):
        cams = [walks[i][k] for i in range(n)]
        res = vgr.render_batch(batch, cams, [3.0] * n)
        for i in range(n):
            r = solo[i].render(cams[i], 3.0)
            np.testing.assert_array_equal(res[i].cut().cpu().numpy(), r.cut().cpu().numpy())
            assert np.array_equal(res[i].image().cpu().numpy(), r.image().cpu().numpy())
        ref = oracle.render(small_sh3_scene, cams[2], 3.0, frustum_guard=2.0, interp=True)
        np.testing.assert_array_equal(res[2].cut().cpu().numpy().view(np.uint32), ref["cut"])
        check_image(res[2].image().cpu().numpy(), ref)
    for v in batch + solo:
        v.close()


def test_busy_first_frames_equal_solo():
    """Many clients admitted at once on a busy GPU (1M leaves at 1080p and
    720p, every first frame in flight together, buffers growing): each
    client's first frame equals the same camera rendered alone.  New views'
    buffers are zero-filled before any of their frames may run, whatever the
    other streams are doing."""
    sc = scenegen.make_scene("m1")
    h = vgr.Hierarchy(sc)
    C = 12
    sizes = [(1920, 1080) if c % 2 else (1280, 720) for c in range(C)]
    cams = [scenegen.camera((20.0 + 7.0 * c, 100.0 - 3.0 * c, 10.0), 0.3 * c, W, H, 1100.0 * W / 1920.0)
            for c, (W, H) in enumerate(sizes)]
    for round_ in range(2):  # the second server reuses the first one's freed memory
        sv = vgr.Server(h, C, max_inflight=0, host_images=True)
        res = sv.serve([dict(client=c, arrival_s=0.0, tau=3.0, cam=cams[c]) for c in range(C)])
        assert (res["status"] == 0).all(), res
        for c in range(C):
            v = vgr.View(h)
            r = v.render(cams[c], 3.0)
            W, H = sizes[c]
            assert np.array_equal(sv.client_host_image(c, H, W), r.image().cpu().numpy()), (round_, c)
            v.close()
        sv.close()
    h.close()
