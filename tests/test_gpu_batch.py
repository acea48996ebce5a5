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
    """Every client's first request at t = 0 (a burst), then Poisson arrivals."""
    rng = np.random.default_rng(seed)
    reqs = []
    for c in range(n_clients):
        t = np.concatenate([[0.0], np.cumsum(rng.exponential(1.0 / rate, per_client - 1))])
        for k, cam in enumerate(_cams(c, per_client, SIZES[c % len(SIZES)])):
            reqs.append(dict(client=c, arrival_s=float(t[k]), cam=cam, tau=3.0, k=k))
    reqs.sort(key=lambda r: (r["arrival_s"], r["client"]))
    return reqs


def _solo_walks(h, n_clients, per_client):
    """Each client's walk rendered alone: images and (cut, pairs) per frame."""
    out = {}
    for c in range(n_clients):
        v = vgr.View(h)
        imgs, counts = [], []
        for cam in _cams(c, per_client, SIZES[c % len(SIZES)]):
            r = v.render(cam, 3.0)
            imgs.append(r.image().cpu().numpy().copy())
            counts.append((r.cut_count, r.stats["pair_count"]))
        v.close()
        out[c] = (imgs, counts)
    return out


def _overlapping_clients(res):
    """Pairs of requests of different clients whose [start, finish) intersect."""
    n = len(res)
    return [(i, j) for i in range(n) for j in range(i + 1, n)
            if res["client"][i] != res["client"][j] and res["start_s"][i] < res["finish_s"][j]
            and res["start_s"][j] < res["finish_s"][i]]


def _max_concurrent(res) -> int:
    """Most frames in flight at one instant ([start, finish) intervals)."""
    ev = sorted([(s, 1) for s in res["start_s"]] + [(f, -1) for f in res["finish_s"]], key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


@pytest.mark.parametrize("max_inflight", [0, 1, 2, None])
def test_server_trace_equals_solo(h_small, max_inflight):
    """Continuous batching (max_inflight 0: every client; 2, also the
    default) keeps frames of different clients in flight together, never more
    than the cap; one frame at a time (1) never does.  Either way every served
    frame -- not only each client's last -- equals the same client's walk
    rendered alone, bit for bit, through per-request host images."""
    C, K = 4, 6
    reqs = _trace(C, K, 200.0, 5)
    sv = vgr.Server(h_small, C, max_inflight=max_inflight, host_images=True)
    res, imgs = sv.serve(reqs, images=True)
    assert (res["status"] == 0).all()
    assert (res["finish_s"] >= res["start_s"]).all() and (res["start_s"] >= res["arrival_s"] - 1e-9).all()
    # per client: requests started in arrival order and never overlapped
    for c in range(C):
        rc = res[res["client"] == c]
        assert (np.diff(rc["start_s"]) >= 0).all()
        assert (rc["start_s"][1:] >= rc["finish_s"][:-1]).all()
        assert rc["lod_from_scratch"][0] == 1 and (rc["lod_from_scratch"][1:] == 0).all()
    overlap = _overlapping_clients(res)
    if max_inflight == 1:
        assert not overlap
        order = np.argsort(res["start_s"])
        assert (res["start_s"][order][1:] >= res["finish_s"][order][:-1]).all()
    elif max_inflight == 0:
        # the t = 0 burst: all four first frames are submitted before any completes
        assert len(overlap) >= C - 1, overlap
    else:
        assert overlap and _max_concurrent(res) <= 2, (overlap, _max_concurrent(res))
    solo = _solo_walks(h_small, C, K)
    for i, r in enumerate(reqs):
        simg, scounts = solo[r["client"]]
        assert np.array_equal(imgs[i], simg[r["k"]]), (i, r["client"], r["k"])
        assert (res["cut_count"][i], res["pair_count"][i]) == scounts[r["k"]]
    sv.close()


def test_server_admission_refusal(h_small):
    sv = vgr.Server(h_small, 2, hbm_reserve=1 << 62)
    res = sv.serve(_trace(2, 2, 500.0, 6))
    assert (res["status"] == 2).all()  # VGR_E_NOMEM: cannot fit even alone, nothing rendered
    sv.close()


def test_server_memory_pressure_serves_every_request(h_small):
    """The clients' views together need more device memory than admission
    allows (the reserve leaves room for about two of four): requests wait for
    memory instead of being refused, idle clients' views are released least
    recently used first, and every request is served with the image its
    client gets rendering the walk alone (a released client's next frame finds
    its cut top-down: the same cut)."""
    C, K = 4, 5
    est = max(vgr.view_bytes_estimate(h_small, W, H) for W, H in SIZES)
    free = torch.cuda.mem_get_info()[0]
    sv = vgr.Server(h_small, C, max_inflight=0, hbm_reserve=int(free - 2.5 * est))
    reqs = _trace(C, K, 300.0, 7)
    res, imgs = sv.serve(reqs, images=True)
    assert (res["status"] == 0).all(), res["status"]
    assert res["views_released"].sum() > 0 and res["admission_waits"].sum() > 0, res
    assert res["lod_from_scratch"].sum() >= C
    solo = _solo_walks(h_small, C, K)
    for i, r in enumerate(reqs):
        simg, scounts = solo[r["client"]]
        assert np.array_equal(imgs[i], simg[r["k"]]), (i, r["client"], r["k"])
        assert (res["cut_count"][i], res["pair_count"][i]) == scounts[r["k"]]
    sv.close()


def test_server_without_release_waits_for_memory(h_small):
    """With evict_idle off, views are never released: once two views exist a
    third client can never be admitted, and its request completes with
    VGR_E_NOMEM as soon as nothing else is in flight; the others are served."""
    C = 3
    est = max(vgr.view_bytes_estimate(h_small, W, H) for W, H in SIZES[:C])
    free = torch.cuda.mem_get_info()[0]
    sv = vgr.Server(h_small, C, max_inflight=0, hbm_reserve=int(free - 2.5 * est), evict_idle=False)
    reqs = _trace(C, 2, 300.0, 8)
    res = sv.serve(reqs)
    ok = res["status"] == 0
    assert ok.sum() >= 2 and (res["status"][~ok] == 2).all()
    assert (res["views_released"] == 0).all()
    sv.close()


@pytest.mark.parametrize("chains", [0, 1, 2, 3])
def test_whole_batch_graph_equals_individual(small_sh3_scene, h_small, chains):
    """Every view replays captured frames on its own stream: the batch runs
    as one captured graph (re-captured when a view's buffers grow, reused
    when the combination repeats) and each frame equals the view rendered
    alone, over several frames and both buffer parities, with the views in
    one branch each (chains 0) or in 1, 2 or 3 chains."""
    vgr.set_batch_chains(chains)
    try:
        _whole_batch_equals_individual(h_small)
    finally:
        vgr.set_batch_chains(0)


def _whole_batch_equals_individual(h_small):
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


def test_batch_single_blend_launch(small_sh3_scene, h_small):
    """A captured batch runs one blend launch over the tiles of every view
    with the exact exponential at the first such view's staging depth (one
    view here has another depth, one the Eq. 5 table: those two blend in their
    own branch).  Every frame equals the view alone, bit for bit, and the
    kernels launched are the views' own minus one blend per shared view plus
    the batch's three (class offsets, tile placement, blend)."""
    n = len(SIZES)
    kinds = [dict(), dict(blend_depth=16), dict(exp_mode=vgr.EXP_LUT), dict()]
    batch = [vgr.View(h_small, use_graph=True, **kinds[i]) for i in range(n)]
    solo = [vgr.View(h_small, **kinds[i]) for i in range(n)]
    walks = [_cams(i, 3, SIZES[i]) for i in range(n)]
    for k in range(3):
        cams = [walks[i][k] for i in range(n)]
        res = vgr.render_batch(batch, cams, [3.0] * n)
        alone = [solo[i].render(cams[i], 3.0) for i in range(n)]
        for i in range(n):
            np.testing.assert_array_equal(res[i].cut().cpu().numpy(), alone[i].cut().cpu().numpy())
            assert np.array_equal(res[i].image().cpu().numpy(), alone[i].image().cpu().numpy()), (k, i)
            assert res[i].stats["pixel_pair_evals"] == alone[i].stats["pixel_pair_evals"]
            assert res[i].stats["pixel_pair_contribs"] == alone[i].stats["pixel_pair_contribs"]
        shared = 2  # views 0 and 3
        assert sum(r.stats["kernels"] for r in res) == sum(a.stats["kernels"] for a in alone) - shared + 3
        if k == 0:
            ref = oracle.render(small_sh3_scene, cams[3], 3.0)
            check_image(res[3].image().cpu().numpy(), ref)
    for v in batch + solo:
        v.close()


@pytest.mark.parametrize("tile", [8, 32])
def test_batch_blend_at_other_tile_sizes(small_sh3_scene, h_small, tile):
    """The batch blend over views with 8- or 32-pixel tiles (one of another
    size blends in its own branch): every frame equals the view alone."""
    n = len(SIZES)
    sizes = [tile, tile, 16, tile]
    batch = [vgr.View(h_small, use_graph=True, tile_size=sizes[i]) for i in range(n)]
    solo = [vgr.View(h_small, tile_size=sizes[i]) for i in range(n)]
    walks = [_cams(i, 2, SIZES[i]) for i in range(n)]
    for k in range(2):
        cams = [walks[i][k] for i in range(n)]
        res = vgr.render_batch(batch, cams, [3.0] * n)
        alone = [solo[i].render(cams[i], 3.0) for i in range(n)]
        for i in range(n):
            assert np.array_equal(res[i].image().cpu().numpy(), alone[i].image().cpu().numpy()), (k, i)
        assert sum(r.stats["kernels"] for r in res) == sum(a.stats["kernels"] for a in alone) - 3 + 3
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
