"""Pins of the oracle's frustum-aware granularity test (the variant in which
the LoD tree also identifies the Gaussians inside the view frustum, Sec. 3.1).

The planes are checked against direct pinhole projection, the box test
against brute force over the box's eight corners, the cut against the
ancestor-chain definition and a hand-derived tree, and the variant against
the distance-only cut (the relations the definition implies, and equality
when every box lies inside the frustum).
"""
import itertools

import numpy as np
import pytest

import oracle
import scenegen

F32 = np.float32


def _rand_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q.astype(np.float32)


def _rand_camera(rng):
    W, H = int(rng.integers(1, 2000)), int(rng.integers(1, 1200))
    fx, fy = F32(rng.uniform(50, 2000)), F32(rng.uniform(50, 2000))
    return dict(R=_rand_rotation(rng), pos=rng.uniform(-50, 50, 3).astype(np.float32), fx=fx, fy=fy,
                cx=F32(rng.uniform(0, W)), cy=F32(rng.uniform(0, H)), width=W, height=H,
                z_near=F32(rng.uniform(0.05, 2.0)))


def test_planes_match_projection():
    """w . x - o >= 0 for all five planes iff x is beyond the near plane and
    projects into the image widened by the guard (FP64 pinhole projection)."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(40):
        cam = _rand_camera(rng)
        g = float(rng.choice([0.0, 2.0, 37.5]))
        pl = oracle.frustum_planes(cam, g).astype(np.float64)
        R = np.asarray(cam["R"], np.float64)
        C = np.asarray(cam["pos"], np.float64)
        x = C + rng.normal(size=(2000, 3)) * rng.uniform(1, 100)
        p = (x - C) @ R.T
        z = p[:, 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = cam["fx"] * p[:, 0] / z + cam["cx"]
            v = cam["fy"] * p[:, 1] / z + cam["cy"]
        want = (z >= cam["z_near"]) & (u >= -g) & (u <= cam["width"] + g) & (v >= -g) & (v <= cam["height"] + g)
        s = x @ pl[:, :3].T - pl[:, 3]
        got = (s >= 0).all(axis=1)
        scale = np.abs(pl[:, :3]).sum(axis=1) * (np.abs(x).max() + np.abs(C).max() + 1.0)
        clear = (np.abs(s) > 1e-4 * scale).all(axis=1)
        np.testing.assert_array_equal(got[clear], want[clear])
        checked += int(clear.sum())
    assert checked > 50000


def test_box_test_matches_corner_brute_force():
    rng = np.random.default_rng(12)
    n_in = n_out = 0
    for _ in range(30):
        cam = _rand_camera(rng)
        pl = oracle.frustum_planes(cam, float(rng.uniform(0, 8)))
        pd = pl.astype(np.float64)
        for _ in range(60):
            c = np.asarray(cam["pos"], np.float64) + rng.normal(size=3) * 30
            h = np.abs(rng.normal(size=3)) * rng.uniform(0.01, 10)
            box = np.concatenate([c - h, c + h]).astype(np.float32)
            corners = np.array([[box[3 * i + 0], box[3 * j + 1], box[3 * k + 2]]
                                for i, j, k in itertools.product((0, 1), repeat=3)], np.float64)
            smax = (corners @ pd[:, :3].T - pd[:, 3]).max(axis=0)  # per plane
            scale = np.abs(pd[:, :3]).sum(axis=1) * (np.abs(corners).max() + 1.0)
            if (np.abs(smax) < 1e-5 * scale).any():
                continue  # a near-tie: the FP32 test may take either side
            want = bool((smax >= 0).all())
            assert oracle.box_meets(box, pl) == want
            n_in += want
            n_out += not want
    assert n_in > 50 and n_out > 50


def _hand_tree(x2_hi):
    """root 0 -> {1, 2}; 1 -> leaves {3, 4} in front at z ~ 10; 2 -> leaves
    {5, 6} in a box with x in [x2_hi - 1, x2_hi], z in [9, 11]."""
    n = 7
    mean = np.array([[0, 0, 0], [0, 0, 10], [x2_hi - 0.5, 0, 10], [-0.5, 0, 10], [0.5, 0, 10],
                     [x2_hi - 0.7, 0, 10], [x2_hi - 0.3, 0, 10]], np.float32)
    box = np.zeros((n, 6), np.float32)
    box[1] = [-1, -1, 9, 1, 1, 11]
    box[2] = [x2_hi - 1, -1, 9, x2_hi, 1, 11]
    box[3] = box[4] = box[1]
    box[5] = box[6] = box[2]
    box[0] = [min(-1, x2_hi - 1), -1, 9, 1, 1, 11]
    return dict(parent=np.array([0xFFFFFFFF, 0, 0, 1, 1, 2, 2], np.uint32),
                first_child=np.array([1, 3, 5, 0, 0, 0, 0], np.uint32),
                n_child=np.array([2, 2, 2, 0, 0, 0, 0], np.uint8), mean=mean,
                cov6=np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (n, 1)),
                opacity=np.full(n, 0.5, np.float32), sh=np.zeros((n, 1, 3), np.float32),
                radius2=np.full(n, 1e6, np.float32), bbox=box, sh_degree=0, n_nodes=n)


def test_hand_derived_tree():
    """Camera at the origin looking down +z, fx = fy = 100, 100 x 100 image.
    Node 2's box corner nearest the view (x = x2_hi, z = 11) projects to
    u = 100 x2_hi / 11 + 50 = -1 for x2_hi = -5.61: outside the image, inside
    it widened by 2 pixels.  Sizes never stop expansion (radius2 = 1e6)."""
    cam = dict(R=np.eye(3, dtype=np.float32), pos=np.zeros(3, np.float32), fx=100.0, fy=100.0, cx=50.0, cy=50.0,
               width=100, height=100, z_near=0.2)
    k = oracle.lod_k(3.0, 100.0)
    sc = _hand_tree(-5.61)
    assert oracle.cut(sc, cam["pos"], k).tolist() == [3, 4, 5, 6]  # distance-only
    for g, want in ((0.0, [2, 3, 4]), (2.0, [3, 4, 5, 6])):
        pl = oracle.frustum_planes(cam, g)
        assert oracle.cut(sc, cam["pos"], k, planes=pl).tolist() == want
        assert oracle.cut(sc, cam["pos"], k, bruteforce=True, planes=pl).tolist() == want
    # behind the camera: node 2 fails the near plane whatever the guard
    sc = _hand_tree(-5.61)
    sc["bbox"][2] = sc["bbox"][5] = sc["bbox"][6] = [-1, -1, -11, 1, 1, -9]
    sc["bbox"][0] = [-1, -1, -11, 1, 1, 11]
    pl = oracle.frustum_planes(cam, 1000.0)
    assert oracle.cut(sc, cam["pos"], k, planes=pl).tolist() == [2, 3, 4]


@pytest.fixture(scope="module")
def tiny_cams():
    cams = [scenegen.trajectory("tiny", f) for f in (0, 5, 11)]
    c = dict(scenegen.trajectory("tiny", 3))
    c["R"] = scenegen.look_rotation(2.5, -0.4).astype(np.float32)
    cams.append(c)
    return cams


def test_topdown_equals_bruteforce(tiny_scene, tiny_cams):
    for cam in tiny_cams:
        for g in (0.0, 2.0, 40.0):
            pl = oracle.frustum_planes(cam, g)
            k = oracle.lod_k(3.0, float(cam["fx"]))
            a = oracle.cut(tiny_scene, cam["pos"], k, planes=pl)
            b = oracle.cut(tiny_scene, cam["pos"], k, bruteforce=True, planes=pl)
            np.testing.assert_array_equal(a, b)


def test_monotone_under_nested_boxes(tiny_scene, tiny_cams):
    """child expands => parent expands, node by node (what the temporal
    update relies on)."""
    sc = tiny_scene
    par = sc["parent"]
    for cam in tiny_cams:
        pl = oracle.frustum_planes(cam, 2.0)
        for tau in (1.0, 3.0):
            k = oracle.lod_k(tau, float(cam["fx"]))
            e = np.array([oracle.expand(sc, n, cam["pos"], k, planes=pl) for n in range(sc["n_nodes"])])
            kids = np.nonzero(e[1:])[0] + 1
            assert e[par[kids]].all()
            assert e.any() and not e.all()


def test_relation_to_distance_cut(tiny_scene, tiny_cams):
    """The frustum-aware cut is the distance cut with every subtree whose root
    box misses the frustum collapsed into that root: each of its nodes is an
    ancestor-or-self of distance-cut nodes, equal to one of them exactly when
    its box meets the frustum, and a node of the distance cut whose whole
    ancestor chain meets the frustum is in it."""
    sc = tiny_scene
    par, box = sc["parent"], sc["bbox"]
    for cam in tiny_cams:
        pl = oracle.frustum_planes(cam, 2.0)
        k = oracle.lod_k(3.0, float(cam["fx"]))
        cd = oracle.cut(sc, cam["pos"], k)
        cf = oracle.cut(sc, cam["pos"], k, planes=pl)
        assert cf.size < cd.size
        in_cf = np.zeros(sc["n_nodes"], bool)
        in_cf[cf] = True
        meets = np.array([oracle.box_meets(box[n], pl) for n in range(sc["n_nodes"])])
        for n in cd:
            a, hit, chain_in = int(n), 0, True
            while a != 0xFFFFFFFF:
                hit += in_cf[a]
                if a != n:
                    chain_in &= bool(meets[a])
                a = int(par[a])
            assert hit == 1
            if chain_in:
                assert in_cf[n]
        extra = np.setdiff1d(cf, cd)
        assert extra.size > 0 and not meets[extra].any()


def test_all_boxes_inside_reduces_to_distance_cut(tiny_scene):
    """Camera high above the scene looking straight down with a wide field
    of view: every box meets the frustum, so the variant is the distance test."""
    sc = tiny_scene
    cam = dict(R=np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float32),
               pos=np.array([10.0, 10.0, 60.0], np.float32), fx=20.0, fy=20.0, cx=64.0, cy=64.0,
               width=128, height=128, z_near=0.2)
    pl = oracle.frustum_planes(cam, 0.0)
    assert all(oracle.box_meets(sc["bbox"][n], pl) for n in range(0, sc["n_nodes"], 7))
    for tau in (0.5, 3.0):
        k = oracle.lod_k(tau, 20.0)
        np.testing.assert_array_equal(oracle.cut(sc, cam["pos"], k, planes=pl), oracle.cut(sc, cam["pos"], k))


def test_cut_depends_on_orientation(tiny_scene):
    base = scenegen.trajectory("tiny", 5)
    turned = dict(base)
    turned["R"] = scenegen.look_rotation(np.pi, 0.0).astype(np.float32)
    k = oracle.lod_k(3.0, float(base["fx"]))
    a = oracle.cut(tiny_scene, base["pos"], k, planes=oracle.frustum_planes(base, 2.0))
    b = oracle.cut(tiny_scene, base["pos"], k, planes=oracle.frustum_planes(turned, 2.0))
    assert not np.array_equal(a, b)


def test_scene_boxes_nest_and_cover(tiny_scene):
    sc = tiny_scene
    box, par = sc["bbox"], sc["parent"]
    n = np.arange(1, sc["n_nodes"])
    assert (box[par[n], :3] <= box[n, :3]).all() and (box[par[n], 3:] >= box[n, 3:]).all()
    h = 3.34 * np.sqrt(sc["cov6"][:, [0, 3, 5]].astype(np.float64))
    m = sc["mean"].astype(np.float64)
    assert (box[:, :3] <= m - h).all() and (box[:, 3:] >= m + h).all()


def test_render_frustum_guard(tiny_scene):
    """orc_render with a guard uses the frustum-aware cut."""
    cam = dict(scenegen.trajectory("tiny", 2))
    k = oracle.lod_k(3.0, float(cam["fx"]))
    r = oracle.render(tiny_scene, cam, 3.0, frustum_guard=2.0)
    np.testing.assert_array_equal(r["cut"], oracle.cut(tiny_scene, cam["pos"], k,
                                                       planes=oracle.frustum_planes(cam, 2.0)))
