"""Pins of the oracle's parent-child weight interpolation (Sec. 3.1 'Weight
Interpolation'; the paper gives no formula, the reading is stated in the
oracle's header): the weight against its FP64 closed form from projected
sizes, its limits at the two LoD transitions, the special cases where it
vanishes, and the opacity share that keeps a node's appearance at the
moment its parent collapses into it.
"""
import numpy as np

import oracle
import scenegen


def _w64(sc, n, cam, t):
    p = int(sc["parent"][n])
    if p == 0xFFFFFFFF:
        return 0.0
    pos = np.asarray(cam, np.float64)
    an = np.sqrt(float(sc["radius2"][n])) / np.linalg.norm(pos - sc["mean"][n].astype(np.float64))
    ap = np.sqrt(float(sc["radius2"][p])) / np.linalg.norm(pos - sc["mean"][p].astype(np.float64))
    if not ap > an:
        return 0.0
    return float(np.clip((t - an) / (ap - an), 0.0, 1.0))


def test_weight_matches_projected_sizes(tiny_scene):
    sc = tiny_scene
    rng = np.random.default_rng(3)
    checked = inner = 0
    for fr in (0, 7, 13):
        cam = scenegen.trajectory("tiny", fr)
        t = np.float32(np.float32(3.0) / np.float32(cam["fx"]))
        cut = oracle.cut(sc, cam["pos"], oracle.lod_k(3.0, float(cam["fx"])))
        for n in rng.choice(cut, size=min(300, cut.size), replace=False):
            w = float(oracle.interp_weight(sc, int(n), cam["pos"], t))
            w64 = _w64(sc, int(n), cam["pos"], float(t))
            assert 0.0 <= w <= 1.0
            assert abs(w - w64) < 2e-3, (n, w, w64)
            checked += 1
            inner += 0.05 < w64 < 0.95
    assert checked > 500 and inner > 50


def test_weight_limits_at_the_transitions(tiny_scene):
    """Camera on the line through a cut node's parent: just inside the
    distance where the parent would collapse, w -> 1; placed so the node is
    just short of expanding, w -> 0."""
    sc = tiny_scene
    cam0 = scenegen.trajectory("tiny", 4)
    tau, f = 3.0, float(cam0["fx"])
    t = float(np.float32(np.float32(tau) / np.float32(f)))
    cut = oracle.cut(sc, cam0["pos"], oracle.lod_k(tau, f))
    done_hi = done_lo = 0
    for n in cut[::37]:
        n = int(n)
        p = int(sc["parent"][n])
        if p == 0xFFFFFFFF or sc["n_child"][n] == 0:
            continue
        for target, which in ((p, "hi"), (n, "lo")):
            c = sc["mean"][target].astype(np.float64)
            u = cam0["pos"] - c
            u /= np.linalg.norm(u)
            R = np.sqrt(float(sc["radius2"][target]))
            # 'hi': the parent just expands; 'lo': the node just does not
            d = R / t * (1 - 1e-5 if which == "hi" else 1 + 1e-5)
            pos = (c + u * d).astype(np.float32)
            k = oracle.lod_k(tau, f)
            if n not in oracle.cut(sc, pos, k):
                continue  # another ancestor changed its mind at this pose
            w = float(oracle.interp_weight(sc, n, pos, np.float32(t)))
            if which == "hi":
                assert w > 0.99, (n, w)
                done_hi += 1
            else:
                assert w < 0.01, (n, w)
                done_lo += 1
    assert done_hi >= 3 and done_lo >= 3


def test_vanishing_weight_renders_own_gaussians(tiny_scene):
    """tau = 0 puts every leaf in the cut with size ratio above t = 0, and a
    far camera leaves only the root: both render exactly as without
    interpolation."""
    sc = tiny_scene
    cam = scenegen.trajectory("tiny", 6)
    a = oracle.render(sc, cam, 0.0)
    b = oracle.render(sc, cam, 0.0, interp=True)
    np.testing.assert_array_equal(a["image"], b["image"])
    far = dict(cam)
    r = float(np.sqrt(sc["radius2"][0]))
    far["pos"] = (sc["mean"][0] + np.array([-100.0 * r, 0, 0])).astype(np.float32)  # t = 3 / 120
    a = oracle.render(sc, far, 3.0)
    b = oracle.render(sc, far, 3.0, interp=True)
    assert a["cut"].tolist() == [0]
    np.testing.assert_array_equal(a["image"], b["image"])


def _two_copies_tree(theta):
    """A root with two leaf children, all three the same Gaussian (sigma
    0.1 m at the origin, colour from SH DC); R_root = 0.6, R_leaf = 0.3."""
    n = 3
    return dict(parent=np.array([0xFFFFFFFF, 0, 0], np.uint32), first_child=np.array([1, 0, 0], np.uint32),
                n_child=np.array([2, 0, 0], np.uint8), mean=np.zeros((n, 3), np.float32),
                cov6=np.tile(np.array([0.01, 0, 0, 0.01, 0, 0.01], np.float32), (n, 1)),
                opacity=np.full(n, theta, np.float32), sh=np.tile(np.array([[[0.6, 0.2, -0.1]]], np.float32), (n, 1, 1)),
                radius2=np.array([0.36, 0.09, 0.09], np.float32), sh_degree=0, n_nodes=n)


def test_opacity_share_keeps_the_collapse_smooth():
    """At the distance where the root collapses into the cut, the two
    children (weight -> 1) render like the root alone at the Gaussian's
    centre pixel; without interpolation they are visibly more opaque."""
    sc = _two_copies_tree(0.6)
    tau, f = 30.0, 120.0
    t = float(np.float32(np.float32(tau) / np.float32(f)))
    d_star = 0.6 / t
    cams = {}
    for side, s in (("inside", 1 - 1e-5), ("outside", 1 + 1e-5)):
        cams[side] = dict(R=np.eye(3, dtype=np.float32), pos=np.array([0, 0, -d_star * s], np.float32),
                          fx=np.float32(f), fy=np.float32(f), cx=np.float32(32.5), cy=np.float32(32.5),
                          width=64, height=64, z_near=np.float32(0.2))
    inside = oracle.render(sc, cams["inside"], tau, interp=True)
    outside = oracle.render(sc, cams["outside"], tau, interp=True)
    plain = oracle.render(sc, cams["inside"], tau)
    assert inside["cut"].tolist() == [1, 2] and outside["cut"].tolist() == [0]
    ci, co, cp = inside["image"][32, 32], outside["image"][32, 32], plain["image"][32, 32]
    np.testing.assert_allclose(ci, co, rtol=2e-4, atol=1e-6)
    assert np.abs(cp - co).max() > 0.05
    # and the whole image moves far less with interpolation than without
    assert np.abs(inside["image"] - outside["image"]).max() < 0.25 * np.abs(plain["image"] - outside["image"]).max()


def test_interpolated_render_moves_towards_parents(tiny_scene):
    """Every interpolated depth lies between the node's and its parent's
    (the mean moves along the segment), and some move."""
    sc = tiny_scene
    cam = scenegen.trajectory("tiny", 9)
    a = oracle.render(sc, cam, 3.0)
    b = oracle.render(sc, cam, 3.0, interp=True)
    np.testing.assert_array_equal(a["cut"], b["cut"])
    R = np.asarray(cam["R"], np.float64)
    C = np.asarray(cam["pos"], np.float64)
    z = lambda n: float(R[2] @ (sc["mean"][n].astype(np.float64) - C))
    moved = 0
    for i, n in enumerate(a["cut"]):
        if not b["proj"]["valid"][i]:
            continue
        p = int(sc["parent"][n])
        zn, zp = z(n), z(p) if p != 0xFFFFFFFF else z(n)
        zi = float(b["proj"]["z"][i])
        assert min(zn, zp) - 1e-4 <= zi <= max(zn, zp) + 1e-4
        moved += abs(zi - zn) > 1e-4
    assert moved > 10


def test_interpolation_takes_the_parents_colour_and_size():
    """Children of another colour and a quarter of the parent's size: at
    the collapse distance (weight -> 1) they render with the parent's colour
    at the centre pixel and the parent's footprint."""
    sc = _two_copies_tree(0.6)
    sc["sh"][0, 0] = [0.8, -0.3, 0.1]
    sc["sh"][1:, 0] = [-0.2, 0.5, 0.4]
    sc["cov6"][0] = [0.04, 0, 0, 0.04, 0, 0.04]          # sigma 0.2 m
    sc["cov6"][1:] = [0.0025, 0, 0, 0.0025, 0, 0.0025]  # sigma 0.05 m
    sc["radius2"][:] = [0.36, 0.0225, 0.0225]
    tau, f = 30.0, 120.0
    t = float(np.float32(np.float32(tau) / np.float32(f)))
    imgs = {}
    for side, s in (("inside", 1 - 1e-5), ("outside", 1 + 1e-5)):
        cam = dict(R=np.eye(3, dtype=np.float32), pos=np.array([0, 0, -0.6 / t * s], np.float32),
                   fx=np.float32(f), fy=np.float32(f), cx=np.float32(32.5), cy=np.float32(32.5),
                   width=64, height=64, z_near=np.float32(0.2))
        imgs[side] = oracle.render(sc, cam, tau, interp=True)["image"]
        if side == "inside":
            imgs["plain"] = oracle.render(sc, cam, tau)["image"]
    np.testing.assert_allclose(imgs["inside"][32, 32], imgs["outside"][32, 32], rtol=1e-3, atol=1e-6)
    assert np.abs(imgs["plain"][32, 32] - imgs["outside"][32, 32]).max() > 0.1
    lit = {k: int((v.max(axis=2) > 0.02).sum()) for k, v in imgs.items()}
    assert abs(lit["inside"] - lit["outside"]) <= 0.15 * lit["outside"], lit
    assert lit["plain"] < 0.5 * lit["outside"], lit
