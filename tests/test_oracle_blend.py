"""Pins of the oracle's preemptive alpha filter (paper Sec. 4.2, Eq. 3, 4),
tile binning, sort and front-to-back blending (Sec. 3.1 'Rasterization').

* exhaustive per-pixel blending of every cut Gaussian (no tiles, boxes or
  filters) must give exactly the tiled, filtered image;
* every dropped Gaussian-tile pair has alpha < alpha* at all its pixels
  (brute-force scan);
* rho_max over a tile rectangle bounds rho at every pixel and is attained;
* single- and multi-Gaussian images are checked against hand-computed
  values, including the T < 1e-4 termination rule and the 0.99 alpha cap;
* every candidate's margin is the maximum of rho over its tile's pixel-centre
  hull (found by a bounded solver), Gaussians below alpha* get no tile, and
  equal depth keys blend in node-id order.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen


def _cam(pos=(0, 0, 0), f=100.0, W=64, H=48, cx=None, cy=None, R=None):
    return dict(R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                pos=np.asarray(pos, np.float32), fx=np.float32(f), fy=np.float32(f),
                cx=np.float32(W / 2 if cx is None else cx), cy=np.float32(H / 2 if cy is None else cy),
                width=W, height=H, z_near=np.float32(0.2))


def _flat_scene(means, covs, opac, dcs):
    """A root whose children are the given Gaussians; tau = 0 selects them all."""
    n = len(means)
    sc = dict(parent=np.array([0xFFFFFFFF] + [0] * n, np.uint32),
              first_child=np.array([1] + [0] * n, np.uint32),
              n_child=np.array([n] + [0] * n, np.uint8),
              mean=np.array([[0, 0, 0]] + list(means), np.float32),
              cov6=np.array([[1, 0, 0, 1, 0, 1]] + list(covs), np.float32),
              opacity=np.array([0.5] + list(opac), np.float32),
              sh=np.array([[[0, 0, 0]]] + [[d] for d in dcs], np.float32),
              radius2=np.full(n + 1, 1e6, np.float32), sh_degree=0, n_nodes=n + 1)
    return sc


C0 = 1.0 / (2.0 * math.sqrt(math.pi))


def _dc_for(rgb):
    return [(c - 0.5) / C0 for c in rgb]


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_exhaustive_equals_tiled(tiny_scene, tile):
    for fr in (0, 7, 15):
        cam = scenegen.trajectory("tiny", fr)
        a = oracle.render(tiny_scene, cam, 3.0, tile=tile)
        b = oracle.render(tiny_scene, cam, 3.0, exhaustive=True)
        assert np.array_equal(a["image"], b["image"])
        assert a["image"].max() > 0.05
        assert a["tiles"] == ((128 + tile - 1) // tile,) * 2


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_exhaustive_equals_tiled_sh3(small_sh3_scene, tile):
    """Binning is exact at every tile size: the image is the exhaustive one
    bit for bit; smaller tiles give more, tighter pairs."""
    cam = scenegen.camera((2.0, 15.0, 3.0), 0.2, 96, 80, 90.0)
    a = oracle.render(small_sh3_scene, cam, 3.0, tile=tile)
    b = oracle.render(small_sh3_scene, cam, 3.0, exhaustive=True)
    assert np.array_equal(a["image"], b["image"])
    assert a["n_pairs"] > 1000
    assert len(a["tile_start"]) == a["tiles"][0] * a["tiles"][1] + 1
    if tile == 8:
        c = oracle.render(small_sh3_scene, cam, 3.0, tile=16)
        assert a["n_pairs"] > c["n_pairs"] and a["n_eval_total"] < c["n_eval_total"]


def _alpha_at(p, x, y):
    dx, dy = p["u"] - x, p["v"] - y
    a, b, c = p["conic"]
    rho = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    return np.minimum(0.99, p["theta"] * np.exp(rho)), rho


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_dropped_pairs_never_reach_alpha_min(tiny_scene, tile):
    cam = scenegen.trajectory("tiny", 3)
    r = oracle.render(tiny_scene, cam, 3.0, tile=tile)
    TW = r["tiles"][0]
    dropped = np.nonzero(r["cand_margin"] < 0)[0]
    assert len(dropped) > 10
    for c in dropped:
        p = r["proj"][r["cand_idx"][c]]
        t = int(r["cand_tile"][c])
        tx, ty = t % TW, t // TW
        xs = np.arange(tx * tile, min(tx * tile + tile, cam["width"])) + 0.5
        ys = np.arange(ty * tile, min(ty * tile + tile, cam["height"])) + 0.5
        X, Y = np.meshgrid(xs, ys)
        alpha, _ = _alpha_at(p, X, Y)
        assert alpha.max() < oracle.ALPHA_MIN


def test_rho_max_bounds_and_is_attained():
    rng = np.random.default_rng(11)
    for _ in range(200):
        A = rng.normal(size=(2, 2))
        S = A @ A.T * rng.uniform(1, 50) + 0.3 * np.eye(2)
        conic = np.linalg.inv(S)
        con = np.array([conic[0, 0], conic[0, 1], conic[1, 1]])
        u, v = rng.uniform(-40, 60, size=2)
        x0, y0 = 16 * 1 + 0.5, 16 * 0 + 0.5
        x1, y1 = x0 + 15, y0 + 15
        rm = oracle.rho_max_rect(con, u, v, x0, x1, y0, y1)
        g = np.linspace(0, 1, 301)
        X, Y = np.meshgrid(x0 + (x1 - x0) * g, y0 + (y1 - y0) * g)
        dx, dy = X - u, Y - v
        rho = -0.5 * (con[0] * dx * dx + con[2] * dy * dy) - con[1] * dx * dy
        assert rm >= rho.max() - 1e-12
        assert rm <= rho.max() + 2e-3 * (1 + abs(rho.max()))  # the grid gets close to the maximum


def test_rho_max_closed_form_axis_aligned():
    # mean left of the rectangle and inside its y-range: the max is at x0, dy = 0
    con = [0.25, 0.0, 0.5]
    assert oracle.rho_max_rect(con, 10.0, 8.0, 16.5, 31.5, 0.5, 15.5) == pytest.approx(-0.5 * 0.25 * 6.5 ** 2)
    # mean inside: 0
    assert oracle.rho_max_rect(con, 20.0, 8.0, 16.5, 31.5, 0.5, 15.5) == 0.0
    # mean below-left: the corner (x0, y1) for an axis-aligned conic
    r = oracle.rho_max_rect(con, 10.0, 20.0, 16.5, 31.5, 0.5, 15.5)
    assert r == pytest.approx(-0.5 * (0.25 * 6.5 ** 2 + 0.5 * 4.5 ** 2))


def test_opacity_zero_gives_black(tiny_scene):
    sc = dict(tiny_scene)
    sc["opacity"] = np.zeros_like(tiny_scene["opacity"])
    r = oracle.render(sc, scenegen.trajectory("tiny", 2), 3.0)
    assert r["n_pairs"] == 0 and r["n_visible"] == 0
    assert not r["image"].any()


def test_empty_frustum_gives_black(tiny_scene):
    fwd = scenegen.trajectory("tiny", 4)
    back = dict(fwd)
    back["R"] = scenegen.look_rotation(math.pi).astype(np.float32)
    # behind the start position (x = 2 m, looking toward -x) there is almost nothing
    back["pos"] = np.array([-30.0, 10.0, 2.5], np.float32)
    fwd2 = dict(fwd)
    fwd2["pos"] = back["pos"]
    rb, rf = oracle.render(tiny_scene, back, 3.0), oracle.render(tiny_scene, fwd2, 3.0)
    assert not rb["image"].any() and rb["n_pairs"] == 0
    np.testing.assert_array_equal(rb["cut"], rf["cut"])
    assert rf["image"].any()


def test_single_gaussian_image_closed_form():
    f, z, s1, s2 = 100.0, 4.0, 0.05, 0.03
    cam = _cam(f=f, W=64, H=48)
    rgb = (0.9, 0.4, 0.2)
    theta = 0.7
    sc = _flat_scene([(0.1, -0.05, z)], [[s1 * s1, 0, 0, s2 * s2, 0, 0.0004]], [theta], [_dc_for(rgb)])
    r = oracle.render(sc, cam, 0.0)
    u, v = f * 0.1 / z + 32, f * -0.05 / z + 24
    tx = 0.1 / z
    S00 = f * f / z / z * (float(np.float32(s1 * s1)) + tx * tx * float(np.float32(0.0004))) + 0.3
    S11 = f * f / z / z * (float(np.float32(s2 * s2)) + (0.05 / z) ** 2 * float(np.float32(0.0004))) + 0.3
    S01 = f * f / z / z * (tx * (-0.05 / z) * float(np.float32(0.0004)))
    S = np.array([[S00, S01], [S01, S11]])
    Ci = np.linalg.inv(S)
    X, Y = np.meshgrid(np.arange(64) + 0.5, np.arange(48) + 0.5)
    dx, dy = X - u, Y - v
    rho = -0.5 * (Ci[0, 0] * dx * dx + Ci[1, 1] * dy * dy) - Ci[0, 1] * dx * dy
    alpha = np.minimum(0.99, float(np.float32(theta)) * np.exp(rho))
    alpha[alpha < 1 / 255] = 0.0
    rgbf = [0.5 + C0 * np.float64(np.float32(d)) for d in _dc_for(rgb)]
    want = alpha[..., None] * np.array(rgbf)
    np.testing.assert_allclose(r["image"], want, rtol=1e-6, atol=1e-9)


def test_front_to_back_order_and_termination():
    """Four wide on-axis Gaussians of opacity 0.95 at increasing depth, all
    centred on pixel (32, 24): alpha = 0.95 there and T runs 1, 0.05,
    0.0025, 1.25e-4; the fourth would take T to 6.25e-6 < 1e-4, so it is
    excluded.  Colour = 0.95 c1 + 0.0475 c2 + 0.002375 c3."""
    cam = _cam(f=100.0, W=64, H=48, cx=32.5, cy=24.5)
    cols = [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1), (0.1, 0.1, 0.9), (0.7, 0.7, 0.7)]
    zs = [3.0, 3.5, 4.0, 4.5]
    # listed far-to-near so that the sort, not the input order, decides
    order = [3, 1, 0, 2]
    sc = _flat_scene([(0, 0, zs[i]) for i in order], [[0.04, 0, 0, 0.04, 0, 0.04]] * 4,
                     [0.95] * 4, [_dc_for(cols[i]) for i in order])
    r = oracle.render(sc, cam, 0.0)
    rgbf = [np.array([0.5 + C0 * np.float64(np.float32(d)) for d in _dc_for(c)]) for c in cols]
    a = np.float64(np.float32(0.95))
    want = a * rgbf[0] + a * (1 - a) * rgbf[1] + a * (1 - a) ** 2 * rgbf[2]
    np.testing.assert_allclose(r["image"][24, 32], want, rtol=1e-12)
    assert r["n_contrib"][24, 32] == 3


def test_sorted_pairs_are_ordered(tiny_scene):
    r = oracle.render(tiny_scene, scenegen.trajectory("tiny", 9), 3.0)
    t, g = r["pair_tile"], r["pair_idx"]
    zk = r["proj"]["zkey"][g]
    node = r["cut"][g]
    key = np.lexsort((node, zk, t))
    np.testing.assert_array_equal(key, np.arange(len(t)))
    # tile ranges partition the pair list
    ts = r["tile_start"]
    assert ts[0] == 0 and ts[-1] == len(t)
    for tile in range(0, r["n_tiles"], 5):
        assert np.all(t[ts[tile]:ts[tile + 1]] == tile)


def test_alpha_is_capped_at_0_99():
    """An opaque Gaussian (theta = 1) centred on a pixel centre: alpha is
    capped at 0.99 there, so the pixel is 0.99 rgb and T ends at 0.01 (an
    uncapped alpha of 1 would take T to 0 < 1e-4 and stop before adding)."""
    cam = _cam(f=100.0, W=64, H=48, cx=32.5, cy=24.5)
    rgb = (0.8, 0.3, 0.6)
    sc = _flat_scene([(0, 0, 3.0)], [[0.04, 0, 0, 0.04, 0, 0.04]], [1.0], [_dc_for(rgb)])
    r = oracle.render(sc, cam, 0.0)
    rgbf = np.array([0.5 + C0 * np.float64(np.float32(d)) for d in _dc_for(rgb)])
    np.testing.assert_allclose(r["image"][24, 32], 0.99 * rgbf, rtol=1e-12)
    assert r["n_contrib"][24, 32] == 1


def test_gaussian_level_filter_drops_faint_gaussians():
    """alpha <= theta everywhere, so a Gaussian with theta < alpha* = 1/255
    can never contribute and gets no candidate tile at all; just above
    alpha* it gets the tiles around its centre, and the tile holding the
    centre is kept (rho_max = 0 >= ln alpha* - ln theta)."""
    cam = _cam(f=100.0, W=64, H=48)
    for theta, has in ((0.0035, False), (0.0045, True)):
        sc = _flat_scene([(0.05, 0.02, 3.0)], [[0.04, 0, 0, 0.04, 0, 0.04]], [theta], [_dc_for((1, 1, 1))])
        r = oracle.render(sc, cam, 0.0)
        assert (r["n_cand"] > 0) == has
        assert (r["n_pairs"] > 0) == has
        assert r["n_visible"] == int(has)


def test_equal_depth_ties_go_to_the_lower_node_id():
    """Two coincident Gaussians with the same FP32 depth key: the pair order
    is (tile, depth key, node id), so the lower node id is blended first."""
    cam = _cam(f=100.0, W=64, H=48, cx=32.5, cy=24.5)
    red, green = (0.9, 0.1, 0.1), (0.1, 0.9, 0.1)
    a = np.float64(np.float32(0.9))
    for first, second in ((red, green), (green, red)):
        sc = _flat_scene([(0, 0, 3.0), (0, 0, 3.0)], [[0.04, 0, 0, 0.04, 0, 0.04]] * 2, [0.9, 0.9],
                         [_dc_for(first), _dc_for(second)])
        r = oracle.render(sc, cam, 0.0)
        f1 = np.array([0.5 + C0 * np.float64(np.float32(d)) for d in _dc_for(first)])
        f2 = np.array([0.5 + C0 * np.float64(np.float32(d)) for d in _dc_for(second)])
        np.testing.assert_allclose(r["image"][24, 32], a * f1 + a * (1 - a) * f2, rtol=1e-12)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tile_margin_is_the_max_over_the_pixel_centre_hull(tiny_scene, tile):
    """For every candidate pair, margin + (ln alpha* - ln theta) is the maximum
    of rho over the convex hull of the tile's pixel centres, clipped to the
    image (the ragged last column and row included).  rho is concave, so a
    bounded quasi-Newton solve finds that maximum independently."""
    opt = pytest.importorskip("scipy.optimize")
    cam = scenegen.camera((2.0, 10.0, 2.5), 0.1, 88 if tile < 32 else 100, 56 if tile < 32 else 70, 60.0)
    r = oracle.render(tiny_scene, cam, 3.0, tile=tile)
    TW, TH = r["tiles"]
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(3)
    cands = np.arange(len(r["cand_tile"]))
    edge = cands[(r["cand_tile"] % TW == TW - 1) | (r["cand_tile"] // TW == TH - 1)]
    assert len(edge) > 20
    pick = np.concatenate([rng.choice(cands, min(150, len(cands)), replace=False),
                           rng.choice(edge, 50, replace=False)])
    for c in pick:
        p = r["proj"][r["cand_idx"][c]]
        t = int(r["cand_tile"][c])
        tx, ty = t % TW, t // TW
        lo = (tile * tx + 0.5, tile * ty + 0.5)
        hi = (min(tile * tx + tile - 0.5, W - 0.5), min(tile * ty + tile - 0.5, H - 0.5))
        a, b, cc = p["conic"]

        def neg(x):
            dx, dy = x[0] - p["u"], x[1] - p["v"]
            val = 0.5 * (a * dx * dx + cc * dy * dy) + b * dx * dy
            return val, np.array([a * dx + b * dy, cc * dy + b * dx])

        x0 = np.clip([p["u"], p["v"]], lo, hi)
        res = opt.minimize(neg, x0, jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                           options=dict(ftol=1e-15, gtol=1e-12, maxiter=200))
        want = -res.fun
        got = r["cand_margin"][c] + p["thr"]
        assert got == pytest.approx(want, rel=1e-7, abs=1e-7), (c, tx, ty)
