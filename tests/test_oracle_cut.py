"""Pins of the oracle's cut finding (paper Sec. 3.1 'Cut Finding').

The oracle's cut is checked against: a hand-derived golden tree, a pure
Python brute force of the definition, and the special cases the definition
fixes (tau = 0 gives all leaves; a far camera gives the root; the cut does
not depend on the camera orientation).
"""
import json
import os

import numpy as np
import pytest

import oracle
import scenegen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cut_small_tree.json")


def _golden_scene():
    g = json.load(open(GOLDEN))
    t = g["tree"]
    n = len(t["parent"])
    sc = dict(parent=np.array(t["parent"], np.uint32), first_child=np.array(t["first_child"], np.uint32),
              n_child=np.array(t["n_child"], np.uint8), mean=np.array(t["mean"], np.float32),
              cov6=np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (n, 1)),
              opacity=np.full(n, 0.5, np.float32), sh=np.zeros((n, 1, 3), np.float32),
              radius2=np.array(t["radius2"], np.float32), sh_degree=0, n_nodes=n)
    return g, sc


def test_golden_small_tree():
    g, sc = _golden_scene()
    for case in g["cases"]:
        k = oracle.lod_k(case["tau"], case["f"])
        got = oracle.cut(sc, case["cam"], k)
        assert got.tolist() == case["cut"], case["why"]
        got_bf = oracle.cut(sc, case["cam"], k, bruteforce=True)
        assert got_bf.tolist() == case["cut"], case["why"]


def _python_cut(sc, cam, k):
    """The definition, in plain Python with float32 scalars."""
    f32 = np.float32
    cam = np.asarray(cam, np.float32)
    mean, r2, nch, par = sc["mean"], sc["radius2"], sc["n_child"], sc["parent"]

    def expand(n):
        if nch[n] == 0:
            return False
        dx, dy, dz = f32(cam[0] - mean[n, 0]), f32(cam[1] - mean[n, 1]), f32(cam[2] - mean[n, 2])
        d2 = f32(f32(f32(dx * dx) + f32(dy * dy)) + f32(dz * dz))
        return bool(f32(d2 * f32(k)) < r2[n])

    out = []
    for n in range(int(sc["n_nodes"])):
        if expand(n):
            continue
        a, ok = int(par[n]), True
        while a != 0xFFFFFFFF:
            if not expand(a):
                ok = False
                break
            a = int(par[a])
        if ok:
            out.append(n)
    return np.array(out, np.uint32)


def test_cut_matches_python_bruteforce(tiny_scene):
    rng = np.random.default_rng(3)
    for _ in range(12):
        cam = rng.uniform([-5, -5, -2], [25, 25, 8]).astype(np.float32)
        tau = float(rng.choice([0.5, 3.0, 15.0, 60.0]))
        k = oracle.lod_k(tau, 120.0)
        got = oracle.cut(tiny_scene, cam, k)
        want = _python_cut(tiny_scene, cam, k)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(oracle.cut(tiny_scene, cam, k, bruteforce=True), want)


def test_cut_is_a_cover(tiny_scene):
    """Every leaf has exactly one ancestor-or-self in the cut."""
    sc = tiny_scene
    cam = np.array([3.0, 9.0, 2.0], np.float32)
    c = oracle.cut(sc, cam, oracle.lod_k(3.0, 120.0))
    inc = np.zeros(sc["n_nodes"], bool)
    inc[c] = True
    par = sc["parent"]
    for leaf in np.nonzero(sc["n_child"] == 0)[0][::7]:
        hits, a = 0, int(leaf)
        while a != 0xFFFFFFFF:
            hits += inc[a]
            a = int(par[a])
        assert hits == 1


def test_tau_zero_gives_all_leaves(tiny_scene):
    cam = np.array([10.0, 10.0, 2.0], np.float32)
    c = oracle.cut(tiny_scene, cam, oracle.lod_k(0.0, 120.0))
    np.testing.assert_array_equal(c, np.nonzero(tiny_scene["n_child"] == 0)[0].astype(np.uint32))


def test_far_camera_gives_root(tiny_scene):
    r = float(np.sqrt(tiny_scene["radius2"][0]))
    cam = tiny_scene["mean"][0] + np.array([r * 40.0 + 1.0, 0, 0], np.float32)  # tau/f = 3/120
    c = oracle.cut(tiny_scene, cam, oracle.lod_k(3.0, 120.0))
    assert c.tolist() == [0]


def test_cut_depends_on_position_only(tiny_scene):
    base = scenegen.trajectory("tiny", 5)
    r1 = oracle.render(tiny_scene, base, 3.0)
    cam2 = dict(base)
    cam2["R"] = scenegen.look_rotation(2.0, 0.3).astype(np.float32)
    r2 = oracle.render(tiny_scene, cam2, 3.0)
    np.testing.assert_array_equal(r1["cut"], r2["cut"])


def test_lod_k_is_fp32():
    # tau / f and its square are single-rounded FP32 operations
    t = np.float32(np.float32(3.0) / np.float32(1100.0))
    assert oracle.lod_k(3.0, 1100.0) == np.float32(t * t)


def test_granularity_boundary_is_strict():
    """A node is refined only while its projected size R f / d is above tau,
    i.e. d^2 (tau / f)^2 < R^2; at equality it stays in the cut.  With tau = f
    (k = 1) and d = 2 the boundary is R^2 = 4, exactly representable."""
    sc = dict(parent=np.array([0xFFFFFFFF, 0, 0], np.uint32), first_child=np.array([1, 0, 0], np.uint32),
              n_child=np.array([2, 0, 0], np.uint8),
              mean=np.array([[0, 0, 2], [0, 0.5, 2], [0, -0.5, 2]], np.float32),
              cov6=np.tile(np.array([1, 0, 0, 1, 0, 1], np.float32), (3, 1)),
              opacity=np.full(3, 0.5, np.float32), sh=np.zeros((3, 1, 3), np.float32),
              radius2=np.array([4.0, 1.0, 1.0], np.float32), sh_degree=0, n_nodes=3)
    cam = np.zeros(3, np.float32)
    k = oracle.lod_k(100.0, 100.0)
    assert k == np.float32(1.0)
    assert not oracle.expand(sc, 0, cam, k)
    assert oracle.cut(sc, cam, k).tolist() == [0]
    sc["radius2"] = np.array([np.nextafter(np.float32(4.0), np.float32(5.0)), 1.0, 1.0], np.float32)
    assert oracle.expand(sc, 0, cam, k)
    assert oracle.cut(sc, cam, k).tolist() == [1, 2]
