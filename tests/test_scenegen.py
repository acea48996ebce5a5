"""Checks of the seeded input generator (not part of the method): tree shape
invariants, the moment-matched merge against its closed form, radius nesting,
and determinism."""
import os
import subprocess
import sys

import numpy as np

import scenegen


def test_bfs_tree_invariants(tiny_scene):
    sc = tiny_scene
    N = sc["n_nodes"]
    par, fc, nch = sc["parent"].astype(np.int64), sc["first_child"].astype(np.int64), sc["n_child"]
    assert par[0] == 0xFFFFFFFF
    assert (nch == 0).sum() == sc["n_leaves"] == 4096
    assert nch.max() <= 8
    inner = np.nonzero(nch > 0)[0]
    assert (nch[inner] >= 2).all()  # single-child chains are collapsed
    for n in inner:
        kids = np.arange(fc[n], fc[n] + nch[n])
        assert (kids > n).all() and (par[kids] == n).all()
    # children blocks are contiguous and in parent order (BFS numbering)
    starts = fc[inner]
    assert (np.diff(starts) > 0).all() and starts[0] == 1
    assert (np.diff(par[1:]) >= 0).all()


def test_moment_match_two_gaussians():
    m = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, -1.0]], np.float32)
    c = np.array([[0.04, 0.01, 0.0, 0.09, 0.0, 0.01], [0.01, 0.0, 0.0, 0.02, 0.005, 0.03]], np.float32)
    op = np.array([0.3, 0.6], np.float32)
    sh = np.array([[[0.1, 0.2, 0.3]], [[-0.5, 0.4, 0.0]]], np.float32)
    leaves = dict(mean=m, cov6=c, opacity=op, sh=sh, rad2=np.array([0.01, 0.04], np.float32), sh_degree=0)
    sc = scenegen.build_tree(leaves)
    assert sc["n_nodes"] == 3 and sc["n_child"][0] == 2
    w = op.astype(np.float64)
    W = w.sum()
    mu = (w[:, None] * m).sum(0) / W
    S = np.zeros((3, 3))
    for i in range(2):
        Si = np.array([[c[i, 0], c[i, 1], c[i, 2]], [c[i, 1], c[i, 3], c[i, 4]], [c[i, 2], c[i, 4], c[i, 5]]], np.float64)
        d = (m[i] - mu)[:, None]
        S += w[i] * (Si + d @ d.T)
    S /= W
    np.testing.assert_allclose(sc["mean"][0], mu, rtol=1e-6)
    np.testing.assert_allclose(sc["cov6"][0], [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]], rtol=1e-6)
    np.testing.assert_allclose(sc["opacity"][0], 1 - (1 - 0.3) * (1 - 0.6), rtol=1e-6)
    np.testing.assert_allclose(sc["sh"][0, 0], (w[:, None] * sh[:, 0]).sum(0) / W, rtol=1e-6)


def test_radius_nesting(tiny_scene):
    sc = tiny_scene
    R = np.sqrt(sc["radius2"].astype(np.float64))
    kids = np.arange(1, sc["n_nodes"])
    p = sc["parent"][kids].astype(np.int64)
    d = np.linalg.norm(sc["mean"][kids].astype(np.float64) - sc["mean"][p].astype(np.float64), axis=1)
    assert (R[p] >= (R[kids] + d) * (1 + 2.0 ** -12) * (1 - 1e-12)).all()


def test_leaf_distributions(tiny_scene):
    sc = tiny_scene
    leaf = sc["n_child"] == 0
    m = sc["mean"][leaf]
    assert (m >= 0).all() and (m[:, :2] <= 20).all() and (m[:, 2] <= 5).all()
    op = sc["opacity"][leaf]
    assert (op > 0).all() and (op < 1).all()
    dc = sc["sh"][leaf][:, 0, :]
    assert 0.25 < dc.std() < 0.35


def test_deterministic_across_thread_counts():
    code = ("import scenegen, hashlib;"
            "s = scenegen.make_scene('tiny');"
            "print(hashlib.sha256(b''.join(s[k].tobytes() for k in "
            "('parent','first_child','n_child','mean','cov6','opacity','sh','radius2'))).hexdigest())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=nt, PYTHONPATH=root)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env, cwd=root).strip())
    assert outs[0] == outs[1]


def _yaw(cam):
    # camera forward axis (third row of R) in the z-up world
    f = np.asarray(cam["R"], np.float64).reshape(3, 3)[2]
    return np.arctan2(f[1], f[0])


def test_walks_follow_the_stated_motion():
    """Each workload's walk moves at its speed on its height and keeps the yaw
    rate within 2 pi A / period (18.9 deg/s for the 1M box and the city)."""
    for name in ("tiny", "m1", "city"):
        c = scenegen.CONFIGS[name]
        cams = [scenegen.trajectory(name, f) for f in range(0, min(c["frames"], 120))]
        pos = np.array([np.asarray(x["pos"], np.float64) for x in cams])
        step = np.linalg.norm(np.diff(pos, axis=0), axis=1)
        np.testing.assert_allclose(step, c["speed"] / c["fps"], rtol=1e-3)
        np.testing.assert_allclose(pos[:, 2], c["start"][2], atol=1e-5)
        yaw = np.unwrap([_yaw(x) for x in cams])
        rate = np.abs(np.diff(yaw)) * c["fps"]
        bound = 2 * np.pi * np.radians(c["yaw_amp_deg"]) / c["yaw_period"]
        assert rate.max() <= bound * 1.001
        assert cams[0]["width"] == c["width"] and cams[0]["fx"] == np.float32(c["focal"])


def test_street_walks_stay_on_streets():
    """The per-view and per-client walks run along a street of the 40 m grid
    (one coordinate fixed at 40 k, k in 1..36) at the city's height, with the
    focal length scaled with the image width."""
    c = scenegen.CONFIGS["city"]
    for seed in (200, 201, 237, 300, 331):
        for (W, H) in scenegen.RESOLUTIONS.values():
            cams = [scenegen.street_trajectory("city", seed, f, W, H) for f in (0, 150, 300)]
            pos = np.array([np.asarray(x["pos"], np.float64) for x in cams])
            fixed = [np.allclose(pos[:, a], pos[0, a], atol=1e-3) for a in (0, 1)]
            assert sum(fixed) == 1
            a = fixed.index(True)
            k = pos[0, a] / 40.0
            assert abs(k - round(k)) < 1e-4 and 1 <= round(k) <= 36
            np.testing.assert_allclose(pos[:, 2], c["start"][2], atol=1e-5)
            assert cams[0]["width"] == W and np.isclose(cams[0]["fx"], c["focal"] * W / c["width"])
