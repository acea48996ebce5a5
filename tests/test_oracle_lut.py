"""Pins of the oracle's lookup-table variant (paper Sec. 4.2, Eq. 5): e^rho
replaced by the nearest of the samples e^(-5.55 i / m), i = 0..m, after the
Eq. 4 test has decided which pixels a Gaussian reaches.

* the nearest sample is within half an interval, so the table's value and
  e^rho differ by a factor of at most e^(5.55 / (2m)) either way, and both
  extremes are approached over a Gaussian's footprint;
* at rho = 0 the table is exact;
* the set of pixels a Gaussian reaches is the exact mode's (Eq. 4 decides);
* as m grows the image converges to the exact one.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen

C0 = 1.0 / (2.0 * math.sqrt(math.pi))


def _cam(f=100.0, W=96, H=80):
    return dict(R=np.eye(3, dtype=np.float32), pos=np.zeros(3, np.float32), fx=np.float32(f), fy=np.float32(f),
                cx=np.float32(W / 2 + 0.5), cy=np.float32(H / 2 + 0.5), width=W, height=H,
                z_near=np.float32(0.2))


def _one(theta=0.9, s=(0.25, 0.15), dc=1.0):
    cov = [s[0] ** 2, 0.0, 0.0, s[1] ** 2, 0.0, 0.0004]
    return scenegen.single_node_scene((0.0, 0.0, 3.0), cov, theta, np.array([[dc, dc, dc]], np.float32))


@pytest.mark.parametrize("m", [8, 32])
def test_table_within_half_an_interval(m):
    sc, cam = _one(), _cam()
    ex = oracle.render(sc, cam, 0.0)
    lt = oracle.render(sc, cam, 0.0, lut_m=m)
    a, b = ex["image"][..., 0], lt["image"][..., 0]
    np.testing.assert_array_equal(a > 0, b > 0)           # Eq. 4 decides the footprint
    assert (a > 0).sum() > 1000
    r = b[a > 0] / a[a > 0]
    h = 5.55 / (2 * m)
    assert r.max() <= math.exp(h) * (1 + 1e-12) and r.min() >= math.exp(-h) * (1 - 1e-12)
    assert r.max() >= math.exp(0.9 * h) and r.min() <= math.exp(-0.9 * h)  # both extremes are reached
    # the mean sits on the centre of pixel (48, 40): rho = 0 there, e^0 is a table entry
    assert b[40, 48] == a[40, 48]


def test_table_values_are_samples_of_the_range():
    """With a single Gaussian at T = 1 every lit pixel is theta e^(-5.55 i/m) rgb."""
    m = 16
    theta = np.float64(np.float32(0.9))
    rgb = 0.5 + C0 * np.float64(np.float32(1.0))
    lt = oracle.render(_one(), _cam(), 0.0, lut_m=m)
    v = lt["image"][..., 0]
    lit = v[v > 0] / (theta * rgb)
    i = -np.log(lit) * m / 5.55
    np.testing.assert_allclose(i, np.round(i), atol=1e-9)
    assert set(np.round(i).astype(int)) <= set(range(m + 1))
    assert len(set(np.round(i).astype(int))) == m + 1  # rho reaches -5.44 here: every entry is used


def test_converges_to_the_exact_image(tiny_scene):
    cam = scenegen.trajectory("tiny", 6)
    ex = oracle.render(tiny_scene, cam, 3.0)
    errs = [np.abs(oracle.render(tiny_scene, cam, 3.0, lut_m=m)["image"] - ex["image"]).max()
            for m in (8, 64, 512, 4096)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 2e-3
    assert errs[0] > 0.05


def test_table_alpha_is_capped():
    # theta = 1 at the pixel centre on the mean: entry 0 is 1, alpha is capped at 0.99
    lt = oracle.render(_one(theta=1.0), _cam(), 0.0, lut_m=32)
    rgb = 0.5 + C0 * np.float64(np.float32(1.0))
    assert lt["image"][40, 48, 0] == pytest.approx(0.99 * rgb, rel=1e-12)


def test_tiled_equals_exhaustive_with_the_table(tiny_scene):
    """Eq. 4 still decides which pixels a Gaussian reaches, so the tile filter
    stays exact under the table: binned and exhaustive images are equal."""
    for fr in (0, 9):
        cam = scenegen.trajectory("tiny", fr)
        a = oracle.render(tiny_scene, cam, 3.0, lut_m=32)
        b = oracle.render(tiny_scene, cam, 3.0, lut_m=32, exhaustive=True)
        assert np.array_equal(a["image"], b["image"])
        assert a["image"].max() > 0.05
