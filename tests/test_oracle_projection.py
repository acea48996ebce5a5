"""Pins of the oracle's projection (EWA conventions, paper Sec. 3.1
'Culling & Projection') and its spherical-harmonic colour.

Closed forms used:
* a Gaussian on the optical axis with axis-aligned scales projects to
  Sigma' = diag(fx^2 sx^2 / z^2 + 0.3, fy^2 sy^2 / z^2 + 0.3) at (cx, cy);
* an isotropic Gaussian at camera-space (x, 0, z) has
  Sigma'_00 = s^2 fx^2 / z^2 (1 + x^2 / z^2) + 0.3, with x / z clamped to
  1.3 (W/2) / fx inside the Jacobian;
* rotating camera and scene together changes nothing;
* an image-plane rotation phi of an on-axis Gaussian rotates Sigma'.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen


def _cam(R=None, pos=(0, 0, 0), f=100.0, W=128, H=96, cx=None, cy=None):
    return dict(R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                pos=np.asarray(pos, np.float32), fx=np.float32(f), fy=np.float32(f),
                cx=np.float32(W / 2 if cx is None else cx), cy=np.float32(H / 2 if cy is None else cy),
                width=W, height=H, z_near=np.float32(0.2))


def _one(mean, cov6, opacity=0.8, sh=(0.0, 0.0, 0.0)):
    return scenegen.single_node_scene(mean, cov6, opacity, np.asarray(sh, np.float32).reshape(1, 3))


def test_on_axis_closed_form():
    z, sx, sy, sz = 4.0, 0.05, 0.02, 0.03
    cam = _cam(pos=(1.0, 2.0, 3.0), f=100.0)
    sc = _one((1.0, 2.0, 3.0 + z), [sx * sx, 0, 0, sy * sy, 0, sz * sz])
    p = oracle.render(sc, cam, 0.0)["proj"][0]
    assert p["valid"] == 1
    assert p["u"] == pytest.approx(64.0) and p["v"] == pytest.approx(48.0)
    s00 = 100.0 ** 2 * float(np.float32(sx * sx)) / z ** 2 + 0.3
    s11 = 100.0 ** 2 * float(np.float32(sy * sy)) / z ** 2 + 0.3
    np.testing.assert_allclose(p["cov"], [s00, 0.0, s11], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p["conic"], [1 / s00, 0.0, 1 / s11], rtol=1e-12)
    assert p["z"] == pytest.approx(z)


def test_off_axis_isotropic_and_clamp():
    s = 0.05
    cov = [s * s, 0, 0, s * s, 0, s * s]
    for x, z in [(0.5, 3.0), (-1.2, 2.0), (9.0, 4.0)]:  # the last is beyond the clamp
        cam = _cam(f=100.0, W=128, H=96)
        sc = _one((x, 0.0, z), cov)
        p = oracle.render(sc, cam, 0.0)["proj"][0]
        lim = 1.3 * (128 / 2) / 100.0
        xf = float(np.float32(x))
        t = max(-lim, min(lim, xf / z))
        s2 = np.float64(np.float32(s * s))
        want00 = s2 * 100.0 ** 2 / z ** 2 * (1 + t * t) + 0.3
        want11 = s2 * 100.0 ** 2 / z ** 2 + 0.3
        assert p["u"] == pytest.approx(100.0 * xf / z + 64.0)
        np.testing.assert_allclose([p["cov"][0], p["cov"][2]], [want00, want11], rtol=1e-9)
        assert abs(p["cov"][1]) < 1e-12


def _rot(axis, ang):
    axis = np.asarray(axis, np.float64)
    axis /= np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_rotating_camera_and_scene_together():
    """World rotation Q applied to the scene and the camera leaves the image
    unchanged: catches a transposed rotation or a wrong Sigma_cam = R Sigma R^T."""
    Q = _rot([0.3, -0.5, 0.8], 0.9)
    Qf = Q.astype(np.float32).astype(np.float64)  # the rotation actually used
    S0 = np.diag([0.09, 0.01, 0.04])
    A = _rot([1, 2, 3], 0.4)
    S0 = A @ S0 @ A.T
    m0 = np.array([0.3, -0.2, 3.0])
    c6 = lambda S: [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]]
    p0 = oracle.render(_one(m0, c6(S0)), _cam(), 0.0)["proj"][0]
    # camera R' = Q^T (world->camera), scene point Q m0, covariance Q S0 Q^T
    cam = _cam(R=Qf.T)
    Rcam = np.asarray(cam["R"], np.float64)
    m1 = Q @ m0
    S1 = Q @ S0 @ Q.T
    p1 = oracle.render(_one(m1, c6(S1)), cam, 0.0)["proj"][0]
    # the FP32 rounding of R', m1 and S1 limits agreement to ~1e-6 relative
    np.testing.assert_allclose([p1["u"], p1["v"]], [p0["u"], p0["v"]], rtol=2e-6)
    np.testing.assert_allclose(p1["cov"], p0["cov"], rtol=5e-5, atol=5e-5)
    assert np.allclose(Rcam @ Rcam.T, np.eye(3), atol=1e-6)


def test_image_plane_rotation_sign_of_b():
    """On-axis Gaussian whose covariance is rotated by phi about the optical
    axis: Sigma' = (f/z)^2 Rot(phi) diag(s1^2, s2^2) Rot(phi)^T + 0.3 I."""
    f, z, s1, s2, phi = 100.0, 5.0, 0.2, 0.04, 0.6
    Rz = _rot([0, 0, 1], phi)
    S = Rz @ np.diag([s1 * s1, s2 * s2, 0.01]) @ Rz.T
    sc = _one((0, 0, z), [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]])
    p = oracle.render(sc, _cam(f=f), 0.0)["proj"][0]
    R2 = Rz[:2, :2]
    want = (f / z) ** 2 * (R2 @ np.diag([s1 * s1, s2 * s2]) @ R2.T) + 0.3 * np.eye(2)
    np.testing.assert_allclose(p["cov"], [want[0, 0], want[0, 1], want[1, 1]], rtol=1e-6)
    inv = np.linalg.inv(want)
    np.testing.assert_allclose(p["conic"], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6)
    assert p["cov"][1] > 0  # phi in (0, pi/2) tilts the long axis into +x +y


def test_near_plane_cull():
    cov = [0.01, 0, 0, 0.01, 0, 0.01]
    assert oracle.render(_one((0, 0, 0.19), cov), _cam(), 0.0)["proj"][0]["valid"] == 0
    assert oracle.render(_one((0, 0, 0.21), cov), _cam(), 0.0)["proj"][0]["valid"] == 1
    assert oracle.render(_one((0, 0, -3.0), cov), _cam(), 0.0)["proj"][0]["valid"] == 0


def test_depth_key_is_fp32_expression():
    cam = _cam(R=_rot([0.2, 1.0, 0.1], 0.3), pos=(1000.25, 700.5, 1.7))
    m = np.array([1003.1, 702.2, 2.9], np.float32)
    p = oracle.render(_one(m, [0.01, 0, 0, 0.01, 0, 0.01]), cam, 0.0)["proj"][0]
    R = cam["R"]
    f32 = np.float32
    d = [f32(m[i] - cam["pos"][i]) for i in range(3)]
    want = f32(f32(f32(R[2, 0] * d[0]) + f32(R[2, 1] * d[1])) + f32(R[2, 2] * d[2]))
    assert p["zkey"] == want


# ------------------------------------------------------------------- colour
def test_sh_degree0_colour():
    for dc in (0.0, 0.7, -3.0):
        sc = _one((0, 0, 2.0), [0.01, 0, 0, 0.01, 0, 0.01], sh=(dc, dc / 2, -dc))
        p = oracle.render(sc, _cam(), 0.0)["proj"][0]
        c0 = 1.0 / (2.0 * math.sqrt(math.pi))
        want = [max(0.0, 0.5 + np.float64(np.float32(v)) * c0) for v in (dc, dc / 2, -dc)]
        np.testing.assert_allclose(p["rgb"], want, rtol=1e-12, atol=1e-15)


def test_sh_closed_forms():
    rng = np.random.default_rng(5)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        x, y, z = d
        Y = oracle.sh_basis(3, d)
        c1 = math.sqrt(3 / (4 * math.pi))
        np.testing.assert_allclose(Y[0], 1 / (2 * math.sqrt(math.pi)), rtol=1e-14)
        np.testing.assert_allclose(Y[1:4], [-c1 * y, c1 * z, -c1 * x], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Y[6], math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Y[8], math.sqrt(15 / (16 * math.pi)) * (x * x - y * y), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Y[4], math.sqrt(15 / (4 * math.pi)) * x * y, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(Y[12], math.sqrt(7 / (16 * math.pi)) * z * (5 * z * z - 3), rtol=1e-12, atol=1e-14)


def test_sh_orthonormal_by_quadrature():
    xs, ws = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phis = 2 * math.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = oracle.sh_basis(3, [st * math.cos(ph), st * math.sin(ph), ct])
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(9)
    for _ in range(8):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(sp.sph_harm_y(l, abs(m), theta, phi))  # includes the Condon-Shortley phase
                want = c.real if m == 0 else math.sqrt(2) * (c.real if m > 0 else c.imag)
                assert Y[l * l + l + m] == pytest.approx(want, abs=1e-12)


def test_near_plane_boundary_is_strict():
    # kept iff the FP32 depth key is above z_near: a mean exactly on the plane is culled
    cov = [0.01, 0, 0, 0.01, 0, 0.01]
    zn = np.float32(0.2)
    assert oracle.render(_one((0, 0, zn), cov), _cam(), 0.0)["proj"][0]["valid"] == 0
    above = np.nextafter(zn, np.float32(1.0))
    assert oracle.render(_one((0, 0, above), cov), _cam(), 0.0)["proj"][0]["valid"] == 1


def test_sh_view_direction_is_camera_to_mean():
    """Degree-1 colour at a mean seen along d = (0.6, 0, 0.8) from the camera:
    the Y_10 (c1 z) coefficient in red and the Y_11 (-c1 x) coefficient in
    green give 0.5 + 0.8 c1 and 0.5 - 0.6 c1; the opposite direction would
    swap the signs."""
    sh = np.zeros((4, 3), np.float32)
    sh[2, 0] = 1.0
    sh[3, 1] = 1.0
    sc = scenegen.single_node_scene((0.75, 0.0, 1.0), [0.01, 0, 0, 0.01, 0, 0.01], 0.8, sh, sh_degree=1)
    p = oracle.render(sc, _cam(f=40.0), 0.0)["proj"][0]
    assert p["valid"] == 1
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(p["rgb"], [0.5 + 0.8 * c1, 0.5 - 0.6 * c1, 0.5], rtol=1e-12)
    # seen from the far side of the mean, the odd band changes sign
    cam = _cam(f=40.0, pos=(1.5, 0.0, 2.0), R=np.diag([-1.0, 1.0, -1.0]))
    q = oracle.render(sc, cam, 0.0)["proj"][0]
    assert q["valid"] == 1
    np.testing.assert_allclose(q["rgb"], [0.5 - 0.8 * c1, 0.5 + 0.6 * c1, 0.5], rtol=1e-12)


def test_off_axis_xz_covariance_closed_form():
    """Mean at camera-space (x, 0, z) with an x-z covariance term: with t = x/z,
    Sigma'_00 = f^2/z^2 (Sxx - 2 t Sxz + t^2 Szz) + 0.3 (the sign of J's
    third column decides the middle term), Sigma'_11 = f^2/z^2 Syy + 0.3 and
    Sigma'_01 = 0."""
    f, x, z = 100.0, 0.5, 2.0
    Sxx, Syy, Sxz, Szz = (float(np.float32(v)) for v in (0.04, 0.03, 0.01, 0.02))
    p = oracle.render(_one((x, 0.0, z), [Sxx, 0.0, Sxz, Syy, 0.0, Szz]), _cam(f=f), 0.0)["proj"][0]
    t = x / z
    k = f * f / (z * z)
    np.testing.assert_allclose(p["cov"], [k * (Sxx - 2 * t * Sxz + t * t * Szz) + 0.3, 0.0, k * Syy + 0.3],
                               rtol=1e-12, atol=1e-12)
