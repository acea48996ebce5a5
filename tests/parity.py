"""Comparison helpers for the GPU-vs-oracle parity tests (not a test module).

Bars (spec tolerances): the cut bit-exact; images within 2e-3 max-abs
per channel on every pixel, and PSNR >= 55 dB over all pixels.  The oracle's
flag (pixels where an FP32 renderer may take the other side of an alpha*
decision) is only reported, unless a test passes ``flip_allow`` explicitly.
The pair set must equal the oracle's except within the FP32 test slack: every
extra GPU pair has an oracle margin (rho_max - threshold) in
[-(slack + delta), 0) and every missing oracle pair a margin below delta.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

IMG_TOL = 2e-3
PSNR_MIN = 55.0
TILE_SLACK = 2e-3      # the renderer's FP32 tile-test slack (nats)
MARGIN_DELTA = 2e-3    # FP32-vs-FP64 error allowance on rho_max (nats)
FP32_U = 2.0 ** -24    # unit roundoff of FP32
# Conic bound: the FP32 EWA (Sigma' = J R Sigma R^T J^T + 0.3 I, a few dozen
# single-rounded operations) perturbs Sigma' by ~c u ||Sigma'||, and inverting
# amplifies that by the condition number: ||d conic|| / ||conic|| <~ c u kappa(Sigma').
# A float32 emulation of the kernel's arithmetic on the 1M-leaf box gives
# max |d conic| / max(|a|, |c|) = 9.1 u kappa (median 0.7); 64 u kappa leaves 7x.
CONIC_K = 64.0


def cond2(cov3: np.ndarray) -> np.ndarray:
    """Condition number lambda_max / lambda_min of 2x2 symmetric (00, 01, 11) matrices."""
    cov3 = np.asarray(cov3, np.float64).reshape(-1, 3)
    half_tr = 0.5 * (cov3[:, 0] + cov3[:, 2])
    disc = np.sqrt(0.25 * (cov3[:, 0] - cov3[:, 2]) ** 2 + cov3[:, 1] ** 2)
    return (half_tr + disc) / (half_tr - disc)


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((a.astype(np.float64) - b) ** 2))
    return math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)


def image_report(img: np.ndarray, ref: dict, tile_mask=None) -> dict:
    H, W = ref["image"].shape[:2]
    sel = np.ones((H, W), bool)
    if tile_mask is not None:
        T = int(ref.get("tile", 16))
        TW = (W + T - 1) // T
        ty, tx = np.mgrid[0:H, 0:W]
        sel = np.asarray(tile_mask).reshape(-1)[(ty // T) * TW + tx // T]
    ok = sel & (ref["flags"] == 0)
    diff = np.abs(img.astype(np.float64) - ref["image"])
    flagged = sel & (ref["flags"] != 0)
    return dict(max_abs=float(diff[ok].max()) if ok.any() else 0.0,
                psnr=psnr(img[sel], ref["image"][sel]),
                flagged=int(flagged.sum()), pixels=int(sel.sum()),
                flagged_over_tol=int((flagged & (diff.max(axis=2) > IMG_TOL)).sum()),
                max_abs_all=float(diff[sel].max()) if sel.any() else 0.0)


FLIP_BOUND = 1e-2  # a flipped alpha* decision moves a pixel by at most ~2 alpha* max(rgb)


def check_image(img, ref, tile_mask=None, tol=IMG_TOL, psnr_min=PSNR_MIN, flip_allow=0.0):
    """Every pixel within ``tol`` (2e-3 per channel) of the FP64 oracle and
    PSNR >= ``psnr_min`` over all pixels.  The oracle's flagged pixels (some
    Gaussian within 2e-3 nats of the alpha* threshold while T >= 0.05) are
    counted and returned, not excused.  A test that needs the allowance for
    flipped alpha* decisions passes ``flip_allow`` (a fraction of the pixels,
    at most 1 %): then up to that many flagged pixels may err beyond ``tol``,
    each within FLIP_BOUND."""
    assert 0.0 <= flip_allow <= 0.01, flip_allow
    r = image_report(img, ref, tile_mask)
    if flip_allow > 0.0:
        assert r["max_abs"] <= tol, r
        assert r["max_abs_all"] <= FLIP_BOUND, r
        assert r["flagged_over_tol"] <= flip_allow * r["pixels"], r
    else:
        assert r["max_abs_all"] <= tol, r
    assert r["psnr"] >= psnr_min, r
    return r


def pair_margin(ref: dict, tile: int, node: int) -> float:
    """Oracle margin rho_max - (ln alpha* - ln theta) of (tile, node) in FP64,
    for any pair (also outside the oracle's candidate rectangle)."""
    cut = ref["cut"]
    g = int(np.searchsorted(cut, node))
    assert cut[g] == node
    p = ref["proj"][g]
    H, W = ref["image"].shape[:2]
    T = int(ref.get("tile", 16))
    TW = (W + T - 1) // T
    tx, ty = tile % TW, tile // TW
    x0, y0 = T * tx + 0.5, T * ty + 0.5
    x1, y1 = min(T * tx + T - 0.5, W - 0.5), min(T * ty + T - 0.5, H - 0.5)
    return oracle.rho_max_rect(p["conic"], p["u"], p["v"], x0, x1, y0, y1) - p["thr"]


def _pairkey(tile, node):
    return (np.asarray(tile, np.int64) << 32) | np.asarray(node, np.int64)


def _rows_needed(A, B, tile, TW, T=16, chunk=8192):
    """Bit w set when some pixel of the pair's tile in rows w r .. w r + r - 1
    (r = max(1, T / 8) rows per bit) has rho >= thr - 1e-3 (FP64, from the
    pair's FP32 record)."""
    out = np.zeros(len(tile), np.int64)
    cT = np.arange(T, dtype=np.float64) + 0.5
    mr = max(1, T // 8)
    for s0 in range(0, len(tile), chunk):
        sl = slice(s0, s0 + chunk)
        t = tile[sl]
        a, b, c = (A[sl, 2].astype(np.float64), A[sl, 3].astype(np.float64), B[sl, 0].astype(np.float64))
        dx = A[sl, 0].astype(np.float64)[:, None] - ((t % TW) * T)[:, None] - cT[None, :]   # [P, col]
        dy = A[sl, 1].astype(np.float64)[:, None] - ((t // TW) * T)[:, None] - cT[None, :]  # [P, row]
        rho = (a[:, None, None] * dx[:, None, :] ** 2 + b[:, None, None] * dx[:, None, :] * dy[:, :, None]
               + c[:, None, None] * dy[:, :, None] ** 2)                                     # [P, row, col]
        rows = (rho >= B[sl, 1].astype(np.float64)[:, None, None] - 1e-3).any(axis=2)       # [P, row]
        groups = rows.reshape(len(t), T // mr, mr).any(axis=2)
        out[sl] = (groups * (1 << np.arange(T // mr))).sum(axis=1)
    return out


def check_stages(dbg: dict, ref: dict, tile_mask=None, theta_rtol: float = 0.0) -> dict:
    """Stage-by-stage parity of one frame.  With tile_mask, pair checks are
    restricted to the masked tiles (the oracle binned only those).  The
    opacity is the stored FP32 value, passed through exactly, unless the
    Gaussians are interpolated (then it is computed: theta_rtol > 0)."""
    cut = ref["cut"]
    np.testing.assert_array_equal(dbg["cut"], cut)
    assert int(dbg.get("tile_size", 16)) == int(ref.get("tile", 16)), "renderer and oracle tile sizes differ"
    proj = ref["proj"]
    # per-cut-index best candidate margin
    best = np.full(len(cut), -np.inf)
    if len(ref["cand_idx"]):
        np.maximum.at(best, ref["cand_idx"], ref["cand_margin"])
    # ---- visible set, in ascending node order
    gv = dbg["vis_node"]
    assert np.all(np.diff(gv.astype(np.int64)) > 0), "visible list not in ascending node order"
    idx = np.searchsorted(cut, gv)
    assert np.all(cut[np.minimum(idx, len(cut) - 1)] == gv), "visible node not in the cut"
    if tile_mask is None:
        ov = cut[proj["visible"] == 1]
        extra = np.setdiff1d(gv, ov)
        missing = np.setdiff1d(ov, gv)
        if len(extra):
            # every pair of such a Gaussian is a slack-band extra; the pair
            # check below bounds each one's oracle margin
            be = best[np.searchsorted(cut, extra)]
            assert np.all(be < 0), be
        if len(missing):
            bm = best[np.searchsorted(cut, missing)]
            assert np.all(bm < MARGIN_DELTA), bm
    # ---- depth keys: the FP32 formula, bit-exact
    zk = proj["zkey"][idx].view(np.uint32)
    np.testing.assert_array_equal(dbg["vis_depth"], zk)
    # ---- records against the FP64 projection
    p = proj[idx]
    A, B = dbg["vis_recA"], dbg["vis_recB"]
    H, W = ref["image"].shape[:2]
    for j, key, half in ((0, "u", W / 2.0), (1, "v", H / 2.0)):
        # u = fx x/z + cx: the FP32 error scales with the larger of the two terms
        err = np.abs(A[:, j] - p[key]) / np.maximum(np.maximum(1.0, half), np.abs(p[key]))
        w = np.argsort(err)[-4:]
        assert err.max() < 2e-5, (key, err[w], A[w, j], p[key][w], p["z"][w], p["cov"][w])
    con = np.stack([-2.0 * A[:, 2], -A[:, 3], -2.0 * B[:, 0]], 1)
    cref = p["conic"]
    cs = np.maximum(np.abs(cref[:, 0]), np.abs(cref[:, 2]))
    rel = np.max(np.abs(con - cref), axis=1) / cs
    kappa = cond2(p["cov"])
    bound = CONIC_K * FP32_U * kappa
    worst = int(np.argmax(rel / bound)) if len(rel) else 0
    assert np.all(rel <= bound), (float(rel[worst]), float(kappa[worst]), float((rel / (FP32_U * kappa)).max()))
    rgb = dbg["vis_rgb"][:, :3]
    assert np.max(np.abs(rgb - p["rgb"])) < 2e-5
    if theta_rtol > 0:
        np.testing.assert_allclose(B[:, 2], p["theta"], rtol=theta_rtol, atol=0)
    else:
        np.testing.assert_array_equal(B[:, 2], p["theta"].astype(np.float32))
    assert np.max(np.abs(B[:, 1] - p["thr"])) < 1e-5
    # ---- depth order: sorted by (depth key, node id)
    order = dbg["depth_order"]
    assert np.array_equal(np.sort(order), np.arange(len(gv)))
    zs, ns = dbg["vis_depth"][order], gv[order]
    ok = (zs[1:] > zs[:-1]) | ((zs[1:] == zs[:-1]) & (ns[1:] > ns[:-1]))
    assert np.all(ok), "depth order not (key, node) ascending"
    # ---- pairs: sorted by tile, depth rank ascending within a tile
    pt, pr = dbg["pair_tile"].astype(np.int64), dbg["pair_rank"].astype(np.int64)
    assert np.all(np.diff(pt) >= 0)
    same = pt[1:] == pt[:-1]
    assert np.all(pr[1:][same] > pr[:-1][same])
    rng = dbg["tile_range"]
    starts = np.flatnonzero(np.r_[True, pt[1:] != pt[:-1]]) if len(pt) else np.zeros(0, np.int64)
    for s0 in starts[:: max(1, len(starts) // 200)]:
        t = pt[s0]
        assert rng[t, 0] == s0 and np.all(pt[rng[t, 0]:rng[t, 1]] == t)
    gnode = gv[order[pr]] if len(pr) else np.zeros(0, np.int64)
    gkeys = _pairkey(pt, gnode)
    okeys = _pairkey(ref["pair_tile"], cut[ref["pair_idx"]])
    ckeys = _pairkey(ref["cand_tile"], cut[ref["cand_idx"]])
    if tile_mask is not None:
        m = np.asarray(tile_mask).reshape(-1)
        gkeys = gkeys[m[pt]]
    extra = np.setdiff1d(gkeys, okeys)
    missing = np.setdiff1d(okeys, gkeys)
    if len(extra):
        em = np.array([pair_margin(ref, int(k) >> 32, int(k) & 0xFFFFFFFF) for k in extra])
        assert np.all(em >= -(TILE_SLACK + MARGIN_DELTA)) and np.all(em < 0), (em.min(), em.max())
    if len(missing):
        marg = dict(zip(ckeys.tolist(), ref["cand_margin"].tolist()))
        mm = np.array([marg[int(k)] for k in missing])
        assert np.all(mm < MARGIN_DELTA), mm.max()
    # ---- row masks: a pair's bit w must be set wherever some pixel of the
    # tile's rows 2w, 2w+1 passes the Eq. 4 test (or misses it by < 1e-3)
    # with the pair's own record; otherwise the blend would skip a pixel
    # the Gaussian contributes to
    if "pair_rowmask" in dbg and len(pr):
        TW = int(dbg["tiles"][0])
        vis = order[pr]
        need = _rows_needed(A[vis], B[vis], pt, TW, int(dbg.get("tile_size", 16)))
        got = dbg["pair_rowmask"].astype(np.int64)
        bad = (got & need) != need
        assert not bad.any(), (int(bad.sum()), got[bad][:5], need[bad][:5])
    # ---- per-tile order of the common pairs equals the oracle's
    common = np.intersect1d(gkeys, okeys)
    g_common = gkeys[np.isin(gkeys, common)]
    o_common = okeys[np.isin(okeys, common)]
    np.testing.assert_array_equal(g_common, o_common)
    return dict(extra_pairs=int(len(extra)), missing_pairs=int(len(missing)), pairs=int(len(gkeys)))


def quantize_scene(sc: dict) -> dict:
    """The scene as the reduced-precision store holds it: SH rounded to FP16
    and covariances to BF16 (round to nearest even), back in FP32."""
    q = dict(sc)
    q["sh"] = sc["sh"].astype(np.float16).astype(np.float32)
    b = sc["cov6"].astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    q["cov6"] = (((b + r) & 0xFFFF0000) & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return q


def oracle_render(sc, cam, tau, **kw):
    return oracle.render(sc, cam, tau, **kw)
