"""Comparison of the CUDA render with the FP64 oracle (test helper).

FP32 (GPU) and FP64 (oracle) can disagree on a discrete decision whose
decision value sits within rounding of its threshold: a tile-rect edge, a
cull (near plane, alpha_cond >= 1/255), the order of two near-equal depths,
a per-pixel skip (alpha >= 1/255) or stop (T(1-alpha) < 1e-4).  Either
outcome is then correct.  These helpers compare what is unique exactly and
accept a borderline decision only when the GPU result equals the oracle's
result under one of the valid outcomes, computed by the oracle itself.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from oracle import sixdgs_oracle as O

# Rounding margins (FP32 decision value vs FP64): a decision is borderline
# when its FP64 decision value is within these of the threshold.
RECT_TOL_PX = 2e-3          # tile-rect edge (u +- r) vs a tile boundary, pixels
L2_TOL = 4e-4               # 2 ln(255 alpha_cond) (the alpha box's squared scale), absolute
LOG_ALPHA_COND_TOL = 1e-4   # ln(alpha_cond) vs ln(1/255)
NEAR_TOL = 1e-5             # t_z vs znear
DEPTH_REL_TOL = 1e-5        # relative depth gap of two list neighbours
LOG_SKIP_TOL = 5e-4         # ln(alpha) vs ln(1/255), per pixel
LOG_STOP_TOL = 2e-2         # ln(T (1 - alpha)) vs ln(1e-4), per pixel

IMAGE_TOL = 2e-4            # max-abs on [0, 1] colour


def oracle_prep(scene, cam, settings):
    with torch.no_grad():
        return O.prepare_view(O.to_params(scene), scene.sh_degree, cam, settings)


def membership_sets(prep: O.ViewPrep, cam, settings):
    """Per Gaussian: 'certain' rect (member for every valid outcome) and
    'possible' rect (member for some valid outcome)."""
    tx, ty = O.tile_grid(cam, settings)
    e = prep.rect_edges.numpy()
    # where the alpha box sets an extent, its FP32 error follows that of
    # L2 = 2 ln(255 alpha_cond) through d(extent)/d(L2)
    gain = prep.rect_box_gain.numpy() if prep.rect_box_gain is not None else np.zeros((e.shape[0], 2))
    tol = RECT_TOL_PX + L2_TOL * gain
    lim = [tx, tx, ty, ty]
    lo_hi = []
    for k in range(4):
        v = e[:, k]
        f = np.floor(v)
        near_int = np.minimum(v - f, f + 1 - v) * (settings.tile_w if k < 2 else settings.tile_h) < tol[:, k // 2]
        nearest = np.round(v)
        alt = np.where(near_int, np.where(v - f < 0.5, f - 1, f + 1), f)  # the other floor value
        base = f + (1 if k in (1, 3) else 0)
        altv = alt + (1 if k in (1, 3) else 0)
        base = np.clip(base, 0, lim[k])
        altv = np.clip(altv, 0, lim[k])
        lo_hi.append((base, altv, near_int))
    x0, x0a, _ = lo_hi[0]
    x1, x1a, _ = lo_hi[1]
    y0, y0a, _ = lo_hi[2]
    y1, y1a, _ = lo_hi[3]
    cert = np.stack([np.maximum(x0, x0a), np.minimum(x1, x1a), np.maximum(y0, y0a), np.minimum(y1, y1a)], 1)
    poss = np.stack([np.minimum(x0, x0a), np.maximum(x1, x1a), np.minimum(y0, y0a), np.maximum(y1, y1a)], 1)
    near_ok = prep.near_margin.numpy()
    la = prep.alpha_cond_logmargin.numpy()
    sure_vis = (near_ok > NEAR_TOL) & (la > LOG_ALPHA_COND_TOL)
    maybe_vis = (near_ok > -NEAR_TOL) & (la > -LOG_ALPHA_COND_TOL) & np.isfinite(la)
    return cert.astype(np.int64), poss.astype(np.int64), sure_vis, maybe_vis


def tile_membership(cert, poss, sure_vis, maybe_vis, x, y):
    def inside(r):
        return (r[:, 0] <= x) & (x < r[:, 1]) & (r[:, 2] <= y) & (y < r[:, 3])
    certain = np.nonzero(inside(cert) & sure_vis)[0]
    possible = np.nonzero(inside(poss) & maybe_vis)[0]
    return set(certain.tolist()), set(possible.tolist())


def check_tile_list(gpu_ids, certain, possible, depth):
    """GPU list: a valid set (certain <= set <= possible) ordered by depth,
    with near-equal depths in either order and exact ties by id."""
    s = set(gpu_ids.tolist())
    missing = certain - s
    extra = s - possible
    assert not missing, f"GPU list misses {sorted(missing)[:8]}"
    assert not extra, f"GPU list has extra {sorted(extra)[:8]}"
    assert len(s) == len(gpu_ids), "duplicate entries"
    z = depth[gpu_ids]
    for a, b, za, zb in zip(gpu_ids[:-1], gpu_ids[1:], z[:-1], z[1:]):
        if abs(zb - za) <= DEPTH_REL_TOL * abs(za):
            continue
        assert zb > za, f"order {a}->{b} depths {za} {zb}"
    return len(s ^ certain)


def gpu_tile_list(sorted_pairs, ranges, tile_offset, tiles_x, x, y, n):
    gt = tile_offset + y * tiles_x + x
    s, e = int(ranges[gt, 0]), int(ranges[gt, 1])
    return (sorted_pairs[s:e] % n).astype(np.int64)


def pixel_candidates(prep, cam, st, x, y, ids):
    """Nominal block of a tile and, per pixel, the values under each single
    borderline skip/stop flip (NaN where not borderline)."""
    block, _, alpha, T_final, walked = O.render_tile(prep, cam, st, x, y, ids=ids)
    cands = [block.numpy()]
    a = alpha.numpy()
    if a.shape[1] == 0:
        return cands
    h, w = block.shape[1], block.shape[2]
    rgb = prep.rgb.detach().numpy()[np.asarray(ids, dtype=np.int64)]
    skip = a < O.ALPHA_MIN
    keep_a = np.where(skip, 0.0, a)
    prod = np.cumprod(1.0 - keep_a, axis=1)
    n = a.shape[1]
    idx = np.arange(n)[None, :]
    live = idx <= walked.numpy()[:, None]
    with np.errstate(divide="ignore"):
        skip_m = np.abs(np.log(a) - math.log(O.ALPHA_MIN)) < LOG_SKIP_TOL
        stop_m = (~skip) & (np.abs(np.log(prod) - math.log(O.T_MIN)) < LOG_STOP_TOL)
    flags = (skip_m | stop_m) & live
    pix = np.nonzero(flags.any(1))[0]
    for p in pix:
        for i in np.nonzero(flags[p])[0]:
            for kind, m in (("skip", skip_m), ("stop", stop_m)):
                if not m[p, i]:
                    continue
                val = O.blend_pixel_sequential(a[p], rgb, st.bg, flip=(kind, int(i)))
                c = np.full((3, h, w), np.nan)
                c[:, p // w, p % w] = val
                cands.append(c)
    return cands


def tile_variants(nominal, certain, possible, depth):
    """Lists of a tile under each single borderline membership or order flip."""
    out = [list(nominal)]
    for g in sorted(possible - certain):
        if g in nominal:
            out.append([i for i in nominal if i != g])
        else:
            v = list(nominal) + [g]
            v.sort(key=lambda i: (depth[i], i))
            out.append(v)
    for k in range(len(nominal) - 1):
        a, b = nominal[k], nominal[k + 1]
        if abs(depth[b] - depth[a]) <= DEPTH_REL_TOL * abs(depth[a]):
            v = list(nominal)
            v[k], v[k + 1] = b, a
            out.append(v)
    return out


def compare_tile_image(gpu_block, prep, cam, st, x, y, certain, possible):
    """Max over pixels of the smallest |GPU - oracle candidate|."""
    depth = prep.depth.detach().numpy()
    nominal = O.tile_list(prep, x, y).tolist()
    best = None
    for ids in tile_variants(nominal, certain, possible, depth):
        cands = pixel_candidates(prep, cam, st, x, y, np.asarray(ids, dtype=np.int64))
        err = np.full(gpu_block.shape, np.inf)
        for c in cands:
            e = np.abs(gpu_block - c)
            err = np.where(np.isnan(e), err, np.minimum(err, e))
        best = err if best is None else np.minimum(best, err)
    return best


def assert_within(err, bound, what=""):
    """Every |error| strictly below its bound (bound broadcast to err's shape)."""
    err = np.asarray(err, dtype=np.float64)
    bound = np.broadcast_to(np.asarray(bound, dtype=np.float64), err.shape)
    bad = ~(err < bound)
    if bad.any():
        i = np.unravel_index(np.argmax(np.where(bad, err / np.maximum(bound, 1e-300), -np.inf)), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {err.size} above bound; worst at {i}: "
                             f"{err[i]:.3e} vs {bound[i]:.3e}")


def validate_image(img_gpu, ref, prep, cam, st):
    """Whole-image check of a GPU render (3, H, W) against the oracle's
    full image ``ref``: every pixel within IMAGE_TOL, except pixels whose
    value the oracle reproduces (within IMAGE_TOL) under a borderline
    decision flip (tile membership, depth order, skip or stop).  Returns the
    mask (H, W) of those borderline pixels and the largest plain error."""
    img_gpu = np.asarray(img_gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(img_gpu - ref).max(axis=0)
    over = err > IMAGE_TOL
    border = np.zeros_like(over)
    if over.any():
        cert, poss, sure, maybe = membership_sets(prep, cam, st)
        ys, xs = np.nonzero(over)
        for (x, y) in sorted({(int(x) // st.tile_w, int(y) // st.tile_h) for x, y in zip(xs, ys)}):
            certain, possible = tile_membership(cert, poss, sure, maybe, x, y)
            x0, y0 = x * st.tile_w, y * st.tile_h
            block = img_gpu[:, y0:y0 + st.tile_h, x0:x0 + st.tile_w]
            e = compare_tile_image(block, prep, cam, st, x, y, certain, possible).max(axis=0)
            assert_within(e, IMAGE_TOL, f"tile ({x}, {y})")
            border[y0:y0 + st.tile_h, x0:x0 + st.tile_w] |= over[y0:y0 + st.tile_h, x0:x0 + st.tile_w]
    return border, float(err[~over].max()) if (~over).any() else 0.0
