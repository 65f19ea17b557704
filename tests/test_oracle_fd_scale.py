"""Finite-difference pin of the oracle's gradients at the scale of the
training workload: 300,000 coupled 6D Gaussians seen by 8 cameras at
800 x 800 (CPU only).

The oracle's gradients are autograd of its forward definition; the small
scenes of test_oracle_pins.py check them against central differences.  Here
the same check runs on the benchmark's own scene: the lowest-id visible
Gaussians (64 in the default suite, 512 with --runslow), two seeded
parameters each, L = sum_v <G_v, I_v> with seeded dL/dI images G_v that are
non-zero on the tiles those Gaussians touch.  Agreement: |fd - analytic| <=
1e-6 |analytic| + 1e-6 rms(analytic).

Every Gaussian's slice, colour and projection depend on its own parameters
only, so moving one parameter of Gaussian k changes only the tiles whose
lists hold k.  Each stencil re-renders just those tiles (the Gaussians of
their lists prepared as a sub-scene, ids kept in order for the depth
tie-break) at theta + h and theta - h, and differences the two blocks pixel
by pixel before summing against G, so that FP64 rounding of the unchanged
terms cancels.  A stencil whose decisions differ between the two sides (a
tile list, a skip or the walk length of a pixel) is discarded and counted.
"""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import sixdgs_oracle as O

PARAMS_PER_GAUSSIAN = 2
REL = 1e-6


def _planes(scene):
    out = []
    for name, arr in scene.planes().items():
        for i in range(arr.shape[0] if arr.ndim == 2 else 1):
            out.append((name, i if arr.ndim == 2 else None))
    return out


def _render_tiles(scene, ids, k, name, plane, value, cam, st, tiles):
    """Blocks and decision signatures of `tiles` with parameter (name, plane)
    of Gaussian k at `value`; float64 parameters, no float32 rounding."""
    p = O.to_params(scene, idx=ids)
    j = int(np.searchsorted(ids, k))
    with torch.no_grad():
        if plane is None:
            p[name][j] = value
        else:
            p[name][plane, j] = value
        prep = O.prepare_view(p, scene.sh_degree, cam, st)
        out = []
        for (x, y) in tiles:
            block, lst, alpha, _, walked = O.render_tile(prep, cam, st, x, y)
            sig = (tuple(ids[lst].tolist()), (alpha.numpy() < O.ALPHA_MIN).tobytes(), walked.numpy().tobytes())
            out.append((block.numpy(), sig))
    return out


def _check(N_GAUSS):
    w = synth.make_workload(2)
    scene, cams = w.scene, w.cameras
    st = O.Settings(lambda_opa=w.lambda_opa, bg=w.bg)
    base = O.to_params(scene)
    with torch.no_grad():
        preps = [O.prepare_view(base, scene.sh_degree, c, st) for c in cams]
    visible = np.zeros(scene.n, bool)
    for pr in preps:
        visible |= pr.valid.numpy()
    sample = np.nonzero(visible)[0][:N_GAUSS]
    assert len(sample) == N_GAUSS

    # tiles each sampled Gaussian touches, per view, and the union per view
    touched = [{} for _ in cams]
    union = [set() for _ in cams]
    for v, pr in enumerate(preps):
        rect, valid = pr.rect.numpy(), pr.valid.numpy()
        for k in sample:
            if valid[k]:
                x0, x1, y0, y1 = rect[k]
                t = [(x, y) for y in range(y0, y1) for x in range(x0, x1)]
                touched[v][k] = t
                union[v].update(t)
    rng = np.random.default_rng(2024)
    G = []
    for v, cam in enumerate(cams):
        g = np.zeros((3, cam.height, cam.width))
        for (x, y) in union[v]:
            blk = g[:, y * st.tile_h:(y + 1) * st.tile_h, x * st.tile_w:(x + 1) * st.tile_w]
            blk[...] = rng.normal(size=blk.shape)
        G.append(g)
    analytic = O.gradients(scene, cams, G, st, tiles=[sorted(u) for u in union])

    planes = _planes(scene)
    picks = rng.choice(len(planes), size=(N_GAUSS, PARAMS_PER_GAUSSIAN))
    fd, an, discarded = [], [], 0
    for gi, k in enumerate(sample):
        for pi in picks[gi]:
            name, plane = planes[pi]
            arr = np.asarray(getattr(scene, name), dtype=np.float64)
            theta = float(arr[k] if plane is None else arr[plane, k])
            h = 1e-6 * max(1.0, abs(theta))
            total, flipped = 0.0, False
            for v, cam in enumerate(cams):
                if k not in touched[v]:
                    continue
                tiles = touched[v][k]
                ids = set([int(k)])
                for (x, y) in tiles:
                    ids.update(O.tile_list(preps[v], x, y).tolist())
                ids = np.array(sorted(ids), dtype=np.int64)
                plus = _render_tiles(scene, ids, k, name, plane, theta + h, cam, st, tiles)
                minus = _render_tiles(scene, ids, k, name, plane, theta - h, cam, st, tiles)
                for (x, y), (bp, sp), (bm, sm) in zip(tiles, plus, minus):
                    if sp != sm:
                        flipped = True
                        break
                    gblk = G[v][:, y * st.tile_h:y * st.tile_h + bp.shape[1], x * st.tile_w:x * st.tile_w + bp.shape[2]]
                    total += float((gblk * (bp - bm)).sum())
                if flipped:
                    break
            if flipped:
                discarded += 1
                continue
            fd.append(total / (2.0 * h))
            an.append(float(analytic[name][k] if plane is None else analytic[name][plane, k]))
    fd, an = np.array(fd), np.array(an)
    assert discarded <= 0.02 * N_GAUSS * PARAMS_PER_GAUSSIAN, discarded
    scale = math.sqrt(float(np.mean(an ** 2)))
    err = np.abs(fd - an)
    bound = REL * np.abs(an) + REL * scale
    worst = int(np.argmax(err / bound))
    print(f"{len(fd)} stencils, {discarded} discarded; worst |fd - an| {err[worst]:.3e} vs bound {bound[worst]:.3e}; "
          f"median relative {np.median(err / np.maximum(np.abs(an), 1e-300)):.2e}")
    assert np.all(err <= bound), (worst, fd[worst], an[worst])


def test_finite_differences_on_the_300k_eight_view_workload_64_gaussians():
    """The 64 lowest-id visible Gaussians (part of the default CPU suite)."""
    _check(64)


@pytest.mark.slow
def test_finite_differences_on_the_300k_eight_view_workload_512_gaussians():
    """The 512 lowest-id visible Gaussians (about 6 minutes on 8 cores; run
    with --runslow)."""
    _check(512)
