"""GPU forward parity: CUDA render vs the FP64 oracle, element by element."""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import sixdgs_oracle as O
from tests import parity as PT

pytestmark = pytest.mark.gpu

sx = pytest.importorskip("paper_2410_04974_gb300")


def _settings(w, tile=(16, 16), lam=0.35, bg=(1.0, 1.0, 1.0)):
    return O.Settings(tile_w=tile[0], tile_h=tile[1], lambda_opa=lam, bg=bg)


def _render(scene, cams, tile=(16, 16), batch=256, lam=0.35, bg=(1.0, 1.0, 1.0), store_aux=False,
            persistent=False):
    r = sx.Renderer(scene.n, scene.sh_degree, cams, tile=tile, batch=batch, lambda_opa=lam, bg=bg,
                    store_aux=store_aux, persistent=persistent)
    params = sx.params_to_device(scene)
    img = r.forward(params)
    torch.cuda.synchronize()
    return r, params, img


def _check_records(r, scene, cams, st, view):
    """Per (view, Gaussian) record vs the oracle's slice/colour/projection."""
    prep = PT.oracle_prep(scene, cams[view], st)
    n = scene.n
    rec = r.records()[view * n:(view + 1) * n].cpu().numpy().astype(np.float64)
    nt = r.ntiles()[view * n:(view + 1) * n].cpu().numpy()
    cert, poss, sure, maybe = PT.membership_sets(prep, cams[view], st)
    gvis = nt > 0
    certain_vis = sure & (cert[:, 0] < cert[:, 1]) & (cert[:, 2] < cert[:, 3])
    possible_vis = maybe & (poss[:, 0] < poss[:, 1]) & (poss[:, 2] < poss[:, 3])
    assert np.all(gvis[certain_vis]), np.nonzero(certain_vis & ~gvis)[0][:10]
    assert not np.any(gvis & ~possible_vis), np.nonzero(gvis & ~possible_vis)[0][:10]
    both = gvis & prep.valid.numpy()
    assert both.sum() > 0
    o = {k: v.detach().numpy() for k, v in dict(mean=prep.mean2d, conic=prep.conic, ac=prep.alpha_cond,
                                                rgb=prep.rgb, depth=prep.depth, radius=prep.radius).items()}
    lg = -0.5 * math.log2(math.e)
    np.testing.assert_allclose(rec[both, 0], o["mean"][both, 0], rtol=1e-5, atol=2e-3)
    np.testing.assert_allclose(rec[both, 1], o["mean"][both, 1], rtol=1e-5, atol=2e-3)
    np.testing.assert_allclose(rec[both, 2] / lg, o["conic"][both, 0], rtol=2e-4, atol=1e-7)
    np.testing.assert_allclose(rec[both, 3] / (2 * lg), o["conic"][both, 1], rtol=2e-4,
                               atol=2e-4 * np.abs(o["conic"][both, 0]).max())
    np.testing.assert_allclose(rec[both, 4] / lg, o["conic"][both, 2], rtol=2e-4, atol=1e-7)
    np.testing.assert_allclose(rec[both, 5], np.log2(o["ac"][both]), atol=2e-4)
    np.testing.assert_allclose(rec[both, 6:8], o["rgb"][both, :2], atol=2e-6)
    np.testing.assert_allclose(rec[both, 8], o["rgb"][both, 2], atol=2e-6)
    np.testing.assert_allclose(rec[both, 11], o["depth"][both], rtol=2e-6)
    # (hx, hy): box of the alpha >= 1/255 ellipse, never smaller than the exact one
    con = o["conic"][both]
    det = con[:, 0] * con[:, 2] - con[:, 1] ** 2
    L2 = 2.0 * np.log(255.0 * o["ac"][both])
    hx_exact = np.sqrt(L2 * con[:, 2] / det)
    hy_exact = np.sqrt(L2 * con[:, 0] / det)
    assert np.all(rec[both, 9] >= hx_exact) and np.all(rec[both, 10] >= hy_exact)
    assert np.all(rec[both, 9] <= 1.001 * hx_exact + 0.02) and np.all(rec[both, 10] <= 1.001 * hy_exact + 0.02)
    return prep, (cert, poss, sure, maybe)


def _check_tiles(r, scene, cams, st, view, tiles, prep, member, img_gpu):
    cert, poss, sure, maybe = member
    sorted_pairs = r.sorted_pairs().cpu().numpy().astype(np.int64)
    ranges = r.ranges().cpu().numpy().astype(np.int64)
    toff = r.tile_offsets()[view]
    tiles_x, _ = O.tile_grid(cams[view], st)
    depth = prep.depth.detach().numpy()
    worst = 0.0
    flips = 0
    for (x, y) in tiles:
        ids = PT.gpu_tile_list(sorted_pairs, ranges, toff, tiles_x, x, y, scene.n)
        # every listed entry belongs to this view
        gt = toff + y * tiles_x + x
        s, e = ranges[gt]
        assert np.all(sorted_pairs[s:e] // scene.n == view)
        certain, possible = PT.tile_membership(cert, poss, sure, maybe, x, y)
        flips += PT.check_tile_list(ids, certain, possible, depth)
        x0, y0 = x * st.tile_w, y * st.tile_h
        block = img_gpu[:, y0:y0 + st.tile_h, x0:x0 + st.tile_w].astype(np.float64)
        err = PT.compare_tile_image(block, prep, cams[view], st, x, y, certain, possible)
        worst = max(worst, float(err.max()))
        assert err.max() <= PT.IMAGE_TOL, (x, y, float(err.max()), np.unravel_index(err.argmax(), err.shape))
    return worst, flips


def _all_tiles(cam, st):
    tx, ty = O.tile_grid(cam, st)
    return [(x, y) for y in range(ty) for x in range(tx)]


def _sample_tiles(cam, st, k, seed):
    tx, ty = O.tile_grid(cam, st)
    rng = np.random.default_rng(seed)
    pick = {(tx // 2, ty // 2), (0, 0), (tx - 1, ty - 1)}
    while len(pick) < k:
        pick.add((int(rng.integers(0, tx)), int(rng.integers(0, ty))))
    return sorted(pick)


@pytest.mark.parametrize("persistent", [False, True])
def test_small_cube_scene_matches_oracle_everywhere(persistent):
    w = synth.make_workload(0)
    st = _settings(w)
    r, params, img = _render(w.scene, w.cameras, persistent=persistent)
    assert int(r.status.item()) == 0
    prep, member = _check_records(r, w.scene, w.cameras, st, 0)
    counts = r.counts()
    assert counts[0] == int((r.ntiles().cpu().numpy() > 0).sum())
    worst, flips = _check_tiles(r, w.scene, w.cameras, st, 0, _all_tiles(w.cameras[0], st), prep, member,
                                img.cpu().numpy().reshape(3, 128, 128))
    print(f"worst pixel error {worst:.2e}, borderline membership flips {flips}")


@pytest.mark.parametrize("size,tile,batch,persistent", [((100, 70), (16, 16), 256, False),
                                                        ((72, 40), (8, 8), 32, True),
                                                        ((130, 50), (32, 16), 128, False),
                                                        ((64, 64), (16, 8), 64, True),
                                                        ((90, 120), (8, 16), 1024, False)])
def test_ragged_images_and_tile_shapes(size, tile, batch, persistent):
    scene = synth.scene_cube(1500, 31)
    scene.l_raw[:3] += math.log(2.0)
    cams = [synth.look_at_camera((4.0, 0.5, -0.3), size[0], size[1])]
    st = _settings(None, tile=tile, bg=(0.1, 0.5, 0.9))
    r, params, img = _render(scene, cams, tile=tile, batch=batch, bg=(0.1, 0.5, 0.9), persistent=persistent)
    assert int(r.status.item()) == 0
    prep, member = _check_records(r, scene, cams, st, 0)
    _check_tiles(r, scene, cams, st, 0, _all_tiles(cams[0], st), prep, member,
                 img.cpu().numpy().reshape(3, size[1], size[0]))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_lower_sh_degrees(deg):
    scene = synth.scene_cube(800, 40 + deg, sh_degree=deg)
    cams = [synth.look_at_camera((0.0, 4.0, 1.0), 96, 80)]
    st = _settings(None)
    r, params, img = _render(scene, cams)
    prep, member = _check_records(r, scene, cams, st, 0)
    _check_tiles(r, scene, cams, st, 0, _all_tiles(cams[0], st), prep, member, img.cpu().numpy().reshape(3, 80, 96))


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_lambda_extremes(lam):
    scene = synth.scene_shell(3000, 50, dp_sigma=0.1)
    scene.l_raw[:3] += math.log(4.0)
    cams = [synth.look_at_camera((4.0, 0.0, 0.0), 64, 64)]
    st = _settings(None, lam=lam)
    r, params, img = _render(scene, cams, lam=lam)
    prep, member = _check_records(r, scene, cams, st, 0)
    _check_tiles(r, scene, cams, st, 0, _all_tiles(cams[0], st), prep, member, img.cpu().numpy().reshape(3, 64, 64))


def test_empty_and_fully_culled_scenes_give_background():
    cams = [synth.look_at_camera((4.0, 0.0, 0.0), 40, 24)]
    bg = (0.25, 0.5, 0.75)
    empty = synth.scene_cube(0, 1)
    r, _, img = _render(empty, cams, bg=bg)
    assert int(r.status.item()) == 0
    np.testing.assert_array_equal(img.cpu().numpy().reshape(3, 24, 40), np.broadcast_to(np.array(bg, np.float32)[:, None, None], (3, 24, 40)))
    # every Gaussian behind the camera
    behind = synth.scene_cube(500, 2)
    behind.mu_p[0] = 10.0
    r, _, img = _render(behind, cams, bg=bg)
    assert r.counts()[0] == 0 and r.counts()[1] == 0
    np.testing.assert_array_equal(img.cpu().numpy().reshape(3, 24, 40), np.broadcast_to(np.array(bg, np.float32)[:, None, None], (3, 24, 40)))


def test_single_gaussian_footprint_on_gpu():
    scene = synth.scene_cube(1, 0, sh_degree=0)
    scene.mu_p[:, 0] = (0.0, 0.0, 0.0)
    scene.mu_d[:, 0] = (-1.0, 0.0, 0.0)
    scene.l_raw[:] = 0.0
    scene.l_raw[:3, 0] = math.log(0.03)
    scene.l_raw[3:6, 0] = math.log(0.3)
    scene.opacity_logit[0] = 1.5
    scene.sh[:, 0] = 0.4
    cams = [synth.look_at_camera((4.0, 0.0, 0.0), 64, 64)]
    st = _settings(None)
    r, _, img = _render(scene, cams)
    ref, _ = O.render_view(scene, cams[0], st)
    np.testing.assert_allclose(img.cpu().numpy().reshape(3, 64, 64), ref.numpy(), atol=1e-6)


def test_shell_200k_800sq_sampled_tiles():
    w = synth.make_workload(1)
    st = _settings(w)
    r, params, img = _render(w.scene, w.cameras)
    assert int(r.status.item()) == 0
    prep, member = _check_records(r, w.scene, w.cameras, st, 0)
    tiles = _sample_tiles(w.cameras[0], st, 24, 5)
    worst, flips = _check_tiles(r, w.scene, w.cameras, st, 0, tiles, prep, member,
                                img.cpu().numpy().reshape(3, 800, 800))
    print(f"worst pixel error {worst:.2e}, borderline membership flips {flips}")


def test_coupled_300k_eight_views_sampled_tiles():
    w = synth.make_workload(2)
    st = _settings(w)
    r, params, img = _render(w.scene, w.cameras)
    assert int(r.status.item()) == 0
    views = r.split(img)
    for v in (0, 3, 6):
        prep, member = _check_records(r, w.scene, w.cameras, st, v)
        tiles = _sample_tiles(w.cameras[v], st, 10, 100 + v)
        _check_tiles(r, w.scene, w.cameras, st, v, tiles, prep, member, views[v].cpu().numpy())


def test_mixed_resolution_batch():
    w = synth.make_workload(3, n_override=20_000)
    cams = w.cameras[:12]
    st = _settings(w)
    r, params, img = _render(w.scene, cams)
    assert int(r.status.item()) == 0
    views = r.split(img)
    for v in (0, 5, 11):
        prep, member = _check_records(r, w.scene, cams, st, v)
        tiles = _sample_tiles(cams[v], st, 8, 200 + v)
        _check_tiles(r, w.scene, cams, st, v, tiles, prep, member, views[v].cpu().numpy())


def test_store_aux_does_not_change_the_image():
    w = synth.make_workload(0)
    _, _, a = _render(w.scene, w.cameras, store_aux=False)
    r, _, b = _render(w.scene, w.cameras, store_aux=True)
    torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_plain_three_sigma_footprint_and_equal_images():
    """alpha_footprint=0 (the 3-sigma square of the 3DGS rasteriser) against
    the oracle's same rule, and the default alpha-aware footprint gives the
    same image bit for bit with fewer duplicates."""
    w = synth.make_workload(0)
    st = O.Settings(alpha_footprint=0)
    params = sx.params_to_device(w.scene)
    r0 = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, alpha_footprint=False)
    img0 = r0.forward(params)
    r1 = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras)
    img1 = r1.forward(params)
    torch.cuda.synchronize()
    assert int(r0.status.item()) == 0 and int(r1.status.item()) == 0
    prep, member = _check_records(r0, w.scene, w.cameras, st, 0)
    _check_tiles(r0, w.scene, w.cameras, st, 0, _all_tiles(w.cameras[0], st), prep, member,
                 img0.cpu().numpy().reshape(3, 128, 128))
    assert torch.equal(img0, img1)
    k0, k1 = int(r0.counts()[1]), int(r1.counts()[1])
    assert k1 < 0.85 * k0, (k0, k1)


def test_plane_length_not_a_multiple_of_four():
    """4,099 Gaussians: the parameter planes cannot be staged with 16-byte
    bulk copies, so the projection loads them with plain loads; records,
    lists and images still match the oracle, and the per-Gaussian lambda and
    the cached slice state take the same path."""
    scene = synth.with_learnable_lambda(synth.scene_cube(4099, 77), 3)
    cams = [synth.look_at_camera((4.0, 0.5, 0.2), 96, 72), synth.look_at_camera((-1.0, 3.8, 0.5), 64, 80)]
    st = _settings(None)
    r, params, img = _render(scene, cams)
    assert int(r.status.item()) == 0
    views = r.split(img)
    for v in range(2):
        prep, member = _check_records(r, scene, cams, st, v)
        _check_tiles(r, scene, cams, st, v, _all_tiles(cams[v], st), prep, member, views[v].cpu().numpy())
    params["cond_cache"] = sx.condition_cache(params)
    img_c = r.forward(params)
    torch.cuda.synchronize()
    assert torch.equal(img_c, img)
