"""GPU backward parity: hand-written gradients vs autograd of the FP64 oracle."""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import sixdgs_oracle as O
from tests import parity as PT

pytestmark = pytest.mark.gpu

sx = pytest.importorskip("paper_2410_04974_gb300")

GROUPS = ("mu_p", "mu_d", "l_raw", "opacity_logit", "sh")
REL_L2 = 1e-3        # per parameter group, ||g - g_ref|| / ||g_ref||
ELEM_REL = 1e-3      # per element: |g - g_ref| <= ELEM_REL |g_ref| + ELEM_FLOOR rms(g_ref)
ELEM_FLOOR = 1e-3


def _compare(gpu, ref, tag, max_outliers=0.0, groups=GROUPS):
    report = {}
    for k in groups:
        g = gpu[k].astype(np.float64)
        r = ref[k]
        norm = np.linalg.norm(r)
        assert norm > 0, (tag, k)
        rel = np.linalg.norm(g - r) / norm
        rms = norm / math.sqrt(r.size)
        bad = np.abs(g - r) > ELEM_REL * np.abs(r) + ELEM_FLOOR * rms
        report[k] = (rel, int(bad.sum()))
        assert rel <= REL_L2, (tag, k, rel)
        assert bad.sum() <= max_outliers * r.size, (tag, k, int(bad.sum()), np.argwhere(bad)[:5])
    print(tag, {k: (f"{v[0]:.1e}", v[1]) for k, v in report.items()})
    return report


def _gpu_grads(scene, cams, g_imgs, tile=(16, 16), store_aux=False, lam=0.35, persistent=False):
    r = sx.Renderer(scene.n, scene.sh_degree, cams, tile=tile, store_aux=store_aux, lambda_opa=lam,
                    persistent=persistent)
    params = sx.params_to_device(scene)
    img = r.forward(params)
    g = r.backward(params, img, r.pack(g_imgs))
    torch.cuda.synchronize()
    r.raise_status()
    return {k: v.cpu().numpy() for k, v in g.items()}, r


@pytest.mark.parametrize("store_aux", [False, True])
def test_small_cube_scene_gradients(store_aux):
    w = synth.make_workload(0)
    g_imgs = synth.random_grad_images(w.cameras, 7)
    gpu, _ = _gpu_grads(w.scene, w.cameras, g_imgs, store_aux=store_aux)
    ref = O.gradients(w.scene, w.cameras, g_imgs, O.Settings())
    _compare(gpu, ref, f"cube4k store_aux={store_aux}", max_outliers=2e-3)


def test_multi_view_ragged_gradients_sum_over_views():
    scene = synth.scene_shell(2000, 61, dp_sigma=0.1)
    scene.l_raw[:3] += math.log(3.0)
    cams = [synth.look_at_camera((4.0, 0.0, 0.5), 72, 56), synth.look_at_camera((0.0, -4.0, 0.0), 40, 88),
            synth.look_at_camera((-2.5, 2.5, 1.5), 64, 64)]
    g_imgs = synth.random_grad_images(cams, 8)
    gpu, _ = _gpu_grads(scene, cams, g_imgs, tile=(8, 16), persistent=True)
    ref = O.gradients(scene, cams, g_imgs, O.Settings(tile_w=8, tile_h=16))
    _compare(gpu, ref, "shell2k 3 views", max_outliers=2e-3)


def test_coupled_300k_gradients_on_sampled_tiles():
    """Full-size scene and ring of 8 views; dL/dI is non-zero on a few tiles
    per view only, so the oracle needs just the Gaussians listed there."""
    w = synth.make_workload(2)
    st = O.Settings()
    rng = np.random.default_rng(9)
    g_imgs, tiles = [], []
    for v, cam in enumerate(w.cameras):
        g = np.zeros((3, cam.height, cam.width), np.float32)
        pick = [(25, 25), (int(rng.integers(15, 35)), int(rng.integers(15, 35))),
                (int(rng.integers(0, 50)), int(rng.integers(0, 50)))]
        for (x, y) in pick:
            g[:, y * 16:(y + 1) * 16, x * 16:(x + 1) * 16] = rng.normal(size=(3, 16, 16))
        g_imgs.append(g)
        tiles.append(pick)
    gpu, _ = _gpu_grads(w.scene, w.cameras, g_imgs)
    ref = O.gradients(w.scene, w.cameras, g_imgs, st, tiles=tiles)
    touched = np.any(ref["sh"] != 0, axis=0)
    assert touched.sum() > 100
    sub = {k: v[..., touched] for k, v in ref.items()}
    gsub = {k: v[..., touched] for k, v in gpu.items()}
    _compare(gsub, sub, "coupled300k sampled", max_outliers=2e-3)
    # Gaussians on none of the sampled tiles get exactly zero gradient
    for k in GROUPS:
        assert np.all(gpu[k][..., ~touched] == 0.0), k


def test_autograd_function_matches_direct_call():
    w = synth.make_workload(0)
    r = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras)
    params = sx.params_to_device(w.scene)
    leaves = {k: v.clone().requires_grad_(True) for k, v in params.items()}
    img = sx.render(r, leaves)
    target = torch.rand_like(img)
    loss = (img - target).abs().mean()
    loss.backward()
    g_img = torch.sign(img.detach() - target) / img.numel()
    r2 = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras)
    img2 = r2.forward(params)
    direct = r2.backward(params, img2, g_img)
    for k in GROUPS:
        torch.testing.assert_close(leaves[k].grad, direct[k], rtol=1e-4, atol=1e-9)


def test_learnable_lambda_forward_and_gradients():
    """Per-Gaussian lambda_opa = sigmoid(raw) (section 4.2): every pixel of
    the images (borderline decisions validated by the oracle) and every
    gradient element, lambda_raw included."""
    scene = synth.with_learnable_lambda(synth.scene_shell(3000, 71, dp_sigma=0.1), 5, spread=1.0)
    scene.l_raw[:3] += math.log(3.0)
    cams = [synth.look_at_camera((4.0, 0.0, 0.5), 64, 56), synth.look_at_camera((0.0, -4.0, 0.0), 48, 64)]
    st = O.Settings()
    g_imgs = synth.random_grad_images(cams, 9)
    r = sx.Renderer(scene.n, scene.sh_degree, cams, lambda_opa=0.9)   # global value unused
    params = sx.params_to_device(scene)
    img = r.forward(params)
    torch.cuda.synchronize()
    for cam, im in zip(cams, r.split(img)):
        ref, prep = O.render_view(scene, cam, st)
        PT.validate_image(im.cpu().numpy(), ref.numpy(), prep, cam, st)
    g = r.backward(params, img, r.pack(g_imgs))
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in g.items()}
    assert "lambda_raw" in gpu
    ref = O.gradients(scene, cams, g_imgs, st)
    _compare(gpu, ref, "learnable lambda", max_outliers=2e-3, groups=GROUPS + ("lambda_raw",))


def test_one_call_driver_equals_the_stages():
    """sixdgs_render_batched = condition_project, bin_sort, raster_fwd (L1),
    raster_bwd; forward-only without targets (also on an inference plan)."""
    w = synth.make_workload(0)
    tgt = synth.perturb(w.scene, synth.target_seed(0))
    params = sx.params_to_device(w.scene)
    r = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras)
    targets = r.forward(sx.params_to_device(tgt))
    img_s, gi_s, loss_s = r.forward(params, targets)
    grads_s = r.backward(params, img_s, gi_s)
    loss_s = float(loss_s.item())
    img = r.new_images()
    gi = torch.empty_like(img)
    grads = r.new_grads(params)
    r.status.zero_()
    r.step(params, img, targets, gi, grads)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    assert torch.equal(img, img_s) and torch.equal(gi, gi_s)
    assert abs(float(r.loss.item()) - loss_s) <= 1e-12 * abs(loss_s)
    for k in GROUPS:      # equal up to the order of the record atomics
        rel = float((grads[k] - grads_s[k]).norm() / grads_s[k].norm())
        assert rel < 1e-5, (k, rel)
    ri = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, inference=True)
    img_i = ri.new_images()
    ri.step(params, img_i)
    torch.cuda.synchronize()
    assert int(ri.status.item()) == 0 and torch.equal(img_i, img_s)


@pytest.mark.parametrize("batch,persistent", [(512, False), (32, False), (64, True)])
def test_fused_forward_backward_equals_separate_kernels(batch, persistent):
    """sixdgs_raster_fwd_bwd (one kernel: forward, L1, backward replay from
    registers and, for single-batch lists, from the staged shared memory)
    against raster_fwd + blend_bwd: images, dL/dC and loss bit for bit, record
    and parameter gradients up to the order of the atomic additions.  Batch 32
    makes most lists span several batches (the reloading path)."""
    w = synth.make_workload(0)
    tgt = synth.perturb(w.scene, synth.target_seed(0))
    params = sx.params_to_device(w.scene)
    r = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, batch=batch, persistent=persistent)
    targets = r.forward(sx.params_to_device(tgt))
    img_s, gi_s, loss_s = r.forward(params, targets)
    grads_s = r.backward(params, img_s, gi_s)
    rec_s = r.grad_records().clone()
    loss_s = float(loss_s.item())
    ranges = r.ranges().cpu().numpy()
    lengths = ranges[:, 1] - ranges[:, 0]
    if batch == 32:
        assert (lengths > 32).mean() > 0.3          # the multi-batch path is exercised
    r.status.zero_()
    r.loss.zero_()
    r.condition_project(params)
    r.bin_sort()
    img = r.new_images()
    gi = torch.empty_like(img)
    r.raster_fwd_bwd(img, targets, gi)
    grads = r.new_grads(params)
    r.project_bwd(params, grads)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    assert torch.equal(img, img_s) and torch.equal(gi, gi_s)
    assert abs(float(r.loss.item()) - loss_s) <= 1e-12 * abs(loss_s)
    rec = r.grad_records()
    vis = r.ntiles() > 0
    scale = rec_s[vis].abs().amax(dim=0).clamp_min(1e-30)
    assert float(((rec[vis] - rec_s[vis]).abs() / scale).max()) < 1e-5
    for k in GROUPS:
        rel = float((grads[k] - grads_s[k]).norm() / grads_s[k].norm())
        assert rel < 1e-5, (k, rel)
