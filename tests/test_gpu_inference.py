"""Inference mode (forward only, view-independent slice state cached once per
scene; the caption of Algorithm 1) on scenes shaped like the paper's Table 2:
the cache against the oracle's Algorithm 1 steps 1-3, the cached projection
bit for bit against the uncached one, and the rendered views against the
FP64 oracle on sampled tiles."""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import sixdgs_oracle as O
from tests import parity as PT
from tests.test_gpu_forward import _check_records, _check_tiles, _sample_tiles, _settings

pytestmark = pytest.mark.gpu

sx = pytest.importorskip("paper_2410_04974_gb300")


def test_condition_cache_matches_oracle():
    scene = synth.scene_shell(3000, 17, dp_sigma=0.1)          # 23 blocks of 128 and a ragged tail
    params = sx.params_to_device(scene)
    cache = sx.condition_cache(params).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    p = O.to_params(scene)
    S = O.covariance(O.cholesky_factor(p["l_raw"]))
    A, Sdi, Sc = (t.numpy() for t in O.condition(S))
    alpha = torch.sigmoid(p["opacity_logit"]).numpy()
    n = scene.n
    A_g = cache[0:9].T.reshape(n, 3, 3)
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    Sdi_g = cache[9:15].T
    Sc_g = cache[15:24].T.reshape(n, 3, 3)
    # FP32 arithmetic on O(1) quantities: errors are a few hundred eps of each matrix's scale
    scale_a = np.abs(A).max(axis=(1, 2))[:, None, None]
    PT.assert_within(np.abs(A_g - A), 1e-4 * scale_a + 1e-30, "A")
    sdi_ref = np.stack([Sdi[:, i, j] for i, j in iu], axis=1)
    PT.assert_within(np.abs(Sdi_g - sdi_ref), 1e-4 * np.abs(sdi_ref).max(axis=1, keepdims=True), "Sigma_d^-1")
    norm_p = np.linalg.norm(S[:, :3, :3].numpy(), ord=2, axis=(1, 2))[:, None, None]
    PT.assert_within(np.abs(Sc_g - Sc), 1e-5 * norm_p, "Sigma_cond")
    np.testing.assert_allclose(cache[24], alpha, rtol=1e-6)


@pytest.mark.parametrize("index,n,views", [(0, None, 3), (4, 30000, 2)])
def test_cached_inference_projection_is_bit_identical(index, n, views):
    w = synth.table2_workload(index, n_override=n, views=views)
    params = sx.params_to_device(w.scene)
    train = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras)
    img_t = train.forward(params)
    cached = dict(params, cond_cache=sx.condition_cache(params))
    inf = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, inference=True)
    img_i = inf.forward(cached)
    torch.cuda.synchronize()
    assert int(inf.status.item()) == 0
    nt_t, nt_i = train.ntiles(), inf.ntiles()
    assert torch.equal(nt_t, nt_i)
    vis = nt_t > 0
    assert int(vis.sum()) > 0
    assert torch.equal(train.records()[vis], inf.records()[vis])
    assert torch.equal(train.sorted_pairs(), inf.sorted_pairs())
    assert torch.equal(img_t, img_i)


@pytest.mark.parametrize("index", [0, 3, 2])
def test_inference_render_matches_oracle(index):
    w = synth.table2_workload(index, views=2)
    st = _settings(w)
    params = sx.params_to_device(w.scene)
    params["cond_cache"] = sx.condition_cache(params)
    r = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, inference=True)
    img = r.forward(params)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    views = r.split(img)
    for v in range(len(w.cameras)):
        prep, member = _check_records(r, w.scene, w.cameras, st, v)
        tiles = _sample_tiles(w.cameras[v], st, 24, seed=100 + v)
        _check_tiles(r, w.scene, w.cameras, st, v, tiles, prep, member, views[v].cpu().numpy())


def test_inference_183k_sampled():
    w = synth.table2_workload(5, views=1)
    st = _settings(w)
    params = sx.params_to_device(w.scene)
    params["cond_cache"] = sx.condition_cache(params)
    r = sx.Renderer(w.scene.n, w.scene.sh_degree, w.cameras, inference=True, batch=256)
    img = r.forward(params)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    prep, member = _check_records(r, w.scene, w.cameras, st, 0)
    tiles = _sample_tiles(w.cameras[0], st, 12, seed=5)
    _check_tiles(r, w.scene, w.cameras, st, 0, tiles, prep, member, r.split(img)[0].cpu().numpy())


def test_nonfinite_cached_state_is_reported():
    scene = synth.scene_cube(300, 3)
    # row 3 of L of Gaussian 7 is zero (L_33 underflows, L_30..L_32 = 0): Sigma_d is singular
    scene.l_raw[3, 7] = -200.0
    scene.l_raw[9:12, 7] = 0.0
    params = sx.params_to_device(scene)
    cache = sx.condition_cache(params)
    assert math.isnan(float(cache[24, 7]))
    cams = [synth.look_at_camera((4.0, 0.0, 0.0), 64, 64)]
    r = sx.Renderer(scene.n, scene.sh_degree, cams, inference=True)
    r.forward(dict(params, cond_cache=cache), check=False)
    torch.cuda.synchronize()
    assert int(r.status.item()) & (1 << sx._lib.ERR_NONFINITE)
    assert int(r.ntiles()[7]) == 0


def test_cached_projection_with_learnable_lambda():
    """The per-Gaussian lambda_opa plane is read beside the cached state: the
    cached inference render equals the uncached one bit for bit."""
    w = synth.table2_workload(1, n_override=8000, views=2)
    scene = synth.with_learnable_lambda(w.scene, 77)
    params = sx.params_to_device(scene)
    assert "lambda_raw" in params
    train = sx.Renderer(scene.n, scene.sh_degree, w.cameras)
    img_t = train.forward(params)
    inf = sx.Renderer(scene.n, scene.sh_degree, w.cameras, inference=True)
    img_i = inf.forward(dict(params, cond_cache=sx.condition_cache(params)))
    torch.cuda.synchronize()
    assert int(inf.status.item()) == 0
    assert torch.equal(img_t, img_i)
    # and the plane matters: the global-lambda render differs
    plain = {k: v for k, v in params.items() if k != "lambda_raw"}
    assert not torch.equal(train.forward(plain), img_t)
