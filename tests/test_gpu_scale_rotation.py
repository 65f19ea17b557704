"""GPU parity of the scale / rotation extraction (section 4.3; Algorithm 1
steps 4-5) against the FP64 oracle, through the C ABI.

What is unique is compared element by element: the scales (eigenvalues of
Sigma_cond) and, where the eigenvalue gap is wide enough, each axis up to its
sign.  What is not unique (the signs, the axes of a repeated eigenvalue) is
checked for validity: R orthonormal with det R = +1 and R diag(S^2) R^T
rebuilding Sigma_cond.

Tolerances come from the arithmetic.  The kernel forms Sigma_cond in FP32
through the Schur complement; the rounding error of that matrix is a small
multiple of eps_32 * |Sigma_p| (eps_32 = 6e-8), so by Weyl's theorem every
eigenvalue is within EIG_TOL * |Sigma_p|_2 (EIG_TOL = 1e-5, about 170 eps)
and an axis with eigenvalue gap g turns by at most EIG_TOL * |Sigma_p|_2 / g
radians (Davis-Kahan).
"""

import numpy as np
import pytest
import torch

import synth
from oracle import sixdgs_oracle as O
from tests import parity as PT

pytestmark = pytest.mark.gpu

sx = pytest.importorskip("paper_2410_04974_gb300")
from paper_2410_04974_gb300 import _lib  # noqa: E402

EIG_TOL = 1e-5
ORTHO_TOL = 2e-6
NONFINITE = 1 << _lib.ERR_NONFINITE


def _oracle(l_raw_f32, idx=None):
    raw = torch.as_tensor(np.asarray(l_raw_f32, dtype=np.float64))
    if idx is not None:
        raw = raw[:, idx]
    L = O.cholesky_factor(raw)
    S = O.covariance(L)
    _, _, S_cond = O.condition(S)
    R, scale = O.scale_rotation(S_cond)
    norm_p = torch.linalg.matrix_norm(S[:, :3, :3], ord=2)
    return R.numpy(), scale.numpy(), S_cond.numpy(), norm_p.numpy()


def _gpu(l_raw):
    raw = torch.as_tensor(np.ascontiguousarray(l_raw, dtype=np.float32)).cuda()
    rot, scale, status = sx.scale_rotation(raw)
    torch.cuda.synchronize()
    n = raw.shape[1]
    R = rot.cpu().numpy().T.reshape(n, 3, 3).astype(np.float64)
    return R, scale.cpu().numpy().T.astype(np.float64), int(status.item())


def _check(Rg, sg, Ro, so, S_cond, norm_p, min_separated=0.5):
    tol = EIG_TOL * norm_p
    # eigenvalues: unique, in decreasing order
    PT.assert_within(np.abs(sg ** 2 - so ** 2), tol[:, None] + 1e-30, "eigenvalues")
    assert np.all(sg[:, :-1] >= sg[:, 1:])
    # validity of what is not unique
    eye = np.broadcast_to(np.eye(3), Rg.shape)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", Rg, Rg), eye, atol=ORTHO_TOL)
    np.testing.assert_allclose(np.linalg.det(Rg), 1.0, atol=3 * ORTHO_TOL)
    rebuilt = np.einsum("nik,nk,njk->nij", Rg, sg ** 2, Rg)
    PT.assert_within(np.abs(rebuilt - S_cond).max(axis=(1, 2)), 4 * tol + 1e-30, "R S^2 R^T")
    # each axis whose eigenvalue is separated from the others, up to its sign
    lam = so ** 2
    gaps = np.stack([lam[:, 0] - lam[:, 1], np.minimum(lam[:, 0] - lam[:, 1], lam[:, 1] - lam[:, 2]),
                     lam[:, 1] - lam[:, 2]], axis=1)
    angle = 2 * tol[:, None] / np.maximum(gaps, 1e-300)
    dots = np.abs(np.einsum("nij,nij->nj", Rg, Ro))
    sel = angle < 0.1
    assert sel.mean() >= min_separated
    PT.assert_within(1.0 - dots[sel], (angle[sel] ** 2) / 2 + 1e-6, "axes")


@pytest.mark.parametrize("dp", [0.0, 0.02, 0.3])
def test_scale_rotation_matches_oracle(dp):
    scene = synth.scene_shell(5000, 31, dp_sigma=dp)   # 40 blocks of 128 and a ragged tail
    Rg, sg, status = _gpu(scene.l_raw)
    assert status == 0
    _check(Rg, sg, *_oracle(scene.l_raw))


def test_scale_rotation_isotropic_and_axis_aligned():
    n = 130
    raw = np.zeros((21, n), np.float32)
    raw[:6] = np.log(0.1)                       # Sigma_p = 0.01 I, uncoupled: repeated eigenvalue
    raw[0, 64:] = np.log(0.3)                   # axis-aligned, distinct first axis
    raw[2, 96:] = np.log(0.02)
    Rg, sg, status = _gpu(raw)
    assert status == 0
    Ro, so, S_cond, norm_p = _oracle(raw)
    _check(Rg, sg, Ro, so, S_cond, norm_p, min_separated=0.3)
    np.testing.assert_allclose(sg[:64], 0.1, rtol=1e-6)
    np.testing.assert_allclose(sg[64:96], [[0.3, 0.1, 0.1]] * 32, rtol=1e-6)
    np.testing.assert_allclose(sg[96:], [[0.3, 0.1, 0.02]] * 34, rtol=1e-6)


def test_scale_rotation_full_size_sampled():
    w = synth.make_workload(2)
    Rg, sg, status = _gpu(w.scene.l_raw)
    assert status == 0
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(w.scene.n, 4096, replace=False))
    _check(Rg[idx], sg[idx], *_oracle(w.scene.l_raw, idx))
    # properties at every Gaussian
    assert np.all(np.isfinite(sg)) and np.all(sg > 0)
    np.testing.assert_allclose(np.linalg.det(Rg), 1.0, atol=3 * ORTHO_TOL)


def test_scale_rotation_empty_and_nonfinite():
    raw = torch.zeros((21, 0), dtype=torch.float32, device="cuda")
    rot, scale, status = sx.scale_rotation(raw)
    assert rot.shape == (9, 0) and scale.shape == (3, 0) and int(status.item()) == 0
    raw = np.zeros((21, 4), np.float32)
    raw[0, 2] = np.inf
    Rg, sg, status = _gpu(raw)
    assert status & NONFINITE
    assert np.all(sg[2] == 0) and np.all(Rg[2] == 0)
    np.testing.assert_allclose(sg[[0, 1, 3]], 1.0, rtol=1e-6)
