"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks one oracle function against something it does not share
code with: a closed form the paper states, an identity of Gaussian algebra,
a library routine (scipy), a brute-force loop, or central finite
differences.  A plausible slip in the oracle (dropped term, wrong sign,
transposed block, wrong SH index, wrong stop rule) fails at least one.
"""

import math

import numpy as np
import pytest
import torch

import synth
from oracle import sixdgs_oracle as O

F64 = torch.float64


def _coupled_scene(n=64, seed=11, dp=0.1):
    return synth.scene_shell(n, seed, dp_sigma=dp)


def _sigma(scene):
    p = O.to_params(scene)
    L = O.cholesky_factor(p["l_raw"])
    return L, O.covariance(L)


# --------------------------------------------------------------------------
# Section 3.1: Cholesky activation and Sigma = L L^T
# --------------------------------------------------------------------------

def test_cholesky_activation_matches_tanh_form():
    scene = _coupled_scene()
    L, _ = _sigma(scene)
    raw = scene.l_raw.astype(np.float64)
    L = L.numpy()
    assert np.all(np.triu(L, 1) == 0.0)
    np.testing.assert_allclose(np.diagonal(L, axis1=1, axis2=2).T, np.exp(raw[:6]), rtol=1e-14)
    for k, (i, j) in enumerate(O.OFFDIAG):
        # 2*sigmoid(x) - 1 == tanh(x/2): an independent form of the map into (-1, 1)
        np.testing.assert_allclose(L[:, i, j], np.tanh(raw[6 + k] / 2.0), rtol=1e-12, atol=1e-16)


def test_covariance_cholesky_roundtrip():
    scene = _coupled_scene()
    L, S = _sigma(scene)
    # The Cholesky factor with positive diagonal is unique: numpy must give L back.
    np.testing.assert_allclose(np.linalg.cholesky(S.numpy()), L.numpy(), rtol=1e-9, atol=1e-14)
    assert np.all(np.linalg.eigvalsh(S.numpy()) > 0)


# --------------------------------------------------------------------------
# Section 3.2, Eq. (mu), (sigma): conditional Gaussian
# --------------------------------------------------------------------------

def test_conditional_density_factorises():
    """log N6([x; d]) - log N3(x | mu_cond, Sigma_cond) = log N3(d | mu_d, Sigma_d) for every x."""
    stats = pytest.importorskip("scipy.stats")
    scene = _coupled_scene(n=16)
    p = O.to_params(scene)
    _, S = _sigma(scene)
    A, S_d_inv, S_cond = O.condition(S)
    rng = np.random.default_rng(5)
    mu_p, mu_d = p["mu_p"].T, p["mu_d"].T
    for g in range(16):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        mu_cond, D, _ = O.slice_at(mu_p[g:g + 1], mu_d[g:g + 1], A[g:g + 1], S_d_inv[g:g + 1],
                                   torch.ones(1, dtype=F64), torch.tensor(d[None]), 0.35)
        mu6 = np.concatenate([mu_p[g].numpy(), mu_d[g].numpy()])
        S6 = S[g].numpy()
        ref = stats.multivariate_normal(mu_d[g].numpy(), S6[3:, 3:]).logpdf(d)
        vals = []
        for _ in range(5):
            x = mu_p[g].numpy() + rng.normal(scale=0.05, size=3)
            joint = stats.multivariate_normal(mu6, S6).logpdf(np.concatenate([x, d]))
            cond = stats.multivariate_normal(mu_cond[0].numpy(), S_cond[g].numpy()).logpdf(x)
            vals.append(joint - cond)
        assert np.ptp(vals) < 1e-9
        assert abs(vals[0] - ref) < 1e-9
        # D is the Mahalanobis term of the direction marginal (appendix, Eq. for D)
        logdet = np.linalg.slogdet(2 * np.pi * S6[3:, 3:])[1]
        assert abs(float(D[0]) - (-2.0 * (ref + 0.5 * logdet))) < 1e-8 * max(1.0, float(D[0]))


def test_schur_complement_matches_woodbury_form():
    """With L = [[P, 0], [Q, R]]: Sigma_cond = P (I + Q^T (R R^T)^-1 Q)^-1 P^T and
    A = P Q^T (Q Q^T + R R^T)^-1 -- a second route to the same matrices."""
    scene = _coupled_scene(n=32)
    L, S = _sigma(scene)
    A, S_d_inv, S_cond = O.condition(S)
    for g in range(32):
        P = L[g, :3, :3].numpy(); Q = L[g, 3:, :3].numpy(); R = L[g, 3:, 3:].numpy()
        inner = np.eye(3) + Q.T @ np.linalg.inv(R @ R.T) @ Q
        np.testing.assert_allclose(S_cond[g].numpy(), P @ np.linalg.inv(inner) @ P.T,
                                   rtol=1e-9, atol=1e-16)
        np.testing.assert_allclose(A[g].numpy(), P @ Q.T @ np.linalg.inv(Q @ Q.T + R @ R.T),
                                   rtol=1e-9, atol=1e-16)
        assert np.all(np.linalg.eigvalsh(S_cond[g].numpy()) > 0)   # SPD (section 4.1)


def test_uncoupled_reduces_to_3d():
    """Sigma_pd = 0 gives mu_cond = mu_p and Sigma_cond = Sigma_p; lambda = 0 gives alpha_cond = alpha."""
    scene = _coupled_scene(n=8)
    for k, (i, j) in enumerate(O.OFFDIAG):
        if i >= 3 and j < 3:
            scene.l_raw[6 + k] = 0.0
    p = O.to_params(scene)
    L, S = _sigma(scene)
    A, S_d_inv, S_cond = O.condition(S)
    assert torch.all(A == 0)
    np.testing.assert_array_equal(S_cond.numpy(), S[:, :3, :3].numpy())
    d = O.view_direction(p["mu_p"].T, (4.0, 0.0, 0.0))
    alpha = torch.sigmoid(p["opacity_logit"])
    mu_cond, D, a0 = O.slice_at(p["mu_p"].T, p["mu_d"].T, A, S_d_inv, alpha, d, 0.0)
    np.testing.assert_array_equal(mu_cond.numpy(), p["mu_p"].T.numpy())
    np.testing.assert_array_equal(a0.numpy(), alpha.numpy())


@pytest.mark.parametrize("lam", [0.0, 0.35, 1.0])
def test_fcond_curve(lam):
    """f_cond = exp(-lambda D) (Eq. pdfv2; appendix figure of f_cond against D)."""
    scene = _coupled_scene(n=16)
    p = O.to_params(scene)
    A, S_d_inv, _ = O.condition(_sigma(scene)[1])
    d = O.view_direction(p["mu_p"].T, (0.0, 4.0, 0.0))
    alpha = torch.sigmoid(p["opacity_logit"])
    _, D, ac = O.slice_at(p["mu_p"].T, p["mu_d"].T, A, S_d_inv, alpha, d, lam)
    delta = (d - p["mu_d"].T).numpy()
    Sd = _sigma(scene)[1][:, 3:, 3:].numpy()
    D_ref = np.array([delta[g] @ np.linalg.solve(Sd[g], delta[g]) for g in range(16)])
    np.testing.assert_allclose(D.numpy(), D_ref, rtol=1e-10)
    np.testing.assert_allclose((ac / alpha).numpy(), np.exp(-lam * D_ref), rtol=1e-10)
    assert np.all(D_ref >= 0)


# --------------------------------------------------------------------------
# Section 4.2: spherical-harmonic colour
# --------------------------------------------------------------------------

def _real_sh_scipy(l, m, d):
    special = pytest.importorskip("scipy.special")
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = special.sph_harm_y(l, abs(m), theta, phi)   # complex, with Condon-Shortley phase
    cs = (-1.0) ** abs(m)
    if m == 0:
        return Y.real
    if m > 0:
        return math.sqrt(2.0) * cs * Y.real
    return math.sqrt(2.0) * cs * Y.imag


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(torch.tensor(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, l * l + l + m], _real_sh_scipy(l, m, d), atol=1e-12)


def test_sh_basis_orthonormal():
    """Quadrature of Y_a Y_b over the sphere: Gauss-Legendre in z, uniform in phi."""
    z, wz = np.polynomial.legendre.leggauss(16)
    phi = np.arange(32) * (2 * np.pi / 32)
    Z, PHI = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z ** 2)
    d = np.stack([s * np.cos(PHI), s * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full_like(PHI, 2 * np.pi / 32)).reshape(-1)
    Y = O.sh_basis(torch.tensor(d), 3).numpy()
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_colour_degree0_is_constant():
    scene = synth.scene_cube(10, 2, sh_degree=0)
    p = O.to_params(scene)
    rng = np.random.default_rng(1)
    d = rng.normal(size=(10, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    rgb = O.sh_colour(p["sh"], torch.tensor(d), 0).numpy()
    ref = 1.0 / (1.0 + np.exp(-scene.sh.astype(np.float64).T * (0.5 / math.sqrt(math.pi))))
    np.testing.assert_allclose(rgb, ref, rtol=1e-14)


# --------------------------------------------------------------------------
# Projection and footprint: a single isotropic Gaussian has a closed form
# --------------------------------------------------------------------------

def _single_gaussian_scene(s, pos, alpha_logit, beta0):
    """One Gaussian with Sigma_cond = s^2 I, delta = 0 (mu_d = view dir), SH degree 0."""
    scene = synth.scene_cube(1, 0, sh_degree=0)
    scene.mu_p[:, 0] = pos
    dvec = np.asarray(pos, dtype=np.float64) - np.array([4.0, 0.0, 0.0])
    scene.mu_d[:, 0] = dvec / np.linalg.norm(dvec)
    scene.l_raw[:] = 0.0
    scene.l_raw[:3, 0] = math.log(s)
    scene.l_raw[3:6, 0] = math.log(0.3)
    scene.opacity_logit[0] = alpha_logit
    scene.sh[:, 0] = beta0
    return scene


@pytest.mark.parametrize("s,depth,logit", [(0.02, 4.0, 0.5), (0.05, 3.5, 2.0), (0.01, 4.5, -1.0)])
def test_single_gaussian_footprint(s, depth, logit):
    cam = synth.look_at_camera((4.0, 0.0, 0.0), 64, 64)
    pos = (4.0 - depth, 0.0, 0.0)
    scene = _single_gaussian_scene(s, pos, logit, 0.7)
    st = O.Settings(tile_w=16, tile_h=16, lambda_opa=0.35)
    img, prep = O.render_view(scene, cam, st)
    img = img.numpy()
    # use the float32-stored parameters
    s = math.exp(float(scene.l_raw[0, 0]))
    depth = 4.0 - float(scene.mu_p[0, 0])
    var = (cam.fx * s / depth) ** 2 + O.DILATION        # isotropic 2D variance, px^2
    alpha = 1.0 / (1.0 + math.exp(-float(scene.opacity_logit[0])))
    rgb = 1.0 / (1.0 + math.exp(-float(scene.sh[0, 0]) * 0.5 / math.sqrt(math.pi)))
    r = 3.0 * math.sqrt(var)
    t0, t1 = math.floor((32 - r) / 16), math.floor((32 + r) / 16) + 1
    for py in range(64):
        for px in range(64):
            rho2 = (px + 0.5 - 32) ** 2 + (py + 0.5 - 32) ** 2
            a = min(0.99, alpha * math.exp(-0.5 * rho2 / var))
            inside = t0 <= px // 16 < t1 and t0 <= py // 16 < t1
            exp_val = (a * rgb + (1 - a) * 1.0) if (inside and a >= 1 / 255) else 1.0
            assert abs(img[0, py, px] - exp_val) < 1e-12, (px, py)


@pytest.mark.parametrize("l21,l10,logit", [(0.6, 0.0, 1.5), (-0.7, 0.02, 3.0), (0.45, -0.03, 0.0)])
def test_rotated_anisotropic_footprint(l21, l10, logit):
    """One Gaussian on the optical axis whose conditional covariance is
    anisotropic and tilted in the image plane, so that the conic's cross term
    is large.  Its image must be the 3DGS blend of one entry (section 4.4)
    with alpha(pixel) = min(0.99, alpha_cond N(x; m, S2) / N(m; m, S2)), the
    Gaussian ratio taken from scipy's bivariate normal density with
    S2 = (f/z)^2 (R Sigma_cond R^T)_xy + 0.3 I, and its extent the 3-sigma
    square of the largest eigenvalue of S2 (numpy).  A sign or factor slip in
    the cross term of the quadratic form mirrors or reshapes the ellipse."""
    from scipy.stats import multivariate_normal

    cam = synth.look_at_camera((4.0, 0.0, 0.0), 64, 64)
    scene = _single_gaussian_scene(0.05, (0.0, 0.0, 0.0), logit, 0.4)
    # position block of L: rows/cols (x, y, z) of the world; camera x = world
    # +y, camera y = world -z, so the (y, z) block sets the image ellipse
    scene.l_raw[1, 0] = math.log(0.06)      # L_yy
    scene.l_raw[2, 0] = math.log(0.015)     # L_zz
    k21 = synth.OFFDIAG_ORDER.index((2, 1))
    k10 = synth.OFFDIAG_ORDER.index((1, 0))
    scene.l_raw[6 + k21, 0] = 2.0 * math.atanh(l21)
    scene.l_raw[6 + k10, 0] = 2.0 * math.atanh(l10)
    st = O.Settings(tile_w=16, tile_h=16, lambda_opa=0.35)
    img = O.render_view(scene, cam, st)[0].numpy()
    # Sigma_p from the float32-stored raw values: exp on the diagonal,
    # 2 sigmoid - 1 below it (Sigma_pd = 0, so Sigma_cond = Sigma_p)
    raw = scene.l_raw[:, 0].astype(np.float64)
    Lp = np.diag(np.exp(raw[:3]))
    for k, (i, j) in enumerate(synth.OFFDIAG_ORDER):
        if i < 3:
            Lp[i, j] = 2.0 / (1.0 + math.exp(-raw[6 + k])) - 1.0
    S = Lp @ Lp.T
    R = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, -1.0]])    # world -> camera x, y rows
    f, z = cam.fx, 4.0
    S2 = (f / z) ** 2 * (R @ S @ R.T) + 0.3 * np.eye(2)
    assert abs(S2[0, 1]) > 0.3 * math.sqrt(S2[0, 0] * S2[1, 1])   # strongly tilted
    m = np.array([32.0, 32.0])
    mvn = multivariate_normal(mean=m, cov=S2)
    alpha_cond = 1.0 / (1.0 + math.exp(-float(scene.opacity_logit[0])))
    rgb = 1.0 / (1.0 + math.exp(-float(scene.sh[0, 0]) * 0.5 / math.sqrt(math.pi)))
    r = 3.0 * math.sqrt(np.linalg.eigvalsh(S2).max())
    t0, t1 = math.floor((32 - r) / 16), math.floor((32 + r) / 16) + 1
    ys, xs = np.mgrid[0:64, 0:64]
    pts = np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5], 1)
    ratio = (mvn.pdf(pts) / mvn.pdf(m)).reshape(64, 64)
    a = np.minimum(0.99, alpha_cond * ratio)
    inside = (t0 <= xs // 16) & (xs // 16 < t1) & (t0 <= ys // 16) & (ys // 16 < t1)
    expect = np.where(inside & (a >= 1 / 255), a * rgb + (1 - a), 1.0)
    assert (expect < 1.0).sum() > 40
    np.testing.assert_allclose(img[0], expect, rtol=0, atol=1e-12)
    # the mirrored ellipse (cross term of the other sign) is far away
    mirror = multivariate_normal(mean=m, cov=S2 * np.array([[1, -1], [-1, 1]]))
    a_m = np.minimum(0.99, alpha_cond * (mirror.pdf(pts) / mirror.pdf(m)).reshape(64, 64))
    assert np.abs(a_m - a).max() > 0.05


def test_off_axis_jacobian():
    """Gaussian off the optical axis: Sigma_2D = s^2 J J^T + 0.3 I with
    J = [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]] (no guard clamp hit)."""
    cam = synth.look_at_camera((4.0, 0.0, 0.0), 64, 64)
    s = 0.03
    # camera x axis is world +y, camera y axis is world -z
    scene = _single_gaussian_scene(s, (0.5, 0.4, -0.3), 0.0, 0.0)
    st = O.Settings()
    p = O.to_params(scene)
    prep = O.prepare_view(p, 0, cam, st)
    s = math.exp(float(scene.l_raw[0, 0]))               # float32-stored values
    x, y, z = float(scene.mu_p[1, 0]), -float(scene.mu_p[2, 0]), 4.0 - float(scene.mu_p[0, 0])
    f = cam.fx
    J = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
    cov = s * s * J @ J.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    np.testing.assert_allclose(prep.conic[0].numpy(), [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-12)
    np.testing.assert_allclose(prep.mean2d[0].numpy(), [f * x / z + 32, f * y / z + 32], rtol=1e-14)
    assert abs(float(prep.depth[0]) - z) < 1e-14


def test_tile_rect_rule():
    cam = synth.look_at_camera((4.0, 0.0, 0.0), 100, 40)   # 7 x 3 tiles of 16
    mean = torch.tensor([[20.0, 20.0], [0.5, 39.0], [99.0, 1.0], [-40.0, 20.0]], dtype=F64)
    r = torch.tensor([4.0, 2.0, 30.0, 10.0], dtype=F64)
    rect = O.tile_rect(mean, r, cam, 16, 16).numpy()
    assert rect[0].tolist() == [1, 2, 1, 2]
    assert rect[1].tolist() == [0, 1, 2, 3]
    assert rect[2].tolist() == [4, 7, 0, 2]
    assert rect[3].tolist() == [0, 0, 0, 2]       # fully off-screen: empty x range


# --------------------------------------------------------------------------
# Blend: closed-form invariants, the sequential loop, brute force
# --------------------------------------------------------------------------

def test_blend_weights_sum_to_one():
    rng = np.random.default_rng(9)
    alpha = torch.tensor(np.minimum(0.99, rng.uniform(0, 1, (64, 200)) ** 3), dtype=F64)
    rgb = torch.tensor(rng.uniform(0, 1, (200, 3)), dtype=F64)
    C, T, first, w = O.blend(alpha, rgb, (1.0, 1.0, 1.0))
    np.testing.assert_allclose((w.sum(1) + T).numpy(), 1.0, atol=1e-12)
    # with white background and white splats every pixel is exactly white
    C2, _, _, _ = O.blend(alpha, torch.ones((200, 3), dtype=F64), (1.0, 1.0, 1.0))
    np.testing.assert_allclose(C2.numpy(), 1.0, atol=1e-12)


def test_blend_matches_sequential_loop():
    rng = np.random.default_rng(4)
    for trial in range(20):
        n = int(rng.integers(0, 60))
        alpha = np.minimum(0.99, rng.uniform(0, 1, (8, n)) ** rng.uniform(0.5, 6))
        alpha[rng.uniform(size=alpha.shape) < 0.2] = 0.002       # some skipped entries
        rgb = rng.uniform(0, 1, (n, 3))
        bg = (0.2, 0.5, 1.0)
        C, T, first, _ = O.blend(torch.tensor(alpha), torch.tensor(rgb), bg)
        for pix in range(8):
            ref = O.blend_pixel_sequential(alpha[pix], rgb, bg)
            np.testing.assert_allclose(C[pix].numpy(), ref, atol=1e-13)


def test_blend_stop_excludes_current_entry():
    alpha = torch.tensor([[0.99, 0.99, 0.5]], dtype=F64)
    rgb = torch.tensor([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]], dtype=F64)
    C, T, first, _ = O.blend(alpha, rgb, (0.0, 0.0, 0.0))
    # T after the first entry is 0.01; 0.01 * 0.01 = 1e-4 is not < 1e-4, so the
    # second entry is kept; T would become 1e-4 * 0.5 < 1e-4 at the third: stop.
    np.testing.assert_allclose(C[0].numpy(), [0.99, 0.0099, 0.0], rtol=1e-12)
    assert int(first[0]) == 2
    np.testing.assert_allclose(float(T[0]), 1e-4, rtol=1e-12)


def _brute_force_image(prep, cam, st):
    """Every pixel walks all Gaussians, membership evaluated per pixel."""
    n = prep.valid.shape[0]
    depth = prep.depth.detach().numpy()
    H, W = cam.height, cam.width
    out = np.zeros((3, H, W))
    for py in range(H):
        for px in range(W):
            tx, ty = px // st.tile_w, py // st.tile_h
            members = []
            for g in range(n):
                if not bool(prep.valid[g]):
                    continue
                x0, x1, y0, y1 = [int(v) for v in prep.rect[g]]
                if x0 <= tx < x1 and y0 <= ty < y1:
                    members.append(g)
            members.sort(key=lambda g: (depth[g], g))
            alphas, cols = [], []
            for g in members:
                u, v = float(prep.mean2d[g, 0]), float(prep.mean2d[g, 1])
                a_, b_, c_ = [float(t) for t in prep.conic[g]]
                dx, dy = u - (px + 0.5), v - (py + 0.5)
                power = -0.5 * (a_ * dx * dx + c_ * dy * dy) - b_ * dx * dy
                alphas.append(min(0.99, float(prep.alpha_cond[g]) * math.exp(power)))
                cols.append([float(t) for t in prep.rgb[g]])
            out[:, py, px] = O.blend_pixel_sequential(alphas, cols, st.bg)
    return out


@pytest.mark.parametrize("seed,w,h,tw,th", [(1, 32, 32, 16, 16), (2, 40, 24, 8, 16), (3, 48, 36, 32, 8)])
def test_tiled_render_equals_brute_force(seed, w, h, tw, th):
    scene = synth.scene_cube(8, seed)
    scene.l_raw[:3] += math.log(5.0)          # bigger splats at this resolution
    scene.mu_p *= 0.5
    scene.opacity_logit[:] = 2.0
    cam = synth.look_at_camera((4.0, 0.3, 0.2), w, h)
    # the per-pixel reference uses the 3DGS 3-sigma membership; both tile
    # footprints must reproduce it (the alpha-aware one drops only tiles where
    # the Gaussian composites no pixel)
    st0 = O.Settings(tile_w=tw, tile_h=th, lambda_opa=0.35, bg=(1.0, 0.9, 0.8), alpha_footprint=0)
    _, prep0 = O.render_view(scene, cam, st0)
    assert int(prep0.valid.sum()) >= 2
    ref = _brute_force_image(prep0, cam, st0)
    for fp in (0, 1):
        st = O.Settings(tile_w=tw, tile_h=th, lambda_opa=0.35, bg=(1.0, 0.9, 0.8), alpha_footprint=fp)
        img, _ = O.render_view(scene, cam, st)
        np.testing.assert_allclose(img.numpy(), ref, atol=1e-12)


def test_alpha_footprint_keeps_every_compositing_pixel():
    """Every pixel centre where a Gaussian's alpha reaches 1/255 lies in a
    tile of its alpha-aware footprint, which is never larger than the 3-sigma
    square and is much smaller on average."""
    w = synth.make_workload(0)
    cam = w.cameras[0]
    p0 = O.prepare_view(O.to_params(w.scene), w.scene.sh_degree, cam, O.Settings(alpha_footprint=0))
    p1 = O.prepare_view(O.to_params(w.scene), w.scene.sh_degree, cam, O.Settings(alpha_footprint=1))
    assert torch.equal(p0.valid, p1.valid)
    r0, r1 = p0.rect.numpy(), p1.rect.numpy()
    v = p0.valid.numpy()
    assert np.all(r1[v, 0] >= r0[v, 0]) and np.all(r1[v, 1] <= r0[v, 1])
    assert np.all(r1[v, 2] >= r0[v, 2]) and np.all(r1[v, 3] <= r0[v, 3])
    area = lambda r: np.maximum(r[:, 1] - r[:, 0], 0) * np.maximum(r[:, 3] - r[:, 2], 0)
    assert area(r1[v]).sum() < 0.85 * area(r0[v]).sum()
    m = p0.mean2d.detach().numpy()
    con = p0.conic.detach().numpy()
    ac = p0.alpha_cond.detach().numpy()
    checked = 0
    for g in np.nonzero(v)[0]:
        x0, x1, y0, y1 = r0[g]
        px = np.arange(x0 * 16, x1 * 16) + 0.5
        py = np.arange(y0 * 16, y1 * 16) + 0.5
        dx = m[g, 0] - px[None, :]
        dy = m[g, 1] - py[:, None]
        a = ac[g] * np.exp(-0.5 * (con[g, 0] * dx * dx + 2 * con[g, 1] * dx * dy + con[g, 2] * dy * dy))
        yy, xx = np.nonzero(a >= 1.0 / 255.0)
        tx, ty = (px[xx] // 16).astype(int), (py[yy] // 16).astype(int)
        assert np.all((r1[g, 0] <= tx) & (tx < r1[g, 1]) & (r1[g, 2] <= ty) & (ty < r1[g, 3])), g
        checked += len(xx)
    assert checked > 10000


def test_render_lists_sorted_by_depth():
    w = synth.make_workload(0)
    st = O.Settings()
    _, prep = O.render_view(w.scene, w.cameras[0], st, tiles=[(3, 3)])
    ids = O.tile_list(prep, 3, 3)
    z = prep.depth.detach().numpy()[ids]
    assert len(ids) > 10 and np.all(np.diff(z) >= 0)


# --------------------------------------------------------------------------
# L1 loss and gradients
# --------------------------------------------------------------------------

def test_l1_loss_closed_form():
    a = [np.array([[[0.0, 1.0], [2.0, 3.0]]]), np.array([[[1.0]]])]
    b = [np.array([[[1.0, 1.0], [0.0, 5.0]]]), np.array([[[0.5]]])]
    loss, g = O.l1_loss(a, b)
    assert abs(loss - (1 + 0 + 2 + 2 + 0.5) / 5) < 1e-15
    np.testing.assert_array_equal(g[0], np.array([[[-1, 0], [1, -1]]]) / 5)
    np.testing.assert_array_equal(g[1], np.array([[[1]]]) / 5)


def _loss_and_decisions(scene, cams, st, g_imgs):
    """<g, image> summed over views, and every discrete decision of the render
    (culls, rects, lists, skips, stops, clamps)."""
    sig = []
    total = 0.0
    for cam, g in zip(cams, g_imgs):
        img, prep = O.render_view(scene, cam, st)
        total += float((img.numpy() * g.astype(np.float64)).sum())
        sig.append(prep.valid.numpy().tobytes())
        sig.append(prep.rect.numpy().tobytes())
        tx, ty = O.tile_grid(cam, st)
        for y in range(ty):
            for x in range(tx):
                _, ids, alpha, _, walked = O.render_tile(prep, cam, st, x, y)
                a = alpha.numpy()
                sig.append(np.asarray(ids).tobytes())
                sig.append((a < O.ALPHA_MIN).tobytes())
                sig.append((a >= O.ALPHA_MAX).tobytes())
                sig.append(walked.numpy().tobytes())
    return total, b"".join(sig)


def _fd_scene():
    scene = synth.scene_shell(6, 21, dp_sigma=0.1)
    scene.l_raw[:3] += math.log(8.0)
    scene.mu_p *= 0.4
    scene.opacity_logit[:] = np.array([0.5, 1.0, -0.5, 2.0, 0.0, 3.0], dtype=np.float32)
    # point the direction means at the cameras so that alpha_cond stays visible
    # (d runs from the camera to the Gaussian, i.e. roughly along -x here)
    scene.mu_d[:] = (np.array([[-1.0], [0.1], [-0.1]]) / np.linalg.norm([1.0, 0.1, 0.1])).astype(np.float32)
    return scene


def test_gradients_match_finite_differences():
    scene = _fd_scene()
    cams = [synth.look_at_camera((4.0, 0.5, 0.3), 32, 32),
            synth.look_at_camera((3.5, -1.5, 0.5), 24, 32)]
    st = O.Settings(lambda_opa=0.35)
    g_imgs = synth.random_grad_images(cams, 77)
    grads = O.gradients(scene, cams, g_imgs, st)

    base = {k: np.asarray(v, dtype=np.float64) for k, v in scene.planes().items()}
    checked = discarded = 0
    nonzero = 0
    for name, arr in base.items():
        flat = arr.reshape(-1)
        for idx in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[idx]))
            vals = []
            sigs = []
            for sgn in (+1, -1):
                pert = {k: v.copy() for k, v in base.items()}
                pert[name].reshape(-1)[idx] += sgn * h
                sc = synth.Scene(pert["mu_p"], pert["mu_d"], pert["l_raw"], pert["opacity_logit"],
                                 pert["sh"], scene.sh_degree)
                v, sg = _loss_and_decisions(sc, cams, st, g_imgs)
                vals.append(v)
                sigs.append(sg)
            if sigs[0] != sigs[1]:
                discarded += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            ad = grads[name].reshape(-1)[idx]
            assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-8, (name, idx, fd, ad)
            checked += 1
            nonzero += abs(ad) > 1e-8
    assert discarded <= 0.02 * (checked + discarded)
    assert nonzero > 100


# --------------------------------------------------------------------------
# Section 4.2: per-Gaussian learnable lambda_opa = sigmoid(raw)
# --------------------------------------------------------------------------

def test_constant_lambda_plane_equals_global_lambda():
    scene = synth.scene_cube(300, 5)
    scene.l_raw[:3] += math.log(3.0)
    cam = synth.look_at_camera((4.0, 0.2, 0.1), 48, 40)
    plane = synth.Scene(scene.mu_p, scene.mu_d, scene.l_raw, scene.opacity_logit, scene.sh, scene.sh_degree,
                        np.full(scene.n, math.log(0.35 / 0.65), np.float32))
    a, _ = O.render_view(scene, cam, O.Settings(lambda_opa=0.35))
    lam_f32 = 1.0 / (1.0 + math.exp(-float(plane.lambda_raw[0])))   # the float32-stored raw value
    b_ref, _ = O.render_view(scene, cam, O.Settings(lambda_opa=lam_f32))
    b, _ = O.render_view(plane, cam, O.Settings(lambda_opa=0.9))   # global value ignored
    np.testing.assert_allclose(b.numpy(), b_ref.numpy(), atol=1e-14)
    np.testing.assert_allclose(b.numpy(), a.numpy(), atol=1e-6)


def test_lambda_gradient_matches_finite_differences():
    scene = synth.with_learnable_lambda(_fd_scene(), 12, spread=1.0)
    cams = [synth.look_at_camera((4.0, 0.5, 0.3), 32, 32)]
    st = O.Settings()
    g_imgs = synth.random_grad_images(cams, 78)
    grads = O.gradients(scene, cams, g_imgs, st)
    base = np.asarray(scene.lambda_raw, dtype=np.float64)
    checked = 0
    for i in range(scene.n):
        h = 1e-6 * max(1.0, abs(base[i]))
        vals, sigs = [], []
        for sgn in (+1, -1):
            lam = base.copy()
            lam[i] += sgn * h
            sc = synth.Scene(scene.mu_p, scene.mu_d, scene.l_raw, scene.opacity_logit, scene.sh, scene.sh_degree, lam)
            v, sg = _loss_and_decisions(sc, cams, st, g_imgs)
            vals.append(v)
            sigs.append(sg)
        if sigs[0] != sigs[1]:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = grads["lambda_raw"][i]
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-8, (i, fd, ad)
        checked += 1
    assert checked >= scene.n - 1 and np.abs(grads["lambda_raw"]).max() > 1e-6


# --------------------------------------------------------------------------
# Section 4.3, Algorithm 1 steps 4-5: scale and rotation of Sigma_cond
# --------------------------------------------------------------------------

def _rodrigues(axis, angle):
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


def test_scale_rotation_recovers_known_ellipsoid():
    rng = np.random.default_rng(5)
    Qs, ss = [], []
    for _ in range(16):
        Qs.append(_rodrigues(rng.normal(size=3), rng.uniform(0.1, 3.0)))
        ss.append(rng.permutation([0.5, 0.05, 0.005]) * rng.uniform(0.5, 2.0))
    Q = np.stack(Qs)
    s = np.stack(ss)
    S = torch.as_tensor(Q @ (s[:, :, None] ** 2 * np.transpose(Q, (0, 2, 1))))
    R, scale = O.scale_rotation(S)
    R, scale = R.numpy(), scale.numpy()
    order = np.argsort(-s, axis=1)
    np.testing.assert_allclose(scale, np.take_along_axis(s, order, 1), rtol=1e-10)
    for i in range(16):
        Qo = Q[i][:, order[i]]
        # each column is the ellipsoid axis of that scale, up to its sign
        np.testing.assert_allclose(np.abs(np.sum(R[i] * Qo, axis=0)), 1.0, rtol=1e-10)
        assert abs(np.linalg.det(R[i]) - 1.0) < 1e-12


def test_scale_rotation_matches_svd_and_reconstructs():
    scene = _coupled_scene(n=128, seed=21, dp=0.3)
    _, S = _sigma(scene)
    _, _, S_cond = O.condition(S)
    R, scale = O.scale_rotation(S_cond)
    U, sv, _ = np.linalg.svd(S_cond.numpy())
    np.testing.assert_allclose(scale.numpy() ** 2, sv, rtol=1e-9)
    np.testing.assert_allclose(np.abs(np.einsum("nij,nij->nj", R.numpy(), U)), 1.0, rtol=1e-6)
    rebuilt = R @ torch.diag_embed(scale ** 2) @ R.transpose(1, 2)
    np.testing.assert_allclose(rebuilt.numpy(), S_cond.numpy(), rtol=1e-9, atol=1e-16)
    np.testing.assert_allclose(np.linalg.det(R.numpy()), 1.0, atol=1e-12)
    np.testing.assert_allclose(R.transpose(1, 2) @ R, np.broadcast_to(np.eye(3), (128, 3, 3)), atol=1e-12)


def test_scale_rotation_axis_aligned_case():
    d = np.array([[4.0, 9.0, 1.0], [1e-4, 1e-6, 1e-2]])
    R, scale = O.scale_rotation(torch.as_tensor(np.stack([np.diag(r) for r in d])))
    np.testing.assert_allclose(scale.numpy(), np.sqrt(-np.sort(-d, axis=1)), rtol=1e-12)
    np.testing.assert_allclose(np.abs(R.numpy()).sum(axis=1), 1.0, atol=1e-12)  # signed permutation
    np.testing.assert_allclose(np.linalg.det(R.numpy()), 1.0, atol=1e-12)


def test_symmetric_eigen_matches_lapack():
    rng = np.random.default_rng(8)
    M = rng.normal(size=(64, 3, 3))
    S = M @ np.transpose(M, (0, 2, 1))
    S[:8] = np.diag([2.0, 2.0, 0.5])            # repeated eigenvalue
    w, V = O.symmetric_eigen(torch.as_tensor(S))
    w, V = w.numpy(), V.numpy()
    np.testing.assert_allclose(np.sort(w, axis=1), np.linalg.eigvalsh(S), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.einsum("nik,nk,njk->nij", V, w, V), S, atol=1e-12)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", V, V), np.broadcast_to(np.eye(3), S.shape), atol=1e-13)
