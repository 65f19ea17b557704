"""FP64 CPU oracle of the differentiable 6D Gaussian render (6DGS, arXiv 2410.04974).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this file: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it.  It shares no code with the CUDA
library; the only common module is the seeded input generator ``synth``.

Everything is plain PyTorch CPU arithmetic in float64, written in the order
of the paper's definitions so that it can be checked against the paper by
eye.  Gradients are the exact derivatives of this forward definition, taken
by autograd (``gradients``); the test suite pins them to central finite
differences.

Definition followed, stage by stage:

* Representation and Cholesky activation -- section 3.1: Sigma = L L^T with
  exp on the diagonal and a sigmoid map into (-1, 1) off the diagonal, read
  as v = 2*sigmoid(raw) - 1.
* Slice -- section 3.2, Eq. (mu), Eq. (sigma), Eq. (pdf)/(alpha) and the
  refined Eq. (pdfv2) of section 4.2; Algorithm 1 steps 1-3.
* View-dependent colour -- section 4.2, the sigmoid of a degree-<=3 real
  spherical-harmonic expansion of the view direction.
* Projection, tiling, sorting and blending -- section 4.4: after slicing,
  the pipeline is the 3DGS rasteriser.  Its conventions (0.3 px^2 dilation,
  3-sigma extent, 1/255 skip, 0.99 clamp, 1e-4 transmittance stop, 1.3x
  frustum guard on the Jacobian, near plane 0.2) are named constants below.
* Loss -- section 4.4 keeps the 3DGS losses; the L1 term is used here.

Readings where the paper is silent or garbled:
view direction d = normalize(mu_p - campos) per Gaussian (used for both the
slice and the SH colour); f_cond = exp(-lambda * D) without a factor 1/2, as
printed; mu_d is used unnormalised; opacity alpha = sigmoid(logit); real
orthonormal SH without the Condon-Shortley phase, index k = l*l + l + m; no
+0.5 offset before the sigmoid; pixel centres at +0.5; ties in depth broken
by Gaussian id; a Gaussian whose alpha_cond < 1/255 is culled before binning
(it would be skipped at every pixel anyway since the per-pixel alpha never
exceeds alpha_cond).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

F64 = torch.float64

# ---- constants of the inherited 3DGS rasteriser (section 4.4) ------------
DILATION = 0.3          # px^2 added to the 2D covariance diagonal
RADIUS_SIGMAS = 3.0     # screen extent = 3 * sqrt(largest 2D eigenvalue)
ALPHA_MIN = 1.0 / 255.0 # per-pixel alpha below this is skipped
ALPHA_MAX = 0.99        # per-pixel alpha clamp
T_MIN = 1e-4            # stop once transmittance would drop below this
FRUSTUM_GUARD = 1.3     # x/z, y/z clamp (in units of the half-fov tangent) for J
LAMBDA_OPA = 0.35       # section 5.1
# tile footprint (settings.alpha_footprint = 1): the 3-sigma square intersected
# with the bounding box of the alpha >= 1/255 ellipse, widened by these
ALPHA_BOX_REL = 1e-4
ALPHA_BOX_ABS = 0.01    # px


@dataclasses.dataclass
class Settings:
    tile_w: int = 16
    tile_h: int = 16
    lambda_opa: float = LAMBDA_OPA
    bg: tuple = (1.0, 1.0, 1.0)
    # 1: tile rectangle = 3-sigma square (3DGS) intersected with the widened
    # bounding box of the alpha >= 1/255 ellipse (tiles outside it hold no
    # pixel that composites the Gaussian, so renders are unchanged); 0: the
    # 3-sigma square alone
    alpha_footprint: int = 1


# ==========================================================================
# Per-Gaussian, view-independent part (Algorithm 1 steps 1-3, Eq. sigma)
# ==========================================================================

OFFDIAG = [(i, j) for i in range(6) for j in range(i)]


def cholesky_factor(l_raw: torch.Tensor) -> torch.Tensor:
    """(21, n) raw -> (n, 6, 6) lower-triangular L (section 3.1)."""
    n = l_raw.shape[1]
    L = torch.zeros((n, 6, 6), dtype=F64)
    rows, cols = [], []
    vals = []
    for k in range(6):
        rows.append(k); cols.append(k)
        vals.append(torch.exp(l_raw[k]))
    for k, (i, j) in enumerate(OFFDIAG):
        rows.append(i); cols.append(j)
        vals.append(2.0 * torch.sigmoid(l_raw[6 + k]) - 1.0)
    L = L.index_put((torch.arange(n).repeat_interleave(len(rows)),
                     torch.tensor(rows).repeat(n), torch.tensor(cols).repeat(n)),
                    torch.stack(vals, dim=1).reshape(-1))
    return L


def covariance(L: torch.Tensor) -> torch.Tensor:
    """Sigma = L L^T (Algorithm 1 step 1)."""
    return L @ L.transpose(1, 2)


def partition(S: torch.Tensor):
    """Blocks Sigma_p, Sigma_pd, Sigma_d (Algorithm 1 step 2)."""
    return S[:, :3, :3], S[:, :3, 3:], S[:, 3:, 3:]


def condition(S: torch.Tensor):
    """Regression matrix A = Sigma_pd Sigma_d^-1, Sigma_d^-1 and the Schur
    complement Sigma_cond = Sigma_p - Sigma_pd Sigma_d^-1 Sigma_pd^T
    (Eq. sigma; Algorithm 1 step 3).  Sigma_d^-1 comes from a Cholesky
    solve of Sigma_d."""
    S_p, S_pd, S_d = partition(S)
    C = torch.linalg.cholesky(S_d)
    S_d_inv = torch.cholesky_inverse(C)
    A = S_pd @ S_d_inv
    S_cond = S_p - A @ S_pd.transpose(1, 2)
    return A, S_d_inv, S_cond


def symmetric_eigen(S: torch.Tensor, tol=1e-15, max_sweeps=50):
    """Eigenvalues (n, 3) and orthonormal eigenvectors (columns, n x 3 x 3) of
    symmetric 3x3 matrices by the cyclic Jacobi method (Golub and Van Loan,
    "Matrix Computations", section 8.5): each rotation J in the (p, q) plane
    is chosen so that (J^T A J)_pq = 0; sweeps over the pairs (0,1), (0,2),
    (1,2) repeat until the off-diagonal mass is below tol times the norm.
    No LAPACK: the result is checked against a library decomposition by the
    tests."""
    A = S.clone()
    n = A.shape[0]
    V = torch.eye(3, dtype=A.dtype).repeat(n, 1, 1)
    scale = torch.linalg.matrix_norm(A).clamp_min(1e-300)
    for _ in range(max_sweeps):
        off = A[:, 0, 1] ** 2 + A[:, 0, 2] ** 2 + A[:, 1, 2] ** 2
        if bool(torch.all(off.sqrt() <= tol * scale)):
            break
        for p, q in ((0, 1), (0, 2), (1, 2)):
            apq = A[:, p, q]
            live = apq.abs() > 1e-300
            theta = (A[:, q, q] - A[:, p, p]) / torch.where(live, 2.0 * apq, torch.ones_like(apq))
            sgn = torch.where(theta >= 0, 1.0, -1.0).to(A.dtype)
            t = torch.where(live, sgn / (theta.abs() + torch.sqrt(theta * theta + 1.0)), torch.zeros_like(apq))
            c = 1.0 / torch.sqrt(t * t + 1.0)
            s_ = t * c
            J = torch.eye(3, dtype=A.dtype).repeat(n, 1, 1)
            J[:, p, p] = c
            J[:, q, q] = c
            J[:, p, q] = s_
            J[:, q, p] = -s_
            A = J.transpose(1, 2) @ A @ J
            V = V @ J
    return torch.diagonal(A, dim1=1, dim2=2), V


def scale_rotation(S_cond: torch.Tensor):
    """Rotation R (n, 3, 3) and scale S (n, 3) of the conditional Gaussian
    (section 4.3; Algorithm 1 steps 4-5): Sigma_cond = U D U^T, R = U,
    S = sqrt(diag D), then the third column of R multiplied by sign(det R).
    Sigma_cond is symmetric positive definite, so its singular value
    decomposition is its eigen-decomposition with the eigenvalues in
    decreasing order (the order a singular value decomposition returns)."""
    w, U = symmetric_eigen(S_cond)
    order = torch.argsort(w, dim=1, descending=True)
    D = torch.gather(w, 1, order)
    R = torch.gather(U, 2, order[:, None, :].expand(-1, 3, -1)).clone()
    sign = torch.sign(torch.linalg.det(R))
    R[:, :, 2] = R[:, :, 2] * sign[:, None]
    return R, torch.sqrt(D)


# ==========================================================================
# Per-view slice (Eq. mu, Eq. pdfv2, Eq. alpha)
# ==========================================================================

def view_direction(mu_p: torch.Tensor, campos) -> torch.Tensor:
    """d = normalize(mu_p - campos), one per Gaussian; (n, 3)."""
    c = torch.as_tensor(np.asarray(campos, dtype=np.float64))
    v = mu_p - c[None, :]
    return v / torch.linalg.norm(v, dim=1, keepdim=True)


def slice_at(mu_p, mu_d, A, S_d_inv, alpha, d, lambda_opa):
    """mu_cond = mu_p + A (d - mu_d); D = (d - mu_d)^T Sigma_d^-1 (d - mu_d);
    f_cond = exp(-lambda_opa * D); alpha_cond = alpha * f_cond."""
    delta = d - mu_d
    mu_cond = mu_p + (A @ delta[:, :, None])[:, :, 0]
    D = torch.einsum("ni,nij,nj->n", delta, S_d_inv, delta)
    f_cond = torch.exp(-lambda_opa * D)
    return mu_cond, D, alpha * f_cond


# ==========================================================================
# Spherical harmonics (section 4.2), from associated Legendre functions
# ==========================================================================

def _legendre_deriv_coeffs(l: int, m: int) -> np.ndarray:
    """Power-series coefficients (ascending) of d^m/dz^m P_l(z)."""
    leg = np.polynomial.legendre.Legendre.basis(l).deriv(m)
    return np.polynomial.legendre.leg2poly(leg.coef)


def sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Real orthonormal spherical harmonics Y_k(d), k = l*l + l + m, (n, K).

    For a unit vector (x, y, z): with P_l^(m) the m-th derivative of the
    Legendre polynomial P_l and N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
      Y_l^0  = N_l0 P_l(z)
      Y_l^m  = sqrt(2) N_lm P_l^(m)(z) Re((x + i y)^m)      (m > 0)
      Y_l^-m = sqrt(2) N_lm P_l^(m)(z) Im((x + i y)^m)      (m > 0)
    using sin^m(theta) e^{i m phi} = (x + i y)^m; no Condon-Shortley phase.
    """
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    cols = {}
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, degree + 1):
        re.append(re[-1] * x - im[-1] * y)
        im.append(re[-2] * y + im[-1] * x)
    for l in range(degree + 1):
        for m in range(0, l + 1):
            coeffs = _legendre_deriv_coeffs(l, m)
            p = torch.zeros_like(z)
            for c in coeffs[::-1]:
                p = p * z + float(c)
            norm = math.sqrt((2 * l + 1) / (4.0 * math.pi)
                             * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                cols[l * l + l] = norm * p
            else:
                cols[l * l + l + m] = math.sqrt(2.0) * norm * p * re[m]
                cols[l * l + l - m] = math.sqrt(2.0) * norm * p * im[m]
    return torch.stack([cols[k] for k in range((degree + 1) ** 2)], dim=1)


def sh_colour(sh: torch.Tensor, d: torch.Tensor, degree: int) -> torch.Tensor:
    """rgb = sigmoid(sum_k beta_k Y_k(d)); sh is (K*3, n) with plane k*3+c."""
    Y = sh_basis(d, degree)                               # (n, K)
    K = Y.shape[1]
    beta = sh[: K * 3].reshape(K, 3, -1).permute(2, 0, 1) # (n, K, 3)
    return torch.sigmoid(torch.einsum("nk,nkc->nc", Y, beta))


# ==========================================================================
# EWA projection (inherited 3DGS step, section 4.4)
# ==========================================================================

def project(mu_cond, S_cond, cam):
    """Camera-space mean t, 2D mean, 2D covariance (dilated), conic, radius.

    J is the Jacobian of the pinhole map at t, with x/z and y/z clamped to
    +-1.3 tan(half fov) for J only."""
    W = torch.as_tensor(np.asarray(cam.world_to_cam, dtype=np.float64))
    R, tw = W[:, :3], W[:, 3]
    t = mu_cond @ R.T + tw[None, :]
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    limx = FRUSTUM_GUARD * (cam.width / 2.0) / cam.fx
    limy = FRUSTUM_GUARD * (cam.height / 2.0) / cam.fy
    txc = torch.clamp(tx / tz, -limx, limx) * tz
    tyc = torch.clamp(ty / tz, -limy, limy) * tz
    zeros = torch.zeros_like(tz)
    J = torch.stack([
        torch.stack([cam.fx / tz, zeros, -cam.fx * txc / (tz * tz)], dim=1),
        torch.stack([zeros, cam.fy / tz, -cam.fy * tyc / (tz * tz)], dim=1)], dim=1)
    T = J @ R[None]
    cov2d = T @ S_cond @ T.transpose(1, 2)
    a = cov2d[:, 0, 0] + DILATION
    b = cov2d[:, 0, 1]
    c = cov2d[:, 1, 1] + DILATION
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], dim=1)
    mid = 0.5 * (a + c)
    lam_max = mid + torch.sqrt(torch.clamp(mid * mid - det, min=0.0))
    radius = RADIUS_SIGMAS * torch.sqrt(lam_max)
    u = cam.fx * tx / tz + cam.cx
    v = cam.fy * ty / tz + cam.cy
    return t, torch.stack([u, v], dim=1), torch.stack([a, b, c], dim=1), det, conic, radius


def tile_rect(mean2d, radius, cam, tile_w, tile_h, radius_y=None):
    """Tiles whose pixel span meets [u-r, u+r] x [v-ry, v+ry] (ry = r unless
    given): x in [floor((u-r)/tw), floor((u+r)/tw)] clamped to the grid, same
    for y.  Returns int64 (n, 4): x0, x1 (exclusive), y0, y1 (exclusive)."""
    ry = radius if radius_y is None else radius_y
    tiles_x = (cam.width + tile_w - 1) // tile_w
    tiles_y = (cam.height + tile_h - 1) // tile_h
    u, v = mean2d[:, 0], mean2d[:, 1]
    x0 = torch.floor((u - radius) / tile_w).clamp(0, tiles_x)
    x1 = (torch.floor((u + radius) / tile_w) + 1).clamp(0, tiles_x)
    y0 = torch.floor((v - ry) / tile_h).clamp(0, tiles_y)
    y1 = (torch.floor((v + ry) / tile_h) + 1).clamp(0, tiles_y)
    return torch.stack([x0, x1, y0, y1], dim=1).to(torch.int64)


def alpha_box(cov2d, alpha_cond):
    """Half-extents (hx, hy) of the bounding box of the alpha >= 1/255 ellipse
    {Delta : alpha_cond exp(-1/2 Delta^T conic Delta) >= 1/255}, i.e.
    Delta^T Sigma2D^-1 Delta <= L2 = 2 ln(255 alpha_cond): sqrt(L2 Sigma2D_ii)
    per axis (the extent of an ellipse along an axis), widened by
    ALPHA_BOX_REL relative and ALPHA_BOX_ABS pixels.  Also returns
    d(hx)/d(L2), d(hy)/d(L2), the sensitivity of each extent to L2."""
    L2 = torch.clamp(2.0 * torch.log(255.0 * alpha_cond), min=0.0)
    sx, sy = cov2d[:, 0], cov2d[:, 2]
    hx = torch.sqrt(L2 * sx) * (1.0 + ALPHA_BOX_REL) + ALPHA_BOX_ABS
    hy = torch.sqrt(L2 * sy) * (1.0 + ALPHA_BOX_REL) + ALPHA_BOX_ABS
    root = torch.sqrt(torch.clamp(L2, min=1e-300))
    return hx, hy, 0.5 * torch.sqrt(sx) / root, 0.5 * torch.sqrt(sy) / root


# ==========================================================================
# One view, all Gaussians
# ==========================================================================

@dataclasses.dataclass
class ViewPrep:
    depth: torch.Tensor     # t_z (n,)
    mean2d: torch.Tensor    # (n, 2)
    conic: torch.Tensor     # (n, 3)  entries (a, b, c) of the inverse 2D covariance
    radius: torch.Tensor    # (n,)
    alpha_cond: torch.Tensor
    rgb: torch.Tensor       # (n, 3)
    rect: torch.Tensor      # (n, 4) int64
    valid: torch.Tensor     # (n,) bool
    # decision margins (float64, no grad): distance of each cull/rect decision
    near_margin: torch.Tensor
    alpha_cond_logmargin: torch.Tensor
    rect_edges: torch.Tensor  # (n, 4) (u-ex)/tw, (u+ex)/tw, (v-ey)/th, (v+ey)/th
    # d(extent)/d(L2) per axis where the alpha box sets the extent, else 0
    rect_box_gain: torch.Tensor = None


def to_params(scene, requires_grad=False, idx=None):
    """Scene planes as float64 tensors (optionally a subset of Gaussians)."""
    out = {}
    for k, v in scene.planes().items():
        a = np.asarray(v, dtype=np.float64)
        if idx is not None:
            a = a[..., idx]
        t = torch.tensor(a, dtype=F64)
        t.requires_grad_(requires_grad)
        out[k] = t
    return out


def prepare_view(p, sh_degree, cam, settings: Settings) -> ViewPrep:
    """Slice + colour + projection + tile rectangle of every Gaussian."""
    mu_p = p["mu_p"].T
    mu_d = p["mu_d"].T
    L = cholesky_factor(p["l_raw"])
    A, S_d_inv, S_cond = condition(covariance(L))
    alpha = torch.sigmoid(p["opacity_logit"])
    # lambda_opa: the global hyper-parameter, or per Gaussian (section 4.2),
    # parametrised as sigmoid(raw) so that 0 < lambda_opa < 1
    lam = torch.sigmoid(p["lambda_raw"]) if "lambda_raw" in p else settings.lambda_opa
    d = view_direction(mu_p, cam.campos)
    mu_cond, D, alpha_cond = slice_at(mu_p, mu_d, A, S_d_inv, alpha, d, lam)
    rgb = sh_colour(p["sh"], d, sh_degree)
    t, mean2d, cov2d, det, conic, radius = project(mu_cond, S_cond, cam)
    if settings.alpha_footprint:
        hx, hy, gx, gy = alpha_box(cov2d.detach(), alpha_cond.detach())
        ex, ey = torch.minimum(radius.detach(), hx), torch.minimum(radius.detach(), hy)
        gain = torch.stack([torch.where(hx <= radius.detach() + ALPHA_BOX_ABS, gx, 0.0 * gx),
                            torch.where(hy <= radius.detach() + ALPHA_BOX_ABS, gy, 0.0 * gy)], dim=1)
    else:
        ex = ey = radius.detach()
        gain = torch.zeros((radius.shape[0], 2), dtype=radius.dtype)
    rect = tile_rect(mean2d.detach(), ex, cam, settings.tile_w, settings.tile_h, ey)
    depth = t[:, 2]
    with torch.no_grad():
        ok_near = depth > cam.znear
        ok_det = det > 0
        ok_alpha = alpha_cond >= ALPHA_MIN
        ok_rect = (rect[:, 0] < rect[:, 1]) & (rect[:, 2] < rect[:, 3])
        valid = ok_near & ok_det & ok_alpha & ok_rect
        u, v = mean2d[:, 0], mean2d[:, 1]
        edges = torch.stack([(u - ex) / settings.tile_w, (u + ex) / settings.tile_w,
                             (v - ey) / settings.tile_h, (v + ey) / settings.tile_h], dim=1)
        prep = ViewPrep(depth, mean2d, conic, radius, alpha_cond, rgb, rect, valid,
                        (depth - cam.znear).detach(),
                        (torch.log(alpha_cond) - math.log(ALPHA_MIN)).detach(), edges.detach(),
                        torch.nan_to_num(gain.detach(), nan=0.0, posinf=0.0))
    return prep


def tile_grid(cam, settings: Settings):
    tx = (cam.width + settings.tile_w - 1) // settings.tile_w
    ty = (cam.height + settings.tile_h - 1) // settings.tile_h
    return tx, ty


def tile_list(prep: ViewPrep, tile_x: int, tile_y: int) -> np.ndarray:
    """Ids of valid Gaussians whose rect holds the tile, sorted by (depth, id)."""
    rect = prep.rect
    m = (prep.valid & (rect[:, 0] <= tile_x) & (tile_x < rect[:, 1])
         & (rect[:, 2] <= tile_y) & (tile_y < rect[:, 3]))
    ids = torch.nonzero(m).flatten().numpy()
    depth = prep.depth.detach().numpy()[ids]
    order = np.lexsort((ids, depth))
    return ids[order]


# ==========================================================================
# Per-pixel blend (inherited 3DGS step)
# ==========================================================================

def pixel_alpha(prep: ViewPrep, ids, px, py):
    """alpha_i(pixel) = min(0.99, alpha_cond_i * exp(-1/2 Delta^T conic_i Delta))
    for pixel centres (px+0.5, py+0.5); returns (P, n)."""
    mu = prep.mean2d[ids]
    con = prep.conic[ids]
    dx = mu[None, :, 0] - (px[:, None] + 0.5)
    dy = mu[None, :, 1] - (py[:, None] + 0.5)
    power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) - con[None, :, 1] * dx * dy
    g = prep.alpha_cond[ids][None, :] * torch.exp(power)
    return torch.clamp(g, max=ALPHA_MAX)


def blend(alpha: torch.Tensor, rgb: torch.Tensor, bg):
    """Front-to-back compositing of ordered lists, one row per pixel.

    alpha: (P, n) per-pixel alphas in list order; rgb: (n, 3).
    A term with alpha < 1/255 is skipped; the walk stops (excluding the
    current term) as soon as T * (1 - alpha) < 1e-4.  Returns colour (P, 3),
    final transmittance (P,), number of list entries walked (P,) and the
    weights (P, n) with T_i = prod_{j<i, kept} (1 - alpha_j)."""
    P, n = alpha.shape
    bg_t = torch.as_tensor(bg, dtype=F64)
    if n == 0:
        return (bg_t[None, :].expand(P, 3).clone(), torch.ones(P, dtype=F64),
                torch.zeros(P, dtype=torch.int64), alpha)
    skip = alpha < ALPHA_MIN
    a = torch.where(skip, torch.zeros_like(alpha), alpha)
    prod = torch.cumprod(1.0 - a, dim=1)
    stop_here = (~skip) & (prod < T_MIN)
    any_stop = stop_here.any(dim=1)
    first = torch.where(any_stop, torch.argmax(stop_here.to(torch.int8), dim=1),
                        torch.full((P,), n, dtype=torch.int64))
    T_ext = torch.cat([torch.ones((P, 1), dtype=F64), prod], dim=1)
    T_excl = T_ext[:, :n]
    keep = (torch.arange(n)[None, :] < first[:, None]) & (~skip)
    w = torch.where(keep, a * T_excl, torch.zeros_like(a))
    T_final = torch.gather(T_ext, 1, first[:, None])[:, 0]
    C = w @ rgb + T_final[:, None] * bg_t[None, :]
    return C, T_final, first, w


def blend_pixel_sequential(alpha, rgb, bg, flip=None):
    """The compositing loop written out for one pixel with Python floats.

    ``flip`` = (kind, i) inverts one decision: kind 'skip' inverts the
    alpha < 1/255 test at entry i, kind 'stop' inverts the T*(1-alpha) < 1e-4
    test at entry i.  Used by the tests to enumerate borderline outcomes."""
    T = 1.0
    C = [0.0, 0.0, 0.0]
    for i in range(len(alpha)):
        a = float(alpha[i])
        skip = a < ALPHA_MIN
        if flip is not None and flip == ("skip", i):
            skip = not skip
        if skip:
            continue
        test_T = T * (1.0 - a)
        stop = test_T < T_MIN
        if flip is not None and flip == ("stop", i):
            stop = not stop
        if stop:
            break
        for c in range(3):
            C[c] += float(rgb[i][c]) * a * T
        T = test_T
    return [C[c] + T * float(bg[c]) for c in range(3)]


def tile_pixels(cam, settings: Settings, tile_x, tile_y):
    """Pixel coordinates (px, py) of a tile clipped to the image."""
    x0, y0 = tile_x * settings.tile_w, tile_y * settings.tile_h
    xs = torch.arange(x0, min(x0 + settings.tile_w, cam.width), dtype=F64)
    ys = torch.arange(y0, min(y0 + settings.tile_h, cam.height), dtype=F64)
    py, px = torch.meshgrid(ys, xs, indexing="ij")
    return px.reshape(-1), py.reshape(-1), len(xs), len(ys)


def render_tile(prep: ViewPrep, cam, settings: Settings, tile_x, tile_y, ids=None):
    """Colour block (3, h, w) of one tile, plus its list and blend state."""
    if ids is None:
        ids = tile_list(prep, tile_x, tile_y)
    px, py, w, h = tile_pixels(cam, settings, tile_x, tile_y)
    ids_t = torch.as_tensor(np.asarray(ids, dtype=np.int64))
    alpha = pixel_alpha(prep, ids_t, px, py)
    C, T_final, walked, weights = blend(alpha, prep.rgb[ids_t], settings.bg)
    return C.T.reshape(3, h, w), ids, alpha, T_final, walked


def render_view(scene, cam, settings: Settings, tiles=None, params=None):
    """Full image (3, H, W) float64, or only the listed (tile_x, tile_y) tiles
    (other pixels NaN).  Returns the image and the ViewPrep."""
    p = params if params is not None else to_params(scene)
    with torch.set_grad_enabled(params is not None and any(t.requires_grad for t in p.values())):
        prep = prepare_view(p, scene.sh_degree, cam, settings)
    tx, ty = tile_grid(cam, settings)
    if tiles is None:
        tiles = [(x, y) for y in range(ty) for x in range(tx)]
    img = torch.full((3, cam.height, cam.width), float("nan"), dtype=F64)
    with torch.no_grad():
        for (x, y) in tiles:
            block = render_tile(prep, cam, settings, x, y)[0]
            x0, y0 = x * settings.tile_w, y * settings.tile_h
            img[:, y0:y0 + block.shape[1], x0:x0 + block.shape[2]] = block
    return img, prep


def render(scene, cams, settings: Settings | None = None):
    """Images of every camera, float64 numpy (3, H, W) each."""
    settings = settings or Settings()
    return [render_view(scene, c, settings)[0].numpy() for c in cams]


# ==========================================================================
# Loss (section 4.4: the 3DGS L1 term)
# ==========================================================================

def l1_loss(images, targets):
    """L = mean |I - I*| over every value of every image; dL/dI = sign(I - I*)/M
    with sign(0) = 0."""
    M = sum(int(np.asarray(i).size) for i in images)
    loss = sum(float(np.abs(np.asarray(i, np.float64) - np.asarray(t, np.float64)).sum())
               for i, t in zip(images, targets)) / M
    grads = [np.sign(np.asarray(i, np.float64) - np.asarray(t, np.float64)) / M
             for i, t in zip(images, targets)]
    return loss, grads


# ==========================================================================
# Gradients: autograd of the forward definition above
# ==========================================================================

def gradients(scene, cams, grad_images, settings: Settings | None = None, tiles=None):
    """dL/dparams for L = sum_v <grad_images[v], image_v>.

    ``tiles`` optionally restricts each view to a list of tiles (the caller
    guarantees grad_images is zero elsewhere).  Only Gaussians present in a
    used tile list can receive gradient; they are found with a no-grad pass
    and re-evaluated with autograd.  Returns a dict of float64 arrays shaped
    like the scene planes."""
    settings = settings or Settings()
    base = to_params(scene)
    lists = []
    involved = set()
    for vi, cam in enumerate(cams):
        with torch.no_grad():
            prep = prepare_view(base, scene.sh_degree, cam, settings)
        tx, ty = tile_grid(cam, settings)
        tl = tiles[vi] if tiles is not None else [(x, y) for y in range(ty) for x in range(tx)]
        per = []
        for (x, y) in tl:
            ids = tile_list(prep, x, y)
            per.append((x, y, ids))
            involved.update(ids.tolist())
        lists.append(per)
    out = {k: np.zeros(np.asarray(v).shape, dtype=np.float64) for k, v in scene.planes().items()}
    if not involved:
        return out
    sub = np.array(sorted(involved), dtype=np.int64)
    remap = {g: i for i, g in enumerate(sub.tolist())}
    p = to_params(scene, requires_grad=True, idx=sub)
    total = torch.zeros((), dtype=F64)
    for vi, cam in enumerate(cams):
        prep = prepare_view(p, scene.sh_degree, cam, settings)
        g_img = torch.as_tensor(np.asarray(grad_images[vi], dtype=np.float64))
        for (x, y, ids) in lists[vi]:
            if len(ids) == 0:
                continue
            local = np.array([remap[i] for i in ids.tolist()], dtype=np.int64)
            block = render_tile(prep, cam, settings, x, y, ids=local)[0]
            x0, y0 = x * settings.tile_w, y * settings.tile_h
            g = g_img[:, y0:y0 + block.shape[1], x0:x0 + block.shape[2]]
            total = total + (g * block).sum()
    total.backward()
    for k in out:
        gk = p[k].grad
        if gk is not None:
            out[k][..., sub] = gk.numpy()
    return out
