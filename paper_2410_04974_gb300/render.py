"""PyTorch-facing wrapper of the sixdgs C ABI.

PyTorch only provides device memory and streams here: every stage of the
render runs in the CUDA kernels of libsixdgs.so.  There is no CPU path; the
renderer refuses to run without a CUDA device and the library.
"""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

PARAM_NAMES = ("mu_p", "mu_d", "l_raw", "opacity_logit", "sh")


def _camera_struct(cam) -> _lib.Camera:
    c = _lib.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    w2c = np.asarray(cam.world_to_cam, dtype=np.float64).reshape(3, 4)
    for i in range(12):
        c.world_to_cam[i] = float(w2c.reshape(-1)[i])
    for i in range(3):
        c.campos[i] = float(np.asarray(cam.campos, dtype=np.float64)[i])
    c.znear = float(getattr(cam, "znear", 0.2))
    return c


def camera_array(cams):
    arr = (_lib.Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = _camera_struct(c)
    return arr


def make_settings(tile=(16, 16), batch=512, lambda_opa=0.35, bg=(1.0, 1.0, 1.0), store_aux=False,
                  spin_budget=0, loss_norm=0.0, count_pairs=False, persistent=False,
                  inference=False, alpha_footprint=True) -> _lib.Settings:
    s = _lib.Settings()
    s.tile_w, s.tile_h = int(tile[0]), int(tile[1])
    s.batch = int(batch)
    s.lambda_opa = float(lambda_opa)
    for i in range(3):
        s.bg[i] = float(bg[i])
    s.store_aux = 1 if store_aux else 0
    s.spin_budget = int(spin_budget)
    s.loss_norm = float(loss_norm)
    s.count_pairs = 1 if count_pairs else 0
    s.persistent = 1 if persistent else 0
    s.inference = 1 if inference else 0
    s.alpha_footprint = 1 if alpha_footprint else 0
    return s


def make_plan(n, sh_degree, cams, settings, dup_capacity=0) -> _lib.Plan:
    lib = _lib.load()
    plan = _lib.Plan()
    arr = camera_array(cams)
    _lib.check(lib.sixdgs_plan_init(int(n), int(sh_degree), arr, len(cams), ctypes.byref(settings),
                                    int(dup_capacity), ctypes.byref(plan)), "sixdgs_plan_init")
    return plan


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


OPTIONAL_PARAMS = ("lambda_raw",)


def params_to_device(scene, device="cuda"):
    """Scene planes (synth.Scene or dict of arrays) as contiguous float32 device
    tensors; includes the optional per-Gaussian lambda_raw plane when present."""
    planes = scene.planes() if hasattr(scene, "planes") else scene
    names = list(PARAM_NAMES) + [k for k in OPTIONAL_PARAMS if planes.get(k) is not None]
    return {k: torch.as_tensor(np.asarray(planes[k], dtype=np.float32)).to(device).contiguous() for k in names}


class Renderer:
    """Plan + workspace of one frame shape (scene size, cameras, settings).

    One frame may be in flight per renderer: forward() followed by at most
    one backward() on the same stream.
    """

    def __init__(self, n, sh_degree, cameras, tile=(16, 16), batch=512, lambda_opa=0.35,
                 bg=(1.0, 1.0, 1.0), store_aux=False, dup_capacity=0, spin_budget=0, loss_norm=0.0,
                 count_pairs=False, persistent=False, inference=False, alpha_footprint=True,
                 device="cuda"):
        if not torch.cuda.is_available():
            raise _lib.SixDGSError("sixdgs needs a CUDA device; there is no CPU path")
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.cameras = list(cameras)
        self.settings = make_settings(tile, batch, lambda_opa, bg, store_aux, spin_budget, loss_norm,
                                      count_pairs, persistent, inference, alpha_footprint)
        self.cams = camera_array(self.cameras)
        self._make_plan(dup_capacity)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.sizes = [(int(c.height), int(c.width)) for c in self.cameras]

    def _make_plan(self, dup_capacity):
        self.plan = make_plan(self.n, self.sh_degree, self.cameras, self.settings, dup_capacity)
        self.ws = torch.empty(int(self.plan.ws_bytes), dtype=torch.uint8, device=self.device)

    # ---- structs --------------------------------------------------------
    def scene_struct(self, params) -> _lib.Scene:
        s = _lib.Scene()
        s.n, s.sh_degree = self.n, self.sh_degree
        for k in PARAM_NAMES + OPTIONAL_PARAMS + ("cond_cache",):
            t = params.get(k)
            if t is None:
                continue
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous(), k
            setattr(s, k, t.data_ptr())
        return s

    def _stream(self, stream=None):
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _wsargs(self):
        return ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws.numel())

    @property
    def total_pixels(self) -> int:
        return int(self.plan.total_pixels)

    def new_images(self):
        return torch.empty(3 * self.total_pixels, dtype=torch.float32, device=self.device)

    def split(self, flat):
        """Per-camera (3, H, W) views of a packed image buffer."""
        out, o = [], 0
        for (h, w) in self.sizes:
            out.append(flat[o:o + 3 * h * w].view(3, h, w))
            o += 3 * h * w
        return out

    def pack(self, images):
        return torch.cat([torch.as_tensor(i, dtype=torch.float32).reshape(-1) for i in images]).to(self.device)

    # ---- stages -----------------------------------------------------------
    def condition_project(self, params, stream=None):
        ws, nb = self._wsargs()
        sc = self.scene_struct(params)
        _lib.check(self.lib.sixdgs_condition_project(ctypes.byref(self.plan), ctypes.byref(sc), self.cams,
                                                     ws, nb, _ptr(self.status), self._stream(stream)),
                   "sixdgs_condition_project")

    def bin_sort(self, stream=None):
        ws, nb = self._wsargs()
        _lib.check(self.lib.sixdgs_bin_sort(ctypes.byref(self.plan), ws, nb, _ptr(self.status),
                                            self._stream(stream)), "sixdgs_bin_sort")

    def raster_fwd(self, images, targets=None, grad_images=None, loss=None, stream=None):
        ws, nb = self._wsargs()
        _lib.check(self.lib.sixdgs_raster_fwd(ctypes.byref(self.plan), ws, nb, _ptr(images), _ptr(targets),
                                              _ptr(grad_images), _ptr(loss), _ptr(self.status),
                                              self._stream(stream)), "sixdgs_raster_fwd")

    def raster_fwd_bwd(self, images, targets, grad_images=None, loss=None, stream=None):
        """Forward blend, fused L1 loss and backward blend in one kernel
        (sixdgs_raster_fwd_bwd); follow with project_bwd.  The loss
        accumulates into `loss` (default: self.loss, not zeroed here)."""
        ws, nb = self._wsargs()
        loss = self.loss if loss is None else loss
        _lib.check(self.lib.sixdgs_raster_fwd_bwd(ctypes.byref(self.plan), ws, nb, _ptr(images), _ptr(targets),
                                                  _ptr(grad_images), _ptr(loss), _ptr(self.status),
                                                  self._stream(stream)), "sixdgs_raster_fwd_bwd")

    def raster_bwd(self, params, images, grad_images, grads, accumulate=False, stream=None):
        ws, nb = self._wsargs()
        sc = self.scene_struct(params)
        _lib.check(self.lib.sixdgs_raster_bwd(ctypes.byref(self.plan), ctypes.byref(sc), ws, nb,
                                              _ptr(images), _ptr(grad_images), _ptr(grads["mu_p"]),
                                              _ptr(grads["mu_d"]), _ptr(grads["l_raw"]),
                                              _ptr(grads["opacity_logit"]), _ptr(grads["sh"]),
                                              _ptr(grads.get("lambda_raw")), int(accumulate), _ptr(self.status),
                                              self._stream(stream)),
                   "sixdgs_raster_bwd")

    def blend_bwd(self, images, grad_images, stream=None):
        ws, nb = self._wsargs()
        _lib.check(self.lib.sixdgs_blend_bwd(ctypes.byref(self.plan), ws, nb, _ptr(images), _ptr(grad_images),
                                             _ptr(self.status), self._stream(stream)), "sixdgs_blend_bwd")

    def project_bwd(self, params, grads, accumulate=False, stream=None):
        ws, nb = self._wsargs()
        sc = self.scene_struct(params)
        _lib.check(self.lib.sixdgs_project_bwd(ctypes.byref(self.plan), ctypes.byref(sc), ws, nb,
                                               _ptr(grads["mu_p"]), _ptr(grads["mu_d"]), _ptr(grads["l_raw"]),
                                               _ptr(grads["opacity_logit"]), _ptr(grads["sh"]),
                                               _ptr(grads.get("lambda_raw")), int(accumulate),
                                               _ptr(self.status), self._stream(stream)), "sixdgs_project_bwd")

    def step(self, params, images, targets=None, grad_images=None, grads=None, stream=None):
        """The whole frame in one library call (sixdgs_render_batched): forward
        only without targets, else forward + L1 loss (into self.loss) +
        backward into `grads` (overwritten)."""
        ws, nb = self._wsargs()
        sc = self.scene_struct(params)
        g = grads or {}
        _lib.check(self.lib.sixdgs_render_batched(
            ctypes.byref(self.plan), ctypes.byref(sc), self.cams, ws, nb, _ptr(images), _ptr(targets),
            _ptr(grad_images), _ptr(self.loss) if targets is not None else None, _ptr(g.get("mu_p")),
            _ptr(g.get("mu_d")), _ptr(g.get("l_raw")), _ptr(g.get("opacity_logit")), _ptr(g.get("sh")),
            _ptr(g.get("lambda_raw")), _ptr(self.status), self._stream(stream)), "sixdgs_render_batched")

    def set_cameras(self, cameras):
        """Swap in cameras of the same sizes (same plan and workspace)."""
        cameras = list(cameras)
        if [(int(c.height), int(c.width)) for c in cameras] != self.sizes:
            raise _lib.SixDGSError("set_cameras needs cameras of the planned sizes")
        self.cameras = cameras
        self.cams = camera_array(cameras)

    def new_grads(self, params):
        return {k: torch.empty_like(params[k]) for k in PARAM_NAMES + OPTIONAL_PARAMS if k in params}

    # ---- frames -----------------------------------------------------------
    def forward(self, params, targets=None, stream=None, check=True):
        """Render every camera; returns the packed image buffer (and, with
        targets, the L1 gradient image and loss)."""
        for attempt in range(3):
            self.status.zero_()
            images = self.new_images()
            gi = loss = None
            if targets is not None:
                gi = torch.empty_like(images)
                self.loss.zero_()
                loss = self.loss
            self.condition_project(params, stream)
            self.bin_sort(stream)
            self.raster_fwd(images, targets, gi, loss, stream)
            if not check:
                break
            st = int(self.status.item())
            if st & (1 << _lib.ERR_CAPACITY):
                k = int(self.counts()[1])
                self._make_plan(int(k * 1.25) + 4096)
                continue
            self.raise_status(st)
            break
        if targets is not None:
            return images, gi, loss
        return images

    def backward(self, params, images, grad_images, stream=None, grads=None, accumulate=False):
        grads = grads if grads is not None else self.new_grads(params)
        self.raster_bwd(params, images, grad_images, grads, accumulate=accumulate, stream=stream)
        return grads

    def raise_status(self, st=None):
        st = int(self.status.item()) if st is None else st
        if st:
            raise _lib.SixDGSError("device status: " + ", ".join(_lib.status_names(st)))

    # ---- workspace inspection (tests, diagnostics) ----------------------
    def _section(self, idx, dtype, count):
        off = int(self.plan.off[idx])
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype)

    def counts(self):
        """[visible pairs, duplicates K] of the last bin_sort."""
        return self._section(_lib.WS_COUNTS, torch.int32, 2).cpu().numpy().astype(np.int64)

    def pair_counts(self):
        """[evaluated, compositing] (pixel, entry) pairs and (warp, entry)
        pairs walked by the last raster_fwd (needs count_pairs=True)."""
        return self._section(_lib.WS_COUNTS, torch.int64, 5)[2:].cpu().numpy()

    def records(self):
        return self._section(_lib.WS_REC, torch.float32, 12 * int(self.plan.n_pairs)).view(-1, 12)

    def ntiles(self):
        return self._section(_lib.WS_NTILES, torch.int32, int(self.plan.n_pairs))

    def rects(self):
        return self._section(_lib.WS_RECT, torch.int16, 4 * int(self.plan.n_pairs)).view(-1, 4)

    def sorted_pairs(self):
        k = int(self.counts()[1])
        return self._section(_lib.WS_SORTED, torch.int32, int(self.plan.dup_capacity))[:k]

    def ranges(self):
        return self._section(_lib.WS_RANGES, torch.int32, 2 * int(self.plan.total_tiles)).view(-1, 2)

    def grad_records(self):
        return self._section(_lib.WS_GRADREC, torch.float32, 12 * int(self.plan.n_pairs)).view(-1, 12)

    def tile_offsets(self):
        offs, o = [], 0
        tw, th = self.settings.tile_w, self.settings.tile_h
        for (h, w) in self.sizes:
            offs.append(o)
            o += ((w + tw - 1) // tw) * ((h + th - 1) // th)
        return offs


class RenderFunction(torch.autograd.Function):
    """images = render(params); backward through the hand-written kernels.
    lambda_raw (per-Gaussian lambda_opa) is optional: pass None to use the
    renderer's global lambda_opa."""

    @staticmethod
    def forward(ctx, renderer: Renderer, mu_p, mu_d, l_raw, opacity_logit, sh, lambda_raw=None):
        params = {"mu_p": mu_p.contiguous(), "mu_d": mu_d.contiguous(), "l_raw": l_raw.contiguous(),
                  "opacity_logit": opacity_logit.contiguous(), "sh": sh.contiguous()}
        if lambda_raw is not None:
            params["lambda_raw"] = lambda_raw.contiguous()
        images = renderer.forward(params)
        ctx.renderer = renderer
        ctx.params = params
        ctx.save_for_backward(images)
        return images

    @staticmethod
    def backward(ctx, grad_images):
        (images,) = ctx.saved_tensors
        g = ctx.renderer.backward(ctx.params, images, grad_images.contiguous())
        return None, g["mu_p"], g["mu_d"], g["l_raw"], g["opacity_logit"], g["sh"], g.get("lambda_raw")


def render(renderer: Renderer, params):
    """Differentiable render: packed images of every camera."""
    return RenderFunction.apply(renderer, *(params[k] for k in PARAM_NAMES), params.get("lambda_raw"))


def scale_rotation(l_raw, stream=None):
    """Per-Gaussian rotation (9, n) and scale (3, n) of the conditional
    covariance (section 4.3, Algorithm 1 steps 4-5), from the (21, n) raw
    Cholesky planes on the GPU."""
    lib = _lib.load()
    n = int(l_raw.shape[1])
    assert l_raw.is_cuda and l_raw.dtype == torch.float32 and l_raw.is_contiguous()
    rot = torch.empty((9, n), dtype=torch.float32, device=l_raw.device)
    scale = torch.empty((3, n), dtype=torch.float32, device=l_raw.device)
    status = torch.zeros(1, dtype=torch.int32, device=l_raw.device)
    s = stream if stream is not None else torch.cuda.current_stream(l_raw.device)
    _lib.check(lib.sixdgs_scale_rotation(n, _ptr(l_raw), _ptr(rot), _ptr(scale), _ptr(status),
                                         ctypes.c_void_p(s.cuda_stream)), "sixdgs_scale_rotation")
    return rot, scale, status


def condition_cache(params, stream=None):
    """View-independent slice state of every Gaussian (section 3.2, Eq. sigma;
    Algorithm 1 steps 1-3), a (25, n) device tensor.  Put it in the params
    dict under "cond_cache" and the forward projection reads it instead of
    recomputing it (same result, bit for bit); recompute it whenever l_raw or
    opacity_logit change."""
    lib = _lib.load()
    l_raw, logit = params["l_raw"], params["opacity_logit"]
    n = int(l_raw.shape[1])
    for t in (l_raw, logit):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    cache = torch.empty((_lib.COND_CACHE_PLANES, n), dtype=torch.float32, device=l_raw.device)
    s = stream if stream is not None else torch.cuda.current_stream(l_raw.device)
    _lib.check(lib.sixdgs_condition_cache(n, _ptr(l_raw), _ptr(logit), _ptr(cache),
                                          ctypes.c_void_p(s.cuda_stream)), "sixdgs_condition_cache")
    return cache
