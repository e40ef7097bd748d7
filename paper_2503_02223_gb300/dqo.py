"""Thin Python binding of libdqo.so (include/dqo.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes torch tensors'
device pointers and the current CUDA stream through ctypes; all arithmetic runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  There is no
fallback: if the library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

c_f = C.c_float
c_i32 = C.c_int32
c_i64 = C.c_int64
c_p = C.c_void_p

DQO_OK, DQO_EINVAL, DQO_ENOMEM, DQO_ECUDA, DQO_ETIMEOUT, DQO_ENOTIMPL, DQO_ESTATE = range(7)
PHASES = ("project", "depth_sort", "binning", "blend_fwd", "blend_bwd", "project_bwd", "quadric", "blend_step")
(DQO_BUF_PROJ, DQO_BUF_RECT, DQO_BUF_DEPTH_ORDER, DQO_BUF_TILE_RANGES, DQO_BUF_TILE_LIST, DQO_BUF_T_FINAL,
 DQO_BUF_N_CONTRIB, DQO_BUF_GRAD2D) = range(8)


class dqo_settings(C.Structure):
    _fields_ = [("tile_w", c_i32), ("tile_h", c_i32), ("alpha_clamp", c_f), ("alpha_min", c_f), ("t_stop", c_f),
                ("znear", c_f), ("lowpass", c_f), ("radius_sigma", c_f), ("lambda_ins", c_f), ("bg", c_f * 3),
                ("og_filter", c_i32), ("batch", c_i32), ("theta_alpha", c_f), ("theta_d", c_f), ("theta_c", c_f),
                ("grads_zero", c_i32)]


class dqo_camera(C.Structure):
    _fields_ = [("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f), ("width", c_i32), ("height", c_i32),
                ("viewmat", c_f * 12)]


class dqo_gaussians(C.Structure):
    _fields_ = [("n", c_i64), ("num_objects", c_i32), ("means", c_p), ("log_scales", c_p), ("quats", c_p),
                ("opacity_logit", c_p), ("rgb", c_p), ("obj_id", c_p), ("flags", c_p)]


class dqo_targets(C.Structure):
    _fields_ = [("rgb", c_p), ("depth", c_p), ("gt_id", c_p)]


class dqo_render_out(C.Structure):
    _fields_ = [("rgb", c_p), ("depth", c_p), ("alpha", c_p), ("ins", c_p), ("id_map", c_p), ("loss", c_p),
                ("update_mask", c_p)]


class dqo_pixel_grads(C.Structure):
    _fields_ = [("rgb", c_p), ("depth", c_p), ("alpha", c_p), ("ins", c_p)]


class dqo_gaussian_grads(C.Structure):
    _fields_ = [("means", c_p), ("log_scales", c_p), ("quats", c_p), ("opacity_logit", c_p), ("rgb", c_p)]


# Exported entry points and their argument types (must match include/dqo.h).
_SIGS = {
    "dqo_settings_default": (None, [c_p]),
    "dqo_create": (c_i32, [c_p, C.c_int]),
    "dqo_destroy": (None, [c_p]),
    "dqo_status_str": (C.c_char_p, [c_i32]),
    "dqo_last_cuda_error": (C.c_int, [c_p]),
    "dqo_version": (C.c_int, []),
    "dqo_render_forward": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "dqo_render_backward": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "dqo_get_buffer": (c_i32, [c_p, c_i32, c_p, C.c_size_t, c_p, c_p]),
    "dqo_get_counts": (c_i32, [c_p, c_p, c_p, c_p]),
    "dqo_set_timing": (c_i32, [c_p, C.c_int]),
    "dqo_get_timings": (c_i32, [c_p, c_p, c_i32]),
    "dqo_launch_count": (c_i64, [c_p]),
    "dqo_depth_order_noalloc": (c_i32, [c_p, c_i64, c_p, c_p, c_p]),
    "dqo_quadric_project": (c_i32, [c_p, c_i32, c_p, c_i32, c_p, c_p, c_p, c_i32, c_p, c_p, c_p, c_p]),
    "dqo_quadric_bbox_loss": (c_i32, [c_p, c_i32, c_p, c_i32, c_p, c_p, c_p, c_i32, c_p, c_p, c_p, c_p]),
    "dqo_quadric_fit": (c_i32, [c_p, c_i32, c_i32, c_p, c_p, c_p, c_i32, c_p, c_i32, c_f, c_p, c_p, c_p, c_p, c_p,
                                c_p]),
    "dqo_quadric_canonical": (c_i32, [c_i32, c_p, c_p, c_p]),
    "dqo_batch_step": (c_i32, [c_p, c_p, c_i32, c_p, c_p, c_i32, c_i32, c_p]),
    "dqo_batch_check": (c_i32, [c_p, c_p, c_p]),
    "dqo_batch_tune": (c_i32, [c_p, c_p, c_i32, c_p, c_p, c_i32, c_p, c_p, c_p, c_p]),
    "dqo_mlp_features": (c_i32, [c_i32, c_i32, c_p, c_p, c_p, c_i32, c_p, c_p, c_f, c_p, c_p, c_i64, c_p]),
    "dqo_mlp_state_bytes": (C.c_size_t, []),
    "dqo_mlp_set_params": (c_i32, [c_p, c_p, c_p]),
    "dqo_mlp_get_params": (c_i32, [c_p, c_p, c_p]),
    "dqo_mlp_forward": (c_i32, [c_p, c_p, c_i64, c_p, c_p, c_p]),
    "dqo_mlp_gradients": (c_i32, [c_p, c_p, c_i64, c_p, c_p, c_p, c_p, c_p, c_p]),
    "dqo_mlp_train_step": (c_i32, [c_p, c_p, c_p, c_i64, c_p, c_p, c_p, c_p]),
    "dqo_mlp_train_steps": (c_i32, [c_p, c_p, c_p, c_i32, c_i64, c_p, c_p, c_p, c_p]),
    "dqo_mlp_check": (c_i32, [c_p, c_p]),
    "dqo_wait_probe": (c_i32, [c_p, c_p]),
    "dqo_alu_probe": (c_i32, [c_i32, c_i32, c_p, C.POINTER(C.c_double), c_p]),
}

class dqo_keyframe(C.Structure):
    _fields_ = [("gaussians", dqo_gaussians), ("camera", dqo_camera), ("targets", dqo_targets),
                ("out", dqo_render_out), ("grads", dqo_gaussian_grads)]


class dqo_fit_batch(C.Structure):
    _fields_ = [("nq", c_i32), ("nv", c_i32), ("npairs", c_i32), ("iters", c_i32), ("lr", c_f),
                ("P", c_p), ("q_ptr", c_p), ("pair_v", c_p), ("obs_bbox", c_p), ("start", c_p),
                ("init", c_p), ("params", c_p), ("loss", c_p), ("ok", c_p)]


MAX_BATCH = 16
MLP_FEATURES = 128
MLP_PARAMS = 35088
# offsets into the fp32 parameter vector
MLP_LAYOUT = {"W1": (0, (128, 128)), "b1": (16384, (128,)), "W2": (16512, (128, 128)), "b2": (32896, (128,)),
              "W3": (33024, (16, 128)), "b3": (35072, (16,))}


class dqo_mlp_hparams(C.Structure):
    _fields_ = [("lr", c_f), ("lr_final", c_f), ("total_steps", c_i64), ("beta1", c_f), ("beta2", c_f),
                ("eps", c_f), ("loss_w", c_f * 9)]

_lib = None
_lock = threading.Lock()


class DqoError(RuntimeError):
    def __init__(self, fn, status, cuda_err=0):
        msg = f"{fn} failed: status {status}"
        if _lib is not None:
            msg += f" ({_lib.dqo_status_str(status).decode()})"
        if cuda_err:
            msg += f", cudaError {cuda_err}"
        super().__init__(msg)
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libdqo.so; raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with paper_2503_02223_gb300.build.build()")
            _build.build()
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(fn: str, status: int, ctx=None):
    if status != DQO_OK:
        err = _lib.dqo_last_cuda_error(ctx) if ctx else 0
        raise DqoError(fn, status, err)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


# ------------------------------------------------------------------------ structs from python

def settings(**kw) -> dqo_settings:
    lib = load()
    s = dqo_settings()
    lib.dqo_settings_default(C.byref(s))
    for k, v in kw.items():
        if k == "bg":
            s.bg = (c_f * 3)(*v)
        else:
            setattr(s, k, v)
    return s


def camera(cam: dict) -> dqo_camera:
    c = dqo_camera()
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = cam["width"], cam["height"]
    vm = cam["viewmat"]
    vm = vm.reshape(-1).tolist() if hasattr(vm, "reshape") else list(vm)
    c.viewmat = (c_f * 12)(*vm)
    return c


_GAUSS_TYPES = dict(means=torch.float32, log_scales=torch.float32, quats=torch.float32,
                    opacity_logit=torch.float32, rgb=torch.float32, obj_id=torch.int32, flags=torch.uint8)


def gaussians(g: dict, num_objects: int) -> dqo_gaussians:
    """g: dict of contiguous CUDA tensors (means [n,3], log_scales [n,3], quats [n,4],
    opacity_logit [n], rgb [n,3], obj_id [n] int32, flags [n] uint8)."""
    for k, dt in _GAUSS_TYPES.items():
        if g[k].dtype != dt:
            raise ValueError(f"{k} must be {dt}, got {g[k].dtype}")
    s = dqo_gaussians()
    s.n = g["means"].shape[0]
    s.num_objects = num_objects
    for k in _GAUSS_TYPES:
        setattr(s, k, _ptr(g[k]))
    return s


def targets(t: dict | None):
    if t is None:
        return None
    s = dqo_targets()
    s.rgb = _ptr(t["rgb"])
    s.depth = _ptr(t.get("depth"))
    s.gt_id = _ptr(t["gt_id"])
    return s


def render_out(o: dict) -> dqo_render_out:
    s = dqo_render_out()
    for k in ("rgb", "depth", "alpha", "ins", "id_map", "loss", "update_mask"):
        setattr(s, k, _ptr(o.get(k)))
    return s


def pixel_grads(pg: dict | None):
    if pg is None:
        return None
    s = dqo_pixel_grads()
    for k in ("rgb", "depth", "alpha", "ins"):
        setattr(s, k, _ptr(pg.get(k)))
    return s


def gaussian_grads(gg: dict) -> dqo_gaussian_grads:
    s = dqo_gaussian_grads()
    for k in ("means", "log_scales", "quats", "opacity_logit", "rgb"):
        setattr(s, k, _ptr(gg.get(k)))
    return s


# ------------------------------------------------------------------------ entry points

class Context:
    """Owns a dqo_ctx (the library's workspace) on one device."""

    def __init__(self, device: int | None = None):
        lib = load()
        self.device = torch.cuda.current_device() if device is None else device
        h = c_p()
        _check("dqo_create", lib.dqo_create(C.byref(h), self.device))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            torch.cuda.synchronize(self.device)
            _lib.dqo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dqo_render_forward(ctx: Context, st: dqo_settings, g: dqo_gaussians, cam: dqo_camera, t, out: dqo_render_out,
                       stream=None):
    lib = load()
    tp = C.byref(t) if t is not None else None
    _check("dqo_render_forward",
           lib.dqo_render_forward(ctx.handle, C.byref(st), C.byref(g), C.byref(cam), tp, C.byref(out),
                                  _stream(stream)), ctx.handle)


def dqo_render_backward(ctx: Context, st: dqo_settings, g: dqo_gaussians, cam: dqo_camera, t, pg,
                        grads: dqo_gaussian_grads, stream=None):
    lib = load()
    tp = C.byref(t) if t is not None else None
    pp = C.byref(pg) if pg is not None else None
    _check("dqo_render_backward",
           lib.dqo_render_backward(ctx.handle, C.byref(st), C.byref(g), C.byref(cam), tp, pp, C.byref(grads),
                                   _stream(stream)), ctx.handle)


def dqo_get_buffer(ctx: Context, which: int, dst: torch.Tensor | None = None, stream=None):
    """Returns the buffer size in bytes; copies into dst (any device) when given."""
    lib = load()
    nbytes = C.c_size_t(0)
    _check("dqo_get_buffer", lib.dqo_get_buffer(ctx.handle, which, None, 0, C.byref(nbytes), _stream(stream)),
           ctx.handle)
    if dst is not None:
        cap = dst.numel() * dst.element_size()
        _check("dqo_get_buffer", lib.dqo_get_buffer(ctx.handle, which, dst.data_ptr(), cap, C.byref(nbytes),
                                                    _stream(stream)), ctx.handle)
    return nbytes.value


def dqo_get_counts(ctx: Context):
    lib = load()
    m, v, t = c_i64(0), c_i64(0), c_i32(0)
    _check("dqo_get_counts", lib.dqo_get_counts(ctx.handle, C.byref(m), C.byref(v), C.byref(t)), ctx.handle)
    return m.value, v.value, t.value


def dqo_set_timing(ctx: Context, enable: bool):
    _check("dqo_set_timing", load().dqo_set_timing(ctx.handle, 1 if enable else 0), ctx.handle)


def dqo_get_timings(ctx: Context) -> dict:
    """Device milliseconds per phase of the most recent timed calls (-1 if not run)."""
    buf = (c_f * len(PHASES))()
    _check("dqo_get_timings", load().dqo_get_timings(ctx.handle, buf, len(PHASES)), ctx.handle)
    return dict(zip(PHASES, list(buf)))


def dqo_launch_count(ctx: Context) -> int:
    return int(load().dqo_launch_count(ctx.handle))


def dqo_depth_order_noalloc(depth_keys: torch.Tensor, order: torch.Tensor, status: torch.Tensor | None = None,
                            stream=None):
    """Depth order without any device allocation (scratch lives in the library); see
    include/dqo.h.  depth_keys: uint32 bit patterns as an int32 CUDA tensor [n]; order:
    int32 CUDA tensor [n] receiving the sorted indices; status (optional): int32 CUDA
    tensor [1] set to 0 when the order is valid, 1 when a bounded sort wait gave up."""
    if depth_keys.dtype != torch.int32 or order.dtype != torch.int32:
        raise ValueError("depth_keys and order must be int32 tensors (uint32 bit patterns)")
    if order.numel() != depth_keys.numel():
        raise ValueError("order must have as many elements as depth_keys")
    if status is not None and (status.dtype != torch.int32 or status.numel() < 1):
        raise ValueError("status must be an int32 tensor of at least one element")
    _check("dqo_depth_order_noalloc",
           load().dqo_depth_order_noalloc(_ptr(depth_keys), depth_keys.numel(), _ptr(order), _ptr(status),
                                          _stream(stream)))


def dqo_quadric_project(ctx: Context, params, P, q_ptr, pair_v, conic=None, bbox=None, valid=None, stream=None):
    lib = load()
    _check("dqo_quadric_project",
           lib.dqo_quadric_project(ctx.handle, params.shape[0], _ptr(params), P.shape[0], _ptr(P), _ptr(q_ptr),
                                   _ptr(pair_v), pair_v.shape[0], _ptr(conic), _ptr(bbox), _ptr(valid),
                                   _stream(stream)), ctx.handle)


def dqo_quadric_bbox_loss(ctx: Context, params, P, q_ptr, pair_v, obs, loss=None, dparams=None, stream=None):
    lib = load()
    _check("dqo_quadric_bbox_loss",
           lib.dqo_quadric_bbox_loss(ctx.handle, params.shape[0], _ptr(params), P.shape[0], _ptr(P), _ptr(q_ptr),
                                     _ptr(pair_v), pair_v.shape[0], _ptr(obs), _ptr(loss), _ptr(dparams),
                                     _stream(stream)), ctx.handle)


def dqo_quadric_fit(ctx: Context, P, q_ptr, pair_v, obs, iters=100, lr=1e-2, init=None, params=None, loss=None,
                    ok=None, stream=None, start=None):
    lib = load()
    nq = q_ptr.shape[0] - 1
    _check("dqo_quadric_fit",
           lib.dqo_quadric_fit(ctx.handle, nq, P.shape[0], _ptr(P), _ptr(q_ptr), _ptr(pair_v), pair_v.shape[0],
                               _ptr(obs), iters, lr, _ptr(start), _ptr(init), _ptr(params), _ptr(loss), _ptr(ok),
                               _stream(stream)), ctx.handle)


def dqo_quadric_canonical(params, out=None, stream=None):
    out = torch.empty_like(params) if out is None else out
    _check("dqo_quadric_canonical", load().dqo_quadric_canonical(params.shape[0], _ptr(params), _ptr(out),
                                                                 _stream(stream)))
    return out


# ------------------------------------------------------------------------ batched step

def keyframe(g: dict, num_objects: int, cam: dict, t: dict, out: dict, grads: dict) -> dqo_keyframe:
    """One keyframe of a batch (the tensors must stay alive while the batch is used)."""
    k = dqo_keyframe()
    k.gaussians = gaussians(g, num_objects)
    k.camera = camera(cam)
    k.targets = targets(t)
    k.out = render_out(out)
    k.grads = gaussian_grads(grads)
    return k


def fit_batch(P, q_ptr, pair_v, obs, iters=100, lr=1e-2, start=None, init=None, params=None, loss=None,
              ok=None) -> dqo_fit_batch:
    f = dqo_fit_batch(nq=q_ptr.shape[0] - 1, nv=P.shape[0], npairs=pair_v.shape[0], iters=iters, lr=lr)
    for name, t in (("P", P), ("q_ptr", q_ptr), ("pair_v", pair_v), ("obs_bbox", obs), ("start", start),
                    ("init", init), ("params", params), ("loss", loss), ("ok", ok)):
        setattr(f, name, _ptr(t))
    return f


SCHEDULE_FUSED, SCHEDULE_SPLIT, SCHEDULE_PER_KEYFRAME = 0, 1, 2
TUNE_CANDIDATES = 21


def tune_candidate(i: int) -> tuple:
    """(tile_w, tile_h, ctas_per_sm, schedule) of autotuner candidate i."""
    w, h = ((16, 16), (8, 32), (32, 8))[i // 7]
    j = i % 7
    sched = SCHEDULE_FUSED if j < 3 else (SCHEDULE_SPLIT if j < 6 else SCHEDULE_PER_KEYFRAME)
    cps = 2 + j if j < 3 else (j - 1 if j < 6 else 0)
    return w, h, cps, sched


def dqo_batch_step(ctx: Context, st: dqo_settings, kfs: list, fits: dqo_fit_batch | None = None,
                   ctas_per_sm: int = 0, schedule: int = SCHEDULE_FUSED, stream=None):
    arr = (dqo_keyframe * len(kfs))(*kfs)
    _check("dqo_batch_step",
           load().dqo_batch_step(ctx.handle, C.byref(st), len(kfs), arr, None if fits is None else C.byref(fits),
                                 ctas_per_sm, schedule, _stream(stream)), ctx.handle)


def dqo_batch_check(ctx: Context) -> tuple[int, bool]:
    pairs, over = C.c_uint64(0), C.c_int(0)
    _check("dqo_batch_check", load().dqo_batch_check(ctx.handle, C.byref(pairs), C.byref(over)), ctx.handle)
    return int(pairs.value), bool(over.value)


def dqo_batch_tune(ctx: Context, st: dqo_settings, kfs: list, fits: dqo_fit_batch | None = None, reps: int = 3,
                   stream=None) -> tuple[int, int, list]:
    """Picks the fastest tile shape (written into st), CTAs per SM and schedule (returned),
    with every candidate's mean step time in ms (order of tune_candidate)."""
    arr = (dqo_keyframe * len(kfs))(*kfs)
    cps, sched = c_i32(0), c_i32(0)
    ms = (c_f * TUNE_CANDIDATES)()
    _check("dqo_batch_tune",
           load().dqo_batch_tune(ctx.handle, C.byref(st), len(kfs), arr, None if fits is None else C.byref(fits),
                                 reps, C.byref(cps), C.byref(sched), ms, _stream(stream)), ctx.handle)
    return int(cps.value), int(sched.value), list(ms)


# ------------------------------------------------------------------------ learned proposal

def mlp_hparams(lr=2e-3, lr_final=1e-5, total_steps=0, beta1=0.9, beta2=0.999, eps=1e-8,
                loss_w=(1, 1, 1, 1, 1, 1, 0.3, 0.3, 0.3)) -> dqo_mlp_hparams:
    h = dqo_mlp_hparams(lr=lr, lr_final=lr_final, total_steps=total_steps, beta1=beta1, beta2=beta2, eps=eps)
    for i, v in enumerate(loss_w):
        h.loss_w[i] = v
    return h


def dqo_mlp_features(P, q_ptr, pair_v, obs, counts=None, length_scale=1.0, X=None, XT=None, ldt=None,
                     stream=None):
    """Features [nq][128] (bfloat16) and optionally their transpose [128][ldt]."""
    nq = q_ptr.shape[0] - 1
    if X is None:
        X = torch.empty(nq, MLP_FEATURES, dtype=torch.bfloat16, device=q_ptr.device)
    ld = 0 if XT is None else (XT.shape[1] if ldt is None else ldt)
    _check("dqo_mlp_features",
           load().dqo_mlp_features(nq, P.shape[0], _ptr(P), _ptr(q_ptr), _ptr(pair_v), pair_v.shape[0], _ptr(obs),
                                   _ptr(counts), length_scale, _ptr(X), _ptr(XT), ld, _stream(stream)))
    return X


class MlpState:
    """Device buffer holding the network's parameters, gradient, Adam moments and BF16 copies."""

    def __init__(self, device="cuda"):
        nbytes = load().dqo_mlp_state_bytes()
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)

    @property
    def handle(self) -> int:
        return self.buf.data_ptr()


def dqo_mlp_set_params(state: MlpState, params, stream=None):
    _check("dqo_mlp_set_params", load().dqo_mlp_set_params(state.handle, _ptr(params), _stream(stream)))


def dqo_mlp_get_params(state: MlpState, params=None, stream=None):
    params = torch.empty(MLP_PARAMS, device=state.buf.device) if params is None else params
    _check("dqo_mlp_get_params", load().dqo_mlp_get_params(state.handle, _ptr(params), _stream(stream)))
    return params


def dqo_mlp_forward(ctx: Context, state: MlpState, X, out=None, stream=None):
    out = torch.empty(X.shape[0], 9, device=X.device) if out is None else out
    _check("dqo_mlp_forward", load().dqo_mlp_forward(ctx.handle, state.handle, X.shape[0], _ptr(X), _ptr(out),
                                                     _stream(stream)), ctx.handle)
    return out


def dqo_mlp_gradients(ctx: Context, state: MlpState, X, labels, loss_w, grads=None, loss=None, stream=None):
    grads = torch.empty(MLP_PARAMS, device=X.device) if grads is None else grads
    loss = torch.empty(1, device=X.device) if loss is None else loss
    w = (c_f * 9)(*[float(v) for v in loss_w])
    _check("dqo_mlp_gradients",
           load().dqo_mlp_gradients(ctx.handle, state.handle, X.shape[0], _ptr(X), _ptr(labels), C.cast(w, c_p),
                                    _ptr(grads), _ptr(loss), _stream(stream)), ctx.handle)
    return grads, loss


def dqo_mlp_train_step(ctx: Context, state: MlpState, hp: dqo_mlp_hparams, X, labels, loss=None, stream=None):
    """One Adam step on the batch X [n][128] (contiguous rows; may be a row slice of a larger
    feature matrix)."""
    _check("dqo_mlp_train_step",
           load().dqo_mlp_train_step(ctx.handle, state.handle, C.byref(hp), X.shape[0], _ptr(X), _ptr(labels),
                                     _ptr(loss), _stream(stream)), ctx.handle)


def dqo_mlp_train_steps(ctx: Context, state: MlpState, hp: dqo_mlp_hparams, X, labels, batch: int, losses=None,
                        stream=None):
    """X.shape[0] // batch Adam steps in one launch, step k on rows [k batch, (k + 1) batch) of
    X [steps * batch][128] and labels; losses (device, one float per step) may be None."""
    steps = X.shape[0] // batch
    if steps * batch != X.shape[0] or labels.shape[0] != X.shape[0]:
        raise ValueError("X and labels must hold a whole number of batches")
    if losses is not None and losses.numel() < steps:
        raise ValueError("losses must hold one float per step")
    _check("dqo_mlp_train_steps",
           load().dqo_mlp_train_steps(ctx.handle, state.handle, C.byref(hp), steps, batch, _ptr(X), _ptr(labels),
                                      _ptr(losses), _stream(stream)), ctx.handle)


def dqo_mlp_check(ctx: Context) -> bool:
    """True if a tensor-core completion wait ran out since the last check."""
    v = C.c_int(0)
    st = load().dqo_mlp_check(ctx.handle, C.byref(v))
    if st not in (DQO_OK, DQO_ETIMEOUT):
        _check("dqo_mlp_check", st, ctx.handle)
    return bool(v.value)


def dqo_wait_probe(ctx: Context, stream=None) -> int:
    """Runs the bounded-wait probe; returns the status (DQO_ETIMEOUT expected)."""
    return int(load().dqo_wait_probe(ctx.handle, _stream(stream)))


ALU_FMA, ALU_EX2 = 0, 1


def dqo_alu_probe(kind: int, iters: int, sink: torch.Tensor, stream=None) -> float:
    """Launches the FP32 FMA (kind 0) or ex2 (kind 1) throughput probe on every SM;
    returns the launch's operation count (flops, or exponentials)."""
    ops = C.c_double(0.0)
    _check("dqo_alu_probe", load().dqo_alu_probe(kind, iters, _ptr(sink), C.byref(ops), _stream(stream)))
    return ops.value


# ------------------------------------------------------------------------ conveniences

def to_device(arrays: dict, device="cuda") -> dict:
    """numpy dict -> contiguous CUDA tensors (same dtypes)."""
    out = {}
    for k, v in arrays.items():
        if v is None:
            out[k] = None
        elif hasattr(v, "dtype") and hasattr(v, "shape") and not isinstance(v, torch.Tensor):
            out[k] = torch.from_numpy(v.copy() if not v.flags["C_CONTIGUOUS"] else v).to(device)
        else:
            out[k] = v
    return out


def alloc_outputs(W: int, H: int, device="cuda", loss=True, id_map=True, mask=False) -> dict:
    f = dict(dtype=torch.float32, device=device)
    o = dict(rgb=torch.empty(H, W, 3, **f), depth=torch.empty(H, W, **f), alpha=torch.empty(H, W, **f),
             ins=torch.empty(H, W, **f))
    if id_map:
        o["id_map"] = torch.empty(H, W, dtype=torch.int32, device=device)
    if loss:
        o["loss"] = torch.zeros(4, **f)
    if mask:
        o["update_mask"] = torch.empty(H, W, dtype=torch.uint8, device=device)
    return o


def alloc_grads(n: int, device="cuda") -> dict:
    f = dict(dtype=torch.float32, device=device)
    return dict(means=torch.zeros(n, 3, **f), log_scales=torch.zeros(n, 3, **f), quats=torch.zeros(n, 4, **f),
                opacity_logit=torch.zeros(n, **f), rgb=torch.zeros(n, 3, **f))
