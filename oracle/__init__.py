"""FP64 CPU oracle of the DQO-MAP hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg import this
package.  It wraps ``dqo_oracle.cpp`` (plain C++, double precision) through ctypes and
shares nothing with the CUDA library.  Every function cites the passage of DQO-MAP
(arXiv 2503.02223) it restates; the readings where the paper is silent are listed in
the C++ file's header.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dqo_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libdqo_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OSettings(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("alpha_clamp", C.c_double),
                ("alpha_min", C.c_double), ("t_stop", C.c_double), ("znear", C.c_double),
                ("lowpass", C.c_double), ("radius_sigma", C.c_double), ("lambda_ins", C.c_double),
                ("bg", C.c_double * 3), ("og_filter", C.c_int32), ("num_objects", C.c_int32),
                ("amb_rel", C.c_double), ("amb_px", C.c_double), ("theta_alpha", C.c_double),
                ("theta_d", C.c_double), ("theta_c", C.c_double)]


class OCamera(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("viewmat", C.c_double * 12)]


_P = C.c_void_p


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i64 = C.c_int64
            lib.oracle_preprocess.argtypes = [_P, _P, i64] + [_P] * 12
            lib.oracle_render.argtypes = [_P, _P, i64] + [_P] * 10 + [C.c_int] + [_P] * 14 + [C.c_int32] * 2
            lib.oracle_render_alternatives.argtypes = [_P, _P, i64] + [_P] * 8 + [i64, _P, C.c_int32, C.c_int32] + \
                [_P] * 6
            lib.oracle_render_pixels.argtypes = [_P, _P, i64] + [_P] * 8 + [i64] + [_P] * 10
            lib.oracle_render_backward.argtypes = [_P, _P, i64] + [_P] * 19
            lib.oracle_bin_tiles.argtypes = [i64, _P, _P, _P, C.c_int, C.c_int, _P, _P]
            lib.oracle_bin_tiles.restype = i64
            lib.oracle_quadric_project.argtypes = [C.c_int, _P, C.c_int, _P, _P, _P, _P, _P, _P]
            lib.oracle_quadric_bbox_loss.argtypes = [C.c_int, _P, C.c_int, _P, _P, _P, _P, _P, _P]
            lib.oracle_quadric_matrix.argtypes = [C.c_int, _P, _P]
            lib.oracle_quadric_fit.argtypes = [C.c_int, C.c_int, _P, _P, _P, _P, C.c_int, C.c_double,
                                               _P, _P, _P, _P, _P, _P]
            lib.oracle_jacobi_eigen.argtypes = [C.c_int, _P, _P]
            lib.oracle_rot_to_rotvec.argtypes = [_P, _P]
            lib.oracle_round_bf16.argtypes = [C.c_double]
            lib.oracle_round_bf16.restype = C.c_double
            lib.oracle_mlp_features.argtypes = [C.c_int, C.c_int, _P, _P, _P, _P, _P, C.c_double, _P]
            lib.oracle_mlp_forward.argtypes = [i64, _P, _P, C.c_int, _P, _P, _P]
            lib.oracle_mlp_backward.argtypes = [i64, _P, _P, _P, _P, C.c_int, _P, _P]
            lib.oracle_quadric_canonical.argtypes = [C.c_int, _P, _P]
            _lib = lib
    return _lib


# ------------------------------------------------------------------------- settings

DEFAULTS = dict(tile_w=16, tile_h=16, alpha_clamp=0.99, alpha_min=1.0 / 255.0, t_stop=1e-4,
                znear=0.2, lowpass=0.3, radius_sigma=3.0, lambda_ins=1.0, bg=(0.0, 0.0, 0.0),
                og_filter=1, num_objects=64, amb_rel=1e-4, amb_px=2e-3, theta_alpha=0.5, theta_d=0.1,
                theta_c=0.1)

# Smooth settings for finite differences: no skip, no stop, no clamp, wide cutoff.
SMOOTH = dict(alpha_min=0.0, t_stop=0.0, alpha_clamp=1.0, radius_sigma=9.0)


def settings(**kw) -> OSettings:
    d = dict(DEFAULTS)
    d.update(kw)
    s = OSettings()
    for k, v in d.items():
        if k == "bg":
            s.bg = (C.c_double * 3)(*v)
        else:
            setattr(s, k, v)
    return s


def camera(cam: dict) -> OCamera:
    c = OCamera()
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.width, c.height = cam["width"], cam["height"]
    c.viewmat = (C.c_double * 12)(*np.asarray(cam["viewmat"], np.float64).ravel())
    return c


def _d(a):
    return np.ascontiguousarray(a, np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _gauss(g):
    return (_d(g["means"]), _d(g["log_scales"]), _d(g["quats"]), _d(g["opacity_logit"]), _d(g["rgb"]),
            np.ascontiguousarray(g["obj_id"], np.int32), np.ascontiguousarray(g["flags"], np.uint8))


# ------------------------------------------------------------------------- rasterizer

def preprocess(g: dict, cam: dict, st: OSettings | None = None) -> dict:
    """Per-Gaussian EWA projection (3DGS, which the paper builds on; Sec. IV impl.)."""
    st = st or settings()
    m, s, q, o, _, _, _ = _gauss(g)
    n = m.shape[0]
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), z=np.zeros(n), opac=np.zeros(n),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               visible=np.zeros(n, np.uint8), ambiguous=np.zeros(n, np.uint8))
    oc = camera(cam)
    _lib_handle().oracle_preprocess(C.byref(st), C.byref(oc), n, _ptr(m), _ptr(s), _ptr(q), _ptr(o),
                                    *[_ptr(out[k]) for k in ("xy", "conic", "z", "opac", "radius", "rect",
                                                             "visible", "ambiguous")])
    return out


def _targets(t):
    if t is None:
        return None, None, None
    return _d(t["rgb"]), (None if t.get("depth") is None else _d(t["depth"])), np.ascontiguousarray(t["gt_id"], np.int32)


def render(g: dict, cam: dict, st: OSettings | None = None, targets: dict | None = None, mode: int = 0,
           rows: tuple | None = None) -> dict:
    """Front-to-back blend of RGB, depth, alpha, ins (Eq. 15 reading) and the object-id argmax,
    with the losses of Eq. 7-10 (reading: per-pixel L1 means over labelled pixels) and the
    incremental-update masks of Eq. 11 (update_mask bit0 Mask_geo, bit1 Mask_rgb).
    rows = (y0, y1): render only pixel rows y0 <= v < y1 (the others stay zero and add
    nothing to the losses).  last[v, u] = index of the pixel's last blended Gaussian (-1: none)."""
    st = st or settings()
    m, s, q, o, c, i, f = _gauss(g)
    n = m.shape[0]
    W, H = cam["width"], cam["height"]
    tr, td, tg = _targets(targets)
    out = dict(rgb=np.zeros((H, W, 3)), depth=np.zeros((H, W)), alpha=np.zeros((H, W)),
               ins=np.zeros((H, W)), id_map=np.zeros((H, W), np.int32), T_final=np.zeros((H, W)),
               n_contrib=np.zeros((H, W), np.int64), amb=np.zeros((H, W), np.uint8),
               id_margin=np.zeros((H, W)), loss=np.zeros(4), dl=np.zeros((H, W, 6)),
               update_mask=np.zeros((H, W), np.uint8), mask_amb=np.zeros((H, W), np.uint8),
               last=np.zeros((H, W), np.int64))
    oc = camera(cam)
    rc = _lib_handle().oracle_render(C.byref(st), C.byref(oc), n, _ptr(m), _ptr(s), _ptr(q), _ptr(o),
                                     _ptr(c), _ptr(i), _ptr(f), _ptr(tr), _ptr(td), _ptr(tg), mode,
                                     *[_ptr(out[k]) for k in ("rgb", "depth", "alpha", "ins", "id_map",
                                                              "T_final", "n_contrib", "amb", "id_margin",
                                                              "loss", "dl", "update_mask", "mask_amb", "last")],
                                     *(rows if rows is not None else (0, 0)))
    if rc:
        raise ValueError("oracle_render: invalid arguments")
    return out


def render_alternatives(g: dict, cam: dict, pxy, st: OSettings | None = None, gt_id=None, max_alt: int = 64,
                        full_items: int = 4) -> dict:
    """Every outcome a correct single-precision render may give at pixel centres
    pxy[k] = (u, v): the render with each subset of the pixel's near-threshold decisions
    (alpha skip / clamp / stop, uncertain tile membership) taken the other way (all subsets
    of up to `full_items` items, else those of one or two).  Returns count[k] and, per
    (k, alternative), vals[..., 7] = (r, g, b, depth, alpha, ins, T_final), n_contrib, id_map,
    id_margin, last (index of the last blended Gaussian, -1: none); alternative 0 is the render
    as it stands."""
    st = st or settings()
    m, s, q, o, c, i, f = _gauss(g)
    n = m.shape[0]
    pxy = np.ascontiguousarray(pxy, np.int32).reshape(-1, 2)
    k = pxy.shape[0]
    gt = None if gt_id is None else np.ascontiguousarray(gt_id, np.int32)
    out = dict(count=np.zeros(k, np.int32), vals=np.zeros((k, max_alt, 7)), n_contrib=np.zeros((k, max_alt), np.int64),
               id_map=np.zeros((k, max_alt), np.int32), id_margin=np.zeros((k, max_alt)),
               last=np.zeros((k, max_alt), np.int64))
    oc = camera(cam)
    rc = _lib_handle().oracle_render_alternatives(C.byref(st), C.byref(oc), n, _ptr(m), _ptr(s), _ptr(q), _ptr(o),
                                                  _ptr(c), _ptr(i), _ptr(f), _ptr(gt), k, _ptr(pxy), max_alt,
                                                  full_items, *[_ptr(out[x]) for x in ("count", "vals", "n_contrib",
                                                                                       "id_map", "id_margin",
                                                                                       "last")])
    if rc:
        raise ValueError("oracle_render_alternatives: pixel out of range")
    return out


def render_pixels(g: dict, cam: dict, pxy, st: OSettings | None = None, gt_id=None) -> dict:
    """The render at selected pixel centres pxy[k] = (u, v) only."""
    st = st or settings()
    m, s, q, o, c, i, f = _gauss(g)
    n = m.shape[0]
    pxy = np.ascontiguousarray(pxy, np.int32)
    k = pxy.shape[0]
    gt = None if gt_id is None else np.ascontiguousarray(gt_id, np.int32)
    out = dict(rgb=np.zeros((k, 3)), depth=np.zeros(k), alpha=np.zeros(k), ins=np.zeros(k),
               id_map=np.zeros(k, np.int32), T_final=np.zeros(k), n_contrib=np.zeros(k, np.int64),
               amb=np.zeros(k, np.uint8), id_margin=np.zeros(k))
    oc = camera(cam)
    rc = _lib_handle().oracle_render_pixels(C.byref(st), C.byref(oc), n, _ptr(m), _ptr(s), _ptr(q), _ptr(o),
                                            _ptr(c), _ptr(i), _ptr(f), _ptr(gt), k, _ptr(pxy),
                                            *[_ptr(out[x]) for x in ("rgb", "depth", "alpha", "ins", "id_map",
                                                                     "T_final", "n_contrib", "amb", "id_margin")])
    if rc:
        raise ValueError("oracle_render_pixels: pixel out of range")
    return out


def render_backward(g: dict, cam: dict, st: OSettings | None = None, targets: dict | None = None,
                    dl=None) -> dict:
    """Adjoint of the render ("back propagation", Sec. IV impl.).  dl[H,W,6] = upstream
    (dC rgb, dD, dA, dins); if None, the fused L1 losses against the targets are used.
    out["unc"][param] bounds how far a correct single-precision evaluation may differ
    because of decisions within rounding distance of their thresholds."""
    st = st or settings()
    m, s, q, o, c, i, f = _gauss(g)
    n = m.shape[0]
    tr, td, tg = _targets(targets)
    dl = None if dl is None else _d(dl)
    out = dict(g2=np.zeros((n, 10)), means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)),
               quats=np.zeros((n, 4)), opacity_logit=np.zeros(n), rgb=np.zeros((n, 3)),
               amb=np.zeros(n, np.uint8), unc_all=np.zeros((n, 14)))
    oc = camera(cam)
    rc = _lib_handle().oracle_render_backward(C.byref(st), C.byref(oc), n, _ptr(m), _ptr(s), _ptr(q), _ptr(o),
                                              _ptr(c), _ptr(i), _ptr(f), _ptr(tr), _ptr(td), _ptr(tg), _ptr(dl),
                                              *[_ptr(out[k]) for k in ("g2", "means", "log_scales", "quats",
                                                                       "opacity_logit", "rgb", "amb", "unc_all")])
    if rc:
        raise ValueError("oracle_render_backward: invalid arguments")
    u = out.pop("unc_all")
    out["unc"] = dict(means=u[:, 0:3], log_scales=u[:, 3:6], quats=u[:, 6:10], opacity_logit=u[:, 10],
                      rgb=u[:, 11:14])
    return out


def bin_tiles(rect, zbits, visible, ntx: int, nty: int):
    """Per-tile Gaussian lists ordered by (tile, z bits, index) from given projections."""
    rect = np.ascontiguousarray(rect, np.int32)
    zbits = np.ascontiguousarray(zbits, np.uint32)
    visible = np.ascontiguousarray(visible, np.uint8)
    n = rect.shape[0]
    area = np.where(visible > 0, (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]), 0)
    m = int(area.sum())
    ranges = np.zeros((ntx * nty, 2), np.int64)
    lst = np.zeros(max(m, 1), np.int64)
    got = _lib_handle().oracle_bin_tiles(n, _ptr(rect), _ptr(zbits), _ptr(visible), ntx, nty, _ptr(ranges), _ptr(lst))
    assert got == m
    return ranges, lst[:m]


# ------------------------------------------------------------------------- dual quadrics

def quadric_project(params, P, q_ptr, pair_v) -> dict:
    """Eq. 1-4: Q* from parameters, C* = P Q* P^T, and BBox(C*) per (quadric, view) pair."""
    params = _d(params).reshape(-1, 9)
    P = _d(P).reshape(-1, 12)
    q_ptr = np.ascontiguousarray(q_ptr, np.int32)
    pair_v = np.ascontiguousarray(pair_v, np.int32)
    k = pair_v.shape[0]
    out = dict(conic=np.zeros((k, 6)), bbox=np.zeros((k, 4)), valid=np.zeros(k, np.uint8))
    rc = _lib_handle().oracle_quadric_project(params.shape[0], _ptr(params), P.shape[0], _ptr(P), _ptr(q_ptr),
                                              _ptr(pair_v), _ptr(out["conic"]), _ptr(out["bbox"]), _ptr(out["valid"]))
    if rc:
        raise ValueError("oracle_quadric_project: view index out of range")
    return out


def quadric_bbox_loss(params, P, q_ptr, pair_v, obs) -> dict:
    """Eq. 12 reading: per-quadric sum of (1 - IoU) over its valid views, and its gradient."""
    params = _d(params).reshape(-1, 9)
    P = _d(P).reshape(-1, 12)
    q_ptr = np.ascontiguousarray(q_ptr, np.int32)
    pair_v = np.ascontiguousarray(pair_v, np.int32)
    obs = _d(obs).reshape(-1, 4)
    nq = params.shape[0]
    out = dict(loss=np.zeros(nq), dparams=np.zeros((nq, 9)))
    rc = _lib_handle().oracle_quadric_bbox_loss(nq, _ptr(params), P.shape[0], _ptr(P), _ptr(q_ptr), _ptr(pair_v),
                                                _ptr(obs), _ptr(out["loss"]), _ptr(out["dparams"]))
    if rc:
        raise ValueError("oracle_quadric_bbox_loss: view index out of range")
    return out


def quadric_matrix(params) -> np.ndarray:
    """Q* = Z diag(a^2, b^2, c^2, -1) Z^T per parameter vector (Eq. 1-3 reading)."""
    params = _d(params).reshape(-1, 9)
    out = np.zeros((params.shape[0], 4, 4))
    _lib_handle().oracle_quadric_matrix(params.shape[0], _ptr(params), _ptr(out))
    return out


def quadric_fit(P, q_ptr, pair_v, obs, iters: int = 100, lr: float = 1e-2, start=None) -> dict:
    """Plain multi-view fit: Eq. 1 initialisation from the boxes' tangent planes (or the
    given start parameters), then `iters` Adam steps on the Eq. 12 bbox loss (readings in
    the C++ source)."""
    P = _d(P).reshape(-1, 12)
    q_ptr = np.ascontiguousarray(q_ptr, np.int32)
    pair_v = np.ascontiguousarray(pair_v, np.int32)
    obs = _d(obs).reshape(-1, 4)
    nq = q_ptr.shape[0] - 1
    out = dict(init=np.zeros((nq, 9)), params=np.zeros((nq, 9)), init_Q=np.zeros((nq, 4, 4)),
               loss=np.zeros(nq), ok=np.zeros(nq, np.uint8))
    st = None if start is None else _d(start).reshape(nq, 9)
    rc = _lib_handle().oracle_quadric_fit(nq, P.shape[0], _ptr(P), _ptr(q_ptr), _ptr(pair_v), _ptr(obs), iters, lr,
                                          *[_ptr(out[k]) for k in ("init", "params", "init_Q", "loss", "ok")],
                                          _ptr(st))
    if rc:
        raise ValueError("oracle_quadric_fit: view index out of range")
    return out


def jacobi_eigen(A):
    """Cyclic Jacobi eigen-decomposition of a symmetric matrix: (eigenvalues, vectors as columns)."""
    A = _d(A).copy()
    n = A.shape[0]
    V = np.zeros((n, n))
    _lib_handle().oracle_jacobi_eigen(n, _ptr(A), _ptr(V))
    return np.diag(A).copy(), V


def rot_to_rotvec(R):
    R = _d(R).reshape(3, 3)
    r = np.zeros(3)
    _lib_handle().oracle_rot_to_rotvec(_ptr(R), _ptr(r))
    return r


# ------------------------------------------------------------------------- learned proposal
# (an addition to the paper's method: a network proposes each quadric's initial value,
# refined by the Eq. 12 fit; FP64 with bfloat16 rounding at the kernels' rounding points)

MLP_PARAMS = 35088
MLP_LAYOUT = {"W1": (0, (128, 128)), "b1": (16384, (128,)), "W2": (16512, (128, 128)), "b2": (32896, (128,)),
              "W3": (33024, (16, 128)), "b3": (35072, (16,))}


def round_bf16(x) -> np.ndarray:
    """Nearest bfloat16 value of each element (ties to even), as float64."""
    f = _lib_handle().oracle_round_bf16
    a = _d(x)
    return np.array([f(float(v)) for v in a.reshape(-1)]).reshape(a.shape)


def mlp_features(P, q_ptr, pair_v, obs, counts=None, length_scale: float = 1.0) -> np.ndarray:
    """Features [nq][128] of the learned proposal (FP64, unrounded): per view slot
    [xn, yn, hw, hh, r1, r2, d, C / length_scale] from P = K [R | t] and the box."""
    P = _d(P).reshape(-1, 12)
    q_ptr = np.ascontiguousarray(q_ptr, np.int32)
    pair_v = np.ascontiguousarray(pair_v, np.int32)
    obs = _d(obs).reshape(-1, 4)
    nq = q_ptr.shape[0] - 1
    F = np.zeros((nq, 128))
    cnt = None if counts is None else np.ascontiguousarray(counts, np.int32)
    rc = _lib_handle().oracle_mlp_features(nq, P.shape[0], _ptr(P), _ptr(q_ptr), _ptr(pair_v), _ptr(obs),
                                           _ptr(cnt), 1.0 / length_scale, _ptr(F))
    if rc:
        raise ValueError("oracle_mlp_features: view index out of range")
    return F


def mlp_forward(X, params, round_bf16_points: bool = True) -> dict:
    """y [n][9] and hidden activations h1, h2 [n][128] of the network for inputs X [n][128]."""
    X = _d(X).reshape(-1, 128)
    prm = _d(params).reshape(-1)
    n = X.shape[0]
    out = dict(y=np.zeros((n, 9)), h1=np.zeros((n, 128)), h2=np.zeros((n, 128)))
    _lib_handle().oracle_mlp_forward(n, _ptr(X), _ptr(prm), int(round_bf16_points), _ptr(out["y"]),
                                     _ptr(out["h1"]), _ptr(out["h2"]))
    return out


def mlp_backward(X, labels, loss_w, params, round_bf16_points: bool = True):
    """(gradient [35088], loss) of (1/n) sum w_j (y_j - label_j)^2."""
    X = _d(X).reshape(-1, 128)
    lab = _d(labels).reshape(-1, 9)
    w = _d(loss_w).reshape(9)
    prm = _d(params).reshape(-1)
    g = np.zeros(MLP_PARAMS)
    loss = np.zeros(1)
    _lib_handle().oracle_mlp_backward(X.shape[0], _ptr(X), _ptr(lab), _ptr(w), _ptr(prm), int(round_bf16_points),
                                      _ptr(g), _ptr(loss))
    return g, float(loss[0])


def mlp_adam(params, grads, m, v, step: int, lr: float, lr_final: float = 0.0, total_steps: int = 0,
             beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma & Ba, bias-corrected; `step` counts this step, from 1) with the
    learning rate on a cosine schedule from lr to lr_final over total_steps (constant if
    total_steps <= 0).  Returns (params, m, v)."""
    g = _d(grads)
    m = beta1 * _d(m) + (1 - beta1) * g
    v = beta2 * _d(v) + (1 - beta2) * g * g
    prog = min((step - 1) / total_steps, 1.0) if total_steps > 0 else 0.0
    a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * prog))
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return _d(params) - a * mh / (np.sqrt(vh) + eps), m, v


def quadric_canonical(params) -> np.ndarray:
    """Canonical parameters of each quadric (same ellipsoid; axes descending, rotation of
    largest trace among the equivalent ones)."""
    p = _d(params).reshape(-1, 9)
    out = np.zeros_like(p)
    _lib_handle().oracle_quadric_canonical(p.shape[0], _ptr(p), _ptr(out))
    return out
