"""Seeded synthetic inputs shaped like DQO-MAP's indoor RGB-D keyframes (Sec. IV).

This module only draws inputs: Gaussian sets, cameras, dual-quadric parameters,
views and noisy observed boxes, and ray-cast RGB-D/instance targets.  It holds none
of the method's arithmetic (no splatting, no conic projection): observed boxes come
from projecting sampled ellipsoid surface points, targets from exact ray/ellipsoid
and ray/plane hits.  Both the oracle tests and the CUDA path consume these arrays.

All randomness is numpy's Philox counter-based generator, so a seed gives the same
arrays on x86_64 and aarch64.

Layouts (all C-contiguous):
  means f32[N,3], log_scales f32[N,3], quats f32[N,4] (w,x,y,z, not normalised),
  opacity_logit f32[N], rgb f32[N,3], obj_id i32[N], flags u8[N] (bit0 = opaque/OG)
  camera: dict(fx, fy, cx, cy, width, height, viewmat f32[3,4] world->camera, OpenCV axes)
  quadric params f32[Q,9] = (centre xyz, log semi-axes abc, rotation vector)
  views P f32[V,3,4] = K [R|t];  pairs in CSR: q_ptr i32[Q+1], pair_v i32[npairs]
  obs_bbox f32[npairs,4] = (u_min, v_min, u_max, v_max)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1000


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


# ----------------------------------------------------------------------------- cameras

def look_at(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World->camera [R|t] (OpenCV: x right, y down, z forward) looking from eye to target."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    # camera y points "down" in the image; 'up' is the world direction that maps to -y
    x = np.cross(z, -up)
    if np.linalg.norm(x) < 1e-8:
        x = np.cross(z, np.array([1.0, 0.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], 0)
    t = -R @ eye
    return np.concatenate([R, t[:, None]], 1)


def make_camera(fx, fy, cx, cy, width, height, viewmat) -> dict:
    return dict(fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy),
                width=int(width), height=int(height),
                viewmat=np.ascontiguousarray(np.asarray(viewmat, np.float32).reshape(3, 4)))


def intrinsics(fx, fy, cx, cy) -> np.ndarray:
    return np.array([[fx, 0, cx], [0, fy, cy], [0, 0, 1]], np.float64)


# ----------------------------------------------------------------------------- rotations

def random_rotations(rng, n) -> np.ndarray:
    """Uniform random rotations as matrices [n,3,3] (from unit quaternions on S^3)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return quat_to_mat(q)


def quat_to_mat(q) -> np.ndarray:
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def mat_to_quat(R) -> np.ndarray:
    """Rotation matrices [...,3,3] -> unit quaternions (w,x,y,z), Shepperd's method."""
    R = np.asarray(R, np.float64)
    shp = R.shape[:-2]
    R = R.reshape(-1, 3, 3)
    q = np.empty((R.shape[0], 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    for i in range(R.shape[0]):
        m = R[i]
        if tr[i] > 0:
            s = np.sqrt(tr[i] + 1.0) * 2
            q[i] = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
        elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
            s = np.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
            q[i] = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
        elif m[1, 1] > m[2, 2]:
            s = np.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
            q[i] = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
        else:
            s = np.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
            q[i] = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    return q.reshape(shp + (4,))


def mat_to_rotvec(R) -> np.ndarray:
    """Rotation matrices [n,3,3] -> rotation vectors (axis * angle), angle in [0, pi)."""
    q = mat_to_quat(R)
    q = q * np.where(q[:, :1] < 0, -1.0, 1.0)
    s = np.linalg.norm(q[:, 1:], axis=1)
    ang = 2 * np.arctan2(s, q[:, 0])
    fac = np.where(s > 1e-12, ang / np.maximum(s, 1e-300), 2.0)
    return q[:, 1:] * fac[:, None]


def rotvec_to_mat(r) -> np.ndarray:
    r = np.asarray(r, np.float64).reshape(-1, 3)
    out = np.empty((r.shape[0], 3, 3))
    for i, v in enumerate(r):
        th = np.linalg.norm(v)
        K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
        if th < 1e-12:
            out[i] = np.eye(3) + K
        else:
            out[i] = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * (K @ K)
    return out


# ----------------------------------------------------------------------------- Gaussians

def _pack(means, log_scales, quats, opacity_logit, rgb, obj_id, flags) -> dict:
    return dict(
        means=np.ascontiguousarray(means, np.float32),
        log_scales=np.ascontiguousarray(log_scales, np.float32),
        quats=np.ascontiguousarray(quats, np.float32),
        opacity_logit=np.ascontiguousarray(opacity_logit, np.float32),
        rgb=np.ascontiguousarray(rgb, np.float32),
        obj_id=np.ascontiguousarray(obj_id, np.int32),
        flags=np.ascontiguousarray(flags, np.uint8),
    )


def tiny_gaussians(seed: int, n: int = 2000, n_objects: int = 4, og_fraction: float = 1.0) -> dict:
    """2 m cube of Gaussians: means U[-1,1]^3, log-scales N(-4,0.5), quats N(0,1)^4,
    opacity logits N(0,1), rgb U[0,1], ids U{0..n_objects-1}."""
    rng = rng_for(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.normal(-4.0, 0.5, (n, 3))
    quats = rng.standard_normal((n, 4))
    logit = rng.standard_normal(n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    obj_id = rng.integers(0, n_objects, n)
    og = rng.uniform(0.0, 1.0, n) < og_fraction
    return _pack(means, log_scales, quats, logit, rgb, obj_id, og.astype(np.uint8))


def tiny_camera(width=320, height=240, f=300.0, dist=3.0) -> dict:
    """Pinhole camera at (0,0,-dist) looking at the origin, image y along world +y."""
    vm = np.concatenate([np.eye(3), np.array([[0.0], [0.0], [dist]])], 1)
    return make_camera(f, f, width / 2.0, height / 2.0, width, height, vm)


def empty_gaussians() -> dict:
    z3 = np.zeros((0, 3))
    return _pack(z3, z3, np.zeros((0, 4)), np.zeros(0), z3, np.zeros(0), np.zeros(0))


# ----------------------------------------------------------------------------- quadrics

def ellipsoid_surface_points(centre, axes, R, m=4096) -> np.ndarray:
    """m points on the ellipsoid x = centre + R diag(axes) d, d on a Fibonacci sphere."""
    i = np.arange(m) + 0.5
    phi = np.arccos(1 - 2 * i / m)
    th = np.pi * (1 + 5 ** 0.5) * i
    d = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    return centre[None, :] + (d * axes[None, :]) @ R.T


def sampled_bbox(P, pts):
    """Box of the projections of sampled surface points, and whether all are in front."""
    h = pts @ P[:, :3].T + P[:, 3]
    if np.any(h[:, 2] <= 1e-6):
        return None
    u = h[:, 0] / h[:, 2]
    v = h[:, 1] / h[:, 2]
    return np.array([u.min(), v.min(), u.max(), v.max()])


def random_quadrics(rng, q, centre_lo=-1.0, centre_hi=1.0, axis_lo=0.1, axis_hi=0.5):
    centres = rng.uniform(centre_lo, centre_hi, (q, 3))
    axes = rng.uniform(axis_lo, axis_hi, (q, 3))
    Rs = random_rotations(rng, q)
    rv = mat_to_rotvec(Rs)
    params = np.concatenate([centres, np.log(axes), rv], 1)
    return params, centres, axes, Rs


def sphere_views(rng, nv, radius=3.0, target=(0.0, 0.0, 0.0)):
    d = rng.standard_normal((nv, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    eyes = np.asarray(target)[None, :] + radius * d
    mats = []
    for e in eyes:
        up = (0.0, -1.0, 0.0)
        if abs(np.dot((np.asarray(target) - e) / radius, up)) > 0.95:
            up = (0.0, 0.0, 1.0)
        mats.append(look_at(e, target, up))
    return np.stack(mats, 0)


def tiny_quadrics(seed: int, q: int = 4, views_per_q: int = 5, noise_px: float = 2.0,
                  f=300.0, width=320, height=240, perturb=True) -> dict:
    """Ellipsoids (axes U[0.1,0.5], centres U[-1,1]^3, random rotation), each seen from its
    own views on a 3 m sphere around the origin; boxes = sampled silhouette + N(0, noise^2)."""
    rng = rng_for(seed)
    params, centres, axes, Rs = random_quadrics(rng, q)
    K = intrinsics(f, f, width / 2.0, height / 2.0)
    Ps, obs, pair_v, q_ptr = [], [], [], [0]
    for k in range(q):
        pts = ellipsoid_surface_points(centres[k], axes[k], Rs[k])
        got = 0
        while got < views_per_q:
            vm = sphere_views(rng, 1)[0]
            P = K @ vm
            bb = sampled_bbox(P, pts)
            if bb is None:
                continue
            Ps.append(P)
            obs.append(bb + rng.normal(0.0, noise_px, 4))
            pair_v.append(len(Ps) - 1)
            got += 1
        q_ptr.append(len(pair_v))
    init = params.copy()
    if perturb:
        init[:, :3] += rng.normal(0.0, 0.05, (q, 3))
        init[:, 3:6] += rng.normal(0.0, 0.1, (q, 3))
        init[:, 6:] += rng.normal(0.0, 0.1, (q, 3))
    return dict(
        params_true=params.astype(np.float32),
        params=init.astype(np.float32),
        P=np.ascontiguousarray(np.stack(Ps, 0), np.float32),
        q_ptr=np.asarray(q_ptr, np.int32),
        pair_v=np.asarray(pair_v, np.int32),
        obs_bbox=np.ascontiguousarray(np.stack(obs, 0), np.float32),
        width=width, height=height,
    )


# ----------------------------------------------------------------------------- indoor keyframe

ROOM = (6.0, 3.0, 5.0)   # x extent, height (y, pointing down: floor y=0, ceiling y=-3), z extent


def _room_planes():
    """(point, normal, u-axis, v-axis, extent_u, extent_v) for floor, ceiling and 4 walls."""
    X, Y, Z = ROOM
    return [
        (np.array([0, 0.0, 0]), np.array([0, -1.0, 0]), np.array([1.0, 0, 0]), np.array([0, 0, 1.0]), X, Z),
        (np.array([0, -Y, 0]), np.array([0, 1.0, 0]), np.array([1.0, 0, 0]), np.array([0, 0, 1.0]), X, Z),
        (np.array([0, 0.0, 0]), np.array([1.0, 0, 0]), np.array([0, -1.0, 0]), np.array([0, 0, 1.0]), Y, Z),
        (np.array([X, 0.0, 0]), np.array([-1.0, 0, 0]), np.array([0, -1.0, 0]), np.array([0, 0, 1.0]), Y, Z),
        (np.array([0, 0.0, 0]), np.array([0, 0, 1.0]), np.array([1.0, 0, 0]), np.array([0, -1.0, 0]), X, Y),
        (np.array([0, 0.0, Z]), np.array([0, 0, -1.0]), np.array([1.0, 0, 0]), np.array([0, -1.0, 0]), X, Y),
    ]


WALL_RGB = np.array([[0.80, 0.78, 0.72], [0.95, 0.95, 0.95], [0.70, 0.72, 0.80],
                     [0.72, 0.80, 0.70], [0.82, 0.70, 0.70], [0.75, 0.75, 0.62]])


def room_objects(rng, n_obj: int, cam_eyes=()):
    """n_obj non-overlapping ellipsoids (axes U[0.1,0.5], random rotation) inside the room."""
    X, Y, Z = ROOM
    centres, axes, Rs = [], [], []
    tries = 0
    while len(centres) < n_obj:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place objects")
        ax = rng.uniform(0.1, 0.5, 3)
        rb = ax.max()
        c = np.array([rng.uniform(rb + 0.05, X - rb - 0.05),
                      -rng.uniform(rb + 0.02, Y - rb - 0.05),
                      rng.uniform(rb + 0.05, Z - rb - 0.05)])
        if any(np.linalg.norm(c - e) < rb + 0.6 for e in cam_eyes):
            continue
        if any(np.linalg.norm(c - c2) < rb + a2.max() + 0.02 for c2, a2 in zip(centres, axes)):
            continue
        centres.append(c)
        axes.append(ax)
        Rs.append(random_rotations(rng, 1)[0])
    return np.array(centres), np.array(axes), np.array(Rs)


def indoor_keyframe(seed: int, n_total: int = 300_000, n_obj: int = 30, width: int = 1200,
                    height: int = 680, f: float = 600.0, object_total: int = 235_000,
                    n_views: int = 8) -> dict:
    """Indoor keyframe: n_obj ellipsoidal objects (ids 1..n_obj) carrying object_total
    Gaussians (per-object counts log-uniform on [2k,20k], rescaled), walls/floor/ceiling
    (id 0) carrying the rest as flattened Gaussians; a 1200x680 camera inside the room."""
    rng = rng_for(seed)
    X, Y, Z = ROOM
    eye = np.array([1.0, -1.6, 0.8])
    target = np.array([X - 0.4, -1.0, Z - 0.4])
    vm = look_at(eye, target)
    # keyframe trajectory for the quadric views: a short arc near the first camera
    eyes = [eye + np.array([0.35 * k, -0.03 * k, 0.12 * k]) for k in range(n_views)]
    centres, axes, Rs = room_objects(rng, n_obj, cam_eyes=eyes)

    counts = np.exp(rng.uniform(np.log(2000), np.log(20000), n_obj))
    counts = np.maximum(1, np.round(counts * object_total / counts.sum())).astype(np.int64)
    counts[-1] += object_total - counts.sum()
    n_wall = n_total - int(counts.sum())
    assert n_wall > 0

    means, ls, qs, ids, cols = [], [], [], [], []
    base_rgb = rng.uniform(0.1, 0.95, (n_obj, 3))
    for k in range(n_obj):
        m = int(counts[k])
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p = centres[k] + (d * axes[k]) @ Rs[k].T
        p += rng.normal(0.0, 0.004, (m, 3))
        means.append(p)
        ls.append(rng.normal(-4.5, 0.5, (m, 3)))
        qs.append(rng.standard_normal((m, 4)))
        ids.append(np.full(m, k + 1))
        cols.append(np.clip(base_rgb[k] + rng.normal(0, 0.05, (m, 3)), 0, 1))

    planes = _room_planes()
    areas = np.array([eu * ev for (_, _, _, _, eu, ev) in planes])
    wc = np.floor(areas / areas.sum() * n_wall).astype(np.int64)
    wc[0] += n_wall - wc.sum()
    for pi, (o, nrm, uax, vax, eu, ev) in enumerate(planes):
        m = int(wc[pi])
        uu = rng.uniform(0, eu, m)
        vv = rng.uniform(0, ev, m)
        p = o + uu[:, None] * uax + vv[:, None] * vax
        # local frame: columns (u, v, n) rotated in-plane by a random angle
        ang = rng.uniform(0, 2 * np.pi, m)
        ca, sa = np.cos(ang), np.sin(ang)
        a1 = ca[:, None] * uax + sa[:, None] * vax
        a2 = -sa[:, None] * uax + ca[:, None] * vax
        Rw = np.stack([a1, a2, np.cross(a1, a2)], 2)
        s = rng.normal(-3.5, 0.3, (m, 3))
        s[:, 2] -= 2.3
        means.append(p)
        ls.append(s)
        qs.append(mat_to_quat_fast(Rw))
        ids.append(np.zeros(m))
        cols.append(np.clip(WALL_RGB[pi] + rng.normal(0, 0.03, (m, 3)), 0, 1))

    means = np.concatenate(means)
    perm = rng.permutation(means.shape[0])
    g = _pack(means[perm], np.concatenate(ls)[perm], np.concatenate(qs)[perm],
              rng.normal(1.5, 1.0, means.shape[0]), np.concatenate(cols)[perm],
              np.concatenate(ids)[perm], np.ones(means.shape[0]))
    cam = make_camera(f, f, width / 2.0, height / 2.0, width, height, vm)

    # quadrics: the objects' ellipsoids, seen from the keyframes that see them whole
    K = intrinsics(f, f, width / 2.0, height / 2.0)
    Ps = [K @ look_at(e, target + np.array([0.0, 0.0, -0.1 * i])) for i, e in enumerate(eyes)]
    params = np.concatenate([centres, np.log(axes), mat_to_rotvec(Rs)], 1)
    obs, pair_v, q_ptr = [], [], [0]
    for k in range(n_obj):
        pts = ellipsoid_surface_points(centres[k], axes[k], Rs[k], 2048)
        for vi, P in enumerate(Ps):
            bb = sampled_bbox(P, pts)
            if bb is None:
                continue
            obs.append(bb + rng.normal(0.0, 2.0, 4))
            pair_v.append(vi)
        q_ptr.append(len(pair_v))
    init = params.copy()
    init[:, :3] += rng.normal(0.0, 0.03, (n_obj, 3))
    init[:, 3:6] += rng.normal(0.0, 0.08, (n_obj, 3))
    init[:, 6:] += rng.normal(0.0, 0.08, (n_obj, 3))
    quad = dict(params_true=params.astype(np.float32), params=init.astype(np.float32),
                P=np.ascontiguousarray(np.stack(Ps, 0), np.float32),
                q_ptr=np.asarray(q_ptr, np.int32), pair_v=np.asarray(pair_v, np.int32),
                obs_bbox=np.ascontiguousarray(np.stack(obs, 0), np.float32),
                width=width, height=height)
    scene = dict(centres=centres, axes=axes, Rs=Rs, base_rgb=base_rgb)
    return dict(gaussians=g, camera=cam, quadrics=quad, scene=scene)


def mat_to_quat_fast(R) -> np.ndarray:
    """Vectorised rotation matrix -> quaternion (w,x,y,z) for proper rotations."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    c0 = tr > 0
    c1 = (~c0) & (R[:, 0, 0] > R[:, 1, 1]) & (R[:, 0, 0] > R[:, 2, 2])
    c2 = (~c0) & (~c1) & (R[:, 1, 1] > R[:, 2, 2])
    c3 = ~(c0 | c1 | c2)
    m = R
    s = np.sqrt(np.maximum(tr + 1.0, 1e-300)) * 2
    q[c0] = np.stack([0.25 * s, (m[:, 2, 1] - m[:, 1, 2]) / s, (m[:, 0, 2] - m[:, 2, 0]) / s,
                      (m[:, 1, 0] - m[:, 0, 1]) / s], 1)[c0]
    s = np.sqrt(np.maximum(1.0 + m[:, 0, 0] - m[:, 1, 1] - m[:, 2, 2], 1e-300)) * 2
    q[c1] = np.stack([(m[:, 2, 1] - m[:, 1, 2]) / s, 0.25 * s, (m[:, 0, 1] + m[:, 1, 0]) / s,
                      (m[:, 0, 2] + m[:, 2, 0]) / s], 1)[c1]
    s = np.sqrt(np.maximum(1.0 + m[:, 1, 1] - m[:, 0, 0] - m[:, 2, 2], 1e-300)) * 2
    q[c2] = np.stack([(m[:, 0, 2] - m[:, 2, 0]) / s, (m[:, 0, 1] + m[:, 1, 0]) / s, 0.25 * s,
                      (m[:, 1, 2] + m[:, 2, 1]) / s], 1)[c2]
    s = np.sqrt(np.maximum(1.0 + m[:, 2, 2] - m[:, 0, 0] - m[:, 1, 1], 1e-300)) * 2
    q[c3] = np.stack([(m[:, 1, 0] - m[:, 0, 1]) / s, (m[:, 0, 2] + m[:, 2, 0]) / s,
                      (m[:, 1, 2] + m[:, 2, 1]) / s, 0.25 * s], 1)[c3]
    return q


def raycast_targets(kf: dict) -> dict:
    """Ray-cast RGB-D and instance targets of the keyframe's room + ellipsoids:
    nearest exact hit per pixel centre; depth = camera z of the hit (0 where no hit),
    gt_id = object index (0 for walls, -1 where nothing is hit)."""
    cam = kf["camera"]
    sc = kf["scene"]
    W, H = cam["width"], cam["height"]
    vm = cam["viewmat"].astype(np.float64)
    R, t = vm[:, :3], vm[:, 3]
    eye = -R.T @ t
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dc = np.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], np.ones_like(u)], -1)
    dw = dc.reshape(-1, 3) @ R          # world ray directions with camera-z component 1
    best = np.full(dw.shape[0], np.inf)
    gid = np.full(dw.shape[0], -1, np.int64)
    col = np.zeros((dw.shape[0], 3))
    for k in range(len(sc["centres"])):
        Rk, ak, ck = sc["Rs"][k], sc["axes"][k], sc["centres"][k]
        o = (Rk.T @ (eye - ck)) / ak
        d = (dw @ Rk) / ak[None, :]
        a = np.einsum("ij,ij->i", d, d)
        b = 2 * d @ o
        c = o @ o - 1.0
        disc = b * b - 4 * a * c
        ok = disc > 0
        s = np.where(ok, (-b - np.sqrt(np.where(ok, disc, 0))) / (2 * a), np.inf)
        s = np.where(s > 1e-3, s, np.inf)
        hit = s < best
        best = np.where(hit, s, best)
        gid = np.where(hit, k + 1, gid)
        col[hit] = sc["base_rgb"][k]
    for pi, (o, nrm, uax, vax, eu, ev) in enumerate(_room_planes()):
        denom = dw @ nrm
        s = np.where(np.abs(denom) > 1e-12, ((o - eye) @ nrm) / np.where(np.abs(denom) > 1e-12, denom, 1), np.inf)
        s = np.where(s > 1e-3, s, np.inf)
        hit = s < best
        best = np.where(hit, s, best)
        gid = np.where(hit, 0, gid)
        col[hit] = WALL_RGB[pi]
    depth = np.where(np.isfinite(best), best, 0.0)   # ray param = camera z (dc has z = 1)
    return dict(rgb=np.ascontiguousarray(col.reshape(H, W, 3), np.float32),
                depth=np.ascontiguousarray(depth.reshape(H, W), np.float32),
                gt_id=np.ascontiguousarray(gid.reshape(H, W), np.int32))


def batched_quadric_fits(seed: int, nq: int = 512, min_views: int = 3, max_views: int = 40,
                         noise_px: float = 2.0, f: float = 525.0, width: int = 640, height: int = 480,
                         radius: float = 3.5, surface_points: int = 1024) -> dict:
    """nq ellipsoids (axes U[0.1,0.5], centres U[-1,1]^3, random rotation), each seen from
    U{min_views..max_views} views on a sphere of `radius` around the origin; observed boxes =
    box of projected surface samples + N(0, noise^2).  CSR pairs, one view per pair."""
    rng = rng_for(seed)
    params, centres, axes, Rs = random_quadrics(rng, nq)
    counts = rng.integers(min_views, max_views + 1, nq)
    K = intrinsics(f, f, width / 2.0, height / 2.0)
    Ps, obs = [], []
    for k in range(nq):
        pts = ellipsoid_surface_points(centres[k], axes[k], Rs[k], surface_points)
        got = 0
        while got < counts[k]:
            P = K @ sphere_views(rng, 1, radius=radius)[0]
            bb = sampled_bbox(P, pts)
            if bb is None:
                continue
            Ps.append(P)
            obs.append(bb + rng.normal(0.0, noise_px, 4))
            got += 1
    q_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return dict(params_true=params.astype(np.float32),
                P=np.ascontiguousarray(np.stack(Ps, 0), np.float32), q_ptr=q_ptr,
                pair_v=np.arange(len(Ps), dtype=np.int32),
                obs_bbox=np.ascontiguousarray(np.stack(obs, 0), np.float32), counts=counts)


# ----------------------------------------------------------------------------- learned proposal

def look_at_batch(eyes, target=(0.0, 0.0, 0.0)) -> np.ndarray:
    """look_at for an array of eyes [..., 3] (same convention; 'up' = -y unless the view is
    within acos(0.95) of vertical, then +z).  Returns [..., 3, 4]."""
    eyes = np.asarray(eyes, np.float64)
    z = np.asarray(target, np.float64) - eyes
    z /= np.linalg.norm(z, axis=-1, keepdims=True)
    up = np.broadcast_to(np.array([0.0, -1.0, 0.0]), eyes.shape).copy()
    up[np.abs(z[..., 1]) > 0.95] = np.array([0.0, 0.0, 1.0])
    x = np.cross(z, -up)
    x /= np.linalg.norm(x, axis=-1, keepdims=True)
    y = np.cross(z, x)
    R = np.stack([x, y, z], -2)
    t = -np.einsum("...ij,...j->...i", R, eyes)
    return np.concatenate([R, t[..., None]], -1)


def proposal_samples(seed: int, n: int, views: int = 8, noise_px: float = 2.0, f: float = 525.0,
                     width: int = 640, height: int = 480, radius: float = 3.5, points: int = 96,
                     chunk: int = 8192) -> dict:
    """n random ellipsoids (axes U[0.1,0.5] m, centres U[-1,1]^3, random rotation), each seen
    from `views` cameras on a sphere of `radius` around the origin looking at it; observed
    box = box of `points` projected surface samples + N(0, noise^2) px.  CSR pairs with
    exactly `views` views per quadric, in order."""
    rng = rng_for(seed)
    params, centres, axes, Rs = random_quadrics(rng, n)
    d = rng.standard_normal((n, views, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    vm = look_at_batch(radius * d)
    P = intrinsics(f, f, width / 2.0, height / 2.0)[None, None] @ vm           # n, views, 3, 4
    i = np.arange(points) + 0.5
    phi = np.arccos(1 - 2 * i / points)
    th = np.pi * (1 + 5 ** 0.5) * i
    sph = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 0)   # 3, points
    box = np.empty((n, views, 4))
    for s in range(0, n, chunk):
        e = slice(s, s + chunk)
        pts = centres[e, :, None] + Rs[e] @ (axes[e, :, None] * sph[None])                  # q, 3, points
        h = P[e, :, :, :3] @ pts[:, None] + P[e, :, :, 3:]                                 # q, views, 3, points
        u, v = h[:, :, 0] / h[:, :, 2], h[:, :, 1] / h[:, :, 2]
        box[e] = np.stack([u.min(-1), v.min(-1), u.max(-1), v.max(-1)], -1)
    box += rng.normal(0.0, noise_px, box.shape)
    return dict(params_true=params.astype(np.float32),
                P=np.ascontiguousarray(P.reshape(n * views, 12), np.float32),
                q_ptr=(np.arange(n + 1) * views).astype(np.int32),
                pair_v=np.arange(n * views, dtype=np.int32),
                obs_bbox=np.ascontiguousarray(box.reshape(n * views, 4), np.float32),
                views=views, length_scale=radius)


def subset_views(s: dict, k: int) -> dict:
    """The first k views of every quadric of a proposal_samples set, as its own CSR set."""
    n = s["q_ptr"].shape[0] - 1
    v = s["views"]
    sel = (np.arange(n)[:, None] * v + np.arange(k)[None]).reshape(-1)
    return dict(params_true=s["params_true"], P=np.ascontiguousarray(s["P"][sel]),
                q_ptr=(np.arange(n + 1) * k).astype(np.int32), pair_v=np.arange(n * k, dtype=np.int32),
                obs_bbox=np.ascontiguousarray(s["obs_bbox"][sel]), views=k, length_scale=s["length_scale"])


def mlp_init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, for the 128-128-128-9 proposal network (fp32 vector of
    35088 in the library's layout; padding rows zero)."""
    rng = rng_for(seed)
    p = np.zeros(35088, np.float32)
    p[0:16384] = rng.normal(0.0, np.sqrt(2.0 / 128), 16384)
    p[16512:32896] = rng.normal(0.0, np.sqrt(2.0 / 128), 16384)
    p[33024:33024 + 9 * 128] = rng.normal(0.0, np.sqrt(1.0 / 128), 9 * 128)
    return p
