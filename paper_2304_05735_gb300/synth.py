"""Seeded synthetic inputs: object shapes, cameras, ray pools, occupancy grids.

This module generates training data shaped like the paper's workload
(Sec. V-A-1 and Sec. VI "Implementation Details": per-object keyframe
images, instance masks and sparse depth; objects inside cuboid bounding
boxes).  The paper's datasets (Cube-Diorama, Replica, D455 sequences) are
not available, so analytic shapes stand in for them.  It holds none of the
method's arithmetic: no volume rendering, no hash encoding, no MLP.  Targets
are the colour of the analytic surface at the first hit (an opaque-surface
stand-in for a shape of high constant density); masks come from the same
intersection test; sparse depth is the first-hit distance.

Both the CUDA path and the CPU oracle receive the arrays produced here; it is
the only module they share.
"""
from dataclasses import dataclass, field

import numpy as np

CLS_OBJECT, CLS_BACKGROUND, CLS_OCCLUDER = 0, 1, 2


# --------------------------------------------------------------------------
# Cameras (pinhole, OpenCV axes: x right, y down, z forward; world z up)
# --------------------------------------------------------------------------
def look_at(position, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """Camera-to-world rotation (columns: camera x, y, z axes in world)."""
    p = np.asarray(position, np.float64)
    z = np.asarray(target, np.float64) - p
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    if np.linalg.norm(x) < 1e-9:
        x = np.cross(z, np.array([0.0, 1.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def sphere_position(radius, azimuth, elevation, center=(0.0, 0.0, 0.0)):
    c = np.asarray(center, np.float64)
    return c + radius * np.array([np.cos(elevation) * np.cos(azimuth), np.cos(elevation) * np.sin(azimuth),
                                  np.sin(elevation)])


def pixel_rays(R_cw, position, fx, fy, cx, cy, us, vs):
    """World-frame rays through pixel centres (u + 0.5, v + 0.5)."""
    dc = np.stack([(us + 0.5 - cx) / fx, (vs + 0.5 - cy) / fy, np.ones_like(us, dtype=np.float64)], axis=-1)
    dw = dc @ R_cw.T
    dw /= np.linalg.norm(dw, axis=-1, keepdims=True)
    ow = np.broadcast_to(np.asarray(position, np.float64), dw.shape).copy()
    return ow, dw


# --------------------------------------------------------------------------
# Analytic shapes in their object frame
# --------------------------------------------------------------------------
@dataclass
class Shape:
    kind: str                      # "ellipsoid" | "superellipsoid" | "box"
    axes: np.ndarray               # semi-axes
    eps: tuple = (1.0, 1.0)        # superellipsoid exponents (e1, e2)
    colour_kind: str = "sin3"      # "sin3" | "random"
    amp: np.ndarray = field(default_factory=lambda: np.zeros((4, 3)))
    omega: np.ndarray = field(default_factory=lambda: np.zeros((4, 3, 3)))
    phase: np.ndarray = field(default_factory=lambda: np.zeros((4, 3)))

    def inside(self, x):
        a = self.axes
        if self.kind == "ellipsoid":
            return np.sum((x / a) ** 2, axis=-1) <= 1.0
        if self.kind == "box":
            return np.all(np.abs(x) <= a, axis=-1)
        e1, e2 = self.eps
        q = np.abs(x / a)
        f = (q[..., 0] ** (2.0 / e2) + q[..., 1] ** (2.0 / e2)) ** (e2 / e1) + q[..., 2] ** (2.0 / e1)
        return f <= 1.0

    def first_hit(self, o, d):
        """First-hit distance along unit rays (inf for a miss), object frame."""
        a = self.axes
        n = o.shape[0]
        t_hit = np.full(n, np.inf)
        if self.kind == "ellipsoid":
            oa, da = o / a, d / a
            A = np.sum(da * da, -1)
            B = 2.0 * np.sum(oa * da, -1)
            Cc = np.sum(oa * oa, -1) - 1.0
            disc = B * B - 4 * A * Cc
            ok = disc >= 0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            t0 = (-B - sq) / (2 * A)
            t1 = (-B + sq) / (2 * A)
            t = np.where(t0 > 0, t0, t1)
            good = ok & (t > 0)
            t_hit[good] = t[good]
            return t_hit
        # box and superellipsoid: bracket with the bounding box of the shape
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            ta = (-a - o) * inv
            tb = (a - o) * inv
        tmin = np.nanmax(np.minimum(ta, tb), axis=-1)
        tmax = np.nanmin(np.maximum(ta, tb), axis=-1)
        tmin = np.maximum(tmin, 0.0)
        box_hit = tmax > tmin
        if self.kind == "box":
            t_hit[box_hit] = tmin[box_hit]
            return t_hit
        idx = np.nonzero(box_hit)[0]
        if idx.size == 0:
            return t_hit
        oo, dd, t0, t1 = o[idx], d[idx], tmin[idx], tmax[idx]
        steps = 96
        ts = t0[:, None] + (t1 - t0)[:, None] * (np.arange(steps + 1)[None, :] / steps)
        pts = oo[:, None, :] + ts[..., None] * dd[:, None, :]
        ins = self.inside(pts)
        any_in = ins.any(axis=1)
        first = np.argmax(ins, axis=1)
        lo_t = ts[np.arange(idx.size), np.maximum(first - 1, 0)]
        hi_t = ts[np.arange(idx.size), first]
        for _ in range(24):  # bisection on the inside test
            mid = 0.5 * (lo_t + hi_t)
            m_in = self.inside(oo + mid[:, None] * dd)
            hi_t = np.where(m_in, mid, hi_t)
            lo_t = np.where(m_in, lo_t, mid)
        res = np.where(first == 0, ts[:, 0], hi_t)
        t_hit[idx[any_in]] = res[any_in]
        return t_hit

    def colour(self, x):
        if self.colour_kind == "sin3":
            return 0.5 + 0.5 * np.sin(3.0 * x)
        c = np.full(x.shape, 0.5)
        for k in range(self.amp.shape[0]):
            for ch in range(3):
                c[..., ch] += self.amp[k, ch] * np.sin(x @ self.omega[k, ch] + self.phase[k, ch])
        return np.clip(c, 0.0, 1.0)


def random_shape(rng, index):
    kind = ("ellipsoid", "superellipsoid", "box")[index % 3]
    axes = rng.uniform(0.1, 0.5, size=3)
    eps = tuple(rng.uniform(0.3, 2.0, size=2))
    omega = rng.normal(size=(4, 3, 3))
    omega *= (rng.uniform(0.0, 6.0, size=(4, 3, 1)) / np.linalg.norm(omega, axis=-1, keepdims=True))
    return Shape(kind=kind, axes=axes, eps=eps, colour_kind="random", amp=rng.uniform(0.0, 0.15, size=(4, 3)),
                 omega=omega, phase=rng.uniform(0, 2 * np.pi, size=(4, 3)))


# --------------------------------------------------------------------------
# Object pose (translation + yaw about world z, Sec. IV-B)
# --------------------------------------------------------------------------
def yaw_matrix(yaw):
    c, s = np.cos(yaw), np.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


@dataclass
class ObjectScene:
    shape: Shape
    t: np.ndarray          # world translation
    yaw: float
    half: np.ndarray       # AABB half extents (object frame)
    seed: int
    pool: dict             # world-frame SoA: origin, dir, rgb, depth, cls (float32 / uint8)


def _object_rays(shape, t, yaw, half, rng, n_frames, W, H, f, depth_frac, occluder_prob, elev=(0.15, 1.1),
                 radius=2.5, stride=1):
    R = yaw_matrix(yaw)
    outs = {k: [] for k in ("origin", "dir", "rgb", "depth", "cls")}
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * half
    for _ in range(n_frames):
        az = rng.uniform(-np.pi, np.pi)
        el = rng.uniform(*elev)
        cam_o = sphere_position(radius, az, el)                 # object frame
        cam_w = t + R @ cam_o
        R_cw = look_at(cam_w, target=t)
        # detection box: projection of the object's 3D box into the image
        cw = (corners @ R.T) + t
        pc = (cw - cam_w) @ R_cw
        uv = pc[:, :2] / pc[:, 2:3] * f + np.array([W / 2.0, H / 2.0])
        u0, v0 = np.clip(np.floor(uv.min(0)), 0, [W - 1, H - 1]).astype(int)
        u1, v1 = np.clip(np.ceil(uv.max(0)), 0, [W - 1, H - 1]).astype(int)
        us, vs = np.meshgrid(np.arange(u0, u1 + 1, stride), np.arange(v0, v1 + 1, stride))
        us, vs = us.ravel().astype(np.float64), vs.ravel().astype(np.float64)
        ow, dw = pixel_rays(R_cw, cam_w, f, f, W / 2.0, H / 2.0, us, vs)
        oo = (ow - t) @ R          # R^T (x - t)
        do = dw @ R
        th = shape.first_hit(oo, do)
        hit = np.isfinite(th)
        rgb = np.tile(rng.uniform(0, 1, size=3), (us.size, 1))   # background texture (unused by the loss)
        rgb[hit] = shape.colour(oo[hit] + th[hit, None] * do[hit])
        cls = np.where(hit, CLS_OBJECT, CLS_BACKGROUND).astype(np.uint8)
        if occluder_prob > 0 and rng.uniform() < occluder_prob:
            cu, cv = rng.uniform(u0, u1 + 1), rng.uniform(v0, v1 + 1)
            rad = rng.uniform(0.1, 0.3) * max(u1 - u0 + 1, v1 - v0 + 1)
            occ = (us - cu) ** 2 + (vs - cv) ** 2 < rad ** 2
            cls[occ] = CLS_OCCLUDER
            rgb[occ] = 0.3
        depth = np.full(us.size, np.nan)
        obj = np.nonzero(cls == CLS_OBJECT)[0]
        if depth_frac > 0 and obj.size:
            pick = obj[rng.uniform(size=obj.size) < depth_frac]
            depth[pick] = th[pick]
        outs["origin"].append(ow); outs["dir"].append(dw); outs["rgb"].append(rgb)
        outs["depth"].append(depth); outs["cls"].append(cls)
    pool = {k: np.concatenate(v) for k, v in outs.items()}
    for k in ("origin", "dir", "rgb", "depth"):
        pool[k] = np.ascontiguousarray(pool[k], np.float32)
    pool["cls"] = np.ascontiguousarray(pool["cls"], np.uint8)
    return pool


def config0_scene(seed=0, n_rays=256):
    """One object: ellipsoid (0.4, 0.3, 0.2), colour 0.5 + 0.5 sin(3x, 3y, 3z), white background; 4 cameras
    64x64 (fx = fy = 64) at azimuth k*90 deg, elevation 30 deg, radius 2.5; n_rays drawn from pixels whose ray
    hits the AABB [-0.5, 0.5]^3.  All rays are object rays (class 0) without depth."""
    shape = Shape(kind="ellipsoid", axes=np.array([0.4, 0.3, 0.2]), colour_kind="sin3")
    half = np.array([0.5, 0.5, 0.5])
    O, D = [], []
    for k in range(4):
        cam = sphere_position(2.5, np.deg2rad(90.0 * k), np.deg2rad(30.0))
        R_cw = look_at(cam)
        us, vs = np.meshgrid(np.arange(64), np.arange(64))
        ow, dw = pixel_rays(R_cw, cam, 64.0, 64.0, 32.0, 32.0, us.ravel().astype(float), vs.ravel().astype(float))
        O.append(ow); D.append(dw)
    ow, dw = np.concatenate(O), np.concatenate(D)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / dw
        ta, tb = (-half - ow) * inv, (half - ow) * inv
    tmin = np.maximum(np.nanmax(np.minimum(ta, tb), -1), 0.0)
    tmax = np.nanmin(np.maximum(ta, tb), -1)
    cand = np.nonzero(tmax > tmin + 1e-3)[0]
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(cand, size=n_rays, replace=False))
    ow, dw = ow[pick], dw[pick]
    th = shape.first_hit(ow, dw)
    rgb = np.ones((n_rays, 3))
    hit = np.isfinite(th)
    rgb[hit] = shape.colour(ow[hit] + th[hit, None] * dw[hit])
    pool = dict(origin=ow.astype(np.float32), dir=dw.astype(np.float32), rgb=rgb.astype(np.float32),
                depth=np.full(n_rays, np.nan, np.float32), cls=np.zeros(n_rays, np.uint8))
    return ObjectScene(shape=shape, t=np.zeros(3), yaw=0.0, half=half, seed=seed, pool=pool)


def multi_object_scene(n_objects=8, seed0=1, n_frames=30, W=320, H=240, f=320.0, depth_frac=0.02,
                       occluder_prob=0.3, posed=True, stride=1):
    """Objects as seeded random ellipsoids / superellipsoids / boxes (semi-axes U(0.1, 0.5)) in their own
    unit AABB, each with a smooth random colour field, seen in n_frames frames of W x H from random poses on
    a radius-2.5 sphere.  Object k uses seed seed0 + k.  Rays are the pixels of the object's detection box
    (projection of its 3D box); class from the analytic mask, random occluder discs, and depth_frac of the
    object rays carry the first-hit depth."""
    scenes = []
    for k in range(n_objects):
        seed = seed0 + k
        rng = np.random.default_rng(seed)
        shape = random_shape(rng, k)
        t = rng.uniform(-2.0, 2.0, size=3) * np.array([1.0, 1.0, 0.2]) if posed else np.zeros(3)
        yaw = float(rng.uniform(-np.pi, np.pi)) if posed else 0.0
        half = np.array([0.5, 0.5, 0.5])
        pool = _object_rays(shape, t, yaw, half, rng, n_frames, W, H, f, depth_frac, occluder_prob, stride=stride)
        scenes.append(ObjectScene(shape=shape, t=t, yaw=yaw, half=half, seed=seed, pool=pool))
    return scenes


def occupancy_bits(shape, half, dilate=2, p=0.0, seed=0, res=64):
    """64^3 occupancy bitgrid (x fastest, 64-bit words): cells whose centre lies within `dilate` cells of the
    shape, OR'd with Bernoulli(p) cells."""
    g = (np.arange(res) + 0.5) / res
    xs = -half[0] + 2 * half[0] * g
    ys = -half[1] + 2 * half[1] * g
    zs = -half[2] + 2 * half[2] * g
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    occ = shape.inside(np.stack([X, Y, Z], -1))
    for _ in range(dilate):
        o2 = occ.copy()
        for ax in range(3):
            o2 |= np.roll(occ, 1, ax) | np.roll(occ, -1, ax)
        occ = o2
    if p > 0:
        occ |= np.random.default_rng(seed).uniform(size=occ.shape) < p
    flat = occ.reshape(-1).astype(np.uint64)          # index x + 64 y + 4096 z
    words = np.zeros(flat.size // 64, np.uint64)
    for b in range(64):
        words |= flat[b::64] << np.uint64(b)
    return words


def random_params(n, seed, scale=1.0):
    """Uniform U(-scale, scale) parameters (for parity cases with non-trivial densities)."""
    return np.random.default_rng(seed).uniform(-scale, scale, size=n)


# --------------------------------------------------------------------------
# Streaming sequence: objects in a room seen along a camera path
# --------------------------------------------------------------------------
@dataclass
class StreamObject:
    shape: Shape
    t: np.ndarray
    yaw: float
    half: np.ndarray
    seed: int


@dataclass
class StreamScene:
    objects: list
    cam_pos: np.ndarray            # [n_frames, 3] camera centres (world)
    cam_rot: np.ndarray            # [n_frames, 3, 3] camera-to-world rotations
    W: int
    H: int
    f: float
    rate_hz: float


def streaming_scene(n_objects=96, n_frames=600, W=640, H=480, f=525.0, rate_hz=25.0, seed=1000, extent=12.0):
    """Objects (random shapes as in multi_object_scene, unit boxes, random yaw) standing on the floor of a
    2 extent x 2 extent room at least 1.5 apart, and a camera at eye height (1.6) that follows a figure-eight
    around the room over n_frames frames (rate_hz) while looking towards the room's centre region."""
    rng = np.random.default_rng(seed)
    objs = []
    pos = []
    tries = 0
    while len(objs) < n_objects:
        tries += 1
        if tries > 200 * n_objects:
            raise ValueError("the room is too small for the objects at the minimum spacing")
        p = np.array([rng.uniform(-extent, extent), rng.uniform(-extent, extent), 0.5])
        if any(np.linalg.norm(p[:2] - q[:2]) < 1.5 for q in pos):
            continue
        k = len(objs)
        orng = np.random.default_rng(seed + 1 + k)
        objs.append(StreamObject(shape=random_shape(orng, k), t=p, yaw=float(orng.uniform(-np.pi, np.pi)),
                                 half=np.array([0.5, 0.5, 0.5]), seed=seed + 1 + k))
        pos.append(p)
    s = np.arange(n_frames) / n_frames * 2.0 * np.pi
    cam = np.stack([0.85 * extent * np.sin(s), 0.6 * extent * np.sin(2.0 * s), np.full(n_frames, 1.6)], axis=1)
    look = np.stack([0.35 * extent * np.sin(s + 0.9), 0.35 * extent * np.cos(s + 0.4), np.full(n_frames, 0.5)],
                    axis=1)
    rot = np.stack([look_at(c, t) for c, t in zip(cam, look)])
    return StreamScene(objects=objs, cam_pos=cam, cam_rot=rot, W=W, H=H, f=f, rate_hz=rate_hz)


def detection_box(obj, cam_pos, R_cw, W, H, f):
    """Pixel rectangle (u0, v0, u1, v1) of the object's projected 3D box clipped to the image, or None when a box
    corner is behind the camera or the rectangle is empty."""
    R = yaw_matrix(obj.yaw)
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * obj.half
    pc = ((corners @ R.T) + obj.t - cam_pos) @ R_cw
    if np.any(pc[:, 2] <= 0.1):
        return None
    uv = pc[:, :2] / pc[:, 2:3] * f + np.array([W / 2.0, H / 2.0])
    u0, v0 = np.floor(uv.min(0))
    u1, v1 = np.ceil(uv.max(0))
    u0, v0, u1, v1 = max(u0, 0), max(v0, 0), min(u1, W - 1), min(v1, H - 1)
    if u1 < u0 or v1 < v0:
        return None
    return int(u0), int(v0), int(u1), int(v1)


def frame_rays(obj, cam_pos, R_cw, box, f, W, H, rng, stride=2, depth_frac=0.02, occluder_prob=0.3):
    """World-frame rays of the pixels of the detection box (every stride-th pixel), with the object's analytic
    colour and mask class, random occluder discs and sparse first-hit depth, as in multi_object_scene."""
    u0, v0, u1, v1 = box
    us, vs = np.meshgrid(np.arange(u0, u1 + 1, stride), np.arange(v0, v1 + 1, stride))
    us, vs = us.ravel().astype(np.float64), vs.ravel().astype(np.float64)
    ow, dw = pixel_rays(R_cw, cam_pos, f, f, W / 2.0, H / 2.0, us, vs)
    R = yaw_matrix(obj.yaw)
    oo = (ow - obj.t) @ R
    do = dw @ R
    th = obj.shape.first_hit(oo, do)
    hit = np.isfinite(th)
    rgb = np.tile(rng.uniform(0, 1, size=3), (us.size, 1))
    rgb[hit] = obj.shape.colour(oo[hit] + th[hit, None] * do[hit])
    cls = np.where(hit, CLS_OBJECT, CLS_BACKGROUND).astype(np.uint8)
    if occluder_prob > 0 and rng.uniform() < occluder_prob:
        cu, cv = rng.uniform(u0, u1 + 1), rng.uniform(v0, v1 + 1)
        rad = rng.uniform(0.1, 0.3) * max(u1 - u0 + 1, v1 - v0 + 1)
        occ = (us - cu) ** 2 + (vs - cv) ** 2 < rad ** 2
        cls[occ] = CLS_OCCLUDER
        rgb[occ] = 0.3
    depth = np.full(us.size, np.nan)
    idx = np.nonzero(cls == CLS_OBJECT)[0]
    if depth_frac > 0 and idx.size:
        pick = idx[rng.uniform(size=idx.size) < depth_frac]
        depth[pick] = th[pick]
    return dict(origin=np.ascontiguousarray(ow, np.float32), dir=np.ascontiguousarray(dw, np.float32),
                rgb=np.ascontiguousarray(rgb, np.float32), depth=np.ascontiguousarray(depth, np.float32),
                cls=np.ascontiguousarray(cls, np.uint8))
