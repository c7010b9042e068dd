"""Seeded synthetic rectified stereo sequences: the inputs shared by the oracle, the CUDA path,
the tests and the benchmark.

This module holds none of the method's arithmetic (no disparity-space warp, census, matching,
aggregation or Kalman code). It renders static planar scenes by ray-plane intersection:

* a ground plane Y = +h (camera frame: x right, y down, z forward; h = 1.65 m camera height),
* fronto-parallel rectangular boxes standing on the ground (faces Z = const in the world frame),
* a distant textured wall (Z = far) that plays the sky,

each textured with seeded bilinear value noise on a world-anchored lattice, so that texture moves
consistently with the camera. Left camera at the rig origin, right camera at +b along x
(rectified pair), pinhole with principal point cx=(W-1)/2, cy=(H-1)/2 and fx=fy=f.
Ground-truth disparity of the left image is f*b/Z for the nearest hit.

Poses follow the convention M^k = R M^{k-1} + t (previous camera frame to current camera frame):
moving the rig forward by s metres gives t = (0, 0, -s).

All randomness is counter-based (SplitMix64 finaliser over a key built from seed, purpose and
index) so every array is a pure function of its seed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_U64 = np.uint64
_GOLD = _U64(0x9E3779B97F4A7C15)
_M1 = _U64(0xBF58476D1CE4E5B9)
_M2 = _U64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) applied elementwise to uint64 arrays."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLD
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
        return z ^ (z >> _U64(31))


def _key(*parts) -> np.ndarray:
    """Mix integer parts (scalars or arrays, may be negative) into one uint64 key array."""
    acc = np.zeros((), dtype=np.uint64)
    for p in parts:
        a = np.asarray(p)
        a = a.astype(np.int64).astype(np.uint64) if a.dtype != np.uint64 else a
        acc = splitmix64(acc ^ a)
    return acc


def uniform01(*parts) -> np.ndarray:
    """Counter-based uniform draws in [0, 1) with 53-bit resolution."""
    return (_key(*parts) >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Stream:
    """Sequential view of the counter-based generator (for scene layout draws)."""

    def __init__(self, seed: int, purpose: int):
        self.seed, self.purpose, self.n = int(seed), int(purpose), 0

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = float(uniform01(self.seed, self.purpose, self.n))
        self.n += 1
        return lo + (hi - lo) * u


# ----------------------------------------------------------------------------------------------
# Scene description
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    ground_y: float                 # ground plane Y = ground_y (y down)
    far_z: float                    # distant wall Z = far_z
    boxes: np.ndarray               # (n, 4): x0, x1, y_top, z  (face spans x0..x1, y_top..ground_y)
    tex_seed: int
    tex_cell: float = 0.10          # lattice spacing (m) on ground and boxes
    far_cell: float = 2.0           # lattice spacing (m) on the far wall


@dataclasses.dataclass
class Camera:
    W: int
    H: int
    f: float
    b: float

    @property
    def cx(self) -> float:
        return (self.W - 1) / 2.0

    @property
    def cy(self) -> float:
        return (self.H - 1) / 2.0

    @property
    def K(self) -> np.ndarray:
        return np.array([[self.f, 0.0, self.cx], [0.0, self.f, self.cy], [0.0, 0.0, 1.0]],
                        dtype=np.float32)


def rot_y(angle: float) -> np.ndarray:
    c, s = math.cos(angle), math.sin(angle)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_xyz(rx: float, ry: float, rz: float) -> np.ndarray:
    cx_, sx = math.cos(rx), math.sin(rx)
    cy_, sy = math.cos(ry), math.sin(ry)
    cz, sz = math.cos(rz), math.sin(rz)
    Rx = np.array([[1, 0, 0], [0, cx_, -sx], [0, sx, cx_]])
    Ry = np.array([[cy_, 0, sy], [0, 1, 0], [-sy, 0, cy_]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _value_noise(seed: int, pid, a: np.ndarray, b: np.ndarray, cell: float) -> np.ndarray:
    """Bilinear value noise in [0, 1) on a lattice of spacing `cell`, keyed by plane id."""
    ga, gb = a / cell, b / cell
    ia, ib = np.floor(ga), np.floor(gb)
    fa, fb = ga - ia, gb - ib
    ia = ia.astype(np.int64)
    ib = ib.astype(np.int64)
    v00 = uniform01(seed, pid, ia, ib)
    v10 = uniform01(seed, pid, ia + 1, ib)
    v01 = uniform01(seed, pid, ia, ib + 1)
    v11 = uniform01(seed, pid, ia + 1, ib + 1)
    return (v00 * (1 - fa) + v10 * fa) * (1 - fb) + (v01 * (1 - fa) + v11 * fa) * fb


def render(scene: Scene, cam: Camera, R_wc: np.ndarray, c_w: np.ndarray, right: bool = False):
    """Ray-cast one view. Returns (intensity float64 in [0,255], depth Z (camera frame) float64).

    R_wc rotates camera-frame vectors into the world frame, c_w is the left camera centre.
    """
    H, W, f = cam.H, cam.W, cam.f
    u = np.arange(W, dtype=np.float64)
    v = np.arange(H, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    dc = np.stack([(uu - cam.cx) / f, (vv - cam.cy) / f, np.ones_like(uu)], axis=-1)  # z = 1
    dw = dc @ R_wc.T
    o = np.asarray(c_w, dtype=np.float64) + (R_wc @ np.array([cam.b, 0.0, 0.0]) if right else 0.0)
    dx, dy, dz = dw[..., 0], dw[..., 1], dw[..., 2]
    inf = np.inf
    best_t = np.full((H, W), inf)
    pid = np.full((H, W), -1, dtype=np.int64)

    with np.errstate(divide="ignore", invalid="ignore"):
        # ground plane
        tg = (scene.ground_y - o[1]) / dy
        ok = (dy > 1e-12) & (tg > 1e-6)
        upd = ok & (tg < best_t)
        best_t = np.where(upd, tg, best_t)
        pid = np.where(upd, 0, pid)
        # boxes (front faces)
        for k, (x0, x1, ytop, zb) in enumerate(scene.boxes):
            tb = (zb - o[2]) / dz
            X = o[0] + tb * dx
            Y = o[1] + tb * dy
            ok = (dz > 1e-12) & (tb > 1e-6) & (X >= x0) & (X <= x1) & (Y >= ytop) & (Y <= scene.ground_y)
            upd = ok & (tb < best_t)
            best_t = np.where(upd, tb, best_t)
            pid = np.where(upd, k + 1, pid)
        # far wall
        tf = (scene.far_z - o[2]) / dz
        ok = (dz > 1e-12) & (tf > 1e-6)
        upd = ok & (tf < best_t)
        best_t = np.where(upd, tf, best_t)
        pid = np.where(upd, 9999, pid)

    t = np.where(np.isfinite(best_t), best_t, 1e9)
    P = o + t[..., None] * dw
    val = np.zeros((H, W))
    m = pid == 0
    val[m] = _value_noise(scene.tex_seed, 0, P[..., 0][m], P[..., 2][m], scene.tex_cell)
    for k in range(len(scene.boxes)):
        m = pid == k + 1
        if m.any():
            val[m] = _value_noise(scene.tex_seed, k + 1, P[..., 0][m], P[..., 1][m], scene.tex_cell)
    m = pid == 9999
    val[m] = _value_noise(scene.tex_seed, 9999, P[..., 0][m], P[..., 1][m], scene.far_cell)
    m = pid < 0
    val[m] = 0.5
    # dc has unit z, so the ray parameter is the camera-frame depth of the hit
    return 255.0 * val, t


def gaussian_noise(seed: int, frame: int, view: int, shape, sigma: float) -> np.ndarray:
    """Box-Muller normal draws from the counter-based generator."""
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    u1 = uniform01(seed, 0x6E6F, frame, view, 2 * idx)
    u2 = uniform01(seed, 0x6E6F, frame, view, 2 * idx + 1)
    u1 = np.maximum(u1, 1e-300)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return (sigma * z).reshape(shape)


def _to_u8(img: np.ndarray) -> np.ndarray:
    return np.clip(np.floor(img + 0.5), 0, 255).astype(np.uint8)


@dataclasses.dataclass
class Sequence:
    cam: Camera
    left: list          # uint8 (H, W) per frame
    right: list
    gt_disp: list       # float32 (H, W) left ground-truth disparity per frame
    R: list             # float32 (3,3) relative pose frame k-1 -> k, index k (R[0] = identity)
    t: list             # float32 (3,)
    scene: Scene
    R_wc: list = None   # camera-to-world rotation of every frame
    c_w: list = None    # camera centre of every frame

    def pose_between(self, i: int, j: int):
        """Relative pose (R, t) mapping frame i camera coordinates to frame j's (Eq. 2 form)."""
        R = self.R_wc[j].T @ self.R_wc[i]
        t = self.R_wc[j].T @ (self.c_w[i] - self.c_w[j])
        return R.astype(np.float32), t.astype(np.float32)

    @property
    def K(self) -> np.ndarray:
        return self.cam.K


def make_scene(seed: int, cam: Camera, n_boxes: int, z_range, travel: float,
               x_half: float = 8.0) -> Scene:
    rs = Stream(seed, 0x5CE7E)
    boxes = []
    for _ in range(n_boxes):
        z = rs.uniform(z_range[0], z_range[1]) + travel
        # keep the box horizontally inside the first frame's field of view
        half = min(x_half, 0.9 * z * (cam.W / 2.0) / cam.f)
        xc = rs.uniform(-half, half)
        w = rs.uniform(1.0, 3.0)
        h = rs.uniform(1.0, 2.5)
        boxes.append((xc - w / 2, xc + w / 2, 1.65 - h, z))
    return Scene(ground_y=1.65, far_z=400.0, boxes=np.array(boxes, dtype=np.float64).reshape(-1, 4),
                 tex_seed=seed * 7919 + 17)


def make_sequence(seed: int, W: int, H: int, f: float, b: float, n_frames: int, n_boxes: int,
                  z_range=(5.0, 60.0), step_range=(0.5, 1.5), yaw_deg: float = 2.0,
                  noise_sigma: float = 0.0) -> Sequence:
    """Render a static-scene sequence with per-frame forward motion and yaw."""
    cam = Camera(W, H, f, b)
    rs = Stream(seed, 0x9053)
    steps, yaws = [], []
    for _ in range(1, n_frames):
        steps.append(rs.uniform(*step_range))
        yaws.append(math.radians(rs.uniform(-yaw_deg, yaw_deg)))
    scene = make_scene(seed, cam, n_boxes, z_range, travel=float(sum(steps)))
    R_wc = [np.eye(3)]
    c_w = [np.zeros(3)]
    for s, a in zip(steps, yaws):
        c_new = c_w[-1] + R_wc[-1] @ np.array([0.0, 0.0, s])
        R_wc.append(R_wc[-1] @ rot_y(a))
        c_w.append(c_new)
    left, right, gt, Rs, ts = [], [], [], [], []
    for k in range(n_frames):
        Il, Z = render(scene, cam, R_wc[k], c_w[k], right=False)
        Ir, _ = render(scene, cam, R_wc[k], c_w[k], right=True)
        if noise_sigma > 0:
            Il = Il + gaussian_noise(seed, k, 0, Il.shape, noise_sigma)
            Ir = Ir + gaussian_noise(seed, k, 1, Ir.shape, noise_sigma)
        left.append(_to_u8(Il))
        right.append(_to_u8(Ir))
        gt.append((f * b / Z).astype(np.float32))
        if k == 0:
            Rs.append(np.eye(3, dtype=np.float32))
            ts.append(np.zeros(3, dtype=np.float32))
        else:
            Rrel = R_wc[k].T @ R_wc[k - 1]
            trel = R_wc[k].T @ (c_w[k - 1] - c_w[k])
            Rs.append(Rrel.astype(np.float32))
            ts.append(trel.astype(np.float32))
    return Sequence(cam, left, right, gt, Rs, ts, scene, R_wc, c_w)


# ----------------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------------

def small_pair(seed: int = 1) -> Sequence:
    """320x96 two-frame pair: ground + 4 boxes, pure forward translation 0.5 m, no image noise."""
    return make_sequence(seed, 320, 96, 721.0, 0.54, n_frames=2, n_boxes=4,
                         step_range=(0.5, 0.5), yaw_deg=0.0, noise_sigma=0.0)


def kitti_like(seed: int = 2, n_frames: int = 10) -> Sequence:
    """1242x375 driving-shaped sequence: ground + 20 boxes at 5-60 m, noise sigma 2 gray levels,
    forward 0.5-1.5 m and yaw +-2 deg per frame."""
    return make_sequence(seed, 1242, 375, 721.0, 0.54, n_frames=n_frames, n_boxes=20,
                         step_range=(0.5, 1.5), yaw_deg=2.0, noise_sigma=2.0)


MIX_SHAPES = [(640, 480, 64), (1242, 375, 128), (1920, 1080, 256)]


def mix_shape(i: int):
    """(W, H, D) of stream i of the multi-camera workloads: 640x480 D=64, 1242x375 D=128,
    1920x1080 D=256 in turn."""
    return MIX_SHAPES[i % 3]


def camera_mix(n_frames: int) -> dict:
    """One driving-shaped sequence per image size of the multi-camera workloads, keyed (W, H):
    ground + 20 boxes, noise sigma 2, focal length 721 px scaled with the width, baseline 0.54 m."""
    out = {}
    for k, (W, H, _) in enumerate(MIX_SHAPES):
        out[(W, H)] = make_sequence(100 + k, W, H, 721.0 * W / 1242.0, 0.54, n_frames=n_frames,
                                    n_boxes=20, noise_sigma=2.0)
    return out


def shifted_view(seq: Sequence, shift: int):
    """The sequence seen by a camera whose principal point sits `shift` pixels further right:
    both views of every frame rolled right by `shift` columns (the wrapped columns are the only
    pixels not consistent with the geometry) and the intrinsics' cx moved with them. Gives
    streams of one size distinct images with the same motion."""
    K = seq.K.astype(np.float32).copy()
    K[0, 2] += shift
    left = [np.ascontiguousarray(np.roll(x, shift, axis=1)) for x in seq.left]
    right = [np.ascontiguousarray(np.roll(x, shift, axis=1)) for x in seq.right]
    return left, right, K


def random_maps(seed: int, W: int, H: int, d_range=(1.0, 127.0), p_range=(0.1, 4.0),
                invalid_frac: float = 0.0):
    """Random previous disparity/variance maps (float32), optionally with invalid (-1) pixels."""
    n = W * H
    idx = np.arange(n, dtype=np.int64)
    d = d_range[0] + (d_range[1] - d_range[0]) * uniform01(seed, 0xD, idx)
    p = p_range[0] + (p_range[1] - p_range[0]) * uniform01(seed, 0xE, idx)
    d = d.astype(np.float32).reshape(H, W)
    p = p.astype(np.float32).reshape(H, W)
    if invalid_frac > 0:
        bad = (uniform01(seed, 0xF, idx) < invalid_frac).reshape(H, W)
        d[bad] = -1.0
        p[bad] = -1.0
    return d, p


def random_pose(seed: int, max_t: float = 1.5, max_rot_deg: float = 3.0):
    """Random 6-DoF pose with |t| <= max_t and each rotation angle within +-max_rot_deg."""
    rs = Stream(seed, 0x7053)
    ang = [math.radians(rs.uniform(-max_rot_deg, max_rot_deg)) for _ in range(3)]
    t = np.array([rs.uniform(-1, 1) for _ in range(3)])
    t = t / max(np.linalg.norm(t), 1e-12) * rs.uniform(0.0, max_t)
    return rot_xyz(*ang).astype(np.float32), t.astype(np.float32)


def random_images(seed: int, W: int, H: int):
    """Independent uniform-noise uint8 left/right images (no geometry), for cost/census tests."""
    n = W * H
    idx = np.arange(n, dtype=np.int64)
    a = (uniform01(seed, 0x11, idx) * 256).astype(np.uint8).reshape(H, W)
    b = (uniform01(seed, 0x12, idx) * 256).astype(np.uint8).reshape(H, W)
    return a, b


def random_windows(seed: int, W: int, H: int, D: int, w_min: int = 1, w_max: int = 24,
                   full_frac: float = 0.0):
    """Random per-pixel windows [lo, hi] inside [0, D-1] (int16), a fraction of them full range."""
    n = W * H
    idx = np.arange(n, dtype=np.int64)
    w = w_min + np.floor(uniform01(seed, 0x21, idx) * (w_max - w_min + 1)).astype(np.int64)
    w = np.minimum(w, D)
    lo = np.floor(uniform01(seed, 0x22, idx) * (D - w + 1)).astype(np.int64)
    hi = lo + w - 1
    if full_frac > 0:
        full = uniform01(seed, 0x23, idx) < full_frac
        lo[full] = 0
        hi[full] = D - 1
    return lo.astype(np.int16).reshape(H, W), hi.astype(np.int16).reshape(H, W)


def mixed_windows(seed: int, W: int, H: int, D: int, narrow=(1, 16), wide=(17, 40),
                  wide_frac: float = 0.0, full_frac: float = 0.0):
    """Windows centred on a smooth disparity surface, so that neighbouring windows overlap and
    shift by a few labels like windows around a prediction: widths uniform in `narrow`, a fraction
    `wide_frac` uniform in `wide`, a fraction `full_frac` the full range (int16 lo, hi)."""
    n = W * H
    idx = np.arange(n, dtype=np.int64)
    x = (idx % W).astype(np.float64)
    y = (idx // W).astype(np.float64)
    phase = 6.2831853 * uniform01(seed, 0x31, np.zeros(1, np.int64))[0]
    centre = (D - 1) * (0.5 + 0.35 * np.sin(6.2831853 * x / 97.0 + phase) *
                        np.cos(6.2831853 * y / 53.0))
    u = uniform01(seed, 0x32, idx)
    w = narrow[0] + np.floor(u * (narrow[1] - narrow[0] + 1)).astype(np.int64)
    pick = uniform01(seed, 0x33, idx)
    wide_w = wide[0] + np.floor(uniform01(seed, 0x34, idx) * (wide[1] - wide[0] + 1)).astype(np.int64)
    w = np.where(pick < wide_frac, wide_w, w)
    w = np.clip(w, 1, D)
    lo = np.clip(np.round(centre - w / 2.0).astype(np.int64), 0, D - w)
    hi = lo + w - 1
    full = (pick >= wide_frac) & (pick < wide_frac + full_frac)
    lo[full] = 0
    hi[full] = D - 1
    return lo.astype(np.int16).reshape(H, W), hi.astype(np.int16).reshape(H, W)

