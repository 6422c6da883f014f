"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module generates data only (meshes, reflectivities, point scatterers, sensor
parameters, poses, sound-speed profiles). It holds none of the echo-formation
arithmetic. The paper's harbour data and the Water Linked 3D-15 datasheet values are
not available, so every workload is synthetic, shaped like the paper's scenes
(harbour sheet-pile wall over a seabed, Sec. V; sensor grid of Sec. III Eq. 1-3).

Conventions: world frame z up, sea surface at z = 0. Sonar frame x forward, y left,
z up. A pose is {"t": (3,) float64, "q": (4,) float64 unit quaternion (w, x, y, z)}
rotating sonar-frame vectors into the world frame.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_WATER = 1500.0
F0 = 450e3

SCENE_SEED = 20260606
SPECKLE_SEED = 1
TRAJ_SEED = 7


@dataclass
class Scene:
    verts: np.ndarray            # float32 [V, 3]
    tris: np.ndarray             # int32 [T, 3]
    mu: np.ndarray               # float32 [T] backscatter coefficient
    flags: np.ndarray            # uint8 [T] bit0 = specular mirror
    points: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.float32))
    sigma: np.ndarray = field(default_factory=lambda: np.zeros((0,), np.float32))
    planes: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.float64))
    meta: dict = field(default_factory=dict)  # generator facts (e.g. the wall's standoff)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


# ------------------------------------------------------------------------ poses
def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _qaxis(axis, ang):
    s = math.sin(ang / 2)
    return np.array([math.cos(ang / 2), s * axis[0], s * axis[1], s * axis[2]])


def pose(t, yaw_deg=0.0, tilt_down_deg=0.0, roll_deg=0.0) -> dict:
    """Pose from heading (about world z), downward tilt of the forward axis (a positive
    rotation about the sonar y axis, which is left) and roll (about the forward axis)."""
    q = _qmul(_qaxis((0, 0, 1), math.radians(yaw_deg)),
              _qmul(_qaxis((0, 1, 0), math.radians(tilt_down_deg)),
                    _qaxis((1, 0, 0), math.radians(roll_deg))))
    q = q / np.linalg.norm(q)
    return {"t": np.asarray(t, np.float64).reshape(3), "q": q.astype(np.float64)}


# ------------------------------------------------------------------------ sensors
def sensor_params(name: str) -> dict:
    """Sensor and run parameters of the named workload.

    c1: 8x8 array, 32x16 beams, 256 bins to 5 m, 64x32 rays (tiny plain ping).
    c2: 32x32 array, 128x64 beams, 1024 bins to 15 m, 512x256 rays x 4 sub-rays.
    c3: the c1 sensor with 2-bounce routes (used with a linear sound-speed profile).
    c4: the c2 sensor with 512x256 rays and one sub-ray (batched trajectory).
    """
    lam = C_WATER / F0
    base = dict(nx=8, ny=8, pitch=lam / 2, f0=F0, bw=50e3, pulse=100e-6, c_ref=0.0,
                hfov=math.radians(90.0), vfov=math.radians(40.0),
                n_beam_az=32, n_beam_el=16, n_range=256, r_min=0.0, r_max=5.0, r_blank=0.3,
                n_ray_az=64, n_ray_el=32, n_sub=1, max_bounces=1, surface_z=0.0,
                r_surface=-1.0, r_seabed=0.5, alpha=0.0, seed=SPECKLE_SEED,
                thr_mode=1, thr=0.1)
    if name == "c1":
        return base
    if name == "c3":
        return dict(base, max_bounces=2)
    if name in ("c2", "c4"):
        p = dict(base, nx=32, ny=32, n_beam_az=128, n_beam_el=64, n_range=1024, r_max=15.0,
                 r_blank=0.5, n_ray_az=512, n_ray_el=256, n_sub=4)
        if name == "c4":
            p["n_sub"] = 1
        return p
    raise ValueError(name)


def ssp(name: str) -> dict:
    """Sound-speed profile: isovelocity 1500 m/s, or (c3) a linear gradient from
    1500 m/s at z = 0 to 1490 m/s at z = -10 m."""
    if name == "c3":
        return {"z": np.array([0.0, -10.0]), "c": np.array([1500.0, 1490.0])}
    return {"z": np.array([0.0]), "c": np.array([C_WATER])}


# ------------------------------------------------------------------------ meshes
def _grid_mesh(xs, ys, zfun):
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    Z = zfun(X, Y)
    verts = np.stack([X, Y, Z], -1).reshape(-1, 3)
    ny, nx = X.shape
    i = np.arange(nx - 1)
    j = np.arange(ny - 1)
    I, J = np.meshgrid(i, j, indexing="xy")
    v00 = (J * nx + I).ravel()
    v10 = v00 + 1
    v01 = v00 + nx
    v11 = v01 + 1
    tris = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    return verts, tris


def fbm_heightfield(n: int, rng: np.random.Generator, octaves=6, hurst=0.8, sigma=0.1):
    """Fractional Brownian motion on an n x n grid: octaves of bilinearly interpolated
    lattice noise with amplitude 2^(-o H), normalised to zero mean and std sigma."""
    u = np.linspace(0.0, 1.0, n)
    out = np.zeros((n, n))
    for o in range(octaves):
        cells = 4 * 2 ** o
        lat = rng.standard_normal((cells + 1, cells + 1))
        x = u * cells
        i0 = np.minimum(np.floor(x).astype(int), cells - 1)
        f = x - i0
        a = lat[i0][:, i0]
        b = lat[i0][:, i0 + 1]
        c = lat[i0 + 1][:, i0]
        d = lat[i0 + 1][:, i0 + 1]
        fy = f[:, None]
        fx = f[None, :]
        out += 2.0 ** (-o * hurst) * ((1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d))
    out -= out.mean()
    out *= sigma / out.std()
    return out


def corrugated_wall(x0=3.0, length=20.0, z_top=0.0, z_bot=-10.5, pitch=0.5, flange=0.15,
                    web=0.10, depth=0.12, n_vert=64):
    """Trapezoidal sheet-pile wall facing -x, running along y, front flange at x = x0."""
    n_p = int(round(length / pitch))
    ys, xs = [], []
    for k in range(n_p):
        y0 = -length / 2 + k * pitch
        ys += [y0, y0 + flange, y0 + flange + web, y0 + 2 * flange + web]
        xs += [x0, x0, x0 + depth, x0 + depth]
    ys.append(length / 2)
    xs.append(x0)
    ys = np.array(ys)
    xs = np.array(xs)
    zs = np.linspace(z_bot, z_top, n_vert + 1)
    ncol = len(ys)
    verts = np.zeros(((n_vert + 1) * ncol, 3))
    for r, z in enumerate(zs):
        verts[r * ncol:(r + 1) * ncol, 0] = xs
        verts[r * ncol:(r + 1) * ncol, 1] = ys
        verts[r * ncol:(r + 1) * ncol, 2] = z
    tris = []
    for r in range(n_vert):
        for c in range(ncol - 1):
            a = r * ncol + c
            b = a + 1
            cc = a + ncol
            d = cc + 1
            tris.append((a, b, d))
            tris.append((a, d, cc))
    return verts, np.array(tris, np.int64)


def _box(center, size, yaw):
    hx, hy, hz = size[0] / 2, size[1] / 2, size[2] / 2
    corners = np.array([[sx * hx, sy * hy, sz * hz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)])
    c, s = math.cos(yaw), math.sin(yaw)
    rot = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    v = corners @ rot.T + center
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    t = []
    for a, b, cq, d in quads:
        t += [(a, b, cq), (a, cq, d)]
    return v, np.array(t)


def _cylinder(center, radius, height, seg=16):
    ang = np.arange(seg) * 2 * math.pi / seg
    ring = np.stack([radius * np.cos(ang), radius * np.sin(ang)], 1)
    bot = np.concatenate([ring, np.full((seg, 1), -height / 2)], 1)
    top = np.concatenate([ring, np.full((seg, 1), height / 2)], 1)
    v = np.concatenate([bot, top, [[0, 0, -height / 2], [0, 0, height / 2]]], 0) + center
    cb, ct = 2 * seg, 2 * seg + 1
    t = []
    for k in range(seg):
        k2 = (k + 1) % seg
        t += [(k, k2, seg + k2), (k, seg + k2, seg + k)]
        t += [(cb, k2, k), (ct, seg + k, seg + k2)]
    return v, np.array(t)


def _assemble(parts):
    verts, tris, mu, flags = [], [], [], []
    off = 0
    for v, t, m, f in parts:
        verts.append(np.asarray(v, np.float64))
        tris.append(np.asarray(t, np.int64) + off)
        mu.append(np.broadcast_to(np.asarray(m, np.float32), (len(t),)))
        flags.append(np.full((len(t),), f, np.uint8))
        off += len(v)
    return (np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.int32),
            np.concatenate(mu).astype(np.float32), np.concatenate(flags))


def scene_c1(seed: int = SCENE_SEED) -> tuple:
    """Flat mirror seabed (two triangles, 20 m x 20 m at z = -4, reflectivity 0.3) and
    three unit point scatterers uniform over the field of view at ranges U(1, 4.5) m.
    Returns (scene, pose)."""
    rng = np.random.default_rng(seed)
    ps = pose((0.0, 0.0, -2.0), tilt_down_deg=15.0)
    sea = np.array([[-7.0, -9.3, -4.0], [13.0, -9.3, -4.0], [13.0, 10.7, -4.0], [-7.0, 10.7, -4.0]])
    verts, tris, mu, flags = _assemble([(sea, [(0, 1, 2), (0, 2, 3)], 0.3, 1)])
    R = _rot(ps["q"])
    pts = []
    while len(pts) < 3:
        az = rng.uniform(-math.pi / 4, math.pi / 4)
        el = rng.uniform(-math.radians(20), math.radians(20))
        r = rng.uniform(1.0, 4.5)
        u = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        x = R @ (r * u) + ps["t"]
        if x[2] > -3.9:
            pts.append(x)
    sc = Scene(verts, tris, mu, flags, np.array(pts, np.float32), np.ones(3, np.float32),
               np.array([[0.0, 0.0, 1.0, -4.0]]))
    return sc, ps


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def scene_c2(seed: int = SCENE_SEED) -> tuple:
    """Harbour sheet-pile wall (20 m long, ~20.5k triangles, front flange 3 m ahead of
    the sonar) over an fBm seabed (256 x 256 vertices over 30 m x 30 m, std 0.1 m,
    mean z = -10, mirror). Reflectivity U(0.1, 0.6) per triangle. Sonar at z = -8,
    facing the wall, tilted 10 degrees down. Returns (scene, pose)."""
    rng = np.random.default_rng(seed)
    wv, wt = corrugated_wall()
    hf = fbm_heightfield(256, rng)
    xs = np.linspace(-15.0, 15.0, 256)
    sv, st = _grid_mesh(xs, xs, lambda X, Y: -10.0 + hf)
    verts, tris, _, flags = _assemble([(wv, wt, 0.0, 0), (sv, st, 0.0, 1)])
    mu = rng.uniform(0.1, 0.6, size=len(tris)).astype(np.float32)
    sc = Scene(verts, tris, mu, flags, planes=np.array([[0.0, 0.0, 1.0, -10.0]]))
    return sc, pose((0.0, 0.0, -8.0), tilt_down_deg=10.0)


def scene_c4(seed: int = SCENE_SEED) -> Scene:
    """The c2 wall over a coarser fBm seabed (128 x 128 vertices) with a field of 100
    boxes and 100 capped 16-segment cylinders resting on it (~60k triangles)."""
    rng = np.random.default_rng(seed + 4)
    wv, wt = corrugated_wall()
    hf = fbm_heightfield(128, rng)
    xs = np.linspace(-15.0, 15.0, 128)
    sv, st = _grid_mesh(xs, xs, lambda X, Y: -10.0 + hf)
    parts = [(wv, wt, 0.0, 0), (sv, st, 0.0, 1)]
    for _ in range(100):
        size = rng.uniform(0.1, 0.6, 3)
        c = np.array([rng.uniform(-7.0, 2.5), rng.uniform(-14.0, 14.0), -10.0 + size[2] / 2])
        v, t = _box(c, size, rng.uniform(0, math.pi))
        parts.append((v, t, 0.0, 0))
    for _ in range(100):
        r, h = rng.uniform(0.05, 0.3), rng.uniform(0.2, 1.0)
        c = np.array([rng.uniform(-7.0, 2.5), rng.uniform(-14.0, 14.0), -10.0 + h / 2])
        v, t = _cylinder(c, r, h)
        parts.append((v, t, 0.0, 0))
    verts, tris, _, flags = _assemble(parts)
    mu = rng.uniform(0.1, 0.6, size=len(tris)).astype(np.float32)
    return Scene(verts, tris, mu, flags, planes=np.array([[0.0, 0.0, 1.0, -10.0]]))


def trajectory_c4(n: int = 64, seed: int = TRAJ_SEED) -> list:
    """30 m lawnmower past the wall: 14 m leg at 3 m standoff, 2 m turn, 14 m leg at
    6 m standoff. Heading jitter +-5 deg, tilt/roll jitter +-3 deg, position +-0.1 m.
    The turn sweeps the heading through open water."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        s = 30.0 * k / (n - 1)
        if s <= 14.0:
            x, y, yaw = 0.0, -7.0 + s, 0.0
        elif s <= 16.0:
            f = (s - 14.0) / 2.0
            x, y, yaw = -3.0 * f, 7.0, 90.0 * math.sin(math.pi * f)
        else:
            x, y, yaw = -3.0, 7.0 - (s - 16.0), 0.0
        jit = rng.uniform(-1, 1, 6)
        out.append(pose((x + 0.1 * jit[0], y + 0.1 * jit[1], -8.0 + 0.1 * jit[2]),
                        yaw_deg=yaw + 5.0 * jit[3], tilt_down_deg=10.0 + 3.0 * jit[4],
                        roll_deg=3.0 * jit[5]))
    return out


def scene_wall_mirror(seed: int = SCENE_SEED) -> tuple:
    """Scene for out/back cross-term multipath: a flat mirror seabed (z = -4, two
    triangles, reflectivity 0.3); a vertical wall 6 m ahead (x = 6, 16 x 8 quads over
    y in [-5, 5], z in [-4, 0], reflectivity U(0.2, 0.6)) that seabed-reflected rays
    reach from below; a plate at x = 3 (y in [-0.8, 0.8], z in [-2.5, -2.2]) that hides
    part of that wall band from the sonar but not from the reflected routes; three unit
    point scatterers between the sonar and the plate. Sonar at (0, 0, -2) tilted 15
    degrees down. Returns (scene, pose)."""
    rng = np.random.default_rng(seed)
    sea = np.array([[-2.0, -8.0, -4.0], [12.0, -8.0, -4.0], [12.0, 8.0, -4.0], [-2.0, 8.0, -4.0]])
    ys, zs = np.linspace(-5.0, 5.0, 17), np.linspace(-4.0, 0.0, 9)
    wv = np.array([[6.0, y, z] for z in zs for y in ys])
    wt = []
    for j in range(len(zs) - 1):
        for i in range(len(ys) - 1):
            a = j * len(ys) + i
            wt += [(a, a + 1, a + len(ys) + 1), (a, a + len(ys) + 1, a + len(ys))]
    plate = np.array([[3.0, -0.8, -2.5], [3.0, 0.8, -2.5], [3.0, 0.8, -2.2], [3.0, -0.8, -2.2]])
    verts, tris, mu, flags = _assemble([(sea, [(0, 1, 2), (0, 2, 3)], 0.3, 1), (wv, wt, 0.0, 0),
                                        (plate, [(0, 1, 2), (0, 2, 3)], 0.5, 0)])
    mu[2:2 + len(wt)] = rng.uniform(0.2, 0.6, len(wt)).astype(np.float32)
    pts = np.stack([rng.uniform(1.0, 2.0, 3), rng.uniform(-1.5, 1.5, 3), rng.uniform(-3.5, -1.5, 3)], 1)
    sc = Scene(verts, tris, mu, flags, pts.astype(np.float32), np.ones(3, np.float32),
               np.array([[0.0, 0.0, 1.0, -4.0]]))
    return sc, pose((0.0, 0.0, -2.0), tilt_down_deg=15.0)


def workload(name: str):
    """(scene, params, poses, ssp) of a named workload; poses is a list.

    wall_mirror: the c1 sensor to 10 m (512 bins) without a sea surface, over
    scene_wall_mirror, for cross-term multipath."""
    if name == "wall_mirror":
        sc, ps = scene_wall_mirror()
        return sc, dict(sensor_params("c1"), r_max=10.0, n_range=512, surface_z=None), [ps], ssp("c1")
    if name in ("c1", "c3"):
        sc, ps = scene_c1()
        return sc, sensor_params(name), [ps], ssp(name)
    if name == "c2":
        sc, ps = scene_c2()
        return sc, sensor_params(name), [ps], ssp(name)
    if name == "c4":
        return scene_c4(), sensor_params(name), trajectory_c4(), ssp(name)
    raise ValueError(name)


# ------------------------------------------------------------------------ surrogate
SUR_CHANNELS = (4, 64, 64, 64, 64, 64, 1)
SUR_KERNEL = 9


def surrogate_init(seed: int = 11) -> np.ndarray:
    """Initial parameters of the surrogate network, packed layer by layer as
    W_l [cout][cin][9] then b_l [cout] (FP32): He-normal weights for the ReLU layers
    (std sqrt(2 / (cin 9))), std sqrt(1 / (cin 9)) for the linear output layer, zero
    biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(SUR_CHANNELS) - 1):
        cin, cout = SUR_CHANNELS[l], SUR_CHANNELS[l + 1]
        gain = 2.0 if l < len(SUR_CHANNELS) - 2 else 1.0
        parts.append(rng.normal(0.0, math.sqrt(gain / (cin * SUR_KERNEL)), cout * cin * SUR_KERNEL))
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def surrogate_unpack(theta: np.ndarray) -> dict:
    """{"W": [l][cout][cin][9], "b": [l][cout]} (float64) from the packed vector."""
    W, b, off = [], [], 0
    for l in range(len(SUR_CHANNELS) - 1):
        cin, cout = SUR_CHANNELS[l], SUR_CHANNELS[l + 1]
        n = cout * cin * SUR_KERNEL
        W.append(np.asarray(theta[off:off + n], np.float64).reshape(cout, cin, SUR_KERNEL))
        off += n
        b.append(np.asarray(theta[off:off + cout], np.float64))
        off += cout
    return {"W": W, "b": b}


def training_scene(seed: int) -> Scene:
    """A randomised harbour scene for surrogate training: a corrugated sheet-pile wall
    (standoff, pitch, flange, web and depth drawn per scene) over a mirror fBm seabed
    (mean depth 9..12 m, std 0.05..0.3 m, 128 x 128 vertices over 30 x 30 m) with 0..60
    boxes and cylinders; reflectivity U(0.1, 0.6) per triangle."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(2.5, 9.0)
    pitch = rng.uniform(0.35, 0.7)
    flange = pitch * rng.uniform(0.2, 0.35)
    web = pitch * rng.uniform(0.1, 0.25)
    wv, wt = corrugated_wall(x0=x0, pitch=pitch, flange=flange, web=web, depth=rng.uniform(0.05, 0.2))
    depth = rng.uniform(9.0, 12.0)
    hf = fbm_heightfield(128, rng, sigma=rng.uniform(0.05, 0.3))
    xs = np.linspace(-15.0, 15.0, 128)
    sv, st = _grid_mesh(xs, xs, lambda X, Y: -depth + hf)
    parts = [(wv, wt, 0.0, 0), (sv, st, 0.0, 1)]
    for _ in range(int(rng.integers(0, 31))):
        size = rng.uniform(0.1, 0.8, 3)
        c = np.array([rng.uniform(-2.0, x0 - 0.5), rng.uniform(-10.0, 10.0), -depth + size[2] / 2])
        v, t = _box(c, size, rng.uniform(0, math.pi))
        parts.append((v, t, 0.0, 0))
    for _ in range(int(rng.integers(0, 31))):
        r, h = rng.uniform(0.05, 0.4), rng.uniform(0.2, 1.5)
        c = np.array([rng.uniform(-2.0, x0 - 0.5), rng.uniform(-10.0, 10.0), -depth + h / 2])
        v, t = _cylinder(c, r, h)
        parts.append((v, t, 0.0, 0))
    verts, tris, _, flags = _assemble(parts)
    mu = rng.uniform(0.1, 0.6, size=len(tris)).astype(np.float32)
    return Scene(verts, tris, mu, flags, planes=np.array([[0.0, 0.0, 1.0, -depth]]),
                 meta={"wall_x": x0, "depth": depth})


def training_poses(seed: int, n: int, scene: Scene) -> list:
    """n seeded sonar poses in a training scene: 1.5..7 m in front of the wall's front
    face, 1..6 m above the seabed's mean plane, heading within 30 degrees of the wall
    normal, tilted 0..20 degrees down, rolled within 3 degrees."""
    rng = np.random.default_rng(seed)
    x_wall, depth = scene.meta["wall_x"], scene.meta["depth"]
    out = []
    for _ in range(n):
        x = x_wall - rng.uniform(1.5, 7.0)
        z = -depth + rng.uniform(1.0, 6.0)
        out.append(pose((x, rng.uniform(-6.0, 6.0), z), yaw_deg=rng.uniform(-30.0, 30.0),
                        tilt_down_deg=rng.uniform(0.0, 20.0), roll_deg=rng.uniform(-3.0, 3.0)))
    return out
