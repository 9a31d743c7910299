"""Seeded synthetic inputs: scenes, cameras and ray batches.

This module only generates inputs. It holds none of the light-transport
arithmetic (no intersection, sampling, shading or accumulation) and imports
nothing but numpy, so both the CUDA path and the FP64 oracle can be fed from
it. All randomness comes from SplitMix64 (Steele, Lea and Flood 2014) used as
a counter-based generator: draw k of stream s is mix(s + (k + 1) * gamma).

Workloads (stand-ins for the paper's proprietary scenes, which are not
available): a Cornell-style box (34 triangles + a 2-triangle emitter), a field
of 200 noise-displaced tessellated spheres on a displaced plane (1,000,000
triangles, 256 emissive, a 2048 x 1024 procedural sky), a white-furnace
sphere, a parallel-emitter direct-lighting scene and a many-light field of
instanced meshes with textured emitters.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

BASE_SEED = 17050126

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
            z = self.state + k * _GAMMA
            out = _mix(z)
        self.counter += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class Camera:
    eye: tuple
    look_at: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int


@dataclasses.dataclass
class SceneData:
    vertices: np.ndarray                 # V x 3 float32
    indices: np.ndarray                  # T x 3 uint32
    tri_material: np.ndarray             # T uint32
    albedo: np.ndarray                   # M x 3 float32
    roughness: np.ndarray                # M float32
    ggx_weight: np.ndarray               # M float32
    emission: np.ndarray                 # M x 3 float32
    emission_tex: np.ndarray             # M int32 (-1 = constant)
    normals: Optional[np.ndarray] = None  # V x 3 float32
    uvs: Optional[np.ndarray] = None     # V x 2 float32
    textures: Optional[np.ndarray] = None  # K x th x tw x 3 float32
    env: Optional[np.ndarray] = None     # H x W x 3 float32
    env_plain: bool = False              # NEE from the plain environment pyramid only
    light_bvh: bool = False              # NEE picks emitters through the light hierarchy
    # two-level scenes: per-instance mesh id and 3x4 object-to-world transform
    mesh_tri_offset: Optional[np.ndarray] = None   # meshes + 1 (prefix into indices)
    instance_mesh: Optional[np.ndarray] = None     # I uint32
    instance_xform: Optional[np.ndarray] = None    # I x 3 x 4 float32
    name: str = ""

    @property
    def num_triangles(self) -> int:
        return int(self.indices.shape[0])

    def bbox(self):
        v = self.vertices.astype(np.float64)
        return v.min(axis=0), v.max(axis=0)

    def flattened(self) -> "SceneData":
        """World-space single-level copy of an instanced scene."""
        if self.instance_mesh is None:
            return self
        verts, idx, mats, nrm, uvs = [], [], [], [], []
        base = 0
        for inst, m in enumerate(self.instance_mesh):
            t0, t1 = int(self.mesh_tri_offset[m]), int(self.mesh_tri_offset[m + 1])
            tri = self.indices[t0:t1]
            used = np.unique(tri.reshape(-1))
            remap = np.zeros(int(used.max()) + 1, dtype=np.int64)
            remap[used] = np.arange(used.size)
            X = self.instance_xform[inst].astype(np.float32)
            v = self.vertices[used]
            vw = (v @ X[:, :3].T + X[:, 3]).astype(np.float32)
            verts.append(vw)
            idx.append((remap[tri] + base).astype(np.uint32))
            mats.append(self.tri_material[t0:t1])
            if self.normals is not None:
                # normals map with the inverse transpose of the linear part
                nw = self.normals[used].astype(np.float64) @ np.linalg.inv(X[:, :3].astype(np.float64))
                nw /= np.linalg.norm(nw, axis=1, keepdims=True)
                nrm.append(nw.astype(np.float32))
            if self.uvs is not None:
                uvs.append(self.uvs[used])
            base += used.size
        return dataclasses.replace(
            self,
            vertices=np.concatenate(verts), indices=np.concatenate(idx),
            tri_material=np.concatenate(mats),
            normals=np.concatenate(nrm) if nrm else None,
            uvs=np.concatenate(uvs) if uvs else None,
            mesh_tri_offset=None, instance_mesh=None, instance_xform=None)


# --------------------------------------------------------------- helpers
def _oriented_quad(p0, p1, p2, p3, facing):
    """Two triangles of the quad p0 p1 p2 p3 wound so their normal has a
    positive component along `facing`."""
    p = np.array([p0, p1, p2, p3], dtype=np.float64)
    n = np.cross(p[1] - p[0], p[2] - p[0])
    if np.dot(n, facing) < 0:
        p = p[[0, 3, 2, 1]]
    return p, np.array([[0, 1, 2], [0, 2, 3]], dtype=np.uint32)


def _box(center, size, angle_deg):
    """Closed box rotated about +y; outward-facing triangles."""
    cx, cy, cz = center
    sx, sy, sz = size
    c, s = math.cos(math.radians(angle_deg)), math.sin(math.radians(angle_deg))

    def P(x, y, z):
        x, z = x * sx / 2, z * sz / 2
        return (cx + c * x + s * z, cy + y * sy / 2, cz - s * x + c * z)

    def R(v):
        x, y, z = v
        return (c * x + s * z, y, -s * x + c * z)

    faces = [
        ((-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (0, 0, -1)),
        ((-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1), (0, 0, 1)),
        ((-1, -1, -1), (-1, 1, -1), (-1, 1, 1), (-1, -1, 1), (-1, 0, 0)),
        ((1, -1, -1), (1, 1, -1), (1, 1, 1), (1, -1, 1), (1, 0, 0)),
        ((-1, -1, -1), (1, -1, -1), (1, -1, 1), (-1, -1, 1), (0, -1, 0)),
        ((-1, 1, -1), (1, 1, -1), (1, 1, 1), (-1, 1, 1), (0, 1, 0)),
    ]
    verts, idx = [], []
    for a, b, cc, d, n in faces:
        p, t = _oriented_quad(P(*a), P(*b), P(*cc), P(*d), R(n))
        idx.append(t + len(verts) * 4)
        verts.append(p)
    return np.concatenate(verts), np.concatenate(idx)


class _Builder:
    def __init__(self):
        self.v, self.i, self.m, self.n, self.uv = [], [], [], [], []
        self.nv = 0
        self.mats = []

    def material(self, albedo, rough=0.5, w=0.0, emission=(0, 0, 0), tex=-1):
        self.mats.append((albedo, rough, w, emission, tex))
        return len(self.mats) - 1

    def add(self, verts, idx, mat, normals=None, uvs=None):
        verts = np.asarray(verts, dtype=np.float64)
        idx = np.asarray(idx, dtype=np.int64)
        self.v.append(verts)
        self.i.append(idx + self.nv)
        self.m.append(np.full(idx.shape[0], mat, dtype=np.uint32) if np.isscalar(mat) else np.asarray(mat, np.uint32))
        self.n.append(normals)
        self.uv.append(uvs)
        self.nv += verts.shape[0]

    def build(self, env=None, textures=None, name="", with_normals=False, with_uvs=False):
        V = np.concatenate(self.v).astype(np.float32)
        normals = None
        if with_normals:
            parts = []
            for v, n in zip(self.v, self.n):
                parts.append(np.zeros_like(v) if n is None else n)
            normals = np.concatenate(parts).astype(np.float32)
        uvs = None
        if with_uvs:
            parts = []
            for v, u in zip(self.v, self.uv):
                parts.append(np.zeros((v.shape[0], 2)) if u is None else u)
            uvs = np.concatenate(parts).astype(np.float32)
        M = self.mats
        return SceneData(
            vertices=V, indices=np.concatenate(self.i).astype(np.uint32),
            tri_material=np.concatenate(self.m).astype(np.uint32),
            albedo=np.array([m[0] for m in M], np.float32).reshape(-1, 3),
            roughness=np.array([m[1] for m in M], np.float32),
            ggx_weight=np.array([m[2] for m in M], np.float32),
            emission=np.array([m[3] for m in M], np.float32).reshape(-1, 3),
            emission_tex=np.array([m[4] for m in M], np.int32),
            normals=normals, uvs=uvs, textures=textures, env=env, name=name)


# ------------------------------------------------------------ Cornell box
def cornell_box(seed: int = BASE_SEED + 1, light: str = "down"):
    """Box [0,1]^3 open towards -z: 5 walls (10 triangles), two boxes rotated
    +-17 degrees about y resting 1e-3 above the floor (24 triangles) and a
    0.25 x 0.25 emitter quad
    (2 triangles) 1e-3 below the ceiling facing down, radiance (17, 12, 4).
    Lambertian albedo in U[0.2, 0.8]^3 per object. 64 x 64 pinhole camera.
    light="up": the same emitter 0.1 below the ceiling facing up, so that the
    room is lit only through the bright patch it makes on the ceiling (every
    surface but that patch is lit indirectly; next-event estimation cannot
    reach the light from them)."""
    rng = Rng(seed)
    b = _Builder()

    def mat():
        return b.material(tuple(rng.uniform(3, 0.2, 0.8)), 0.5, 0.0)

    walls = [
        (((0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)), (0, 1, 0)),    # floor
        (((0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1)), (0, -1, 0)),   # ceiling
        (((0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)), (0, 0, -1)),   # back
        (((0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)), (1, 0, 0)),    # left
        (((1, 0, 0), (1, 0, 1), (1, 1, 1), (1, 1, 0)), (-1, 0, 0)),   # right
    ]
    for quad, facing in walls:
        p, t = _oriented_quad(*quad, facing)
        b.add(p, t, mat())
    # the boxes float 1e-3 above the floor so that no two triangles are
    # coplanar and overlapping (a tie in t would make the hit ambiguous)
    for center, size, ang in (((0.33, 0.151, 0.62), (0.3, 0.3, 0.3), 17.0),
                              ((0.68, 0.301, 0.42), (0.3, 0.6, 0.3), -17.0)):
        v, t = _box(center, size, ang)
        b.add(v, t, mat())
    lm = b.material((0.78, 0.78, 0.78), 0.5, 0.0, (17.0, 12.0, 4.0))
    if light not in ("down", "up"):
        raise ValueError(light)
    y = 1.0 - 1e-3 if light == "down" else 0.9
    facing = (0, -1, 0) if light == "down" else (0, 1, 0)
    p, t = _oriented_quad((0.375, y, 0.375), (0.625, y, 0.375), (0.625, y, 0.625), (0.375, y, 0.625), facing)
    b.add(p, t, lm)
    scene = b.build(name="cornell-36" if light == "down" else "cornell-36-up")
    cam = Camera((0.5, 0.5, -1.4), (0.5, 0.5, 0.0), (0.0, 1.0, 0.0), 40.0, 64, 64)
    return scene, cam


def door_room(seed: int = BASE_SEED + 1, res: int = 64):
    """The Cornell room lit from a closed side chamber through a door (not a
    configuration of the task; the guiding scene where next-event estimation
    fails for most of the image). Room [0,1]^3 as in cornell_box (same walls,
    boxes, albedos and camera) without its emitter; its right wall (x = 1)
    has a door z in [0.55, 0.75], y in [0, 0.65] into a chamber x in [1, 1.6],
    y in [0, 1], z in [0.35, 1] (white walls, albedo 0.8) whose ceiling
    carries a 0.3 x 0.45 emitter 1e-3 below it facing down, radiance
    (85, 60, 20). Light reaches the room only through the door: from almost
    every visible point a shadow ray towards the emitter is blocked, and a
    path must pass the door (a small solid angle) to reach the lit chamber."""
    rng = Rng(seed)
    b = _Builder()

    def mat():
        return b.material(tuple(rng.uniform(3, 0.2, 0.8)), 0.5, 0.0)

    z0, z1, yd = 0.55, 0.75, 0.65
    right = [((1, 0, 0), (1, 0, z0), (1, 1, z0), (1, 1, 0)),
             ((1, 0, z1), (1, 0, 1), (1, 1, 1), (1, 1, z1)),
             ((1, yd, z0), (1, yd, z1), (1, 1, z1), (1, 1, z0))]
    walls = [
        ([((0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1))], (0, 1, 0)),    # floor
        ([((0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1))], (0, -1, 0)),   # ceiling
        ([((0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1))], (0, 0, -1)),   # back
        ([((0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0))], (1, 0, 0)),    # left
        (right, (-1, 0, 0)),                                              # right, with the door
    ]
    for quads, facing in walls:
        m = mat()
        for quad in quads:
            p, t = _oriented_quad(*quad, facing)
            b.add(p, t, m)
    for center, size, ang in (((0.33, 0.151, 0.62), (0.3, 0.3, 0.3), 17.0),
                              ((0.68, 0.301, 0.42), (0.3, 0.6, 0.3), -17.0)):
        v, t = _box(center, size, ang)
        b.add(v, t, mat())
    white = b.material((0.8, 0.8, 0.8), 0.5, 0.0)
    x0, x1, c0, c1 = 1.0, 1.6, 0.35, 1.0
    chamber = [
        (((x0, 0, c0), (x1, 0, c0), (x1, 0, c1), (x0, 0, c1)), (0, 1, 0)),     # floor
        (((x0, 1, c0), (x1, 1, c0), (x1, 1, c1), (x0, 1, c1)), (0, -1, 0)),    # ceiling
        (((x1, 0, c0), (x1, 0, c1), (x1, 1, c1), (x1, 1, c0)), (-1, 0, 0)),    # far wall
        (((x0, 0, c1), (x1, 0, c1), (x1, 1, c1), (x0, 1, c1)), (0, 0, -1)),    # back
        (((x0, 0, c0), (x1, 0, c0), (x1, 1, c0), (x0, 1, c0)), (0, 0, 1)),     # front
    ]
    for quad, facing in chamber:
        p, t = _oriented_quad(*quad, facing)
        b.add(p, t, white)
    lm = b.material((0.78, 0.78, 0.78), 0.5, 0.0, (85.0, 60.0, 20.0))
    y = 1.0 - 1e-3
    p, t = _oriented_quad((1.15, y, 0.45), (1.45, y, 0.45), (1.45, y, 0.9), (1.15, y, 0.9), (0, -1, 0))
    b.add(p, t, lm)
    scene = b.build(name="cornell-door")
    cam = Camera((0.5, 0.5, -1.4), (0.5, 0.5, 0.0), (0.0, 1.0, 0.0), 40.0, res, res)
    return scene, cam


def glossy_room(res: int = 64):
    """The Cornell room lit through its ceiling (cornell_box(light="up")) with
    glossy boxes (pure GGX coating, roughness 0.05) and a half-glossy floor
    (GGX weight 0.6, roughness 0.08): every visible surface is lit along paths
    that leave the emitter, bounce off the ceiling and often off a glossy
    surface, which next-event estimation from the camera side reaches poorly
    and a light tracer reaches directly."""
    sd, cam = cornell_box(light="up")
    rough = sd.roughness.copy()
    gw = sd.ggx_weight.copy()
    # materials in creation order: floor, ceiling, back, left, right, box, box, emitter
    for mi, (r, w) in {0: (0.08, 0.6), 5: (0.05, 1.0), 6: (0.05, 1.0)}.items():
        rough[mi] = r
        gw[mi] = w
    sd = dataclasses.replace(sd, roughness=rough, ggx_weight=gw, name="cornell-36-up-glossy")
    return sd, dataclasses.replace(cam, width=res, height=res)


# ------------------------------------------------------------ value noise
def _value_noise(p: np.ndarray, seed: int) -> np.ndarray:
    """Trilinear value noise in [0, 1] on the integer lattice (smoothstep)."""
    fl = np.floor(p)
    f = p - fl
    f = f * f * (3.0 - 2.0 * f)
    il = fl.astype(np.int64)
    out = np.zeros(p.shape[0])
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                x = (il[:, 0] + dx).astype(np.uint64)
                y = (il[:, 1] + dy).astype(np.uint64)
                z = (il[:, 2] + dz).astype(np.uint64)
                with np.errstate(over="ignore"):
                    h = _mix(np.uint64(seed) + x * np.uint64(0x8DA6B343) + y * np.uint64(0xD8163841)
                             + z * np.uint64(0xCB1AB31F))
                val = (h >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
                w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * \
                    (f[:, 2] if dz else 1 - f[:, 2])
                out += w * val
    return out


def _vertex_normals(v: np.ndarray, idx: np.ndarray) -> np.ndarray:
    n = np.zeros_like(v)
    fn = np.cross(v[idx[:, 1]] - v[idx[:, 0]], v[idx[:, 2]] - v[idx[:, 0]])
    for k in range(3):
        np.add.at(n, idx[:, k], fn)
    n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-30)
    return n


def uv_sphere(seg: int, rings: int):
    """Unit UV sphere: 2 poles + seg x (rings - 1) ring vertices, outward
    winding; seg * 2 * (rings - 1) triangles (64 x 35 -> 4352)."""
    th = np.pi * np.arange(1, rings) / rings
    ph = 2 * np.pi * np.arange(seg) / seg
    ring = np.stack([np.outer(np.sin(th), np.cos(ph)), np.repeat(np.cos(th)[:, None], seg, 1),
                     np.outer(np.sin(th), np.sin(ph))], -1).reshape(-1, 3)
    v = np.concatenate([[[0, 1, 0]], ring, [[0, -1, 0]]])
    south = v.shape[0] - 1
    tris = []
    j = np.arange(seg)
    jn = (j + 1) % seg
    tris.append(np.stack([np.zeros(seg, np.int64), 1 + jn, 1 + j], 1))
    for r in range(rings - 2):
        a = 1 + r * seg + j
        bb = 1 + r * seg + jn
        c = 1 + (r + 1) * seg + j
        d = 1 + (r + 1) * seg + jn
        tris.append(np.stack([a, bb, d], 1))
        tris.append(np.stack([a, d, c], 1))
    base = 1 + (rings - 2) * seg
    tris.append(np.stack([np.full(seg, south), base + j, base + jn], 1))
    idx = np.concatenate(tris)
    fn = np.cross(v[idx[:, 1]] - v[idx[:, 0]], v[idx[:, 2]] - v[idx[:, 0]])
    cen = v[idx].mean(axis=1)
    flip = np.einsum("ij,ij->i", fn, cen) < 0
    idx[flip] = idx[flip][:, [0, 2, 1]]
    return v, idx


def procedural_sky(width: int, height: int, seed: int, sun_radius_deg: float = 0.27,
                   sun_gain: float = 1e4):
    """Equirectangular RGB32F sky (row 0 = +y): a zenith-to-horizon gradient,
    a dim ground below the horizon and a sun disk ~1e4 times brighter in a
    seeded direction above the horizon."""
    rng = Rng(seed)
    theta = np.pi * (np.arange(height) + 0.5) / height
    phi = 2 * np.pi * (np.arange(width) + 0.5) / width
    st, ct = np.sin(theta)[:, None], np.cos(theta)[:, None]
    d = np.stack([st * np.cos(phi)[None, :], np.broadcast_to(ct, (height, width)),
                  st * np.sin(phi)[None, :]], -1)
    up = np.clip(d[..., 1], -1, 1)
    zen = np.array([0.25, 0.45, 1.0])
    hor = np.array([0.9, 0.85, 0.8])
    t = np.clip(up, 0, 1)[..., None] ** 0.5
    sky = (1 - t) * hor + t * zen
    ground = np.array([0.3, 0.25, 0.2])
    env = np.where(up[..., None] >= 0, sky, ground * (0.5 + 0.5 * np.exp(up[..., None] * 4)))
    sth = math.radians(rng.uniform(1, 25, 60)[0])
    sph = 2 * math.pi * rng.uniform(1)[0]
    sd = np.array([math.sin(sth) * math.cos(sph), math.cos(sth), math.sin(sth) * math.sin(sph)])
    cosang = d @ sd
    sun = cosang >= math.cos(math.radians(sun_radius_deg))
    env[sun] = np.array([1.0, 0.95, 0.85]) * sun_gain
    return env.astype(np.float32), sd


def sphere_field(seed: int = BASE_SEED + 2, n_spheres: int = 200, seg: int = 64, rings: int = 35,
                 plane_res=(360, 180), n_emissive_spheres: int = 8, emissive_per_sphere: int = 32,
                 env_size=(2048, 1024), width: int = 1920, height: int = 1080):
    """200 noise-displaced UV spheres (64 x 35 -> 4,352 triangles each) on a
    360 x 180-quad displaced plane (129,600 triangles): 1,000,000 triangles
    with vertex normals. 256 emissive triangles (the first 32 triangles of
    the top cap of 8 spheres, radiance U[5, 50]). Per-material GGX roughness
    U[0.05, 0.8], GGX weight U[0.2, 0.8], albedo U[0.2, 0.8]^3. Procedural
    2048 x 1024 sky with a sun disk. Smaller counts give the same family."""
    rng = Rng(seed)
    b = _Builder()
    sv, si = uv_sphere(seg, rings)
    px, pz = plane_res
    ext_x, ext_z = 36.0, 18.0
    # plane
    xs = np.linspace(-ext_x, ext_x, px + 1)
    zs = np.linspace(-ext_z, ext_z, pz + 1)
    X, Z = np.meshgrid(xs, zs)
    pts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], 1)
    Y = 0.6 * (_value_noise(pts * np.array([0.35, 0, 0.35]), seed ^ 0x5A5A) - 0.5)
    pv = np.stack([X.ravel(), Y, Z.ravel()], 1)
    ii = np.arange(pz)[:, None] * (px + 1) + np.arange(px)[None, :]
    a, bb, c, d = ii.ravel(), ii.ravel() + 1, ii.ravel() + px + 1, ii.ravel() + px + 2
    pidx = np.concatenate([np.stack([a, c, bb], 1), np.stack([bb, c, d], 1)])
    fn = np.cross(pv[pidx[:, 1]] - pv[pidx[:, 0]], pv[pidx[:, 2]] - pv[pidx[:, 0]])
    flip = fn[:, 1] < 0
    pidx[flip] = pidx[flip][:, [0, 2, 1]]
    pm = b.material(tuple(rng.uniform(3, 0.2, 0.8)), float(rng.uniform(1, 0.05, 0.8)[0]),
                    float(rng.uniform(1, 0.2, 0.8)[0]))
    b.add(pv, pidx, pm, normals=_vertex_normals(pv, pidx))
    # spheres
    radii = rng.uniform(n_spheres, 0.6, 1.8)
    cx = rng.uniform(n_spheres, -30, 30)
    cz = rng.uniform(n_spheres, -15, 15)
    emissive_ids = set(range(0, n_spheres, max(1, n_spheres // max(1, n_emissive_spheres)))[:n_emissive_spheres])
    for s in range(n_spheres):
        r = radii[s]
        ground = 0.6 * (_value_noise(np.array([[cx[s] * 0.35, 0, cz[s] * 0.35]]), seed ^ 0x5A5A)[0] - 0.5)
        center = np.array([cx[s], ground + r * 0.95, cz[s]])
        disp = 1.0 + 0.05 * (2.0 * _value_noise(sv * 2.5 + 17.0 * s, seed + 1000 + s) - 1.0)
        v = center + sv * (r * disp)[:, None]
        n = _vertex_normals(v, si)
        m = b.material(tuple(rng.uniform(3, 0.2, 0.8)), float(rng.uniform(1, 0.05, 0.8)[0]),
                       float(rng.uniform(1, 0.2, 0.8)[0]))
        mats = np.full(si.shape[0], m, dtype=np.uint32)
        if s in emissive_ids:
            le = float(rng.uniform(1, 5.0, 50.0)[0])
            tint = rng.uniform(3, 0.6, 1.0)
            em = b.material((0.5, 0.5, 0.5), 0.5, 0.0, tuple(le * tint))
            mats[:emissive_per_sphere] = em
        b.add(v, si, mats, normals=n)
    env, sun_dir = procedural_sky(env_size[0], env_size[1], seed ^ 0x51CE)
    scene = b.build(env=env, with_normals=True, name=f"sphere-field-{n_spheres}")
    cam = Camera((0.0, 9.0, 26.0), (0.0, 0.5, -2.0), (0.0, 1.0, 0.0), 50.0, width, height)
    return scene, cam


def turntable(res: int = 64, seed: int = BASE_SEED + 7, sun_radius_deg: float = 3.0, sun_gain: float = 300.0):
    """A close-up object on a turntable in an open, sky-lit scene (the setting
    Sec. 2.1.3 describes): a glossy sphere (radius 0.2, pure GGX, roughness
    0.05) resting on a matte stand (0.6 x 0.5 x 0.6) near the camera, a 400 x
    400 ground, three large boxes 100-150 away that make the scene's bound a
    few hundred times the object's; a 256 x 128 sky with a sun disk of
    `sun_radius_deg` whose reflections off the sphere light the stand. Not a
    configuration of the task: the photon-aiming test and bench scene."""
    rng = Rng(seed)
    b = _Builder()
    gm = b.material((0.5, 0.5, 0.5), 0.5, 0.0)
    p, t = _oriented_quad((-200, 0, -200), (200, 0, -200), (200, 0, 200), (-200, 0, 200), (0, 1, 0))
    b.add(p, t, gm)
    v, t = _box((0.0, 0.25, 0.0), (0.6, 0.5, 0.6), 0.0)
    b.add(v, t, b.material((0.75, 0.75, 0.7), 0.5, 0.0))
    sv, si = uv_sphere(48, 24)
    sp = sv * 0.2 + np.array([0.0, 0.7005, 0.0])
    b.add(sp, si, b.material((0.9, 0.9, 0.9), 0.02, 1.0), normals=_vertex_normals(sp, si))
    for k in range(3):
        ang = 2 * np.pi * (k / 3.0 + 0.1)
        dist = float(rng.uniform(1, 100.0, 150.0)[0])
        c = (dist * np.cos(ang), 10.0, dist * np.sin(ang))
        v, t = _box(c, (20.0, 20.0, 20.0), float(rng.uniform(1, 0, 90)[0]))
        b.add(v, t, b.material(tuple(rng.uniform(3, 0.3, 0.7)), 0.5, 0.0))
    env, _ = procedural_sky(256, 128, seed ^ 0x7A7A, sun_radius_deg=sun_radius_deg, sun_gain=sun_gain)
    scene = b.build(env=env, with_normals=True, name="turntable")
    cam = Camera((0.0, 1.1, 1.6), (0.0, 0.55, 0.0), (0.0, 1.0, 0.0), 35.0, res, res)
    return scene, cam


# ---------------------------------------------------------- pin scenes
def furnace_sphere(seg: int = 48, rings: int = 24, env_size=(8, 4), radiance: float = 1.0,
                   res: int = 32, albedo: float = 1.0):
    """Convex, flat-shaded sphere with albedo 1 inside a constant environment
    of radiance 1: every pixel must converge to exactly 1."""
    b = _Builder()
    v, idx = uv_sphere(seg, rings)
    m = b.material((albedo, albedo, albedo), 0.5, 0.0)
    b.add(v, idx, m)
    env = np.full((env_size[1], env_size[0], 3), radiance, np.float32)
    scene = b.build(env=env, name="furnace")
    cam = Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, res, res)
    return scene, cam


def parallel_emitter(h: float = 1.0, a: float = 0.5, b_: float = 0.75, L: float = 3.0,
                     albedo: float = 0.6):
    """Lambertian floor (y = 0) under a 2a x 2b emitter facing down at height
    h, centred above the origin; a 1 x 1 camera with a tiny field of view
    looks at the origin from the side, below the emitter plane."""
    bld = _Builder()
    fm = bld.material((albedo, albedo, albedo), 0.5, 0.0)
    p, t = _oriented_quad((-50, 0, -50), (50, 0, -50), (50, 0, 50), (-50, 0, 50), (0, 1, 0))
    bld.add(p, t, fm)
    lm = bld.material((0.0, 0.0, 0.0), 0.5, 0.0, (L, L, L))
    p, t = _oriented_quad((-a, h, -b_), (a, h, -b_), (a, h, b_), (-a, h, b_), (0, -1, 0))
    bld.add(p, t, lm)
    scene = bld.build(name="parallel-emitter")
    cam = Camera((0.0, 0.5 * h, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.01, 1, 1)
    return scene, cam


# ----------------------------------------------------------- many lights
def many_emitters(seed: int = BASE_SEED + 5, n_lights: int = 256, res: int = 64, light_bvh: bool = True):
    """A 20 x 20 Lambertian floor (albedo 0.7) under `n_lights` small emitter
    triangles (edge ~0.2) scattered over it at heights in [0.3, 3], each facing
    a random direction of the lower hemisphere, radiance lognormal(1, 1) times
    a random RGB tint; three boxes on the floor cast shadows. The lights are
    spread out, so at any floor point a few of them dominate: the case the
    light hierarchy is for. res x res pinhole camera looking down at the
    floor from 14 above."""
    rng = Rng(seed)
    b = _Builder()
    p, t = _oriented_quad((-10, 0, -10), (10, 0, -10), (10, 0, 10), (-10, 0, 10), (0, 1, 0))
    b.add(p, t, b.material((0.7, 0.7, 0.7), 0.5, 0.0))
    for center, size, ang in (((-3.0, 0.5, 2.0), (1.0, 1.0, 1.0), 20.0), ((4.0, 1.0, -3.0), (1.5, 2.0, 1.0), -35.0),
                              ((0.5, 0.4, -6.0), (3.0, 0.8, 0.6), 5.0)):
        v, tt = _box(center, size, ang)
        b.add(v, tt, b.material((0.5, 0.6, 0.4), 0.4, 0.3))
    pos = np.stack([rng.uniform(n_lights, -9.5, 9.5), rng.uniform(n_lights, 0.3, 3.0),
                    rng.uniform(n_lights, -9.5, 9.5)], 1)
    nrm = rng.normal(3 * n_lights).reshape(n_lights, 3)
    nrm[:, 1] = -np.abs(nrm[:, 1])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    radiance = np.exp(1.0 + rng.normal(n_lights))
    tint = rng.uniform(3 * n_lights, 0.3, 1.0).reshape(n_lights, 3)
    for k in range(n_lights):
        n = nrm[k]
        a = np.cross(n, (0.0, 0.0, 1.0) if abs(n[2]) < 0.9 else (1.0, 0.0, 0.0))
        a /= np.linalg.norm(a)
        c = np.cross(n, a)
        q = pos[k] + 0.12 * np.array([a, np.cos(2.1) * a + np.sin(2.1) * c, np.cos(4.2) * a + np.sin(4.2) * c])
        tri = np.array([[0, 1, 2]], np.uint32)
        if np.dot(np.cross(q[1] - q[0], q[2] - q[0]), n) < 0:
            tri = np.array([[0, 2, 1]], np.uint32)
        b.add(q, tri, b.material((0.5, 0.5, 0.5), 0.5, 0.0, tuple(radiance[k] * tint[k])))
    scene = b.build(name=f"many-emitters-{n_lights}")
    scene.light_bvh = light_bvh
    cam = Camera((0.0, 14.0, 6.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0, res, res)
    return scene, cam


def instanced_field(seed: int = BASE_SEED + 3, n_meshes: int = 100, n_instances: int = 1000,
                    total_tris: int = 10_000_000, n_emissive: int = 100_000, n_textures: int = 16,
                    tex_size: int = 64, width: int = 1920, height: int = 1080,
                    min_tris: int = 1000, max_tris: int = 50_000):
    """1000 instances of 100 unique seeded meshes whose sizes are log-uniform
    in [1k, 50k] triangles, rescaled so that the instanced total is
    `total_tris`; `n_emissive` instanced emitter triangles carry one of 16
    64 x 64 lognormal(0, 1) RGB textures (emission scale 20). No
    environment."""
    rng = Rng(seed)
    b = _Builder()
    sizes = np.exp(rng.uniform(n_meshes, math.log(min_tris), math.log(max_tris)))
    inst_mesh = (rng.u64(n_instances) % np.uint64(n_meshes)).astype(np.int64)
    counts = np.bincount(inst_mesh, minlength=n_meshes)
    scale = total_tris / float(np.dot(counts, sizes))
    sizes = np.maximum(8, np.round(sizes * scale)).astype(np.int64)
    mesh_off = [0]
    emissive_mesh = set(range(0, n_meshes, 4))
    em_mats = []
    for t in range(n_textures):
        em_mats.append(b.material((0.5, 0.5, 0.5), 0.5, 0.0, (20.0, 20.0, 20.0), tex=t))
    # emitter triangle budget per emissive mesh, from the instance counts
    em_inst = sum(int(counts[m]) for m in emissive_mesh)
    per_mesh_em = max(1, int(round(n_emissive / max(1, em_inst))))
    for m in range(n_meshes):
        seg = max(4, int(math.sqrt(sizes[m] / 2.0)))
        rings = max(3, int(round(sizes[m] / (2.0 * seg))) + 1)
        v, idx = uv_sphere(seg, rings)
        disp = 1.0 + 0.2 * (2.0 * _value_noise(v * 1.7 + 11.0 * m, seed + 77 + m) - 1.0)
        v = v * disp[:, None]
        mat = b.material(tuple(rng.uniform(3, 0.2, 0.8)), float(rng.uniform(1, 0.05, 0.8)[0]),
                         float(rng.uniform(1, 0.2, 0.8)[0]))
        mats = np.full(idx.shape[0], mat, dtype=np.uint32)
        if m in emissive_mesh:
            k = min(per_mesh_em, idx.shape[0])
            mats[:k] = em_mats[m % n_textures]
        uv = np.stack([0.5 + np.arctan2(v[:, 2], v[:, 0]) / (2 * np.pi),
                       np.arccos(np.clip(v[:, 1] / np.maximum(np.linalg.norm(v, axis=1), 1e-9), -1, 1)) / np.pi], 1)
        b.add(v, idx, mats, normals=_vertex_normals(v, idx), uvs=uv)
        mesh_off.append(mesh_off[-1] + idx.shape[0])
    textures = np.exp(rng.normal(n_textures * tex_size * tex_size * 3)).reshape(
        n_textures, tex_size, tex_size, 3).astype(np.float32)
    scene = b.build(textures=textures, with_normals=True, with_uvs=True, name="instanced-field")
    ang = rng.uniform(n_instances, 0, 2 * math.pi)
    sc = rng.uniform(n_instances, 0.8, 2.5)
    # a dense cluster in front of the camera: about a third of the image is
    # covered by instances at any resolution
    pos = np.stack([rng.uniform(n_instances, -28, 28), rng.uniform(n_instances, 0, 10),
                    rng.uniform(n_instances, -45, 5)], 1)
    xf = np.zeros((n_instances, 3, 4), np.float32)
    c, s = np.cos(ang), np.sin(ang)
    xf[:, 0, 0], xf[:, 0, 2], xf[:, 2, 0], xf[:, 2, 2] = c * sc, s * sc, -s * sc, c * sc
    xf[:, 1, 1] = sc
    xf[:, :, 3] = pos
    scene.mesh_tri_offset = np.array(mesh_off, np.int64)
    scene.instance_mesh = inst_mesh.astype(np.uint32)
    scene.instance_xform = xf
    cam = Camera((0.0, 14.0, 38.0), (0.0, 3.0, -15.0), (0.0, 1.0, 0.0), 55.0, width, height)
    return scene, cam


# ------------------------------------------------------------ ray batches
def random_rays(scene: SceneData, n: int, seed: int, kind: str = "incoherent", cam: Camera = None):
    """n x 8 float32 rays (ox oy oz dx dy dz tmin tmax).
    kind = 'primary': pinhole rays through random film positions;
    'camera': pinhole rays in scanline pixel order (coherent), one jittered
    ray per pixel per pass over the image, as many passes as n needs;
    'incoherent': origins on random triangles (slightly off the surface),
    uniformly random directions; 'shadow': segments between two random
    surface points; 'edges': rays aimed exactly at triangle vertices and edge
    midpoints from random outside points."""
    rng = Rng(seed)
    V = scene.vertices.astype(np.float64)
    I = scene.indices.astype(np.int64)
    lo, hi = V.min(0), V.max(0)
    out = np.zeros((n, 8), np.float32)

    def surf_points(k):
        t = (rng.u64(k) % np.uint64(I.shape[0])).astype(np.int64)
        u, v = rng.uniform(k), rng.uniform(k)
        su = np.sqrt(u)
        bary = np.stack([1 - su, su * (1 - v), su * v], 1)
        p = np.einsum("ik,ikj->ij", bary, V[I[t]])
        nrm = np.cross(V[I[t, 1]] - V[I[t, 0]], V[I[t, 2]] - V[I[t, 0]])
        nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-30)
        return p, nrm

    def unit(k):
        z = rng.uniform(k, -1, 1)
        ph = rng.uniform(k, 0, 2 * math.pi)
        r = np.sqrt(1 - z * z)
        return np.stack([r * np.cos(ph), r * np.sin(ph), z], 1)

    if kind in ("primary", "camera"):
        assert cam is not None
        fwd = np.array(cam.look_at, float) - np.array(cam.eye, float)
        fwd /= np.linalg.norm(fwd)
        right = np.cross(fwd, np.array(cam.up, float))
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        th = math.tan(math.radians(cam.vfov_deg) / 2)
        asp = cam.width / cam.height
        if kind == "primary":
            sx, sy = rng.uniform(n, -1, 1), rng.uniform(n, -1, 1)
        else:
            pix = np.arange(n, dtype=np.int64) % (cam.width * cam.height)
            fx = (pix % cam.width + rng.uniform(n)) / cam.width
            fy = (pix // cam.width + rng.uniform(n)) / cam.height
            sx, sy = 2 * fx - 1, 1 - 2 * fy
        d = fwd + (sx * th * asp)[:, None] * right + (sy * th)[:, None] * up
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        out[:, 0:3] = np.array(cam.eye)
        out[:, 3:6] = d
        out[:, 6], out[:, 7] = 0.0, np.inf
    elif kind == "incoherent":
        p, nrm = surf_points(n)
        d = unit(n)
        flip = np.einsum("ij,ij->i", d, nrm) < 0
        o = p + 1e-4 * (np.linalg.norm(hi - lo)) * np.where(flip[:, None], -nrm, nrm)
        out[:, 0:3], out[:, 3:6] = o, d
        out[:, 6], out[:, 7] = 0.0, np.inf
    elif kind == "shadow":
        p, n1 = surf_points(n)
        q, _ = surf_points(n)
        o = p + 1e-4 * np.linalg.norm(hi - lo) * n1
        dv = q - o
        dist = np.linalg.norm(dv, axis=1)
        dist = np.maximum(dist, 1e-6)
        out[:, 0:3], out[:, 3:6] = o, dv / dist[:, None]
        out[:, 6], out[:, 7] = 0.0, dist * (1 - 1e-4)
    elif kind == "edges":
        t = (rng.u64(n) % np.uint64(I.shape[0])).astype(np.int64)
        which = (rng.u64(n) % np.uint64(6)).astype(np.int64)
        a = V[I[t, which % 3]]
        bpt = V[I[t, (which + 1) % 3]]
        target = np.where((which < 3)[:, None], a, 0.5 * (a + bpt))
        cen = 0.5 * (lo + hi)
        o = cen + unit(n) * (0.75 * np.linalg.norm(hi - lo) + 1.0)
        d = target - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        out[:, 0:3], out[:, 3:6] = o, d
        out[:, 6], out[:, 7] = 0.0, np.inf
    else:
        raise ValueError(kind)
    return out


# ------------------------------------------------------------ batched jobs
def batch_jobs(seed: int = BASE_SEED + 5, n_jobs: int = 64, min_tris: int = 1000, max_tris: int = 500_000,
               resolutions=(256, 512, 1024), spps=(16, 32, 64, 128, 256), depth_range=(4, 16), spp_divisor: int = 1,
               res_divisor: int = 1):
    """Independent seeded jobs for batched rendering: scene family drawn from
    {Cornell-like, sphere field}, triangle count log-uniform in
    [min_tris, max_tris], square resolution, samples per pixel and depth
    drawn uniformly from the given sets. Returns a list of (SceneData,
    Camera, spp, max_depth)."""
    rng = Rng(seed)
    jobs = []
    for j in range(n_jobs):
        fam = int(rng.u64(1)[0] % np.uint64(2))
        target = math.exp(rng.uniform(1, math.log(min_tris), math.log(max_tris))[0])
        res = resolutions[int(rng.u64(1)[0] % np.uint64(len(resolutions)))] // res_divisor
        spp = max(1, spps[int(rng.u64(1)[0] % np.uint64(len(spps)))] // spp_divisor)
        depth = int(depth_range[0] + rng.u64(1)[0] % np.uint64(depth_range[1] - depth_range[0] + 1))
        jseed = seed * 1000 + j
        if fam == 0 or target < 2500:
            sd, cam = cornell_box(jseed)
        else:
            # spheres of seg x rings triangles plus a plane, scaled to the target
            seg = 24
            rings = 12
            per = seg * 2 * (rings - 1)
            plane = (40, 20)
            n_sph = int(max(2, min(400, (target - 2 * plane[0] * plane[1]) / per)))
            if n_sph * per < target / 2:
                seg, rings = 64, 35
                per = seg * 2 * (rings - 1)
                n_sph = int(max(2, min(200, (target - 2 * plane[0] * plane[1]) / per)))
            sd, cam = sphere_field(jseed, n_spheres=n_sph, seg=seg, rings=rings, plane_res=plane,
                                   n_emissive_spheres=max(1, n_sph // 25), env_size=(256, 128))
        cam = Camera(cam.eye, cam.look_at, cam.up, cam.vfov_deg, res, res)
        jobs.append((sd, cam, spp, depth))
    return jobs
