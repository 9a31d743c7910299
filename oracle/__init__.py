"""FP64 CPU oracle for the QMC path tracer and its guiding network.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product library
never does. The C sources next to this file implement, plainly and in double
precision, what the paper defines (each function cites its passage); this
module only marshals numpy arrays to them.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


def _p(a, t=C.c_void_p):
    return None if a is None else a.ctypes.data_as(t)


class _Desc(C.Structure):
    _fields_ = [
        ("nv", C.c_int64), ("nt", C.c_int64),
        ("vertices", C.c_void_p), ("normals", C.c_void_p), ("uvs", C.c_void_p),
        ("indices", C.c_void_p), ("tri_material", C.c_void_p),
        ("nm", C.c_int32), ("albedo", C.c_void_p), ("roughness", C.c_void_p),
        ("ggx_weight", C.c_void_p), ("emission", C.c_void_p), ("emission_tex", C.c_void_p),
        ("ntex", C.c_int32), ("tex_w", C.c_int32), ("tex_h", C.c_int32), ("textures", C.c_void_p),
        ("env_w", C.c_int32), ("env_h", C.c_int32), ("env", C.c_void_p),
        ("env_plain", C.c_int32), ("light_bvh", C.c_int32),
    ]


class _Cam(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("look_at", C.c_double * 3), ("up", C.c_double * 3),
                ("vfov_deg", C.c_double), ("width", C.c_uint32), ("height", C.c_uint32)]


class _Opts(C.Structure):
    _fields_ = [("filter_sigma", C.c_double), ("rr_enable", C.c_int32), ("mis_mode", C.c_int32),
                ("seed", C.c_uint64), ("threads", C.c_int32), ("lt_aim", C.c_int32)]


def _declare(L):
    u32, u64, i64, f64, vp = C.c_uint32, C.c_uint64, C.c_int64, C.c_double, C.c_void_p
    sig = {
        "or_prime": (u32, [C.c_int]),
        "or_scramble_factor": (u32, [u64, u32]),
        "or_radical_inverse_u32": (u32, [u32, u32, u64]),
        "or_pixel_base_index": (u64, [u32, u32, u32, u32]),
        "or_sample_dims_batch": (None, [vp, i64, C.c_int, u32, u32, u64, vp]),
        "or_scene_create": (vp, [C.POINTER(_Desc)]),
        "or_scene_destroy": (None, [vp]),
        "or_trace": (None, [vp, vp, i64, C.c_int, C.c_int, vp, vp, vp, vp]),
        "or_bvh_node_count": (i64, [vp]),
        "or_adapt_shading_normal": (None, [vp, vp, vp, vp]),
        "or_bsdf_eval": (None, [vp, f64, f64, vp, vp, vp, vp, vp]),
        "or_bsdf_sample": (C.c_int, [vp, f64, f64, vp, vp, f64, f64, f64, vp, vp, vp]),
        "or_ggx_D": (f64, [f64, f64]),
        "or_ggx_G1": (f64, [f64, f64]),
        "or_onb": (None, [vp, vp, vp]),
        "or_alias_build": (None, [vp, i64, vp, vp]),
        "or_alias_sample": (i64, [vp, vp, i64, f64]),
        "or_env_pyramid_probs": (None, [vp, C.c_int32, C.c_int32, vp]),
        "or_env_sample": (None, [vp, f64, f64, vp, vp, vp, vp]),
        "or_env_pdf": (f64, [vp, vp]),
        "or_env_lookup": (None, [vp, vp, vp]),
        "or_scene_light_pdf_area": (f64, [vp, u32]),
        "or_scene_env_select_prob": (f64, [vp]),
        "or_camera_ray": (None, [C.POINTER(_Cam), f64, f64, vp, vp]),
        "or_filter_offset": (None, [f64, f64, f64, vp, vp]),
        "or_render": (None, [vp, C.POINTER(_Cam), u32, u32, u32, C.POINTER(_Opts), vp, vp, vp, vp]),
        "or_render_pixels": (None, [vp, C.POINTER(_Cam), vp, vp, vp, i64, u32, C.POINTER(_Opts), vp]),
        "or_render_two_way": (None, [vp, C.POINTER(_Cam), u32, u32, u32, C.POINTER(_Opts), C.c_int32, vp, vp, vp,
                                     vp, vp]),
        "or_render_probes": (None, [vp, vp, vp, u32, u32, u32, u32, C.POINTER(_Opts), vp, vp, vp, vp]),
        "or_env_normal_cell": (C.c_int, [vp]),
        "or_env_sample_n": (None, [vp, vp, f64, f64, vp, vp]),
        "or_env_pdf_n": (f64, [vp, vp, vp]),
        "or_env_texel_probs_n": (None, [vp, C.c_int, vp]),
        "or_lb_sample": (i64, [vp, vp, vp, f64, vp]),
        "or_lb_prob": (f64, [vp, vp, vp, i64]),
        "or_lb_estimate": (f64, [vp, C.c_int32, vp, vp]),
        "or_lb_p_left": (f64, [vp, C.c_int32, vp, vp]),
        "or_lb_num_nodes": (C.c_int32, [vp]),
        "or_lb_node_info": (None, [vp, C.c_int32, vp, vp, vp, vp]),
        "or_lb_region": (C.c_int, [vp]),
        "or_lb_light_of_tri": (i64, [vp, i64]),
        "or_pa_info": (C.c_int32, [vp, vp, vp, vp]),
        "or_pa_eye": (None, [vp, C.POINTER(_Cam), vp]),
        "or_pa_probs": (None, [vp, vp, vp, vp, vp]),
        "or_pa_sample": (C.c_int32, [vp, vp, vp, vp, f64, vp]),
        "or_pa_env_density": (f64, [vp, vp, vp, vp]),
        "or_pa_dir_density": (f64, [vp, vp, vp, vp, vp]),
        "or_pa_cone_sample": (None, [vp, C.c_int32, vp, f64, f64, vp]),
        "or_vmf_pdf": (f64, [f64, vp, vp]),
        "or_vmf_sample": (None, [f64, vp, f64, f64, vp]),
        "or_oneblob": (None, [vp, vp]),
        "or_guide_features": (None, [vp, vp, vp, vp]),
        "or_mlp_forward": (None, [vp, vp, i64, vp, vp]),
        "or_mixture_pdf": (f64, [vp, vp]),
        "or_mixture_sample": (None, [vp, f64, f64, f64, vp]),
        "or_guide_loss_grad": (f64, [vp, vp, vp, vp, i64, vp]),
        "or_guide_nparams": (i64, []),
        "or_adam_step": (None, [vp, vp, vp, vp, i64, i64, f64, f64, f64, f64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ------------------------------------------------------------------ halton
def prime(dim: int) -> int:
    return lib().or_prime(dim)


def scramble_factor(seed: int, base: int) -> int:
    return lib().or_scramble_factor(seed, base)


def radical_inverse_u32(base: int, factor: int, index: int) -> int:
    return lib().or_radical_inverse_u32(base, factor, index)


def pixel_base_index(W: int, H: int, x: int, y: int) -> int:
    return lib().or_pixel_base_index(W, H, x, y)


def sample_dims_u32(indices, ndims: int, W: int, H: int, seed: int) -> np.ndarray:
    idx = np.ascontiguousarray(np.asarray(indices, dtype=np.uint64))
    out = np.zeros((idx.size, ndims), np.uint32)
    lib().or_sample_dims_batch(_p(idx), idx.size, ndims, W, H, seed, _p(out))
    return out


# ------------------------------------------------------------------- scene
class Scene:
    """Oracle scene built from a scenes.SceneData-like object (flattened)."""

    def __init__(self, sd):
        if getattr(sd, "instance_mesh", None) is not None:
            sd = sd.flattened()
        self._keep = []

        def keep(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            self._keep.append(a)
            return a

        v = keep(sd.vertices, np.float32)
        i = keep(sd.indices, np.uint32)
        d = _Desc()
        d.nv, d.nt = v.shape[0], i.shape[0]
        d.vertices = v.ctypes.data
        n = keep(sd.normals, np.float32)
        d.normals = n.ctypes.data if n is not None else None
        uv = keep(sd.uvs, np.float32)
        d.uvs = uv.ctypes.data if uv is not None else None
        d.indices = i.ctypes.data
        d.tri_material = keep(sd.tri_material, np.uint32).ctypes.data
        d.nm = int(np.asarray(sd.roughness).size)
        d.albedo = keep(sd.albedo, np.float32).ctypes.data
        d.roughness = keep(sd.roughness, np.float32).ctypes.data
        d.ggx_weight = keep(sd.ggx_weight, np.float32).ctypes.data
        d.emission = keep(sd.emission, np.float32).ctypes.data
        d.emission_tex = keep(sd.emission_tex, np.int32).ctypes.data
        tex = keep(sd.textures, np.float32)
        if tex is not None:
            d.ntex, d.tex_h, d.tex_w = tex.shape[0], tex.shape[1], tex.shape[2]
            d.textures = tex.ctypes.data
        env = keep(sd.env, np.float32)
        if env is not None:
            d.env_h, d.env_w = env.shape[0], env.shape[1]
            d.env = env.ctypes.data
        d.env_plain = int(getattr(sd, "env_plain", False))
        d.light_bvh = int(getattr(sd, "light_bvh", False))
        self._desc = d
        self.handle = lib().or_scene_create(C.byref(d))

    def __del__(self):
        if getattr(self, "handle", None):
            lib().or_scene_destroy(self.handle)
            self.handle = None

    # ---- ray casting
    def trace(self, rays: np.ndarray, any_hit: bool = False, use_bvh: bool = True):
        r = np.ascontiguousarray(rays, dtype=np.float32)
        n = r.shape[0]
        prim = np.zeros(n, np.uint32)
        t, b1, b2 = np.zeros(n), np.zeros(n), np.zeros(n)
        lib().or_trace(self.handle, _p(r), n, int(any_hit), int(use_bvh), _p(prim), _p(t), _p(b1), _p(b2))
        return prim, t, b1, b2

    def bvh_node_count(self) -> int:
        return lib().or_bvh_node_count(self.handle)

    # ---- lights
    def env_sample(self, u: float, v: float):
        wi = np.zeros(3)
        pdf = C.c_double()
        tx, ty = C.c_int32(), C.c_int32()
        lib().or_env_sample(self.handle, u, v, _p(wi), C.byref(pdf), C.byref(tx), C.byref(ty))
        return wi, pdf.value, tx.value, ty.value

    def env_pdf(self, wi) -> float:
        return lib().or_env_pdf(self.handle, _p(_f64(wi, 3)))

    def env_lookup(self, wi) -> np.ndarray:
        L = np.zeros(3)
        lib().or_env_lookup(self.handle, _p(_f64(wi, 3)), _p(L))
        return L

    def light_pdf_area(self, prim: int) -> float:
        return lib().or_scene_light_pdf_area(self.handle, prim)

    def env_select_prob(self) -> float:
        return lib().or_scene_env_select_prob(self.handle)

    # ---- rendering
    def render(self, cam, spp: int, max_depth: int, iter0: int = 0, sigma: float = 0.5,
               rr: bool = False, mis_mode: int = 0, seed: int = 0, threads: int = 0):
        c = _camera(cam)
        o = _Opts(sigma, int(rr), mis_mode, seed, threads)
        W, H = cam.width, cam.height
        s, s2 = np.zeros((H, W, 3)), np.zeros((H, W, 3))
        cnt = np.zeros((H, W), np.uint32)
        rays = np.zeros(1, np.uint64)
        lib().or_render(self.handle, C.byref(c), iter0, spp, max_depth, C.byref(o), _p(s), _p(s2),
                        _p(cnt), _p(rays))
        return s, s2, cnt, int(rays[0])

    def render_two_way(self, cam, spp: int, max_depth: int, iter0: int = 0, sigma: float = 0.5,
                       mis_mode: int = 0, lt_mode: int = 0, seed: int = 0, threads: int = 0, aim: bool = True):
        """Two-way path tracing (Sec. 2): camera stage sums (with the light
        tracer as a third MIS technique) and the light stage's splats; the
        per-pixel estimate is (sum + splat) / count. aim: photon aiming
        (Sec. 2.1.3), else emission uniform over the scene's bound."""
        c = _camera(cam)
        o = _Opts(sigma, 0, mis_mode, seed, threads, int(aim))
        W, H = cam.width, cam.height
        s, s2, sp = np.zeros((H, W, 3)), np.zeros((H, W, 3)), np.zeros((H, W, 3))
        cnt = np.zeros((H, W), np.uint32)
        rays = np.zeros(1, np.uint64)
        lib().or_render_two_way(self.handle, C.byref(c), iter0, spp, max_depth, C.byref(o), lt_mode, _p(s),
                                _p(s2), _p(cnt), _p(sp), _p(rays))
        return s, s2, cnt, sp, int(rays[0])

    def render_samples(self, cam, px, py, sj, max_depth: int, sigma: float = 0.5, rr: bool = False,
                       mis_mode: int = 0, seed: int = 0):
        c = _camera(cam)
        o = _Opts(sigma, int(rr), mis_mode, seed, 1)
        px = np.ascontiguousarray(px, np.uint32)
        py = np.ascontiguousarray(py, np.uint32)
        sj = np.ascontiguousarray(sj, np.uint32)
        L = np.zeros((px.size, 3))
        lib().or_render_pixels(self.handle, C.byref(c), _p(px), _p(py), _p(sj), px.size, max_depth,
                               C.byref(o), _p(L))
        return L

    def env_sample_n(self, ng, u: float, v: float):
        """Environment direction for a shading point of geometric normal ng
        (normal-oriented top levels) and its solid-angle pdf."""
        n = np.ascontiguousarray(ng, np.float64)
        wi = np.zeros(3)
        pdf = np.zeros(1)
        lib().or_env_sample_n(self.handle, _p(n), u, v, _p(wi), _p(pdf))
        return wi, float(pdf[0])

    def env_pdf_n(self, ng, wi) -> float:
        n = np.ascontiguousarray(ng, np.float64)
        w = np.ascontiguousarray(wi, np.float64)
        return lib().or_env_pdf_n(self.handle, _p(n), _p(w))

    def env_texel_probs_n(self, cell: int, W: int, H: int):
        out = np.zeros((H, W))
        lib().or_env_texel_probs_n(self.handle, cell, _p(out))
        return out

    # ---- probabilistic light hierarchy (light_bvh scenes, Sec. 2.1.1)
    def lb_sample(self, x, n, u: float):
        """(emitter index, its probability) drawn with u for point x, normal n."""
        prob = np.zeros(1)
        e = lib().or_lb_sample(self.handle, _p(_f64(x, 3)), _p(_f64(n, 3)), u, _p(prob))
        return int(e), float(prob[0])

    def lb_prob(self, x, n, e: int) -> float:
        return lib().or_lb_prob(self.handle, _p(_f64(x, 3)), _p(_f64(n, 3)), e)

    def lb_estimate(self, node: int, x, n) -> float:
        return lib().or_lb_estimate(self.handle, node, _p(_f64(x, 3)), _p(_f64(n, 3)))

    def lb_p_left(self, node: int, x, n) -> float:
        return lib().or_lb_p_left(self.handle, node, _p(_f64(x, 3)), _p(_f64(n, 3)))

    def lb_num_nodes(self) -> int:
        return lib().or_lb_num_nodes(self.handle)

    def lb_node(self, node: int):
        box, I, flux = np.zeros(6), np.zeros(6), np.zeros(1)
        links = np.zeros(4, np.int32)
        lib().or_lb_node_info(self.handle, node, _p(box), _p(I), _p(flux), links.ctypes.data)
        return {"lo": box[:3], "hi": box[3:], "I": I, "flux": float(flux[0]), "left": int(links[0]),
                "right": int(links[1]), "parent": int(links[2]), "count": int(links[3])}

    def lb_light_of_tri(self, t: int) -> int:
        return lib().or_lb_light_of_tri(self.handle, t)

    # ------------------------------------------ photon aiming (Sec. 2.1.3)
    def pa_clusters(self):
        """(cluster spheres [n][4]: centre, radius; cluster of every object)."""
        n_obj = C.c_int32()
        n = lib().or_pa_info(self.handle, None, None, C.byref(n_obj))
        cc = np.zeros((n, 4))
        oc = np.zeros(n_obj.value, np.int32)
        lib().or_pa_info(self.handle, _p(cc), _p(oc), None)
        return cc, oc

    def pa_eye(self, cam):
        """Photon aiming's eye vector of a camera: (position, solid angle of its view cone)."""
        out = np.zeros(4)
        c = _camera(cam)
        lib().or_pa_eye(self.handle, C.byref(c), _p(out))
        return out

    def pa_probs(self, eye, y=None, ny=None):
        n = self.pa_clusters()[0].shape[0]
        P = np.zeros(n)
        lib().or_pa_probs(self.handle, _p(_f64(eye, 4)), None if y is None else _p(_f64(y, 3)),
                          None if ny is None else _p(_f64(ny, 3)), _p(P))
        return P

    def pa_sample(self, eye, u, y=None, ny=None):
        p = C.c_double()
        c = lib().or_pa_sample(self.handle, _p(_f64(eye, 4)), None if y is None else _p(_f64(y, 3)),
                               None if ny is None else _p(_f64(ny, 3)), u, C.byref(p))
        return c, p.value

    def pa_env_density(self, eye, x, w):
        return lib().or_pa_env_density(self.handle, _p(_f64(eye, 4)), _p(_f64(x, 3)), _p(_f64(w, 3)))

    def pa_dir_density(self, eye, y, ny, w):
        return lib().or_pa_dir_density(self.handle, _p(_f64(eye, 4)), _p(_f64(y, 3)), _p(_f64(ny, 3)),
                                       _p(_f64(w, 3)))

    def pa_cone_sample(self, c, y, u1, u2):
        w = np.zeros(3)
        lib().or_pa_cone_sample(self.handle, c, _p(_f64(y, 3)), u1, u2, _p(w))
        return w

    def render_probes(self, pos, nrm, spp: int, max_depth: int, iter0: int = 0, mis_mode: int = 0,
                      seed: int = 0, rr: bool = False):
        """Irradiance probes (Sec. 4.2): per probe the sums of E, E^2 and the
        sample count over iterations [iter0, iter0 + spp)."""
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        nrm = np.ascontiguousarray(nrm, np.float64).reshape(-1, 3)
        n = pos.shape[0]
        o = _Opts(0.5, int(rr), mis_mode, seed, 1)
        S, S2 = np.zeros((n, 3)), np.zeros((n, 3))
        cnt = np.zeros(n, np.uint32)
        rays = np.zeros(1, np.uint64)
        lib().or_render_probes(self.handle, _p(pos), _p(nrm), n, iter0, spp, max_depth, C.byref(o), _p(S), _p(S2),
                               _p(cnt), _p(rays))
        return S, S2, cnt, int(rays[0])


def lb_region(w) -> int:
    """Cube-face region of a direction (0..5 = +x, -x, +y, -y, +z, -z)."""
    return lib().or_lb_region(_p(_f64(w, 3)))


def env_normal_cell(n) -> int:
    """Cell of a normal in the 8 x 8 octahedral map of the normal-oriented
    environment levels."""
    a = np.ascontiguousarray(n, np.float64)
    return lib().or_env_normal_cell(_p(a))


def _camera(cam) -> _Cam:
    c = _Cam()
    for k in range(3):
        c.eye[k], c.look_at[k], c.up[k] = cam.eye[k], cam.look_at[k], cam.up[k]
    c.vfov_deg, c.width, c.height = cam.vfov_deg, cam.width, cam.height
    return c


def camera_ray(cam, sx: float, sy: float):
    o, d = np.zeros(3), np.zeros(3)
    c = _camera(cam)
    lib().or_camera_ray(C.byref(c), sx, sy, _p(o), _p(d))
    return o, d


def filter_offset(sigma: float, u0: float, u1: float):
    dx, dy = C.c_double(), C.c_double()
    lib().or_filter_offset(sigma, u0, u1, C.byref(dx), C.byref(dy))
    return dx.value, dy.value


def resolve(sum_, sum2, count):
    """Per-pixel mean and variance of the mean from FP64 film sums."""
    n = np.maximum(count.astype(np.float64), 1.0)[..., None]
    mean = sum_ / n
    var = np.maximum(sum2 / n - mean * mean, 0.0) / np.maximum(n - 1.0, 1.0)
    return mean, var


# ---------------------------------------------------------------- shading
def adapt_shading_normal(ns, ng, wo):
    out = np.zeros(3)
    lib().or_adapt_shading_normal(_p(_f64(ns, 3)), _p(_f64(ng, 3)), _p(_f64(wo, 3)), _p(out))
    return out


def bsdf_eval(albedo, rough, w, ns, wo, wi):
    f = np.zeros(3)
    pdf = C.c_double()
    lib().or_bsdf_eval(_p(_f64(albedo, 3)), rough, w, _p(_f64(ns, 3)), _p(_f64(wo, 3)), _p(_f64(wi, 3)),
                       _p(f), C.byref(pdf))
    return f, pdf.value


def bsdf_sample(albedo, rough, w, ns, wo, u_lobe, u1, u2):
    wi, f = np.zeros(3), np.zeros(3)
    pdf = C.c_double()
    ok = lib().or_bsdf_sample(_p(_f64(albedo, 3)), rough, w, _p(_f64(ns, 3)), _p(_f64(wo, 3)), u_lobe, u1,
                              u2, _p(wi), _p(f), C.byref(pdf))
    return bool(ok), wi, f, pdf.value


def ggx_D(alpha, cos_h):
    return lib().or_ggx_D(alpha, cos_h)


def ggx_G1(alpha, cos_t):
    return lib().or_ggx_G1(alpha, cos_t)


def onb(n):
    t, b = np.zeros(3), np.zeros(3)
    lib().or_onb(_p(_f64(n, 3)), _p(t), _p(b))
    return t, b


# ----------------------------------------------------------------- lights
def alias_build(w):
    w = _f64(w)
    prob = np.zeros(w.size)
    alias = np.zeros(w.size, np.int64)
    lib().or_alias_build(_p(w), w.size, _p(prob), _p(alias))
    return prob, alias


def alias_sample(prob, alias, u: float) -> int:
    return lib().or_alias_sample(_p(prob), _p(alias), prob.size, u)


def env_pyramid_probs(env: np.ndarray) -> np.ndarray:
    e = np.ascontiguousarray(env, np.float32)
    H, W = e.shape[0], e.shape[1]
    out = np.zeros((H, W))
    lib().or_env_pyramid_probs(_p(e), W, H, _p(out))
    return out


# ------------------------------------------------------------------ guide
def vmf_pdf(kappa, mu, w):
    return lib().or_vmf_pdf(kappa, _p(_f64(mu, 3)), _p(_f64(w, 3)))


def vmf_sample(kappa, mu, u1, u2):
    w = np.zeros(3)
    lib().or_vmf_sample(kappa, _p(_f64(mu, 3)), u1, u2, _p(w))
    return w


def oneblob(s7):
    enc = np.zeros(224)
    lib().or_oneblob(_p(_f64(s7, 7)), _p(enc))
    return enc


def guide_features(pos01, wo, n):
    s = np.zeros(7)
    lib().or_guide_features(_p(_f64(pos01, 3)), _p(_f64(wo, 3)), _p(_f64(n, 3)), _p(s))
    return s


def guide_nparams() -> int:
    return lib().or_guide_nparams()


def mlp_forward(params, x):
    p = _f64(params)
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 224))
    out = np.zeros((x.shape[0], 40))
    lib().or_mlp_forward(_p(p), _p(x), x.shape[0], _p(out), None)
    return out


def mlp_forward_acts(params, x):
    """Outputs [n][40] and the four hidden activations [n][4][64]."""
    p = _f64(params)
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 224))
    out = np.zeros((x.shape[0], 40))
    acts = np.zeros((x.shape[0], 4, 64))
    lib().or_mlp_forward(_p(p), _p(x), x.shape[0], _p(out), _p(acts))
    return out, acts


def mixture_pdf(raw, w):
    return lib().or_mixture_pdf(_p(_f64(raw, 40)), _p(_f64(w, 3)))


def mixture_sample(raw, u_sel, u1, u2):
    w = np.zeros(3)
    lib().or_mixture_sample(_p(_f64(raw, 40)), u_sel, u1, u2, _p(w))
    return w


def guide_loss_grad(params, x, wi, weight):
    p = _f64(params)
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 224))
    wi = np.ascontiguousarray(np.asarray(wi, np.float64).reshape(-1, 3))
    wt = _f64(weight)
    g = np.zeros(p.size)
    loss = lib().or_guide_loss_grad(_p(p), _p(x), _p(wi), _p(wt), x.shape[0], _p(g))
    return loss, g


def adam_step(params, grad, m, v, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays params, m, v."""
    lib().or_adam_step(_p(params), _p(_f64(grad)), _p(m), _p(v), params.size, t, lr, b1, b2, eps)
