"""Thin Python binding of the C ABI in include/rt.h (ctypes).

Argument marshalling only: every step of the hot path runs in the CUDA
library. Device buffers are torch CUDA tensors (PyTorch provides device
memory and streams); host buffers are numpy arrays. The library must have
been built (``paper_1705_01263_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

RT_MISS = 0xFFFFFFFF
STATUS = {0: "RT_OK", 1: "RT_INVALID_ARG", 2: "RT_OOM", 3: "RT_CUDA_ERROR", 4: "RT_TIMEOUT",
          5: "RT_QUEUE_OVERFLOW", 6: "RT_STACK_OVERFLOW", 7: "RT_NOT_SUPPORTED"}
RT_OK, RT_TIMEOUT = 0, 4


class RtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class rt_scene_desc(C.Structure):
    _fields_ = [
        ("num_vertices", C.c_int64), ("num_triangles", C.c_int64),
        ("vertices", C.c_void_p), ("normals", C.c_void_p), ("uvs", C.c_void_p),
        ("indices", C.c_void_p), ("tri_material", C.c_void_p),
        ("num_materials", C.c_int32), ("albedo", C.c_void_p), ("roughness", C.c_void_p),
        ("ggx_weight", C.c_void_p), ("emission", C.c_void_p), ("emission_tex", C.c_void_p),
        ("num_textures", C.c_int32), ("tex_width", C.c_int32), ("tex_height", C.c_int32),
        ("textures", C.c_void_p),
        ("env_width", C.c_int32), ("env_height", C.c_int32), ("env", C.c_void_p),
        ("num_meshes", C.c_int32), ("mesh_tri_offset", C.c_void_p),
        ("num_instances", C.c_int32), ("instance_mesh", C.c_void_p), ("instance_xform", C.c_void_p),
        ("env_plain", C.c_int32), ("light_bvh", C.c_int32),
    ]


class rt_rays(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax")]


class rt_hits(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("prim", "inst", "t", "u", "v")]


class rt_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class rt_stats(C.Structure):
    _fields_ = [("paths", C.c_uint64), ("extension_rays", C.c_uint64), ("shadow_rays", C.c_uint64),
                ("waves", C.c_uint32), ("wavefront_steps", C.c_uint32), ("tail_launches", C.c_uint32),
                ("kernel_launches", C.c_uint32), ("trace_ms", C.c_double), ("shade_ms", C.c_double),
                ("shadow_ms", C.c_double), ("megakernel_ms", C.c_double), ("other_ms", C.c_double),
                ("trace_launches", C.c_uint32), ("ext_nodes", C.c_uint64), ("ext_tris", C.c_uint64),
                ("shadow_nodes", C.c_uint64), ("shadow_tris", C.c_uint64), ("regen_sets", C.c_uint32)]


class rt_render_opts(C.Structure):
    _fields_ = [("filter_sigma", C.c_float), ("rr_enable", C.c_int32), ("mis_mode", C.c_int32),
                ("seed", C.c_uint64), ("time_budget_ms", C.c_double), ("max_paths_in_flight", C.c_uint32),
                ("megakernel_only", C.c_int32), ("sort_by_material", C.c_int32),
                ("tail_threshold", C.c_uint32), ("block_size", C.c_uint32),
                ("abort_flag", C.c_void_p), ("guide", C.c_void_p), ("stats", C.POINTER(rt_stats)),
                ("profile", C.c_int32), ("trace_kernel", C.c_int32), ("sort_rays", C.c_int32),
                ("scheduler", C.c_int32), ("regen_fraction", C.c_float), ("lt_emission", C.c_int32),
                ("state_compression", C.c_int32)]


class rt_render_job(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("camera", rt_camera), ("spp", C.c_uint32), ("max_depth", C.c_uint32),
                ("film", C.c_void_p), ("guide", C.c_void_p)]


class rt_guide_opts(C.Structure):
    _fields_ = [("batch", C.c_uint32), ("learning_rate", C.c_float), ("alpha", C.c_float),
                ("train_steps", C.c_uint32), ("seed", C.c_uint64), ("train_every", C.c_uint32),
                ("guide_depth", C.c_uint32), ("warm_steps", C.c_uint32), ("warm_set_batches", C.c_uint32)]


_lib = None

EXPORTED = [
    "rt_scene_create", "rt_scene_destroy", "rt_scene_info", "rt_trace", "rt_film_create", "rt_film_destroy",
    "rt_film_clear", "rt_film_next_iteration", "rt_film_seek", "rt_film_buffers", "rt_film_resolve", "rt_render",
    "rt_render_static", "rt_render_batch", "rt_autotune", "rt_sample_index", "rt_halton", "rt_divide_u64_host", "rt_guide_create", "rt_guide_destroy",
    "rt_guide_num_params", "rt_guide_get_params", "rt_guide_set_params", "rt_guide_state_size", "rt_guide_save",
    "rt_guide_load", "rt_guide_infer", "rt_guide_infer_async", "rt_guide_check", "rt_guide_loss_grad", "rt_guide_train_step", "rt_last_error",
    "rt_status_string", "rt_gemm_bf16", "rt_render_probes", "rt_render_two_way",
]


def lib(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed). Raises if the
    library cannot be built or loaded: there is no CPU fallback."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    vp, i64, u32, u64, i32 = C.c_void_p, C.c_int64, C.c_uint32, C.c_uint64, C.c_int32
    sigs = {
        "rt_scene_create": [C.POINTER(rt_scene_desc), C.POINTER(vp)],
        "rt_debug_scene_create_host": [C.POINTER(rt_scene_desc), C.POINTER(vp)],
        "rt_scene_destroy": [vp],
        "rt_scene_info": [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)],
        "rt_trace": [vp, C.POINTER(rt_rays), i64, C.POINTER(rt_hits), i32, vp],
        "rt_film_create": [u32, u32, C.POINTER(vp)],
        "rt_film_destroy": [vp],
        "rt_film_clear": [vp, vp],
        "rt_film_next_iteration": [vp, C.POINTER(u32)],
        "rt_film_seek": [vp, u32],
        "rt_film_buffers": [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)],
        "rt_film_resolve": [vp, vp, vp, vp],
        "rt_render": [vp, C.POINTER(rt_camera), u32, u32, vp, C.POINTER(rt_render_opts), vp],
        "rt_render_static": [vp, C.POINTER(rt_camera), u32, u32, u32, vp, vp, vp, C.POINTER(rt_render_opts), vp],
        "rt_render_batch": [vp, i32, C.POINTER(rt_render_opts), vp],
        "rt_autotune": [vp, i32, u32, C.POINTER(rt_render_opts), vp],
        "rt_sample_index": [u32, u32, vp, vp, vp, i64, vp, vp],
        "rt_halton": [u32, u32, u64, vp, i64, i32, vp, vp],
        "rt_divide_u64_host": [vp, i64, u32, vp],
        "rt_gemm_bf16": [vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, vp],
        "rt_debug_trace_host": [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp],
        "rt_debug_trace_host_stack": [vp, vp, i64, i32, i32, vp, vp],
        "rt_debug_regen_host": [u32, u32, u32, vp, u32, vp, vp, vp],
        "rt_debug_guided_plan_host": [u32, u32, u32, u32, u32, i32, u32, i32, vp],
        "rt_debug_aim_tree_host": [vp, vp, vp, vp, vp],
        "rt_debug_aim_host": [vp, vp, i32, vp, i64, vp],
        "rt_debug_env_sample_host": [vp, vp, vp, vp, i64, vp, vp, vp],
        "rt_debug_light_bvh_host": [vp, vp, vp, vp, i64, vp, vp, vp],
        "rt_debug_render_host": [vp, C.POINTER(rt_camera), u32, C.POINTER(rt_render_opts), vp, vp, vp, i64, vp],
        "rt_debug_halton_host": [u32, u32, u64, vp, i64, i32, vp],
        "rt_debug_sample_index_host": [u32, u32, u32, u32, u32, C.POINTER(u64)],
        "rt_debug_guide_infer_layers": [vp, vp, i64, vp, vp],
        "rt_debug_guide_mixture": [vp, vp, vp, i64, vp, vp, vp, vp],
        "rt_debug_render_probes_host": [vp, vp, vp, u32, u32, C.POINTER(rt_render_opts), vp, vp, i64, vp],
        "rt_render_probes": [vp, vp, vp, u32, u32, u32, vp, C.POINTER(rt_render_opts), vp],
        "rt_render_two_way": [vp, C.POINTER(rt_camera), u32, u32, vp, C.POINTER(rt_render_opts), C.c_int32, vp,
                              vp, vp],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.rt_last_error.restype = C.c_char_p
    L.rt_status_string.restype = C.c_char_p
    L.rt_status_string.argtypes = [C.c_int]
    if hasattr(L, "rt_guide_num_params"):
        L.rt_guide_num_params.restype = C.c_int64
        L.rt_guide_num_params.argtypes = []
    for name, args in {
        "rt_guide_create": [vp, C.POINTER(rt_guide_opts), C.POINTER(vp)],
        "rt_guide_destroy": [vp],
        "rt_guide_get_params": [vp, vp],
        "rt_guide_set_params": [vp, vp],
        "rt_guide_state_size": [vp, C.POINTER(i64)],
        "rt_guide_save": [vp, vp],
        "rt_guide_load": [vp, vp],
        "rt_guide_infer": [vp, vp, i64, vp, vp],
        "rt_guide_infer_async": [vp, vp, i64, vp, vp],
        "rt_guide_check": [vp, vp],
        "rt_guide_loss_grad": [vp, vp, vp, vp, i64, vp, C.POINTER(C.c_float), vp],
        "rt_guide_train_step": [vp, vp, vp, vp, i64, vp],
    }.items():
        if hasattr(L, name):
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int


def check(status: int):
    if status != RT_OK:
        raise RtError(status, lib().rt_last_error().decode())
    return status


def _ptr(t) -> Optional[int]:
    """Device address of a torch tensor (or host address of a numpy array)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream=None):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------ scene
class Scene:
    """Device scene built from a scenes.SceneData (rt_scene_create)."""

    def __init__(self, sd, host_only: bool = False):
        self._keep = []
        d = rt_scene_desc()

        def arr(a, dt, cols=None):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=dt))
            self._keep.append(a)
            return a.ctypes.data

        d.num_vertices = int(sd.vertices.shape[0])
        d.num_triangles = int(sd.indices.shape[0])
        d.vertices = arr(sd.vertices, np.float32)
        d.normals = arr(sd.normals, np.float32)
        d.uvs = arr(sd.uvs, np.float32)
        d.indices = arr(sd.indices, np.uint32)
        d.tri_material = arr(sd.tri_material, np.uint32)
        d.num_materials = int(np.asarray(sd.roughness).size)
        d.albedo = arr(sd.albedo, np.float32)
        d.roughness = arr(sd.roughness, np.float32)
        d.ggx_weight = arr(sd.ggx_weight, np.float32)
        d.emission = arr(sd.emission, np.float32)
        d.emission_tex = arr(sd.emission_tex, np.int32)
        if sd.textures is not None:
            d.num_textures, d.tex_height, d.tex_width = (int(x) for x in sd.textures.shape[:3])
            d.textures = arr(sd.textures, np.float32)
        if sd.env is not None:
            d.env_height, d.env_width = int(sd.env.shape[0]), int(sd.env.shape[1])
            d.env = arr(sd.env, np.float32)
            d.env_plain = 1 if getattr(sd, "env_plain", False) else 0
        d.light_bvh = 1 if getattr(sd, "light_bvh", False) else 0
        if getattr(sd, "instance_mesh", None) is not None:
            d.num_meshes = int(len(sd.mesh_tri_offset) - 1)
            d.mesh_tri_offset = arr(sd.mesh_tri_offset, np.int64)
            d.num_instances = int(len(sd.instance_mesh))
            d.instance_mesh = arr(sd.instance_mesh, np.uint32)
            d.instance_xform = arr(sd.instance_xform, np.float32)
        self.desc = d
        h = C.c_void_p()
        fn = lib().rt_debug_scene_create_host if host_only else lib().rt_scene_create
        check(fn(C.byref(d), C.byref(h)))
        self.handle = h
        self.host_only = host_only
        self._keep = None  # the library copied everything

    def info(self):
        n, t, b = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().rt_scene_info(self.handle, C.byref(n), C.byref(t), C.byref(b)))
        return {"nodes": n.value, "leaf_tris": t.value, "device_bytes": b.value}

    def close(self):
        if getattr(self, "handle", None):
            lib().rt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rt_scene_create(sd) -> Scene:
    return Scene(sd)


def rt_trace(scene: Scene, rays, any_hit: bool = False, hits=None, stream=None):
    """rays: torch CUDA float32 tensor n x 8 (ox oy oz dx dy dz tmin tmax),
    column-sliced into the SoA pointers (the tensor is transposed to 8 x n).
    Returns (prim, inst, t, u, v) torch tensors."""
    import torch
    soa = rays.t().contiguous() if rays.shape[-1] == 8 else rays
    n = soa.shape[1]
    if hits is None:
        hits = (torch.empty(n, dtype=torch.int32, device=soa.device),
                torch.empty(n, dtype=torch.int32, device=soa.device),
                torch.empty(n, dtype=torch.float32, device=soa.device),
                torch.empty(n, dtype=torch.float32, device=soa.device),
                torch.empty(n, dtype=torch.float32, device=soa.device))
    r = rt_rays(*[soa[k].data_ptr() for k in range(8)])
    h = rt_hits(*[x.data_ptr() for x in hits])
    check(lib().rt_trace(scene.handle, C.byref(r), n, C.byref(h), int(any_hit), _stream(stream)))
    return hits, soa


class Film:
    def __init__(self, width: int, height: int):
        h = C.c_void_p()
        check(lib().rt_film_create(width, height, C.byref(h)))
        self.handle = h
        self.width, self.height = width, height

    def clear(self, stream=None):
        check(lib().rt_film_clear(self.handle, _stream(stream)))

    def next_iteration(self) -> int:
        v = C.c_uint32()
        check(lib().rt_film_next_iteration(self.handle, C.byref(v)))
        return v.value

    def seek(self, next_iteration: int):
        check(lib().rt_film_seek(self.handle, next_iteration))

    def buffers(self):
        """(sum, sum2, count) as torch tensors viewing the film's device memory."""
        import torch
        s, s2, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
        check(lib().rt_film_buffers(self.handle, C.byref(s), C.byref(s2), C.byref(c)))
        n = self.width * self.height
        return (_wrap_device(s.value, (self.height, self.width, 3), torch.float64),
                _wrap_device(s2.value, (self.height, self.width, 3), torch.float64),
                _wrap_device(c.value, (self.height, self.width), torch.int32))

    def download(self):
        import torch
        torch.cuda.synchronize()
        s, s2, c = self.buffers()
        return s.cpu().numpy().copy(), s2.cpu().numpy().copy(), c.cpu().numpy().view(np.uint32).copy()

    def resolve(self, mean=None, var=None, stream=None):
        import torch
        if mean is None:
            mean = torch.empty((self.height, self.width, 3), dtype=torch.float32, device="cuda")
        check(lib().rt_film_resolve(self.handle, mean.data_ptr(), None if var is None else var.data_ptr(),
                                    _stream(stream)))
        return mean, var

    def close(self):
        if getattr(self, "handle", None):
            lib().rt_film_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _wrap_device(ptr: int, shape, dtype):
    """Zero-copy torch view of library-owned device memory."""
    import torch
    n = int(np.prod(shape))
    itemsize = torch.empty((), dtype=dtype).element_size()

    class _Arr:
        __cuda_array_interface__ = {
            "shape": (n,), "typestr": {torch.float64: "<f8", torch.int32: "<i4", torch.float32: "<f4"}[dtype],
            "data": (ptr, False), "version": 3, "strides": None,
        }
    t = torch.as_tensor(_Arr(), device="cuda")
    return t.view(*shape)


def rt_film_create(width: int, height: int) -> Film:
    return Film(width, height)


def make_camera(cam) -> rt_camera:
    c = rt_camera()
    for k in range(3):
        c.eye[k], c.look_at[k], c.up[k] = cam.eye[k], cam.look_at[k], cam.up[k]
    c.vfov_deg, c.width, c.height = cam.vfov_deg, cam.width, cam.height
    return c


def make_opts(sigma: float = 0.5, rr: bool = False, mis_mode: int = 0, seed: int = 0, time_budget_ms: float = 0.0,
              max_paths: int = 0, megakernel_only: bool = False, sort_by_material: bool = False,
              tail_threshold: int = 0, abort_flag=None, guide=None, stats: Optional[rt_stats] = None,
              profile: int = 0, trace_kernel: int = 0, sort_rays: bool = False, block_size: int = 0,
              scheduler: int = 0, regen_fraction: float = 0.0, lt_emission: int = 0,
              state_compression: bool = False):
    o = rt_render_opts()
    o.filter_sigma = sigma if sigma > 0 else -1.0
    o.rr_enable, o.mis_mode, o.seed = int(rr), mis_mode, seed
    o.time_budget_ms, o.max_paths_in_flight = time_budget_ms, max_paths
    o.megakernel_only, o.sort_by_material, o.tail_threshold = int(megakernel_only), int(sort_by_material), tail_threshold
    o.abort_flag = abort_flag
    o.guide = guide.handle if guide is not None else None
    # keep the Python objects whose handles the options point to alive for as
    # long as the options are
    o._keep_alive = (guide, stats)
    if stats is not None:
        o.stats = C.pointer(stats)
    o.profile = profile
    o.trace_kernel = trace_kernel
    o.sort_rays = int(sort_rays)
    o.block_size = block_size
    o.scheduler = scheduler
    o.regen_fraction = regen_fraction
    o.lt_emission = lt_emission
    o.state_compression = int(state_compression)
    return o


def rt_render(scene: Scene, cam, spp: int, max_depth: int, film: Film, opts: Optional[rt_render_opts] = None,
              stream=None, allow_timeout: bool = False) -> int:
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    st = lib().rt_render(scene.handle, C.byref(c), spp, max_depth, film.handle, C.byref(o), _stream(stream))
    if st == RT_TIMEOUT and allow_timeout:
        return st
    return check(st)


def _jobs(jobs):
    """jobs: list of (Scene, camera, spp, max_depth, Film[, Guide or None])."""
    arr = (rt_render_job * len(jobs))()
    for k, job in enumerate(jobs):
        sc, cam, spp, depth, film = job[:5]
        guide = job[5] if len(job) > 5 else None
        arr[k].scene, arr[k].camera, arr[k].spp, arr[k].max_depth, arr[k].film = sc.handle, make_camera(cam), spp, depth, film.handle
        arr[k].guide = guide.handle if guide is not None else None
    return arr


def rt_render_batch(jobs, opts: Optional[rt_render_opts] = None, stream=None, allow_timeout: bool = False) -> int:
    arr = _jobs(jobs)
    o = opts if opts is not None else make_opts()
    st = lib().rt_render_batch(arr, len(jobs), C.byref(o), _stream(stream))
    if st == RT_TIMEOUT and allow_timeout:
        return st
    return check(st)


def rt_autotune(jobs, sample_spp: int = 1, opts: Optional[rt_render_opts] = None, stream=None) -> rt_render_opts:
    arr = _jobs(jobs)
    o = opts if opts is not None else make_opts()
    check(lib().rt_autotune(arr, len(jobs), sample_spp, C.byref(o), _stream(stream)))
    return o


def rt_render_static(scene: Scene, cam, spp: int, max_depth: int, first_iteration: int, sum_, sum2, count,
                     opts: Optional[rt_render_opts] = None, stream=None) -> int:
    """Allocation-free render into caller-owned device tensors (float64
    H x W x 3 sums, int32 H x W count), accumulated in place."""
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    return check(lib().rt_render_static(scene.handle, C.byref(c), spp, max_depth, first_iteration, sum_.data_ptr(),
                                        sum2.data_ptr(), count.data_ptr(), C.byref(o), _stream(stream)))


def rt_sample_index(width, height, px, py, j, out=None, stream=None):
    import torch
    n = px.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.int64, device=px.device)
    check(lib().rt_sample_index(width, height, px.data_ptr(), py.data_ptr(), j.data_ptr(), n, out.data_ptr(),
                                _stream(stream)))
    return out


def rt_halton(width, height, seed, indices, ndims, out=None, stream=None):
    import torch
    n = indices.numel()
    if out is None:
        out = torch.empty((n, ndims), dtype=torch.int32, device=indices.device)
    check(lib().rt_halton(width, height, seed, indices.data_ptr(), n, ndims, out.data_ptr(), _stream(stream)))
    return out


def rt_divide_u64_host(n: np.ndarray, d: int) -> np.ndarray:
    n = np.ascontiguousarray(n, np.uint64)
    q = np.zeros_like(n)
    check(lib().rt_divide_u64_host(n.ctypes.data, n.size, d, q.ctypes.data))
    return q


def rt_gemm_bf16(A, B, C=None, accumulate=False, stream=None):
    """C = A @ B.T on the tensor cores (A: M x K bf16, B: N x K bf16, C: M x N f32)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    check(lib().rt_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, A.stride(0), B.stride(0),
                             C.stride(0), int(accumulate), _stream(stream)))
    return C


class Guide:
    """Online path-guiding network (rt_guide_*)."""

    def __init__(self, scene=None, batch=0, lr=0.0, alpha=0.0, train_steps=0, seed=0, train_every=0, guide_depth=0,
                 warm_steps=0, warm_set_batches=0):
        o = rt_guide_opts(batch, lr, alpha, train_steps, seed, train_every, guide_depth, warm_steps,
                          warm_set_batches)
        h = C.c_void_p()
        check(lib().rt_guide_create(scene.handle if scene is not None else None, C.byref(o), C.byref(h)))
        self.handle = h

    @staticmethod
    def num_params() -> int:
        return lib().rt_guide_num_params()

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.num_params(), np.float32)
        check(lib().rt_guide_get_params(self.handle, p.ctypes.data))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        check(lib().rt_guide_set_params(self.handle, p.ctypes.data))

    def state(self) -> bytes:
        n = C.c_int64()
        check(lib().rt_guide_state_size(self.handle, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        check(lib().rt_guide_save(self.handle, buf.ctypes.data))
        return buf.tobytes()

    def load(self, blob: bytes):
        buf = np.frombuffer(blob, np.uint8).copy()
        check(lib().rt_guide_load(self.handle, buf.ctypes.data))

    def infer(self, features, stream=None):
        import torch
        n = features.shape[0]
        raw = torch.empty((n, 40), dtype=torch.float32, device=features.device)
        check(lib().rt_guide_infer(self.handle, features.data_ptr(), n, raw.data_ptr(), _stream(stream)))
        return raw

    def infer_async(self, features, raw, stream=None):
        """Enqueue the fused inference into `raw` (n x 40, device) without
        waiting; check() reports a completion-wait timeout."""
        check(lib().rt_guide_infer_async(self.handle, features.data_ptr(), features.shape[0], raw.data_ptr(),
                                         _stream(stream)))
        return raw

    def check(self, stream=None):
        check(lib().rt_guide_check(self.handle, _stream(stream)))

    def infer_layers(self, features, stream=None):
        """Test hook: the same outputs layer by layer through the GEMM path
        the training forward pass uses (rt_guide_infer runs the fused kernel)."""
        import torch
        n = features.shape[0]
        raw = torch.empty((n, 40), dtype=torch.float32, device=features.device)
        check(lib().rt_debug_guide_infer_layers(self.handle, features.data_ptr(), n, raw.data_ptr(), _stream(stream)))
        return raw

    def loss_grad(self, features, wi, weight, stream=None):
        import torch
        n = features.shape[0]
        g = torch.empty(self.num_params(), dtype=torch.float32, device=features.device)
        loss = C.c_float()
        check(lib().rt_guide_loss_grad(self.handle, features.data_ptr(), wi.data_ptr(), weight.data_ptr(), n,
                                       g.data_ptr(), C.byref(loss), _stream(stream)))
        return loss.value, g

    def train_step(self, features, wi, weight, stream=None):
        check(lib().rt_guide_train_step(self.handle, features.data_ptr(), wi.data_ptr(), weight.data_ptr(),
                                        features.shape[0], _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            lib().rt_guide_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_guide_mixture(raw, wi, u, stream=None):
    """Test hook: (pdf at wi, sampled direction, pdf at it) from the device
    mixture code of guided shading; torch CUDA float32 inputs [n][40],
    [n][3], [n][3]."""
    import torch
    n = raw.shape[0]
    pdf_wi = torch.empty(n, dtype=torch.float32, device=raw.device)
    ws = torch.empty((n, 3), dtype=torch.float32, device=raw.device)
    pdf_ws = torch.empty(n, dtype=torch.float32, device=raw.device)
    check(lib().rt_debug_guide_mixture(raw.data_ptr(), wi.data_ptr(), u.data_ptr(), n, pdf_wi.data_ptr(),
                                       ws.data_ptr(), pdf_ws.data_ptr(), _stream(stream)))
    return pdf_wi, ws, pdf_ws


# -------------------------------------------------- host test hooks (CPU)
def debug_trace_host(scene: Scene, rays: np.ndarray, any_hit: bool = False, return_inst: bool = False):
    r = np.ascontiguousarray(rays, np.float32)
    n = r.shape[0]
    prim = np.zeros(n, np.uint32)
    t, u, v = np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.float32)
    nodes = np.zeros(n, np.uint32)
    inst = np.zeros(n, np.uint32)
    check(lib().rt_debug_trace_host(scene.handle, r.ctypes.data, n, int(any_hit), prim.ctypes.data, t.ctypes.data,
                                    u.ctypes.data, v.ctypes.data, nodes.ctypes.data, inst.ctypes.data))
    if return_inst:
        return prim, t, u, v, nodes, inst
    return prim, t, u, v, nodes


def debug_trace_host_stack(scene: Scene, rays: np.ndarray, stack_entries: int, any_hit: bool = False):
    """(prim, t) of the traversal run on the host with a stack of only
    `stack_entries` node groups; RtError(RT_STACK_OVERFLOW) when a ray needs more."""
    r = np.ascontiguousarray(rays, np.float32)
    n = r.shape[0]
    prim = np.zeros(n, np.uint32)
    t = np.zeros(n, np.float32)
    check(lib().rt_debug_trace_host_stack(scene.handle, r.ctypes.data, n, int(any_hit), int(stack_entries),
                                          prim.ctypes.data, t.ctypes.data))
    return prim, t


def debug_regen_host(life: np.ndarray, cap: int, regen_min: int, stop_step: int = 0xFFFFFFFF):
    """Host run of the regeneration scheduler's slot bookkeeping with path
    lengths `life` (uint8, >= 1 per task): (step at which each task was
    retired, or 0xFFFFFFFF if never started; steps; refilling steps)."""
    life = np.ascontiguousarray(life, np.uint8)
    n = life.size
    out = np.zeros(n, np.uint32)
    steps, regen = C.c_uint32(), C.c_uint32()
    check(lib().rt_debug_regen_host(n, cap, regen_min, life.ctypes.data, stop_step, out.ctypes.data,
                                    C.byref(steps), C.byref(regen)))
    return out, steps.value, regen.value


GUIDED_PLAN_FIELDS = ("cap", "cap_young", "per_step", "gdepth", "rec_depth", "keep_young", "rec_young",
                      "rec_alloc", "keep_alloc", "keep", "rec_paths", "rec_stride", "set_steps")


def debug_guided_plan_host(batch: int, wsb: int, guide_depth: int, max_depth: int, cap: int, fixed_pool: bool,
                           n: int, young: bool) -> dict:
    """Host run of the guided render's set and buffer arithmetic: a dict of
    GUIDED_PLAN_FIELDS for a pool of `cap` paths per set and a set of n
    paths."""
    out = np.zeros(13, np.uint32)
    check(lib().rt_debug_guided_plan_host(batch, wsb, guide_depth, max_depth, cap, int(fixed_pool), n, int(young),
                                          out.ctypes.data))
    return dict(zip(GUIDED_PLAN_FIELDS, (int(x) for x in out)))


def debug_aim_tree_host(scene: Scene):
    """Photon aiming's hierarchy of a host-only scene: (spheres [n][4], links [n][2], clusters)."""
    nn, nc = C.c_int32(), C.c_int32()
    check(lib().rt_debug_aim_tree_host(scene.handle, None, None, C.byref(nn), C.byref(nc)))
    sph = np.zeros((nn.value, 4), np.float32)
    links = np.zeros((nn.value, 2), np.int32)
    check(lib().rt_debug_aim_tree_host(scene.handle, sph.ctypes.data, links.ctypes.data, None, None))
    return sph, links, nc.value


def debug_aim_host(scene: Scene, eye, kind: int, q):
    """Photon aiming's queries run on the host (see rt_debug_aim_host)."""
    q = np.ascontiguousarray(q, np.float32).reshape(-1, 9)
    out = np.zeros((q.shape[0], 4), np.float32)
    e = np.ascontiguousarray(eye, np.float32)
    check(lib().rt_debug_aim_host(scene.handle, e.ctypes.data, kind, q.ctypes.data, q.shape[0], out.ctypes.data))
    return out


def debug_env_sample_host(scene: Scene, ng, u, v):
    """(wi, cell, pdf) of the environment's NEE sampling for geometric
    normals ng and sample pairs (u, v), run on the host."""
    ng = np.ascontiguousarray(ng, np.float32).reshape(-1, 3)
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    n = ng.shape[0]
    if u.size != n or v.size != n:
        raise ValueError("debug_env_sample_host: ng, u and v must have the same length")
    wi = np.zeros((n, 3), np.float32)
    cell = np.zeros(n, np.uint32)
    pdf = np.zeros(n, np.float32)
    check(lib().rt_debug_env_sample_host(scene.handle, ng.ctypes.data, u.ctypes.data, v.ctypes.data, n,
                                         wi.ctypes.data, cell.ctypes.data, pdf.ctypes.data))
    return wi, cell, pdf


def debug_light_bvh_host(scene: Scene, x, nrm, u):
    """(emitter, probability from the descent, probability by re-traversal)
    of the light hierarchy for points x, normals nrm and numbers u, run on
    the host."""
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    nrm = np.ascontiguousarray(nrm, np.float32).reshape(-1, 3)
    u = np.ascontiguousarray(u, np.float32)
    n = x.shape[0]
    if nrm.shape[0] != n or u.size != n:
        raise ValueError("debug_light_bvh_host: x, nrm and u must have the same length")
    e = np.zeros(n, np.uint32)
    ps, pr = np.zeros(n, np.float32), np.zeros(n, np.float32)
    check(lib().rt_debug_light_bvh_host(scene.handle, x.ctypes.data, nrm.ctypes.data, u.ctypes.data, n,
                                        e.ctypes.data, ps.ctypes.data, pr.ctypes.data))
    return e, ps, pr


def debug_render_host(scene: Scene, cam, max_depth, px, py, j, opts: Optional[rt_render_opts] = None):
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    px = np.ascontiguousarray(px, np.uint32)
    py = np.ascontiguousarray(py, np.uint32)
    j = np.ascontiguousarray(j, np.uint32)
    L = np.zeros((px.size, 3), np.float32)
    check(lib().rt_debug_render_host(scene.handle, C.byref(c), max_depth, C.byref(o), px.ctypes.data,
                                     py.ctypes.data, j.ctypes.data, px.size, L.ctypes.data))
    return L


def rt_render_probes(scene: Scene, pos, nrm, spp: int, max_depth: int, film: "Film",
                     opts: Optional[rt_render_opts] = None, stream=None, allow_timeout: bool = False) -> int:
    """Irradiance probes (rt_render_probes): pos, nrm torch CUDA float32 [n][3];
    film = Film(n, 1). Returns the status (RT_TIMEOUT only with allow_timeout)."""
    pos = pos.contiguous()
    nrm = nrm.contiguous()
    n = pos.shape[0]
    o = opts if opts is not None else make_opts()
    st = lib().rt_render_probes(scene.handle, pos.data_ptr(), nrm.data_ptr(), n, spp, max_depth, film.handle,
                                C.byref(o), _stream(stream))
    if st == RT_TIMEOUT and allow_timeout:
        return st
    check(st)
    return st


def rt_render_two_way(scene: Scene, cam, spp: int, max_depth: int, film: "Film",
                      opts: Optional[rt_render_opts] = None, lt_mode: int = 0, lt_splat=None,
                      stream=None) -> rt_stats:
    """Two-way path tracing (rt_render_two_way): the camera stage into `film`,
    the light stage into `lt_splat` (torch CUDA float64 [H][W][3], added into)
    or, when None, into the film's sums. Returns the call's statistics."""
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    ptr = None
    if lt_splat is not None:
        import torch
        if lt_splat.dtype != torch.float64 or not lt_splat.is_cuda or not lt_splat.is_contiguous():
            raise ValueError("lt_splat must be a contiguous CUDA float64 tensor")
        if tuple(lt_splat.shape) != (cam.height, cam.width, 3):
            raise ValueError("lt_splat must be [H][W][3]")
        ptr = lt_splat.data_ptr()
    stats = rt_stats()
    check(lib().rt_render_two_way(scene.handle, C.byref(c), spp, max_depth, film.handle, C.byref(o), lt_mode, ptr,
                                  C.byref(stats), _stream(stream)))
    return stats


def debug_render_probes_host(scene: Scene, pos, nrm, max_depth, p, j, opts: Optional[rt_render_opts] = None):
    """Host execution of probe paths (test hook): E of sample j[i] of probe p[i]."""
    pos = np.ascontiguousarray(pos, np.float32).reshape(-1, 3)
    nrm = np.ascontiguousarray(nrm, np.float32).reshape(-1, 3)
    p = np.ascontiguousarray(p, np.uint32)
    j = np.ascontiguousarray(j, np.uint32)
    o = opts if opts is not None else make_opts()
    E = np.zeros((p.size, 3), np.float32)
    check(lib().rt_debug_render_probes_host(scene.handle, pos.ctypes.data, nrm.ctypes.data, pos.shape[0], max_depth,
                                            C.byref(o), p.ctypes.data, j.ctypes.data, p.size, E.ctypes.data))
    return E


def debug_halton_host(width, height, seed, indices, ndims):
    idx = np.ascontiguousarray(indices, np.uint64)
    out = np.zeros((idx.size, ndims), np.uint32)
    check(lib().rt_debug_halton_host(width, height, seed, idx.ctypes.data, idx.size, ndims, out.ctypes.data))
    return out


def debug_sample_index_host(width, height, x, y, j) -> int:
    v = C.c_uint64()
    check(lib().rt_debug_sample_index_host(width, height, x, y, j, C.byref(v)))
    return v.value
