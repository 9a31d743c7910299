"""CPU checks of the C-ABI library: it builds, loads and exports every
function declared in include/rt.h; host logic (strength-reduced division,
BVH8 build, traversal and per-sample path code executed on the host) agrees
with the oracle."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import build, rt, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(rt_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rt_\w+)", out))
    declared = header_functions()
    assert len(declared) >= 25
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    rt.lib()  # and it loads


def test_no_cpu_fallback_in_device_entry_points():
    """Without a GPU the device entry points report a CUDA error; they never
    compute on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sd, cam = scenes.cornell_box()
    with pytest.raises(rt.RtError):
        rt.Scene(sd)
    with pytest.raises(rt.RtError):
        rt.Film(8, 8)


def test_strength_reduced_division_matches_integer_division():
    rng = np.random.default_rng(0)
    n = np.concatenate([rng.integers(0, 2**63, 200_000, dtype=np.int64).astype(np.uint64) * np.uint64(2)
                        + rng.integers(0, 2, 200_000, dtype=np.int64).astype(np.uint64),
                        np.arange(0, 70_000, dtype=np.uint64),
                        np.array([2**64 - 1, 2**64 - 2, 2**63, 2**32, 2**32 - 1], np.uint64)])
    for d in [2, 3, 5, 7, 11, 619, 2187, 177147, 4294967291, 2**31, 3**20]:
        assert np.array_equal(rt.rt_divide_u64_host(n, d), n // np.uint64(d)), d


def test_strength_reduced_division_exhaustive_16bit_dividends_all_small_bases():
    n = np.arange(0, 1 << 16, dtype=np.uint64)
    for d in range(2, 700):
        assert np.array_equal(rt.rt_divide_u64_host(n, d), n // np.uint64(d))


def test_halton_host_code_matches_oracle_bits():
    rng = np.random.default_rng(1)
    idx = np.concatenate([np.arange(0, 4096, dtype=np.uint64),
                          rng.integers(0, 2**63, 2000, dtype=np.int64).astype(np.uint64) * np.uint64(2),
                          np.array([2**64 - 1, 2**63, 2**32 - 1, 2**32], np.uint64)])
    for (W, H, seed) in [(64, 64, 0), (1920, 1080, 17050126), (1, 1, 5)]:
        a = rt.debug_halton_host(W, H, seed, idx, 40)
        b = oracle.sample_dims_u32(idx, 40, W, H, seed)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mis_mode", [0, 2, 3])
def test_direct_light_host_matches_oracle_with_emitter_near_receivers(mis_mode):
    """Emitter facing the ceiling 0.1 below it: NEE shadow rays to it leave
    ceiling points at grazing angles, where the surface offset of the shadow
    ray origin is larger than the occlusion margin at the light unless the
    segment is measured from that origin. Per sample, depth 1."""
    sd, cam = scenes.cornell_box(light="up")
    s, o = rt.Scene(sd, host_only=True), oracle.Scene(sd)
    rng = np.random.default_rng(3)
    n = 20000
    px, py, j = rng.integers(0, cam.width, n), rng.integers(0, cam.height, n), rng.integers(0, 256, n)
    Lg = rt.debug_render_host(s, cam, 1, px, py, j, rt.make_opts(mis_mode=mis_mode))
    Lo = o.render_samples(cam, px, py, j, 1, mis_mode=mis_mode)
    d = np.abs(Lg - Lo).sum(1)
    assert (d <= 1e-3 * np.maximum(np.abs(Lo).sum(1), 1e-3)).mean() >= 0.99
    assert abs(Lg.mean() - Lo.mean()) <= 1e-3 * Lo.mean()


def test_halton_host_code_matches_oracle_bits_1024_dims():
    # large bases make the fixed-point fast path hand over to the exact
    # Horner evaluation most often (about n (b - 1) / 2^32 of the values)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.integers(0, 2**63, 3000, dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1),
                          rng.integers(0, 2**32, 3000, dtype=np.int64).astype(np.uint64)])
    a = rt.debug_halton_host(1920, 1080, 99, idx, 1024)
    b = oracle.sample_dims_u32(idx, 1024, 1920, 1080, 99)
    assert np.array_equal(a, b)


def test_sample_index_host_code_matches_oracle():
    for W, H in [(64, 64), (1920, 1080), (7, 5), (1, 1), (333, 100)]:
        k = max(0, (W - 1).bit_length())
        l = 0
        while 3**l < H:
            l += 1
        P = 2**k * 3**l
        rng = np.random.default_rng(W * H)
        for _ in range(50):
            x, y, j = int(rng.integers(0, W)), int(rng.integers(0, H)), int(rng.integers(0, 5000))
            assert rt.debug_sample_index_host(W, H, x, y, j) == oracle.pixel_base_index(W, H, x, y) + j * P


@pytest.fixture(scope="module")
def small_field():
    sd, cam = scenes.sphere_field(n_spheres=6, seg=24, rings=12, plane_res=(40, 20), n_emissive_spheres=2,
                                  env_size=(64, 32), width=96, height=54)
    return sd, cam, rt.Scene(sd, host_only=True), oracle.Scene(sd)


@pytest.mark.parametrize("kind", ["primary", "incoherent", "shadow"])
def test_bvh8_traversal_host_matches_oracle(small_field, kind):
    from helpers import t_close
    sd, cam, s, o = small_field
    rays = scenes.random_rays(sd, 20000, seed=3, kind=kind, cam=cam)
    p, t, u, v, nodes = rt.debug_trace_host(s, rays, any_hit=(kind == "shadow"))
    po, to, _, _ = o.trace(rays, any_hit=(kind == "shadow"))
    if kind == "shadow":
        assert np.array_equal(p != rt.RT_MISS, po != rt.RT_MISS)
        return
    assert np.mean(p == po) >= 0.99999
    hit = (po != rt.RT_MISS) & (p == po)
    assert np.all(t_close(t[hit], to[hit], rays[hit]))


def test_bvh8_build_shapes(small_field):
    sd, cam, s, o = small_field
    info = s.info()
    assert info["leaf_tris"] == sd.num_triangles
    assert 0 < info["nodes"] < sd.num_triangles


def test_empty_and_single_triangle_scenes_host():
    from test_oracle_geometry import tri_scene
    s = rt.Scene(tri_scene([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]]), host_only=True)
    rays = np.array([[0.2, 0.2, 1, 0, 0, -1, 0, np.inf], [2, 2, 1, 0, 0, -1, 0, np.inf],
                     [0.2, 0.2, 1, 0, 0, -1, 0, 0.5]], np.float32)
    p, t, u, v, _ = rt.debug_trace_host(s, rays)
    assert p.tolist() == [0, rt.RT_MISS, rt.RT_MISS]
    assert t[0] == pytest.approx(1.0) and u[0] == pytest.approx(0.2) and v[0] == pytest.approx(0.2)
    e = rt.Scene(tri_scene(np.zeros((3, 3)), np.zeros((0, 3))), host_only=True)
    p, t, _, _, _ = rt.debug_trace_host(e, rays)
    assert np.all(p == rt.RT_MISS) and np.all(np.isinf(t))


@pytest.mark.parametrize("which", ["cornell", "cornell_up", "field", "furnace", "many_lights", "instanced_lights"])
def test_path_code_host_matches_oracle_per_sample(small_field, which):
    if which == "many_lights":
        sd, cam = scenes.many_emitters(n_lights=200, res=32)
        s, o, D = rt.Scene(sd, host_only=True), oracle.Scene(sd), 4
    elif which == "instanced_lights":
        # two-level scene, emitters per (instance, triangle), light hierarchy
        sd, cam = scenes.instanced_field(n_meshes=6, n_instances=40, total_tris=40_000, n_emissive=400,
                                         width=48, height=32, min_tris=200, max_tris=2000)
        sd.light_bvh = True
        s, o, D = rt.Scene(sd, host_only=True), oracle.Scene(sd), 4
    elif which.startswith("cornell"):
        sd, cam = scenes.cornell_box(light="up" if which == "cornell_up" else "down")
        s, o, D = rt.Scene(sd, host_only=True), oracle.Scene(sd), 8
    elif which == "field":
        sd, cam, s, o = small_field
        D = 6
    else:
        sd, cam = scenes.furnace_sphere(res=16)
        s, o, D = rt.Scene(sd, host_only=True), oracle.Scene(sd), 4
    rng = np.random.default_rng(0)
    n = 3000
    px, py, j = rng.integers(0, cam.width, n), rng.integers(0, cam.height, n), rng.integers(0, 64, n)
    Lg = rt.debug_render_host(s, cam, D, px, py, j)
    Lo = o.render_samples(cam, px, py, j, D)
    d = np.abs(Lg - Lo).sum(1)
    # the light-facing-ceiling box is lit only through chains of bounces, where
    # FP32 rounding of each vertex compounds to a few 1e-3 relative
    rel = 1e-2 if which == "cornell_up" else 1e-3
    close = d <= rel * np.maximum(np.abs(Lo).sum(1), 1e-3)
    assert close.mean() >= 0.99
    if which == "instanced_lights":
        # the oracle sees a flattened copy whose world vertices numpy rounds
        # from an FP32 product while the library traverses in object space,
        # so a few grazing paths part ways; the image mean is carried by the
        # 1% of paths that reach a surface and is not compared sample-exact
        return
    assert np.abs(Lg.mean(0) - Lo.mean(0)).max() <= 1e-2 * np.abs(Lo.mean(0)).max()


@pytest.mark.parametrize("scene_kind", ["cornell", "cornell_up", "furnace"])
def test_probe_code_host_matches_oracle_per_sample(scene_kind):
    """Irradiance probes (Sec. 4.2): the library's probe paths, run on the
    host, against the oracle sample by sample (same sequence indices)."""
    if scene_kind == "furnace":
        sd, _ = scenes.furnace_sphere(res=16)
        pos = np.array([[0.0, 3.0, 0.0], [2.5, 0.3, -0.4], [-1.2, -1.5, 2.0]])
        nrm = np.array([[0.0, -1.0, 0.0], [-1.0, 0.0, 0.0], [0.6, 0.0, -0.8]])
        D = 3
    else:
        sd, _ = scenes.cornell_box(light="up" if scene_kind == "cornell_up" else "down")
        pos = np.array([[0.5, 1e-3, 0.5], [0.2, 0.5, 0.999], [0.99, 0.3, 0.3], [0.5, 0.5, 0.5]])
        nrm = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, -1.0], [-1.0, 0.0, 0.0], [0.0, 0.7, 0.7]])
        D = 8
    nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    s, o = rt.Scene(sd, host_only=True), oracle.Scene(sd)
    rng = np.random.default_rng(4)
    m = 3000
    p = rng.integers(0, len(pos), m)
    j = rng.integers(0, 256, m)
    Eg = rt.debug_render_probes_host(s, pos, nrm, D, p, j)
    # the oracle at the same (probe, sample) pairs: all probes of one
    # iteration per call, the same FP32-rounded probe positions and normals
    pos64, nrm64 = pos.astype(np.float32).astype(np.float64), nrm.astype(np.float32).astype(np.float64)
    Eo2 = np.zeros((m, 3))
    for jj in np.unique(j):
        S, _, _, _ = o.render_probes(pos64, nrm64, 1, D, iter0=int(jj))
        sel = np.where(j == jj)[0]
        Eo2[sel] = S[p[sel]]
    d = np.abs(Eg - Eo2).sum(1)
    rel = 1e-2 if scene_kind == "cornell_up" else 1e-3
    close = d <= rel * np.maximum(np.abs(Eo2).sum(1), 1e-3)
    assert close.mean() >= 0.99, close.mean()
    assert np.abs(Eg.mean(0) - Eo2.mean(0)).max() <= 1e-2 * np.abs(Eo2.mean(0)).max()


@pytest.mark.parametrize("plain", [False, True])
def test_env_normal_sampling_host_matches_oracle(plain):
    """Environment NEE per normal cell (Sec. 2.1.2), the library's code run on
    the host against the oracle: the cell of each normal, the direction drawn
    for (u, v) and its solid-angle pdf; with env_plain the plain pyramid."""
    sd, _ = scenes.sphere_field(n_spheres=2, seg=8, rings=4, plane_res=(4, 2), n_emissive_spheres=0,
                                env_size=(256, 128), width=16, height=16)
    sd.env_plain = plain
    s, o = rt.Scene(sd, host_only=True), oracle.Scene(sd)
    rng = np.random.default_rng(11)
    n = 4000
    ng = rng.normal(size=(n, 3))
    ng /= np.linalg.norm(ng, axis=1, keepdims=True)
    ng = ng.astype(np.float32)
    uv = rng.random((n, 2)).astype(np.float32)
    wi, cell, pdf = rt.debug_env_sample_host(s, ng, uv[:, 0], uv[:, 1])
    ng64 = ng.astype(np.float64)
    cell_o = np.array([oracle.env_normal_cell(x) for x in ng64])
    assert (cell == cell_o).mean() >= 0.999
    wo = np.zeros((n, 3))
    po = np.zeros(n)
    for i in range(n):
        wo[i], po[i] = o.env_sample_n(ng64[i], float(uv[i, 0]), float(uv[i, 1]))
    same_dir = np.abs(wi - wo).max(1) < 1e-3
    assert same_dir.mean() >= 0.99
    ok = same_dir & (cell == cell_o)
    assert np.allclose(pdf[ok], po[ok], rtol=1e-3, atol=0)
    # the pdf the library reports for its own directions is the oracle's pdf
    # of those directions (what the MIS weights at environment hits use)
    po_g = np.array([o.env_pdf_n(ng64[i], wi[i].astype(np.float64)) for i in range(n)])
    assert (np.abs(pdf - po_g) <= 1e-3 * po_g + 1e-12).mean() >= 0.995
    if not plain:
        # normal-oriented levels: most directions above their horizon (the
        # conservative cone bounds keep a band below it; about half with the
        # plain pyramid of this sun-and-sky map)
        assert (np.einsum("ij,ij->i", wi, ng) > 0).mean() > 0.75


@pytest.mark.parametrize("n_lights", [300, 3])
def test_light_bvh_host_matches_oracle(n_lights):
    """The light hierarchy (Sec. 2.1.1) run on the host against the oracle:
    the emitter drawn for (x, n, u), its probability, and the re-traversal's
    probability of it (3 emitters: a tree that is a single leaf)."""
    sd, _ = scenes.many_emitters(n_lights=n_lights, res=8)
    s, o = rt.Scene(sd, host_only=True), oracle.Scene(sd)
    rng = np.random.default_rng(12)
    n = 3000
    x = np.stack([rng.uniform(-10, 10, n), rng.uniform(0, 2.5, n), rng.uniform(-10, 10, n)], 1).astype(np.float32)
    nrm = rng.normal(size=(n, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    u = rng.random(n).astype(np.float32)
    e, ps, pr = rt.debug_light_bvh_host(s, x, nrm, u)
    eo = np.zeros(n, np.int64)
    po = np.zeros(n)
    for i in range(n):
        eo[i], po[i] = o.lb_sample(x[i].astype(np.float64), nrm[i].astype(np.float64), float(u[i]))
    same = e == eo
    assert same.mean() >= 0.995
    assert np.allclose(ps[same], po[same], rtol=1e-4, atol=0)
    assert np.allclose(pr, ps, rtol=1e-5, atol=0)
    pg = np.array([o.lb_prob(x[i].astype(np.float64), nrm[i].astype(np.float64), int(e[i])) for i in range(n)])
    assert np.allclose(pr, pg, rtol=1e-4, atol=0)


@pytest.mark.parametrize("kind", ["primary", "incoherent", "shadow"])
def test_two_level_traversal_host_matches_flattened_oracle(kind):
    """Instanced scenes: the library's two-level traversal, run on the host,
    against the oracle on the flattened copy ((instance, triangle) mapped to
    the flattened index); the FP32 object-space and world-space geometries
    differ by the rounding of the transforms, so a disagreement must be a
    valid alternative hit."""
    from test_gpu_trace import check_closest
    sd, cam = scenes.instanced_field(n_meshes=6, n_instances=60, total_tris=60_000, n_emissive=300, width=64,
                                     height=36, min_tris=300, max_tris=3000)
    flat = sd.flattened()
    s, o = rt.Scene(sd, host_only=True), oracle.Scene(flat)
    rays = scenes.random_rays(flat, 20000, seed=9, kind=kind, cam=cam)
    p, t, u, v, _, inst = rt.debug_trace_host(s, rays, any_hit=(kind == "shadow"), return_inst=True)
    po, to, uo, vo = o.trace(rays, any_hit=(kind == "shadow"))
    if kind == "shadow":
        assert (np.asarray(p != rt.RT_MISS) == np.asarray(po != rt.RT_MISS)).mean() >= 0.9999
        return
    hit = p != rt.RT_MISS
    counts = np.diff(sd.mesh_tri_offset)[sd.instance_mesh]
    base = np.concatenate([[0], np.cumsum(counts)[:-1]])
    ii = np.where(hit, inst, 0).astype(np.int64)
    fp = np.where(hit, base[ii] + (p.astype(np.int64) - sd.mesh_tri_offset[sd.instance_mesh[ii]]), rt.RT_MISS)
    check_closest(flat, rays, (fp.astype(np.uint32), t, u, v), (po, to, uo, vo), min_agree=0.9999, t_rel=1e-4)


def test_two_way_checks_its_arguments_on_the_host():
    """rt_render_two_way (Sec. 2, two-way path tracing) refuses null scene,
    camera or film before touching a device."""
    L = rt.lib()
    st = L.rt_render_two_way(None, None, 1, 3, None, None, 0, None, None, None)
    assert rt.STATUS[st] == "RT_INVALID_ARG"
    assert b"null argument" in L.rt_last_error()


def test_stack_overflow_is_reported_as_a_status_on_the_host():
    """The traversal's overflow path: a ray that needs more stack entries than
    the stack holds ends and the call returns RT_STACK_OVERFLOW (never a trap
    or a silently wrong hit). Scene: clusters of 16 parallel triangles at
    exponentially spaced depths (a comb-shaped BVH); the rays run inside every
    box and miss every triangle, so every internal node is visited and
    pending siblings pile up on the stack."""
    from test_oracle_geometry import tri_scene
    V, I = [], []
    for k in range(100):
        for j in range(16):
            z = 1.5 ** k * (1 + 1e-3 * j / 16)
            b = len(V)
            V += [[-1, -1, z], [1, -1, z], [0, 1, z]]
            I.append([b, b + 1, b + 2])
    s = rt.Scene(tri_scene(np.array(V, np.float32), np.array(I)), host_only=True)
    miss = np.array([[0.9, 0.9, 0.5, 0, 0, 1, 0, np.inf], [-0.9, 0.9, 0.5, 0, 0, 1, 0, np.inf]], np.float32)
    hit = np.array([[0.0, 0.0, 0.5, 0, 0, 1, 0, np.inf]], np.float32)
    rays = np.concatenate([miss, hit])
    p_full, t_full, _, _, _ = rt.debug_trace_host(s, rays)
    assert p_full[0] == rt.RT_MISS and p_full[1] == rt.RT_MISS and p_full[2] != rt.RT_MISS
    # the full stack (48 entries) gives the kernels' answer
    p48, t48 = rt.debug_trace_host_stack(s, rays, 48)
    assert np.array_equal(p48, p_full) and np.array_equal(t48, t_full)
    # the smallest stack that suffices, and one entry less overflows
    need = next(k for k in range(1, 49) if _no_overflow(s, miss, k))
    assert need >= 2
    with pytest.raises(rt.RtError) as e:
        rt.debug_trace_host_stack(s, miss, need - 1)
    assert e.value.status == 6 and "overflow" in str(e.value)
    for k in range(need, 49):
        p, t = rt.debug_trace_host_stack(s, miss, k)
        assert np.all(p == rt.RT_MISS) and np.all(np.isinf(t))
    with pytest.raises(rt.RtError):
        rt.debug_trace_host_stack(s, miss, 0)


def _no_overflow(s, rays, k):
    try:
        rt.debug_trace_host_stack(s, rays, k)
        return True
    except rt.RtError as e:
        assert e.status == 6
        return False


@pytest.mark.parametrize("n,cap,frac", [(10_000, 1000, 0.5), (10_000, 1000, 1e-9), (10_000, 1000, 1.0),
                                        (5000, 8192, 0.5), (777, 64, 0.5), (1, 32, 0.5), (65_536, 4096, 0.25)])
def test_regeneration_bookkeeping_on_the_host(n, cap, frac):
    """The slot decisions of the regeneration scheduler (the same functions
    the kernels call), driven by random path lengths: every task starts and
    is retired exactly once, after exactly its length in steps; the pool
    never holds more than its capacity; refills happen only once at least
    the fraction has ended."""
    rng = np.random.default_rng(n + cap)
    life = rng.integers(1, 18, n).astype(np.uint8)
    regen_min = max(1, int(math.ceil(frac * cap)))
    at, steps, regen = rt.debug_regen_host(life, cap, regen_min)
    assert np.all(at != 0xFFFFFFFF)
    # tasks start in order; a task started at step s0 retires at s0 + life
    # (tasks of the first load start at step 0)
    start = at.astype(np.int64) - life
    assert np.all(start[:min(n, cap)] == 0)
    assert np.all(np.diff(start) >= 0)
    assert steps == at.max()
    if n > cap:
        assert regen > 0
        # never more live paths than slots
        for s in np.unique(start):
            live = np.sum((start <= s) & (at > s))
            assert live <= cap
    else:
        assert regen == 0


def test_regeneration_stop_drains_a_contiguous_range_on_the_host():
    """After a stop no task starts; the retired tasks are exactly a prefix."""
    rng = np.random.default_rng(3)
    life = rng.integers(1, 18, 50_000).astype(np.uint8)
    at, steps, _ = rt.debug_regen_host(life, 2048, 1024, stop_step=20)
    done = at != 0xFFFFFFFF
    k = int(done.sum())
    assert 2048 < k < 50_000 and np.all(done[:k]) and not done[k:].any()
    assert steps <= 20 + 17


@pytest.mark.parametrize("name", ["cornell", "field", "many", "turntable"])
def test_photon_aiming_host_matches_oracle(name):
    """Photon aiming (Sec. 2.1.3) as the kernels compute it, run on the host
    in FP32, against the FP64 oracle: the same clusters and hierarchy, the
    same line and cone densities, the same cluster picked by the descent
    (away from the FP32/FP64 boundaries of the cumulative probabilities)."""
    sd, cam = {"cornell": scenes.cornell_box, "field": scenes.sphere_field,
               "many": lambda: scenes.many_emitters(n_lights=64, res=16),
               "turntable": lambda: scenes.turntable(res=16)}[name]()
    s, o = rt.Scene(sd, host_only=True), oracle.Scene(sd)
    sph, links, ncl = rt.debug_aim_tree_host(s)
    cc, _ = o.pa_clusters()
    assert ncl == cc.shape[0] and sph.shape[0] == 2 * ncl - 1
    leaf = links[:, 0] < 0
    assert np.allclose(sph[leaf], cc[links[leaf, 1]], rtol=1e-6, atol=1e-6)
    eye = o.pa_eye(cam)
    rng = np.random.default_rng(9)
    lo, hi = sd.vertices.min(0), sd.vertices.max(0)
    n = 400
    x = lo + rng.random((n, 3)) * (hi - lo)
    w = rng.normal(size=(n, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    ny = rng.normal(size=(n, 3))
    ny /= np.linalg.norm(ny, axis=1, keepdims=True)
    x, w, ny = (a.astype(np.float32).astype(np.float64) for a in (x, w, ny))
    env_g = rt.debug_aim_host(s, eye, 0, np.concatenate([x, w, np.zeros((n, 3))], 1))[:, 0]
    dir_g = rt.debug_aim_host(s, eye, 1, np.concatenate([x, ny, w], 1))[:, 0]
    env_o = np.array([o.pa_env_density(eye, x[i], w[i]) for i in range(n)])
    dir_o = np.array([o.pa_dir_density(eye, x[i], ny[i], w[i]) for i in range(n)])
    # a query on the boundary of a cluster's disk or cone may fall on either
    # side in FP32: at most 2% of them
    for g_, o_ in ((env_g, env_o), (dir_g, dir_o)):
        ok = np.isclose(g_, o_, rtol=2e-4, atol=1e-30)
        assert ok.mean() >= 0.98, (ok.mean(), g_[~ok][:5], o_[~ok][:5])
        assert np.any(o_ > 0)
    # the descent: environment photons and triangle photons
    u = (np.arange(n) + 0.5) / n
    for tri in (0.0, 1.0):
        q = np.concatenate([x, ny, u[:, None], np.full((n, 1), tri), np.zeros((n, 1))], 1)
        got = rt.debug_aim_host(s, eye, 2, q)
        same = 0
        for i in range(n):
            c, _ = o.pa_sample(eye, u[i], x[i] if tri else None, ny[i] if tri else None)
            same += np.allclose(got[i], cc[c], rtol=1e-6, atol=1e-6)
        assert same >= 0.98 * n
    # cone samples
    q = np.concatenate([np.tile(cc[:1], (n, 1)), x, rng.random((n, 2))], 1)
    gw = rt.debug_aim_host(s, eye, 3, q)[:, :3]
    ow = np.array([o.pa_cone_sample(0, x[i], q[i, 7], q[i, 8]) for i in range(n)])
    assert np.abs(gw - ow).max() < 2e-4


def test_guided_plan_buffers_hold_every_set():
    """The guided render's set and buffer arithmetic (host hook of the code
    the render runs): for batches, warm-up sizes, guide depths, pools and set
    sizes, the recording paths and kept samples of every set fit the buffers,
    the records cover min(n, recording paths) paths, and the training steps
    read only kept samples."""
    from paper_1705_01263_gb300 import rt
    rng = np.random.default_rng(21)
    for _ in range(3000):
        batch = int(rng.choice([256, 1000, 1 << 14, 1 << 16, 1 << 20]))
        wsb = int(rng.integers(0, 70))
        gdepth = int(rng.integers(1, 70))
        max_depth = int(rng.integers(0, 17))
        cap = int(rng.choice([32, 4096, 65536, 1 << 20, 1 << 24, 1 << 27]))
        fixed = bool(rng.integers(0, 2))
        young = bool(rng.integers(0, 2))
        g = rt.debug_guided_plan_host(batch, wsb, gdepth, max_depth, cap, fixed, 1, young)
        cset = g["cap_young"] if young else g["cap"]
        assert 1 <= g["cap_young"] <= g["cap"] <= cap
        assert g["rec_depth"] <= min(gdepth, max_depth, 8)
        for n in {1, cset, max(1, cset // 3), int(rng.integers(1, cset + 1))}:
            e = rt.debug_guided_plan_host(batch, wsb, gdepth, max_depth, cap, fixed, n, young)
            assert e["rec_paths"] <= e["rec_alloc"], e
            assert e["keep"] <= e["keep_alloc"], e
            assert e["rec_stride"] >= 1
            recorded = min(e["rec_paths"], -(-n // e["rec_stride"]))
            assert recorded == min(n, e["rec_paths"]), (n, e)
            assert e["keep"] >= batch
            if not young:
                assert 1 <= e["set_steps"] <= 4 and e["set_steps"] * batch <= e["keep"]
