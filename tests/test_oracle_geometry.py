"""Pins for the oracle's ray casting (Sec. 2.3 watertight traversal and
intersection; Sec. 3.1 rays -> hits): closed-form hits, watertightness on
closed meshes, the tie rule, and BVH == brute force."""
import math

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes


def tri_scene(verts, idx):
    n = len(idx)
    return scenes.SceneData(
        vertices=np.asarray(verts, np.float32), indices=np.asarray(idx, np.uint32),
        tri_material=np.zeros(n, np.uint32), albedo=np.full((1, 3), 0.5, np.float32),
        roughness=np.full(1, 0.5, np.float32), ggx_weight=np.zeros(1, np.float32),
        emission=np.zeros((1, 3), np.float32), emission_tex=np.full(1, -1, np.int32))


def ray(o, d, tmin=0.0, tmax=np.inf):
    d = np.asarray(d, float)
    d = d / np.linalg.norm(d)
    return np.array([[*o, *d, tmin, tmax]], np.float32)


def test_closed_form_hit_and_barycentrics():
    s = oracle.Scene(tri_scene([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]]))
    prim, t, b1, b2 = s.trace(ray((0.25, 0.5, 2.0), (0, 0, -1)), use_bvh=False)
    assert prim[0] == 0 and t[0] == pytest.approx(2.0, abs=1e-15)
    assert b1[0] == pytest.approx(0.25, abs=1e-15) and b2[0] == pytest.approx(0.5, abs=1e-15)
    # interval (tmin, tmax) is open at both ends, no back-face culling
    assert s.trace(ray((0.25, 0.5, 2.0), (0, 0, -1), tmax=2.0), use_bvh=False)[0][0] == oracle_miss()
    assert s.trace(ray((0.25, 0.5, -2.0), (0, 0, 1)), use_bvh=False)[0][0] == 0
    assert s.trace(ray((1.25, 0.5, 2.0), (0, 0, -1)), use_bvh=False)[0][0] == oracle_miss()
    assert s.trace(ray((0.25, 0.5, 0.0), (1, 0, 0)), use_bvh=False)[0][0] == oracle_miss()


def oracle_miss():
    return 0xFFFFFFFF


def test_degenerate_triangle_never_hit():
    s = oracle.Scene(tri_scene([[0, 0, 0], [1, 1, 1], [2, 2, 2]], [[0, 1, 2]]))
    assert s.trace(ray((1, 1, 5), (0, 0, -1)), use_bvh=False)[0][0] == oracle_miss()


def test_equal_t_goes_to_lower_prim():
    v = [[0, 0, 0], [1, 0, 0], [0, 1, 0]]
    s = oracle.Scene(tri_scene(v + v, [[3, 4, 5], [0, 1, 2], [3, 5, 4]]))
    for use_bvh in (False, True):
        prim, t, _, _ = s.trace(ray((0.2, 0.2, 1.0), (0, 0, -1)), use_bvh=use_bvh)
        assert prim[0] == 0 and t[0] == pytest.approx(1.0)


@pytest.mark.parametrize("seg,rings", [(12, 7), (64, 35)])
def test_watertight_closed_mesh_vertices_and_edges(seg, rings):
    """Rays through the vertices and edge midpoints of a closed mesh, from
    inside and radially from outside, must never slip through a crack."""
    v, idx = scenes.uv_sphere(seg, rings)
    v = v.astype(np.float32).astype(np.float64)
    sd = tri_scene(v, idx)
    s = oracle.Scene(sd)
    targets = [v]
    for a, b in ((0, 1), (1, 2), (2, 0)):
        targets.append(0.5 * (v[idx[:, a]] + v[idx[:, b]]))
    targets = np.concatenate(targets)
    rng = np.random.default_rng(3)
    centre = rng.uniform(-0.05, 0.05, 3)
    d = targets - centre
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    n = targets.shape[0]
    inside = np.zeros((n, 8), np.float32)
    inside[:, 0:3], inside[:, 3:6], inside[:, 7] = centre, d, np.inf
    outside = inside.copy()
    outside[:, 0:3] = centre + 3.0 * d
    outside[:, 3:6] = -d
    for rays in (inside, outside):
        prim, t, _, _ = s.trace(rays, use_bvh=False)
        assert np.all(prim != oracle_miss())
        assert np.all(np.isfinite(t))


@pytest.mark.parametrize("kind", ["incoherent", "shadow", "edges", "primary"])
def test_bvh_equals_brute_force(kind):
    sd, cam = scenes.sphere_field(n_spheres=6, seg=24, rings=12, plane_res=(40, 20), n_emissive_spheres=2,
                                  env_size=(16, 8))
    s = oracle.Scene(sd)
    assert s.bvh_node_count() > 100
    rays = scenes.random_rays(sd, 3000, seed=11, kind=kind, cam=cam)
    a = s.trace(rays, use_bvh=False)
    b = s.trace(rays, use_bvh=True)
    assert np.array_equal(a[0], b[0])
    hit = a[0] != oracle_miss()
    assert hit.mean() > 0.05
    assert np.array_equal(a[1][hit], b[1][hit])
    if kind == "shadow":
        ah = s.trace(rays, any_hit=True, use_bvh=True)[0] != oracle_miss()
        assert np.array_equal(ah, hit)
