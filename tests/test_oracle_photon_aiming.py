"""Pins of the oracle's photon aiming (Sec. 2.1.3: photons are aimed at
clusters of objects picked through a hierarchy in proportion to an estimate
of their screen-space photon density):

- the clusters do not depend on the order of the objects (the paper's
  property of its merge criterion);
- the cluster hierarchy's descent is measure preserving: sampled cluster
  frequencies equal the product of the branch probabilities, which sum to one;
- the environment photon's line density integrates to one over the plane
  across its direction, and the triangle photon's direction density to one
  over the sphere: a wrong disk or cone area, a missed or doubled cluster
  in the sums, breaks either;
- cone samples are uniform in solid angle inside the cone;
- closed forms for a scene of one object;
- the aimed light tracer gives the path tracer's expectation, and in a
  sky-lit scene whose bound is much larger than the objects in view the
  light tracer alone has a lower error per sample than with uniform
  emission.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes


def _objects(sd):
    """Object of every triangle: connected components over shared vertex
    indices, numbered by first triangle (plain union-find)."""
    parent = list(range(sd.vertices.shape[0]))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for t in sd.indices:
        for k in (1, 2):
            a, b = find(int(t[0])), find(int(t[k]))
            if a != b:
                parent[max(a, b)] = min(a, b)
    num, out = {}, np.zeros(sd.indices.shape[0], np.int64)
    for i, t in enumerate(sd.indices):
        r = find(int(t[0]))
        if r not in num:
            num[r] = len(num)
        out[i] = num[r]
    return out


def _canon(cc):
    return np.array(sorted(map(tuple, np.round(cc, 9))))


@pytest.mark.parametrize("name", ["cornell", "field", "many"])
def test_clusters_do_not_depend_on_object_order(name):
    sd, cam = {"cornell": scenes.cornell_box, "field": scenes.sphere_field,
               "many": lambda: scenes.many_emitters(n_lights=64, res=16)}[name]()
    cc, oc = oracle.Scene(sd).pa_clusters()
    obj = _objects(sd)
    assert obj.max() + 1 == oc.size
    rng = np.random.default_rng(4)
    order = rng.permutation(oc.size)
    tri = np.concatenate([np.where(obj == o)[0] for o in order])
    sd2 = dataclasses.replace(sd, indices=sd.indices[tri], tri_material=sd.tri_material[tri])
    cc2, oc2 = oracle.Scene(sd2).pa_clusters()
    assert np.array_equal(_canon(cc), _canon(cc2))
    # an object's cluster sphere is the same in both orders
    for o in range(oc.size):
        assert np.allclose(cc[oc[o]], cc2[oc2[np.where(order == o)[0][0]]], rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,tri", [("cornell", False), ("cornell", True), ("many", False), ("many", True)])
def test_descent_is_measure_preserving(name, tri):
    sd, cam = scenes.cornell_box() if name == "cornell" else scenes.many_emitters(n_lights=64, res=16)
    s = oracle.Scene(sd)
    y, ny = (np.array([0.5, 0.999, 0.5]), np.array([0.0, -1.0, 0.0])) if tri else (None, None)
    eye = s.pa_eye(cam)
    P = s.pa_probs(eye, y, ny)
    assert P.sum() == pytest.approx(1.0, abs=1e-12) and np.all(P >= 0)
    n = 20000
    hist = np.zeros(P.size)
    for k in range(n):
        c, p = s.pa_sample(eye, (k + 0.5) / n, y, ny)
        hist[c] += 1
        assert p == pytest.approx(P[c], rel=1e-12)
    assert np.abs(hist / n - P).max() <= 2.0 / n * 2


def _plane_grid(center, w, half, m):
    t1 = np.cross(w, [0.0, 1.0, 0.0] if abs(w[1]) < 0.9 else [1.0, 0.0, 0.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(w, t1)
    g = (np.arange(m) + 0.5) / m * 2 * half - half
    return [center + a * t1 + b * t2 for a in g for b in g], (2 * half / m) ** 2


@pytest.mark.parametrize("w", [(0.3, 0.8, -0.52), (-0.7, 0.2, 0.68)])
def test_environment_line_density_integrates_to_one(w):
    sd, cam = scenes.cornell_box()
    s = oracle.Scene(sd)
    w = np.array(w) / np.linalg.norm(w)
    pts, dA = _plane_grid(np.array([0.5, 0.5, 0.5]), w, 1.6, 320)
    eye = s.pa_eye(cam)
    total = sum(s.pa_env_density(eye, x, w) for x in pts) * dA
    assert total == pytest.approx(1.0, abs=0.02)


@pytest.mark.parametrize("y,ny", [((0.5, 0.999, 0.5), (0.0, -1.0, 0.0)),      # inside the walls' sphere
                                  ((0.5, 3.0, 0.5), (0.0, -1.0, 0.0)),        # outside every sphere
                                  ((2.5, 0.5, 0.5), (-0.6, 0.8, 0.0))])
def test_triangle_direction_density_integrates_to_one(y, ny):
    sd, cam = scenes.cornell_box()
    s = oracle.Scene(sd)
    y, ny = np.array(y), np.array(ny) / np.linalg.norm(ny)
    nt, npp = 300, 600
    eye = s.pa_eye(cam)
    tot = 0.0
    for i in range(nt):
        ct = 1 - 2 * (i + 0.5) / nt
        st = math.sqrt(1 - ct * ct)
        for j in range(npp):
            ph = 2 * math.pi * (j + 0.5) / npp
            tot += s.pa_dir_density(eye, y, ny, np.array([st * math.cos(ph), ct, st * math.sin(ph)]))
    tot *= (2.0 / nt) * (2 * math.pi / npp)
    assert tot == pytest.approx(1.0, abs=0.02)


def test_cone_samples_are_uniform_in_the_cone():
    sd, cam = scenes.cornell_box()
    s = oracle.Scene(sd)
    cc, _ = s.pa_clusters()
    y = np.array([0.5, 3.0, 0.5])
    for c in range(cc.shape[0]):
        v = cc[c, :3] - y
        d = np.linalg.norm(v)
        cmax = math.sqrt(1 - (cc[c, 3] / d) ** 2)
        m = 64
        cos = np.array([np.dot(s.pa_cone_sample(c, y, (i + 0.5) / m, (j + 0.5) / m), v / d)
                        for i in range(m) for j in range(m)])
        assert cos.min() >= cmax - 1e-12
        # uniform in solid angle: cos theta uniform on [cmax, 1]
        assert cos.mean() == pytest.approx((1 + cmax) / 2, abs=1e-4 * (1 - cmax) + 1e-12)
        assert np.var(cos) == pytest.approx((1 - cmax) ** 2 / 12, rel=2e-3)


def test_one_object_closed_forms():
    """One triangle: a single cluster of probability 1; its line density is
    1 / (pi r^2) inside the disk and zero outside, its cone density 1 / (2 pi
    (1 - cos theta)) inside the cone."""
    from test_oracle_geometry import tri_scene
    sd = tri_scene([[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[0, 1, 2]])
    s = oracle.Scene(sd)
    cc, oc = s.pa_clusters()
    assert cc.shape == (1, 4) and oc.tolist() == [0]
    c, r = cc[0, :3], cc[0, 3]
    assert np.allclose(c, [0.5, 0.5, 0.0]) and r == pytest.approx(math.sqrt(2) / 2)
    eye = np.array([0.3, 0.2, 5.0, 0.5])   # position, view-cone solid angle
    assert s.pa_probs(eye).tolist() == [1.0]
    w = np.array([0.0, 0.0, 1.0])
    assert s.pa_env_density(eye, c + np.array([0.3, 0.2, -4.0]), w) == pytest.approx(1 / (math.pi * r * r))
    assert s.pa_env_density(eye, c + np.array([0.8, 0.0, 2.0]), w) == 0.0
    y = np.array([0.5, 0.5, 3.0])
    ct = math.sqrt(1 - (r / 3.0) ** 2)
    assert s.pa_dir_density(eye, y, np.array([0, 0, -1.0]), np.array([0, 0, -1.0])) == \
        pytest.approx(1 / (2 * math.pi * (1 - ct)))
    assert s.pa_dir_density(eye, y, np.array([0, 0, -1.0]), np.array([0, 0, 1.0])) == 0.0
    # an emitter facing away from the only cluster: the estimate is zero,
    # the descent falls back to one half at each step (a single leaf here)
    assert s.pa_probs(eye, y, np.array([0, 0, 1.0])).tolist() == [1.0]


def _chunks(s, cam, spp, D, K, **kw):
    return [s.render_two_way(cam, spp, D, iter0=c * spp, **kw) for c in range(K)]


def test_aimed_light_tracer_has_the_path_tracers_expectation():
    """The room lit through its ceiling with the light tracer alone wherever
    it makes the path (lt_mode 1): aimed emission against the path tracer,
    per 4 x 4 block."""
    sd, cam = scenes.glossy_room(16)
    s = oracle.Scene(sd)
    K = 8
    blocks = []
    for S, S2, C, SP, _ in _chunks(s, cam, 64, 3, K, lt_mode=1, aim=True):
        blocks.append(((S + SP) / C[..., None]).reshape(4, 4, 4, 4, 3).mean(axis=(1, 3)))
    blocks = np.array(blocks)
    m_tw, se_tw = blocks.mean(axis=0), blocks.std(axis=0, ddof=1) / np.sqrt(K)
    S, S2, C, _ = s.render(cam, 2048, 3, iter0=1 << 20)
    mean, var = oracle.resolve(S, S2, C)
    m_pt = mean.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3))
    se_pt = np.sqrt(var.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3)) / 16.0)
    z = np.abs(m_tw - m_pt) / np.sqrt(se_tw ** 2 + se_pt ** 2 + 1e-30)
    assert z.max() < 4.5, z.max()


def test_aiming_lowers_the_light_tracers_error_in_an_open_scene():
    """A small near-mirror object on a stand near the camera, in a scene
    whose bound is hundreds of times larger, lit by a sky with a sun. The
    light tracer alone (lt_mode 1: it makes every path it can, so the
    emission decides its error): aimed emission puts photons on the clusters
    in view, uniform emission over the scene's bound spreads them over a disk
    of radius ~280. Mean relative error against a two-way reference of 2048
    iterations from a disjoint range."""
    sd, cam = scenes.turntable(res=24)
    s = oracle.Scene(sd)
    D = 3
    ref = np.mean([(S + SP) / C[..., None] for S, S2, C, SP, _ in
                   [s.render_two_way(cam, 256, D, iter0=(1 << 20) + k * 256) for k in range(8)]], axis=0)
    err = {}
    for aim in (False, True):
        S, S2, C, SP, _ = s.render_two_way(cam, 64, D, aim=aim, lt_mode=1)
        err[aim] = np.abs((S + SP) / C[..., None] - ref).sum() / np.abs(ref).sum()
    assert err[True] < 0.85 * err[False], err
