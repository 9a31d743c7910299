"""Pins of the oracle's probabilistic light hierarchy (Sec. 2.1.1): the
probabilities form a distribution, the descent draws emitters with exactly
those probabilities, the deterministic re-traversal gives the same number, the
tree is well formed, small sets reduce to flux-proportional selection, the
directional values bound the one-sided cosine lobe, the clamp keeps every
emitter reachable, and images rendered with it are unbiased (NEE-only,
BSDF-only and MIS agree) and less noisy than with the alias table where a few
of many lights dominate."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes


@pytest.fixture(scope="module")
def many():
    sd, cam = scenes.many_emitters(n_lights=200, res=24)
    return sd, cam, oracle.Scene(sd)


def random_points(rng, n):
    x = np.stack([rng.uniform(-10, 10, n), rng.uniform(0, 2.5, n), rng.uniform(-10, 10, n)], 1)
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return x, nrm


def test_probabilities_form_a_distribution(many):
    _, _, s = many
    rng = np.random.default_rng(1)
    for x, n in zip(*random_points(rng, 20)):
        P = np.array([s.lb_prob(x, n, e) for e in range(200)])
        assert np.all(P > 0.0)
        assert P.sum() == pytest.approx(1.0, abs=1e-12)


def test_descent_draws_each_emitter_with_its_probability(many):
    """The map u -> emitter is measure preserving: on a fine grid of u the
    share of each emitter is its probability (up to one grid cell per
    boundary of its u-set)."""
    _, _, s = many
    rng = np.random.default_rng(2)
    N = 1 << 16
    for x, n in zip(*random_points(rng, 3)):
        u = (np.arange(N) + 0.5) / N
        picks = np.array([s.lb_sample(x, n, float(v))[0] for v in u])
        freq = np.bincount(picks, minlength=200) / N
        P = np.array([s.lb_prob(x, n, e) for e in range(200)])
        assert np.abs(freq - P).max() <= 8.0 / N


def test_sampled_probability_equals_deterministic_retraversal(many):
    _, _, s = many
    rng = np.random.default_rng(3)
    xs, ns = random_points(rng, 200)
    for x, n, u in zip(xs, ns, rng.random(200)):
        e, p = s.lb_sample(x, n, float(u))
        assert p == pytest.approx(s.lb_prob(x, n, e), rel=1e-12)


def test_tree_is_well_formed(many):
    sd, _, s = many
    nn = s.lb_num_nodes()
    nodes = [s.lb_node(i) for i in range(nn)]
    leaves = [d for d in nodes if d["count"] > 0]
    assert nn == 2 * len(leaves) - 1
    assert all(1 <= d["count"] <= 4 for d in leaves)
    assert sum(d["count"] for d in leaves) == 200
    assert nodes[0]["parent"] == -1
    for i, d in enumerate(nodes):
        if d["count"] == 0:
            L, R = nodes[d["left"]], nodes[d["right"]]
            assert L["parent"] == i and R["parent"] == i
            assert d["flux"] == pytest.approx(L["flux"] + R["flux"], rel=1e-12)
            assert np.allclose(d["I"], L["I"] + R["I"], rtol=1e-12, atol=0)
            for c in (L, R):
                assert np.all(c["lo"] >= d["lo"]) and np.all(c["hi"] <= d["hi"])
    # the root holds every emitter's flux: luminance x area
    lum = sd.emission @ np.array([0.2126, 0.7152, 0.0722])
    V = sd.vertices.astype(np.float64)[sd.indices]
    area = 0.5 * np.linalg.norm(np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]), axis=1)
    assert nodes[0]["flux"] == pytest.approx(float((lum[sd.tri_material] * area).sum()), rel=1e-12)
    # every emitter sits in the leaf its deterministic path names
    ems = [t for t in range(sd.indices.shape[0]) if lum[sd.tri_material[t]] > 0]
    assert [s.lb_light_of_tri(t) for t in ems] == list(range(200))


def test_four_or_fewer_emitters_reduce_to_flux_proportional_selection():
    sd, _ = scenes.many_emitters(n_lights=4, res=8)
    s = oracle.Scene(sd)
    assert s.lb_num_nodes() == 1
    plain = oracle.Scene(dataclasses.replace(sd, light_bvh=False))
    em = [t for t in range(sd.indices.shape[0]) if plain.light_pdf_area(t) > 0]
    V = sd.vertices.astype(np.float64)
    area = np.array([0.5 * np.linalg.norm(np.cross(*(V[sd.indices[t]][1:] - V[sd.indices[t]][0]))) for t in em])
    flux_share = np.array([plain.light_pdf_area(t) for t in em]) * area
    rng = np.random.default_rng(4)
    for x, n in zip(*random_points(rng, 5)):
        P = np.array([s.lb_prob(x, n, e) for e in range(4)])
        assert np.allclose(P, flux_share / flux_share.sum(), rtol=1e-9)


def test_directional_values_bound_the_cosine_lobe():
    """A single one-sided emitter of normal +z: the +z face region holds its
    whole flux, the -z region nothing, the four side regions the lobe's
    maximum over their cones, cos(90 deg - 54.74 deg) = sqrt(2/3). For random
    normals the six values bound flux x max(0, n . w) over sampled directions
    of each region."""
    sd, _ = scenes.many_emitters(n_lights=1, res=8)
    V = sd.vertices.astype(np.float64)
    tri = sd.indices[-1]
    p = V[tri]
    n = np.cross(p[1] - p[0], p[2] - p[0])
    n /= np.linalg.norm(n)
    s = oracle.Scene(sd)
    d = s.lb_node(0)
    flux = d["flux"]
    rng = np.random.default_rng(5)
    w = rng.normal(size=(20000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    reg = np.array([oracle.lb_region(v) for v in w])
    lobe = flux * np.maximum(0.0, w @ n)
    for k in range(6):
        assert d["I"][k] >= lobe[reg == k].max() - 1e-12
    # the axis-aligned case in closed form, with a rotated copy of the scene
    R = _rotation_to(n, np.array([0.0, 0.0, 1.0]))
    sd2 = dataclasses.replace(sd, vertices=(V @ R.T).astype(np.float32))
    d2 = oracle.Scene(sd2).lb_node(0)
    assert d2["I"][4] == pytest.approx(d2["flux"], rel=1e-6)
    assert d2["I"][5] == 0.0
    for k in range(4):
        assert d2["I"][k] == pytest.approx(d2["flux"] * math.sqrt(2.0 / 3.0), rel=1e-5)


def _rotation_to(a, b):
    """Rotation matrix taking unit vector a to unit vector b (Rodrigues)."""
    v = np.cross(a, b)
    c = float(np.dot(a, b))
    K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + K + K @ K / (1.0 + c)


def test_clamp_keeps_emitters_behind_the_surface_reachable(many):
    """A shading point whose normal turns away from every emitter gets
    vanishing estimates everywhere, yet each child keeps at least 0.1."""
    _, _, s = many
    x = np.array([0.0, 0.01, 0.0])
    down = np.array([0.0, -1.0, 0.0])
    for i in range(s.lb_num_nodes()):
        d = s.lb_node(i)
        if d["count"] == 0:
            p = s.lb_p_left(i, x, down)
            assert 0.1 <= p <= 0.9
    assert min(s.lb_prob(x, down, e) for e in range(200)) > 0.0


@pytest.mark.parametrize("depth", [1, 3])
def test_images_agree_across_nee_only_bsdf_only_and_mis(depth):
    """Unbiasedness: with the hierarchy's probabilities NEE-only and MIS images
    match the BSDF-only image (which never uses them) within 4 sigma
    (pixels averaged in 4 x 4 blocks)."""
    sd, cam = scenes.many_emitters(n_lights=64, res=16)
    s = oracle.Scene(sd)
    imgs = {}
    for mode, spp in ((3, 4096), (2, 256), (0, 256)):
        S, S2, cnt, _ = s.render(cam, spp, depth, mis_mode=mode)
        mean, var = oracle.resolve(S, S2, cnt)
        m = mean.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3))
        v = var.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3)) / 16.0
        imgs[mode] = (m, v)
    mb, vb = imgs[3]
    for mode in (2, 0):
        m, v = imgs[mode]
        z = np.abs(m - mb) / np.sqrt(v + vb + 1e-30)
        assert z.max() < 4.5
        assert abs(m.mean() - mb.mean()) <= 4.0 * math.sqrt((v.sum() + vb.sum())) / m.size


def test_hierarchy_beats_the_alias_table_where_few_lights_dominate():
    sd, cam = scenes.many_emitters(n_lights=200, res=16)
    out = {}
    for bvh in (False, True):
        s = oracle.Scene(dataclasses.replace(sd, light_bvh=bvh))
        S, S2, cnt, _ = s.render(cam, 128, 1, mis_mode=2)
        mean, var = oracle.resolve(S, S2, cnt)
        out[bvh] = (mean.mean(), var.mean())
    assert out[True][0] == pytest.approx(out[False][0], rel=0.05)
    assert out[True][1] < 0.7 * out[False][1]
