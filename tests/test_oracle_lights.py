"""Pins for the oracle's light importance sampling (Sec. 2.1.1 triangle
emitters with one flux per triangle, selected here by an alias table;
Sec. 2.1.2 environment pyramid with area-weighted texels)."""
import math

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes


def alias_implied_probs(prob, alias):
    n = prob.size
    p = prob.copy()
    np.add.at(p, alias, 1.0 - prob)
    return p / n


@pytest.mark.parametrize("n", [1, 2, 7, 1000])
def test_alias_table_reproduces_weights(n):
    rng = np.random.default_rng(n)
    w = rng.lognormal(0, 1.5, n)
    w[rng.random(n) < 0.1] = 1e-9
    prob, alias = oracle.alias_build(w)
    assert np.all((prob >= 0) & (prob <= 1))
    assert np.allclose(alias_implied_probs(prob, alias), w / w.sum(), rtol=1e-11, atol=1e-15)
    # a fine regular grid of u reproduces the probabilities to grid resolution
    m = 200_000
    counts = np.zeros(n)
    for u in (np.arange(m) + 0.5) / m:
        counts[oracle.alias_sample(prob, alias, u)] += 1
    assert np.allclose(counts / m, w / w.sum(), atol=2.0 / m * 2 + 1e-12)


def env_scene(env):
    sd = scenes.SceneData(
        vertices=np.zeros((3, 3), np.float32), indices=np.zeros((0, 3), np.uint32),
        tri_material=np.zeros(0, np.uint32), albedo=np.zeros((1, 3), np.float32),
        roughness=np.zeros(1, np.float32), ggx_weight=np.zeros(1, np.float32),
        emission=np.zeros((1, 3), np.float32), emission_tex=np.full(1, -1, np.int32), env=env)
    return oracle.Scene(sd)


def test_constant_env_pdf_is_uniform_sphere():
    s = env_scene(np.full((16, 32, 3), 2.5, np.float32))
    rng = np.random.default_rng(0)
    assert s.env_select_prob() == 1.0
    for _ in range(200):
        u, v = rng.random(2)
        wi, pdf, tx, ty = s.env_sample(u, v)
        assert np.linalg.norm(wi) == pytest.approx(1.0, abs=1e-12)
        assert pdf == pytest.approx(1.0 / (4 * math.pi), rel=1e-12)
        assert s.env_pdf(wi) == pytest.approx(1.0 / (4 * math.pi), rel=1e-12)


def test_env_descent_probabilities_and_texel_placement():
    rng = np.random.default_rng(1)
    W, H = 32, 16
    env = rng.lognormal(0, 2, (H, W, 3)).astype(np.float32)
    env[3, 5] = 0.0  # a black texel is never chosen
    P = oracle.env_pyramid_probs(env)
    th = np.pi * np.arange(H + 1) / H
    om = (2 * np.pi / W) * (np.cos(th[:-1]) - np.cos(th[1:]))
    e64 = env.astype(np.float64)
    lum = 0.2126 * e64[..., 0] + 0.7152 * e64[..., 1] + 0.0722 * e64[..., 2]
    want = lum * om[:, None]
    want /= want.sum()
    assert P.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(P, want, rtol=1e-10, atol=1e-16)
    s = env_scene(env)
    # the preimage of every texel is a rectangle in (u, v): a regular grid of
    # sample pairs lands on each texel in proportion to its probability
    m = 400
    counts = np.zeros((H, W))
    for i in range(m):
        for j in range(m):
            wi, pdf, tx, ty = s.env_sample((i + 0.5) / m, (j + 0.5) / m)
            counts[ty, tx] += 1
            if (i * m + j) % 97 == 0:
                # direction lies in the chosen texel and the pdf is lum / sum(w)
                t = math.acos(max(-1.0, min(1.0, wi[1])))
                p = math.atan2(wi[2], wi[0]) % (2 * math.pi)
                assert th[ty] - 1e-12 <= t <= th[ty + 1] + 1e-12
                assert 2 * math.pi * tx / W - 1e-12 <= p <= 2 * math.pi * (tx + 1) / W + 1e-12
                assert pdf == pytest.approx(lum[ty, tx] / (lum * om[:, None]).sum(), rel=1e-9)
    assert counts[3, 5] == 0
    assert np.abs(counts / m**2 - P).max() < 4.0 / m


def test_env_pdf_integrates_to_one():
    rng = np.random.default_rng(2)
    env = rng.lognormal(0, 1, (8, 16, 3)).astype(np.float32)
    s = env_scene(env)
    # midpoint rule in (theta, phi) with the sin(theta) Jacobian, grid lines
    # on texel boundaries
    n_t, n_p = 8 * 60, 16 * 8
    tt = np.pi * (np.arange(n_t) + 0.5) / n_t
    ph = 2 * np.pi * (np.arange(n_p) + 0.5) / n_p
    tot = 0.0
    for t in tt:
        for p in ph:
            tot += s.env_pdf([math.sin(t) * math.cos(p), math.cos(t), math.sin(t) * math.sin(p)]) * math.sin(t)
    tot *= (np.pi / n_t) * (2 * np.pi / n_p)
    assert tot == pytest.approx(1.0, abs=1e-4)


def test_textured_emitter_flux_is_exact_integral():
    """Two emitters over one texture, covering the lower-left and the
    upper-right half of UV space: selection probabilities are in the ratio of
    the exact mean luminances (texels cut by the diagonal count half)."""
    tw = th = 4
    rng = np.random.default_rng(3)
    tex = rng.lognormal(0, 1, (1, th, tw, 3)).astype(np.float32)
    sd = scenes.SceneData(
        vertices=np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [1, 0, 1]], np.float32),
        indices=np.array([[0, 2, 1], [1, 2, 3]], np.uint32), tri_material=np.zeros(2, np.uint32),
        albedo=np.zeros((1, 3), np.float32), roughness=np.zeros(1, np.float32),
        ggx_weight=np.zeros(1, np.float32), emission=np.ones((1, 3), np.float32),
        emission_tex=np.zeros(1, np.int32),
        uvs=np.array([[0, 0], [1, 0], [0, 1], [1, 1]], np.float32), textures=tex)
    s = oracle.Scene(sd)
    t64 = tex[0].astype(np.float64)
    lum = 0.2126 * t64[..., 0] + 0.7152 * t64[..., 1] + 0.0722 * t64[..., 2]
    lo = hi = 0.0
    for y in range(th):
        for x in range(tw):
            if x + y < tw - 1:
                lo += lum[y, x]
            elif x + y == tw - 1:
                lo += 0.5 * lum[y, x]
                hi += 0.5 * lum[y, x]
            else:
                hi += lum[y, x]
    # equal areas 0.5: pdf_area = P(select) / 0.5
    assert s.light_pdf_area(0) == pytest.approx(2.0 * lo / (lo + hi), rel=1e-12)
    assert s.light_pdf_area(1) == pytest.approx(2.0 * hi / (lo + hi), rel=1e-12)
