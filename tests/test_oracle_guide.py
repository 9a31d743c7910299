"""Pins for the oracle's path-guiding math. The paper has no learned part;
these pin the textbook definitions (vMF density and sampling, one-blob
encoding, backpropagation, Adam) to closed forms and finite differences."""
import math

import numpy as np
import pytest

import oracle


def sphere_grid(n_t=800, n_p=800):
    ct = 1 - 2 * (np.arange(n_t) + 0.5) / n_t
    ph = 2 * np.pi * (np.arange(n_p) + 0.5) / n_p
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C * C)
    return np.stack([S * np.cos(P), C, S * np.sin(P)], -1).reshape(-1, 3), (2.0 / n_t) * (2 * np.pi / n_p)


@pytest.mark.parametrize("kappa", [0.01, 1.0, 10.0, 200.0])
def test_vmf_integrates_to_one(kappa):
    mu = np.array([0.0, 1.0, 0.0])  # aligned with the cos-theta grid axis
    grid, dA = sphere_grid(40000 if kappa > 50 else 800, 8)
    tot = sum(oracle.vmf_pdf(kappa, mu, w) for w in grid[:: 1]) * dA
    assert tot == pytest.approx(1.0, rel=1e-4)


@pytest.mark.parametrize("kappa", [0.5, 5.0, 80.0])
def test_vmf_sampling_mean_cosine(kappa):
    mu = np.array([0.3, -0.5, 0.8])
    mu /= np.linalg.norm(mu)
    m = 200
    cs = []
    for i in range(m):
        for j in range(m // 4):
            w = oracle.vmf_sample(kappa, mu, (i + 0.5) / m, (j + 0.5) / (m // 4))
            assert np.linalg.norm(w) == pytest.approx(1.0, abs=1e-12)
            cs.append(np.dot(w, mu))
    want = 1.0 / math.tanh(kappa) - 1.0 / kappa
    assert np.mean(cs) == pytest.approx(want, abs=2e-3)


def test_oneblob_closed_form():
    s = np.array([0.0, 0.5, 1.0, 0.123, 0.77, 0.999, 0.5001])
    enc = oracle.oneblob(s).reshape(7, 32)
    c = (np.arange(32) + 0.5) / 32
    want = np.exp(-((s[:, None] - c[None, :]) ** 2) / (2 * (1 / 32) ** 2))
    assert np.allclose(enc, want, rtol=1e-14, atol=0)
    assert enc[3].argmax() == int(0.123 * 32)


def random_params(seed, scale=0.15):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, oracle.guide_nparams())


def test_mixture_pdf_integrates_to_one():
    rng = np.random.default_rng(4)
    raw = rng.normal(0, 1.5, 40)
    grid, dA = sphere_grid(600, 600)
    tot = sum(oracle.mixture_pdf(raw, w) for w in grid) * dA
    assert tot == pytest.approx(1.0, rel=2e-3)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(5)
    params = random_params(6)
    B = 6
    s7 = rng.random((B, 7))
    x = np.stack([oracle.oneblob(r) for r in s7])
    wi = rng.normal(size=(B, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    weight = rng.uniform(0.1, 3.0, B)
    loss, g = oracle.guide_loss_grad(params, x, wi, weight)
    assert np.isfinite(loss)
    idx = np.concatenate([rng.choice(14336, 25, replace=False),
                          14336 + rng.choice(12288, 25, replace=False),
                          26624 + rng.choice(2560, 40, replace=False)])
    h = 1e-6
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (oracle.guide_loss_grad(p1, x, wi, weight)[0] - oracle.guide_loss_grad(p2, x, wi, weight)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_forward_matches_plain_matrix_products():
    rng = np.random.default_rng(7)
    params = random_params(8)
    x = rng.random((5, 224))
    dims = [224, 64, 64, 64, 64, 40]
    h = x
    off = 0
    for l in range(5):
        W = params[off: off + dims[l] * dims[l + 1]].reshape(dims[l + 1], dims[l])
        off += W.size
        h = h @ W.T
        if l < 4:
            h = np.maximum(h, 0)
    assert np.allclose(oracle.mlp_forward(params, x), h, rtol=1e-12, atol=1e-14)


def test_adam_first_steps_textbook():
    rng = np.random.default_rng(9)
    p = rng.normal(size=50)
    g1, g2 = rng.normal(size=50), rng.normal(size=50)
    m, v = np.zeros(50), np.zeros(50)
    q = p.copy()
    oracle.adam_step(q, g1, m, v, 1, lr=1e-2)
    # first step: m_hat = g, v_hat = g^2 -> step = lr * g / (|g| + eps)
    assert np.allclose(q, p - 1e-2 * g1 / (np.abs(g1) + 1e-8), rtol=1e-13)
    oracle.adam_step(q, g2, m, v, 2, lr=1e-2)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1**2 + 0.001 * g2**2
    mh, vh = m2 / (1 - 0.81), v2 / (1 - 0.999**2)
    want = p - 1e-2 * g1 / (np.abs(g1) + 1e-8) - 1e-2 * mh / (np.sqrt(vh) + 1e-8)
    assert np.allclose(q, want, rtol=1e-12)


def test_training_reduces_loss_on_a_fixed_target():
    """Sanity of the whole loop: Adam on a batch whose directions cluster
    around one axis lowers the loss."""
    rng = np.random.default_rng(10)
    params = random_params(11, 0.05)
    B = 64
    x = np.stack([oracle.oneblob(r) for r in rng.random((B, 7))])
    wi = np.array([0.0, 1.0, 0.0]) + 0.2 * rng.normal(size=(B, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    weight = np.ones(B)
    m, v = np.zeros_like(params), np.zeros_like(params)
    l0, _ = oracle.guide_loss_grad(params, x, wi, weight)
    for t in range(1, 41):
        _, g = oracle.guide_loss_grad(params, x, wi, weight)
        oracle.adam_step(params, g, m, v, t, lr=1e-2)
    l1, _ = oracle.guide_loss_grad(params, x, wi, weight)
    assert l1 < l0 - 1.0
