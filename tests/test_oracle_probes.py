"""Irradiance probes in the oracle (Sec. 4.2: irradiance at user points from
the hemisphere around a normal, sampled progressively like pixels), pinned to
closed forms: a uniform sky gives E = pi L; a convex white sphere in it
changes nothing (furnace); under a parallel Lambertian rectangle of radiance
L, E = pi L F with F the point-to-rectangle form factor."""
import math

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes
from test_oracle_render import corner_form_factor


def furnace_probes():
    pos = np.array([[0.0, 3.0, 0.0], [0.0, 3.0, 0.0], [2.5, 0.3, -0.4], [-1.2, -1.5, 2.0]])
    nrm = np.array([[0.0, 1.0, 0.0], [0.0, -1.0, 0.0], [-1.0, 0.0, 0.0], [0.6, 0.0, -0.8]])
    return pos, nrm / np.linalg.norm(nrm, axis=1, keepdims=True)


def test_uniform_sky_and_furnace_are_exact_with_bsdf_sampling():
    """Cosine sampling of a constant sky, also through one bounce off a
    convex albedo-1 sphere: every path returns pi L exactly."""
    sd, _ = scenes.furnace_sphere(radiance=2.0)
    s = oracle.Scene(sd)
    pos, nrm = furnace_probes()
    S, S2, cnt, _ = s.render_probes(pos, nrm, 16, 2, mis_mode=3)
    assert np.all(cnt == 16)
    assert np.allclose(S / 16, 2.0 * math.pi, rtol=0, atol=1e-11)


def test_uniform_sky_with_mis_converges_to_pi_l():
    sd, _ = scenes.furnace_sphere(radiance=1.0)
    s = oracle.Scene(sd)
    pos, nrm = furnace_probes()
    S, S2, cnt, _ = s.render_probes(pos, nrm, 2048, 4)
    mean = S / cnt[:, None]
    assert np.allclose(mean, math.pi, rtol=5e-3)


@pytest.mark.parametrize("mis_mode", [0, 2, 3])
def test_probe_under_parallel_rectangle(mis_mode):
    h, a, b, L = 1.0, 0.5, 0.75, 3.0
    sd, _ = scenes.parallel_emitter(h, a, b, L, 0.6)
    s = oracle.Scene(sd)
    F = 4 * corner_form_factor(a / h, b / h)
    spp = 4096 if mis_mode != 3 else 16384
    S, S2, cnt, _ = s.render_probes([[0.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]], spp, 1, mis_mode=mis_mode)
    want = math.pi * L * F
    tol = 3e-3 if mis_mode != 3 else 1.5e-2
    assert S[0, 0] / cnt[0] == pytest.approx(want, rel=tol)


def test_probe_iterations_split_and_merge():
    sd, _ = scenes.cornell_box()
    s = oracle.Scene(sd)
    pos = np.array([[0.5, 0.01, 0.5], [0.2, 0.5, 0.9], [0.99, 0.3, 0.3]])
    nrm = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, -1.0], [-1.0, 0.0, 0.0]])
    A = s.render_probes(pos, nrm, 12, 6)
    B1 = s.render_probes(pos, nrm, 5, 6, iter0=0)
    B2 = s.render_probes(pos, nrm, 7, 6, iter0=5)
    assert np.array_equal(A[2], B1[2] + B2[2])
    assert np.allclose(A[0], B1[0] + B2[0], rtol=1e-13, atol=1e-13)
