"""Pins for the oracle's path tracer (Sec. 2 forward path tracing with NEE
and MIS; Appendix A.1 filter importance sampling; Appendix A.4 per-pixel
sample counts): white furnace, a closed-form direct-lighting pixel,
agreement of the MIS techniques, split-and-merge of iteration ranges."""
import math

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes


def test_camera_ray_geometry():
    cam = scenes.Camera((0, 0, 0), (0, 0, -1), (0, 1, 0), 90.0, 200, 100)
    o, d = oracle.camera_ray(cam, 100.0, 50.0)
    assert np.allclose(d, [0, 0, -1], atol=1e-15) and np.allclose(o, 0)
    _, d = oracle.camera_ray(cam, 200.0, 50.0)   # right edge: tan = aspect * tan(45)
    assert math.atan2(d[0], -d[2]) == pytest.approx(math.atan(2.0), abs=1e-14)
    _, d = oracle.camera_ray(cam, 100.0, 0.0)    # top edge
    assert math.atan2(d[1], -d[2]) == pytest.approx(math.pi / 4, abs=1e-14)


def test_filter_offsets_are_gaussian():
    u = oracle.sample_dims_u32(np.arange(1 << 14, dtype=np.uint64), 2, 1, 1, 0)
    vals = (u >> 8).astype(np.float64) * 2.0**-24
    dx = np.array([oracle.filter_offset(0.5, a, b) for a, b in vals])
    assert abs(dx.mean()) < 1e-3
    assert dx.std(axis=0) == pytest.approx([0.5, 0.5], rel=2e-3)
    # inside 1.5 px (3 sigma) radius: 1 - exp(-4.5) of the mass
    inside = (np.hypot(dx[:, 0], dx[:, 1]) <= 1.5).mean()
    assert inside == pytest.approx(1 - math.exp(-4.5), abs=1e-3)
    assert oracle.filter_offset(0.0, 0.25, 0.75) == (-0.25, 0.25)


def test_white_furnace_bsdf_sampling_is_exact():
    sd, cam = scenes.furnace_sphere(res=16)
    s = oracle.Scene(sd)
    S, S2, cnt, _ = s.render(cam, 8, 4, mis_mode=3)
    mean, _ = oracle.resolve(S, S2, cnt)
    assert np.allclose(mean, 1.0, rtol=0, atol=1e-12)


def test_white_furnace_with_mis_converges_to_one():
    sd, cam = scenes.furnace_sphere(res=32)
    s = oracle.Scene(sd)
    S, S2, cnt, _ = s.render(cam, 64, 4)
    mean, var = oracle.resolve(S, S2, cnt)
    assert abs(mean.mean() - 1.0) < 1e-3
    # every pixel within five of its own standard errors (64 samples)
    assert np.all(np.abs(mean - 1.0) < 5.0 * np.sqrt(var) + 1e-3)


def corner_form_factor(A, B):
    a1, b1 = math.sqrt(1 + A * A), math.sqrt(1 + B * B)
    return (A / a1 * math.atan(B / a1) + B / b1 * math.atan(A / b1)) / (2 * math.pi)


@pytest.mark.parametrize("mis_mode", [0, 1, 2, 3])
def test_direct_light_under_parallel_rectangle(mis_mode):
    """Lambert floor under a parallel 2a x 2b emitter at height h: radiance
    at the point below the centre = albedo * L * F, F = 4 F_corner."""
    h, a, b, L, rho = 1.0, 0.5, 0.75, 3.0, 0.6
    sd, cam = scenes.parallel_emitter(h, a, b, L, rho)
    s = oracle.Scene(sd)
    F = 4 * corner_form_factor(a / h, b / h)
    spp = 4096 if mis_mode != 3 else 16384
    S, S2, cnt, _ = s.render(cam, spp, 1, mis_mode=mis_mode)
    mean, var = oracle.resolve(S, S2, cnt)
    want = rho * L * F
    tol = 3e-3 if mis_mode != 3 else 1.5e-2
    assert mean[0, 0, 0] == pytest.approx(want, rel=tol)


@pytest.mark.parametrize("light", ["down", "up"])
def test_mis_techniques_agree_on_cornell(light):
    # "up": the emitter faces the ceiling 0.1 below it, so most of the light
    # that NEE finds arrives from close by at grazing angles
    sd, cam = scenes.cornell_box(light=light)
    s = oracle.Scene(sd)
    res = {}
    for mode in (0, 2, 3):
        S, S2, cnt, _ = s.render(cam, 32, 4, mis_mode=mode)
        m, v = oracle.resolve(S, S2, cnt)
        res[mode] = (m.mean(), math.sqrt(v.sum()) / m.size)
    for mode in (2, 3):
        d = abs(res[mode][0] - res[0][0])
        sig = math.hypot(res[mode][1], res[0][1])
        assert d < 4 * sig + 1e-3 * res[0][0], (mode, res)


def test_split_and_merge_equals_single_range():
    sd, cam = scenes.cornell_box()
    cam.width = cam.height = 24
    s = oracle.Scene(sd)
    A = s.render(cam, 16, 6)
    B1 = s.render(cam, 7, 6, iter0=0)
    B2 = s.render(cam, 9, 6, iter0=7)
    assert np.array_equal(A[2], B1[2] + B2[2])
    assert np.allclose(A[0], B1[0] + B2[0], rtol=1e-13, atol=1e-13)
    assert np.allclose(A[1], B1[1] + B2[1], rtol=1e-13, atol=1e-13)
    assert A[3] == B1[3] + B2[3]


def test_render_is_deterministic_and_thread_independent():
    sd, cam = scenes.cornell_box()
    cam.width = cam.height = 16
    s = oracle.Scene(sd)
    a = s.render(cam, 4, 8, threads=1)
    b = s.render(cam, 4, 8, threads=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
