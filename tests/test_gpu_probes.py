"""Irradiance probes on the GPU (Sec. 4.2): closed forms (uniform sky and
white furnace exact with cosine sampling; a parallel Lambertian rectangle),
parity with the FP64 oracle at the same sequence indices, resumable iteration
ranges, and argument errors."""
import math

import numpy as np
import pytest

import oracle
from helpers import allowed_4sigma
from paper_1705_01263_gb300 import scenes
from test_oracle_render import corner_form_factor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda")


def probes_render(scene, pos, nrm, spp, depth, film=None, **kw):
    from paper_1705_01263_gb300 import rt
    film = film or rt.Film(len(pos), 1)
    stats = rt.rt_stats()
    rt.rt_render_probes(scene, dev(pos), dev(nrm), spp, depth, film, rt.make_opts(stats=stats, **kw))
    torch.cuda.synchronize()
    return film, stats


def furnace_probes():
    pos = [[0.0, 3.0, 0.0], [0.0, 3.0, 0.0], [2.5, 0.3, -0.4], [-1.2, -1.5, 2.0]]
    nrm = [[0.0, 1.0, 0.0], [0.0, -1.0, 0.0], [-1.0, 0.0, 0.0], [0.6, 0.0, -0.8]]
    return pos, nrm


def test_uniform_sky_and_furnace_exact_with_bsdf_sampling():
    from paper_1705_01263_gb300 import rt
    sd, _ = scenes.furnace_sphere(radiance=2.0)
    pos, nrm = furnace_probes()
    film, st = probes_render(rt.Scene(sd), pos, nrm, 32, 2, mis_mode=3)
    s, s2, c = film.download()
    assert np.all(c == 32) and st.paths == 32 * len(pos)
    assert np.allclose(s / 32, 2.0 * math.pi, rtol=1e-6)


def test_uniform_sky_with_mis():
    from paper_1705_01263_gb300 import rt
    sd, _ = scenes.furnace_sphere(radiance=1.0)
    pos, nrm = furnace_probes()
    film, _ = probes_render(rt.Scene(sd), pos, nrm, 2048, 4)
    s, s2, c = film.download()
    assert np.allclose(s / c[..., None], math.pi, rtol=5e-3)


@pytest.mark.parametrize("mis_mode", [0, 2, 3])
def test_probe_under_parallel_rectangle(mis_mode):
    from paper_1705_01263_gb300 import rt
    h, a, b, L = 1.0, 0.5, 0.75, 3.0
    sd, _ = scenes.parallel_emitter(h, a, b, L, 0.6)
    F = 4 * corner_form_factor(a / h, b / h)
    spp = 4096 if mis_mode != 3 else 16384
    film, _ = probes_render(rt.Scene(sd), [[0.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]], spp, 1, mis_mode=mis_mode)
    s, _, c = film.download()
    tol = 3e-3 if mis_mode != 3 else 1.5e-2
    assert s[0, 0, 0] / c[0, 0] == pytest.approx(math.pi * L * F, rel=tol)


@pytest.mark.parametrize("light", ["down", "up"])
def test_probes_match_the_oracle(light):
    """64 probes on the walls, floor and in the air of both Cornell boxes,
    256 samples each, against the oracle at the same sequence indices."""
    from paper_1705_01263_gb300 import rt
    sd, _ = scenes.cornell_box(light=light)
    rng = np.random.default_rng(7)
    pos = rng.uniform(0.05, 0.95, (64, 3))
    nrm = rng.normal(size=(64, 3))
    pos[:16, 1] = 1e-3
    nrm[:16] = [0.0, 1.0, 0.0]                 # on the floor, facing up
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    pos, nrm = pos.astype(np.float32), nrm.astype(np.float32)
    spp = 256
    film, _ = probes_render(rt.Scene(sd), pos, nrm, spp, 8)
    s, s2, c = film.download()
    mg, vg = oracle.resolve(s, s2, c)
    S, S2, C, _ = oracle.Scene(sd).render_probes(pos.astype(np.float64), nrm.astype(np.float64), spp, 8)
    assert np.array_equal(c[0], C)
    mo, vo = oracle.resolve(S[None], S2[None], C[None])
    sig = np.sqrt(vg + vo)
    out = int((np.abs(mg - mo) > 4 * sig + 1e-6).sum())
    assert out <= allowed_4sigma(mg.size), out
    assert abs(mg.sum() - mo.sum()) <= 0.01 * abs(mo.sum())


def test_probe_iterations_resume_exactly():
    from paper_1705_01263_gb300 import rt
    sd, _ = scenes.cornell_box()
    scene = rt.Scene(sd)
    pos = [[0.5, 0.01, 0.5], [0.2, 0.5, 0.99], [0.99, 0.3, 0.3]]
    nrm = [[0.0, 1.0, 0.0], [0.0, 0.0, -1.0], [-1.0, 0.0, 0.0]]
    a, _ = probes_render(scene, pos, nrm, 12, 6)
    b = rt.Film(3, 1)
    probes_render(scene, pos, nrm, 5, 6, film=b)
    probes_render(scene, pos, nrm, 7, 6, film=b, max_paths=32)   # other set size
    sa, s2a, ca = a.download()
    sb, s2b, cb = b.download()
    assert np.array_equal(ca, cb)
    assert np.allclose(sa, sb, rtol=1e-12, atol=1e-12) and np.allclose(s2a, s2b, rtol=1e-12, atol=1e-12)


def test_probe_argument_errors():
    from paper_1705_01263_gb300 import rt
    sd, _ = scenes.cornell_box()
    scene = rt.Scene(sd)
    pos, nrm = [[0.5, 0.5, 0.5]], [[0.0, 1.0, 0.0]]
    with pytest.raises(rt.RtError):
        rt.rt_render_probes(scene, dev(pos), dev(nrm), 4, 4, rt.Film(2, 1))       # film not n x 1
    with pytest.raises(rt.RtError):
        rt.rt_render_probes(scene, dev(pos), dev(nrm), 4, 0, rt.Film(1, 1))       # max_depth 0
    with pytest.raises(rt.RtError):
        rt.rt_render_probes(scene, dev(pos), dev(nrm), 4, 4, rt.Film(1, 1),
                            rt.make_opts(guide=rt.Guide(scene)))
