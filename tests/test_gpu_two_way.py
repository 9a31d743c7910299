"""GPU parity of two-way path tracing (Sec. 2: path tracer and light tracer
combined by MIS) through the C ABI: the camera stage and the light stage's
splats against the oracle on the same samples (every heuristic, filter and
light-tracer mode), the combined image against the GPU path tracer in
expectation, the error reduction in the ceiling-lit glossy room, and the
refused configurations; scenes with the light hierarchy (Sec. 2.1.1) included."""
import dataclasses

import numpy as np
import pytest

import oracle
from helpers import allowed_4sigma, image_parity
from paper_1705_01263_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _scene(name, res):
    if name == "glossy":
        sd, cam = scenes.glossy_room(res)
    elif name == "many":
        sd, cam = scenes.many_emitters(n_lights=64, res=res)   # light hierarchy
    elif name == "turntable":
        sd, cam = scenes.turntable(res=res)   # open scene: photon aiming at the object in view
    elif name == "cornell-env":
        # open towards the camera and lit by a sky too: environment photons
        sd, cam = scenes.cornell_box()
        sd = dataclasses.replace(sd, env=scenes.procedural_sky(32, 16, seed=3)[0])
        cam = dataclasses.replace(cam, width=res, height=res)
    else:
        sd, cam = scenes.cornell_box()
        cam = dataclasses.replace(cam, width=res, height=res)
    return sd, cam


def two_way_gpu(sd, cam, spp, depth, first=0, lt_mode=0, sigma=0.5, mis_mode=0, scene=None, aim=True):
    from paper_1705_01263_gb300 import rt
    scene = scene or rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    film.seek(first)
    splat = torch.zeros((cam.height, cam.width, 3), dtype=torch.float64, device="cuda")
    opts = rt.make_opts(sigma=sigma, mis_mode=mis_mode, lt_emission=0 if aim else 1)
    stats = rt.rt_render_two_way(scene, cam, spp, depth, film, opts, lt_mode=lt_mode, lt_splat=splat)
    torch.cuda.synchronize()
    s, s2, c = film.download()
    return s, s2, c, splat.cpu().numpy(), stats


@pytest.mark.parametrize("name,depth,lt_mode,mis_mode,sigma,aim", [
    ("glossy", 3, 0, 0, 0.5, True), ("glossy", 3, 0, 1, 0.5, True), ("glossy", 3, 1, 0, 0.5, True),
    ("cornell", 4, 0, 0, 0.5, True), ("cornell", 4, 0, 0, 0.0, True), ("many", 3, 0, 0, 0.5, True),
    ("cornell-env", 3, 0, 0, 0.5, True), ("cornell-env", 3, 1, 0, 0.5, True), ("turntable", 3, 0, 0, 0.5, True),
    ("turntable", 3, 0, 1, 0.5, True), ("glossy", 3, 0, 0, 0.5, False), ("cornell-env", 3, 1, 0, 0.5, False)])
def test_two_way_matches_the_oracle_on_the_same_samples(name, depth, lt_mode, mis_mode, sigma, aim):
    sd, cam = _scene(name, 32)
    s, s2, c, sp, stats = two_way_gpu(sd, cam, 64, depth, lt_mode=lt_mode, sigma=sigma, mis_mode=mis_mode, aim=aim)
    S, S2, C, SP, _ = oracle.Scene(sd).render_two_way(cam, 64, depth, sigma=sigma, mis_mode=mis_mode,
                                                      lt_mode=lt_mode, aim=aim)
    assert np.array_equal(c, C)
    assert stats.paths == 64 * 32 * 32 and stats.extension_rays > 0 and stats.shadow_rays > 0
    # camera stage: per pixel within 4 sigma of its own noise
    mg, vg = oracle.resolve(s, s2, c)
    mo, vo = oracle.resolve(S, S2, C)
    l1, out, n = image_parity(mg, vg, mo, vo)
    assert l1 <= 0.02, l1
    assert out <= allowed_4sigma(n), (out, n)
    # light stage: the splat images agree pixel by pixel (the same light
    # paths; FP32 against FP64 only moves a few paths)
    l1s = np.abs(sp - SP).sum() / SP.sum()
    assert l1s <= 0.02, l1s
    blk_g = sp.reshape(8, 4, 8, 4, 3).sum(axis=(1, 3))
    blk_o = SP.reshape(8, 4, 8, 4, 3).sum(axis=(1, 3))
    assert np.abs(blk_g - blk_o).max() <= 0.05 * blk_o.max(), np.abs(blk_g - blk_o).max() / blk_o.max()
    assert SP.sum() > 0.05 * S.sum()   # the light stage carries part of the image


@pytest.mark.parametrize("name", ["glossy", "cornell-env"])
def test_two_way_has_the_path_tracers_expectation(name):
    """The combined image (8 batches of 256 iterations) against rt_render at
    4096 iterations from a disjoint range, per 4 x 4 pixel block."""
    from paper_1705_01263_gb300 import rt
    sd, cam = _scene(name, 32)
    scene = rt.Scene(sd)
    K = 8
    blocks = []
    for k in range(K):
        s, s2, c, sp, _ = two_way_gpu(sd, cam, 256, 3, first=k * 256, scene=scene)
        blocks.append(((s + sp) / c[..., None]).reshape(8, 4, 8, 4, 3).mean(axis=(1, 3)))
    blocks = np.array(blocks)
    m_tw, se_tw = blocks.mean(axis=0), blocks.std(axis=0, ddof=1) / np.sqrt(K)
    film = rt.Film(cam.width, cam.height)
    film.seek(1 << 20)
    rt.rt_render(scene, cam, 4096, 3, film)
    S, S2, C = film.download()
    mean, var = oracle.resolve(S, S2, C)
    m_pt = mean.reshape(8, 4, 8, 4, 3).mean(axis=(1, 3))
    se_pt = np.sqrt(var.reshape(8, 4, 8, 4, 3).mean(axis=(1, 3)) / 16.0)
    z = np.abs(m_tw - m_pt) / np.sqrt(se_tw ** 2 + se_pt ** 2 + 1e-30)
    assert z.max() < 4.5, z.max()
    assert m_tw.mean() == pytest.approx(m_pt.mean(), rel=0.02)


def test_two_way_lowers_the_error_in_the_glossy_room():
    from paper_1705_01263_gb300 import rt
    sd, cam = _scene("glossy", 64)
    scene = rt.Scene(sd)
    s, s2, c, sp, _ = two_way_gpu(sd, cam, 4096, 4, first=1 << 20, scene=scene)
    ref = (s + sp) / c[..., None]
    film = rt.Film(cam.width, cam.height)
    rt.rt_render(scene, cam, 64, 4, film)
    S, S2, C = film.download()
    e_pt = np.sqrt(((S / C[..., None] - ref) ** 2).mean())
    s, s2, c, sp, _ = two_way_gpu(sd, cam, 64, 4, scene=scene)
    e_tw = np.sqrt((((s + sp) / c[..., None] - ref) ** 2).mean())
    assert e_tw < 0.5 * e_pt, (e_tw, e_pt)


def test_two_way_splats_into_the_film_without_a_buffer():
    from paper_1705_01263_gb300 import rt
    sd, cam = _scene("cornell", 16)
    scene = rt.Scene(sd)
    s, s2, c, sp, _ = two_way_gpu(sd, cam, 16, 3, scene=scene)
    film = rt.Film(cam.width, cam.height)
    rt.rt_render_two_way(scene, cam, 16, 3, film)
    S, S2, C = film.download()
    assert np.array_equal(C, c)
    np.testing.assert_allclose(S, s + sp, rtol=1e-9, atol=1e-12)


def test_two_way_refuses_what_it_does_not_combine():
    from paper_1705_01263_gb300 import rt
    sd, cam = _scene("cornell", 16)
    scene = rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    with pytest.raises(rt.RtError):
        rt.rt_render_two_way(scene, cam, 1, 3, film, rt.make_opts(mis_mode=2))
    with pytest.raises(rt.RtError):
        rt.rt_render_two_way(scene, cam, 1, 3, film, lt_mode=2)


@pytest.mark.parametrize("light_bvh", [False, True])
def test_instanced_two_way_has_the_path_tracers_expectation(light_bvh):
    """Two-level scene (emitters are (instance, triangle) pairs): the combined
    image against rt_render on the same scene, per 4 x 4 pixel block."""
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.instanced_field(n_meshes=6, n_instances=60, total_tris=30_000, n_emissive=300, width=32,
                                     height=32, min_tris=200, max_tris=4000)
    sd.light_bvh = light_bvh
    scene = rt.Scene(sd)
    K = 8
    blocks = []
    for k in range(K):
        s, s2, c, sp, _ = two_way_gpu(sd, cam, 128, 3, first=k * 128, scene=scene)
        blocks.append(((s + sp) / c[..., None]).reshape(8, 4, 8, 4, 3).mean(axis=(1, 3)))
    blocks = np.array(blocks)
    m_tw, se_tw = blocks.mean(axis=0), blocks.std(axis=0, ddof=1) / np.sqrt(K)
    assert sp.sum() > 0.0
    film = rt.Film(cam.width, cam.height)
    film.seek(1 << 20)
    rt.rt_render(scene, cam, 4096, 3, film)
    S, S2, C = film.download()
    mean, var = oracle.resolve(S, S2, C)
    m_pt = mean.reshape(8, 4, 8, 4, 3).mean(axis=(1, 3))
    se_pt = np.sqrt(var.reshape(8, 4, 8, 4, 3).mean(axis=(1, 3)) / 16.0)
    z = np.abs(m_tw - m_pt) / np.sqrt(se_tw ** 2 + se_pt ** 2 + 1e-30)
    assert z.max() < 4.5, z.max()
    assert m_tw.mean() == pytest.approx(m_pt.mean(), rel=0.03)


@pytest.mark.parametrize("name,lt_mode", [("glossy", 0), ("cornell-env", 0), ("cornell-env", 1), ("turntable", 0)])
def test_two_way_splats_match_the_oracle_per_pixel(name, lt_mode):
    """The light stage's splat image against the oracle's on the same light
    paths, pixel by pixel: K batches of iterations give both sides a
    per-pixel mean and a standard error (the spread of the batch splats);
    every pixel channel within 4 sigma, up to the Gaussian allowance."""
    from paper_1705_01263_gb300 import rt
    sd, cam = _scene(name, 32)
    scene = rt.Scene(sd)
    osc = oracle.Scene(sd)
    K, per = 8, 16
    g, o = [], []
    for k in range(K):
        _, _, _, sp, _ = two_way_gpu(sd, cam, per, 3, first=k * per, lt_mode=lt_mode, scene=scene)
        _, _, _, SP, _ = osc.render_two_way(cam, per, 3, iter0=k * per, lt_mode=lt_mode)
        g.append(sp / per)
        o.append(SP / per)
    g, o = np.array(g), np.array(o)
    mg, mo = g.mean(axis=0), o.mean(axis=0)
    var = g.var(axis=0, ddof=1) / K + o.var(axis=0, ddof=1) / K
    out = np.abs(mg - mo) > 4 * np.sqrt(var) + 1e-9 * np.maximum(np.abs(mo), 1e-3)
    assert out.sum() <= allowed_4sigma(out.size), (int(out.sum()), out.size)
    assert mo.sum() > 0 and np.abs(mg - mo).sum() <= 0.02 * mo.sum()
