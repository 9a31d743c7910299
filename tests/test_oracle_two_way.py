"""Pins of the oracle's two-way path tracing (Sec. 2: a path tracer and a light
tracer combined by multiple importance sampling):

- (environment photons included: the scene open to a sky)
- with the light tracer's density set to zero the camera stage, whose weights
  are products of area-measure densities over the stored vertices, is the
  path tracer of render.c, whose weights are a ratio of two solid-angle pdfs;
- every density is the density of the sampler it names: the light tracer's
  mean of p_hit / p_lt and p_nee / p_lt over its camera connections equals
  how often the camera side actually makes those paths (BSDF-sampled emitter
  hits and unoccluded next-event samples); a dropped cosine, a wrong pixel
  filter Jacobian or a misnamed direction in any density breaks the equality;
- the combined image, and the light tracer alone where it can make the path,
  have the path tracer's expectation (the weights sum to one);
- in a room lit through its ceiling with glossy surfaces the combination has
  a far lower error per sample than the path tracer.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes


def _scene(name, res=16):
    if name == "cornell":
        sd, cam = scenes.cornell_box()
    elif name == "cornell-up":
        sd, cam = scenes.cornell_box(light="up")
    elif name == "cornell-env":
        # the box is open towards the camera: a sky lights it too
        sd, cam = scenes.cornell_box()
        sd = dataclasses.replace(sd, env=scenes.procedural_sky(32, 16, seed=3)[0])
    elif name == "glossy":
        sd, cam = scenes.glossy_room()
    else:
        sd, cam = scenes.many_emitters(n_lights=64, res=res)
    return sd, dataclasses.replace(cam, width=res, height=res)


@pytest.mark.parametrize("name,mis_mode", [("cornell", 0), ("cornell", 1), ("glossy", 0), ("many", 0),
                                           ("cornell-env", 0)])
def test_camera_stage_without_the_light_tracer_is_the_path_tracer(name, mis_mode):
    sd, cam = _scene(name)
    s = oracle.Scene(sd)
    S, S2, C, _ = s.render(cam, 16, 4, mis_mode=mis_mode)
    T, T2, TC, SP, _ = s.render_two_way(cam, 16, 4, mis_mode=mis_mode, lt_mode=2)
    assert SP.sum() == 0.0
    assert np.array_equal(C, TC)
    # the two forms differ only by rounding (sharp GGX lobes make the area-measure
    # products large); a dropped or misplaced factor moves weights by O(1)
    np.testing.assert_allclose(T, S, rtol=1e-6, atol=1e-12 * float(S.max()))


def _chunks(s, cam, spp, D, K, lt_mode, first=0, **kw):
    out = []
    for c in range(K):
        S, S2, C, SP, _ = s.render_two_way(cam, spp, D, iter0=first + c * spp, lt_mode=lt_mode, **kw)
        out.append((S, SP, C))
    return out


# The glossy room stops at depth 2: deeper, the ratio of the GGX pdfs of the
# two directions of a vertex grows without bound at grazing angles and the
# light tracer's mean converges too slowly for a short test.
@pytest.mark.parametrize("name,D", [("cornell", 4), ("cornell-up", 3), ("glossy", 2), ("many", 2),
                                    ("cornell-env", 2)])
def test_every_density_is_the_density_of_its_sampler(name, D):
    sd, cam = _scene(name)
    s = oracle.Scene(sd)
    # 16 chunks: photon aiming leaves few photons where the camera looks
    # little, so single light paths there carry large density ratios and the
    # spread of 8 chunks underestimates the standard error
    K = 16
    cam_blk, lt_blk = [], []
    for S, SP, C in _chunks(s, cam, 128, D, K, lt_mode=3):
        n = C.sum()
        # per 4 x 4 pixel block and channel (0: emitter hits, 1: next-event samples)
        cam_blk.append(S[..., :2].reshape(4, 4, 4, 4, 2).sum(axis=(1, 3)) / n)
        lt_blk.append(SP[..., :2].reshape(4, 4, 4, 4, 2).sum(axis=(1, 3)) / n)
    d = np.array(cam_blk) - np.array(lt_blk)
    mean, se = d.mean(axis=0), d.std(axis=0, ddof=1) / np.sqrt(K)
    ref = np.array(cam_blk).mean(axis=0)
    assert np.all(np.abs(mean) <= 4.5 * se + 1e-9), (mean, se)
    tot_cam, tot_diff = ref.sum(axis=(0, 1)), mean.sum(axis=(0, 1))
    # over the image: within 3%, or within 4 standard errors where the counts
    # are rare (BSDF-sampled hits of small emitters: ~0.2% of paths)
    se_tot = d.sum(axis=(1, 2)).std(axis=0, ddof=1) / np.sqrt(K)
    assert np.all(np.abs(tot_diff) <= np.maximum(0.03 * tot_cam, 4.0 * se_tot)), (tot_diff, tot_cam, se_tot)
    assert tot_cam[0] > 0.001 and tot_cam[1] > 0.1   # both techniques were exercised


@pytest.mark.parametrize("name,lt_mode,mis_mode,sigma", [("glossy", 0, 0, 0.5), ("glossy", 0, 1, 0.5),
                                                        ("glossy", 1, 0, 0.5), ("glossy", 0, 0, 0.0),
                                                        ("many", 0, 0, 0.5), ("cornell-env", 0, 0, 0.5)])
def test_two_way_image_has_the_path_tracer_expectation(name, lt_mode, mis_mode, sigma):
    sd, cam = _scene(name)
    s = oracle.Scene(sd)
    K = 8
    blocks = []
    for S, SP, C in _chunks(s, cam, 64, 3, K, lt_mode=lt_mode, mis_mode=mis_mode, sigma=sigma):
        img = (S + SP) / C[..., None]
        blocks.append(img.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3)))
    blocks = np.array(blocks)
    m_tw, se_tw = blocks.mean(axis=0), blocks.std(axis=0, ddof=1) / np.sqrt(K)
    S, S2, C, _ = s.render(cam, 2048, 3, iter0=1 << 20, sigma=sigma, mis_mode=mis_mode)
    mean, var = oracle.resolve(S, S2, C)
    m_pt = mean.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3))
    se_pt = np.sqrt(var.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3)) / 16.0)
    z = np.abs(m_tw - m_pt) / np.sqrt(se_tw ** 2 + se_pt ** 2 + 1e-30)
    assert z.max() < 4.5, z.max()
    assert m_tw.mean() == pytest.approx(m_pt.mean(), rel=0.03)


def test_two_way_lowers_the_error_where_light_tracing_reaches_the_light():
    sd, cam = _scene("glossy")
    s = oracle.Scene(sd)
    D = 4
    ref = np.mean([(S + SP) / C[..., None] for S, SP, C in _chunks(s, cam, 256, D, 4, lt_mode=0, first=1 << 20)],
                  axis=0)
    S, S2, C, _ = s.render(cam, 32, D)
    e_pt = np.sqrt(((S / C[..., None] - ref) ** 2).mean())
    S, S2, C, SP, _ = s.render_two_way(cam, 32, D)
    e_tw = np.sqrt((((S + SP) / C[..., None] - ref) ** 2).mean())
    assert e_tw < 0.5 * e_pt, (e_tw, e_pt)
