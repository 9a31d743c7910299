"""Guided rendering (not in the paper): the one-sample MIS mixture of the
trained vMF proposal and the BSDF keeps the estimator consistent, so the
guided image must agree with the oracle's high-sample reference within its
own Monte Carlo error; training must run during the render."""
import os

import numpy as np
import pytest

import oracle
from helpers import allowed_4sigma
from paper_1705_01263_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cornell_64_depth8_ref.npz")


def reference():
    """Oracle reference of the Cornell configuration (stored, written by
    tests/golden/make_cornell_reference.py); falls back to 1024 spp here."""
    if os.path.exists(GOLDEN):
        d = np.load(GOLDEN)
        return d["mean"], d["var"]
    sd, cam = scenes.cornell_box()
    S, S2, C, _ = oracle.Scene(sd).render(cam, 1024, 8)
    return oracle.resolve(S, S2, C)


def test_guided_render_is_consistent_with_the_oracle():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    guide = rt.Guide(scene, seed=5)
    p0 = guide.get_params()
    film = rt.Film(cam.width, cam.height)
    stats = rt.rt_stats()
    # 1024 spp: the per-pixel 4-sigma test needs the QMC error past its early
    # transient (the plain tracer fails it at 128 spp just the same)
    rt.rt_render(scene, cam, 1024, 8, film, rt.make_opts(guide=guide, stats=stats))
    torch.cuda.synchronize()
    assert stats.waves == 64                     # 16 spp per iteration set
    assert not np.array_equal(p0, guide.get_params())   # trained during the render
    s, s2, c = film.download()
    assert np.all(c == 1024)
    mg, vg = oracle.resolve(s, s2, c)
    mr, vr = reference()
    sig = np.sqrt(vg + vr)
    out = int((np.abs(mg - mr) > 4 * sig + 1e-6).sum())
    assert out <= allowed_4sigma(mg.size), out
    # the image mean agrees within 4 sigma of its estimate
    d = abs(mg.mean() - mr.mean())
    s_tot = np.sqrt(vg.sum() + vr.sum()) / mg.size
    assert d <= 4 * s_tot + 1e-4 * mr.mean(), (d, s_tot)


def test_guided_and_plain_agree_in_mean():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    guide = rt.Guide(scene, seed=6)
    a = rt.Film(cam.width, cam.height)
    b = rt.Film(cam.width, cam.height)
    rt.rt_render(scene, cam, 64, 8, a, rt.make_opts(guide=guide))
    rt.rt_render(scene, cam, 64, 8, b)
    torch.cuda.synchronize()
    ma, va = oracle.resolve(*a.download())
    mb, vb = oracle.resolve(*b.download())
    d = abs(ma.mean() - mb.mean())
    s_tot = np.sqrt(va.sum() + vb.sum()) / ma.size
    assert d <= 4 * s_tot + 1e-4 * mb.mean(), (d, s_tot)
