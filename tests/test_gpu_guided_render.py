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

GOLDEN = {"down": os.path.join(os.path.dirname(__file__), "golden", "cornell_64_depth8_ref.npz"),
          "up": os.path.join(os.path.dirname(__file__), "golden", "cornell_up_64_depth8_ref.npz"),
          "door": os.path.join(os.path.dirname(__file__), "golden", "cornell_door_64_depth8_ref.npz")}


def reference(light="down"):
    """Oracle reference of the Cornell configuration (stored, written by
    tests/golden/make_cornell_reference.py); falls back to 1024 spp here."""
    if os.path.exists(GOLDEN[light]):
        d = np.load(GOLDEN[light])
        return d["mean"], d["var"]
    sd, cam = scenes.cornell_box(light=light)
    S, S2, C, _ = oracle.Scene(sd).render(cam, 1024, 8)
    return oracle.resolve(S, S2, C)


@pytest.mark.parametrize("pool,gdepth,warm", [(0, 0, 0), (65536, 0, 0), (0, 1, 8), (0, 2, 0), (0, 64, 0)])
def test_guided_render_is_consistent_with_the_oracle(pool, gdepth, warm):
    """pool 0: the library's iteration sets; 65536: 16 spp per set, so that
    a training step follows every set; gdepth 1 or 2: only the first vertices
    guided (BSDF sampling and its MIS weights beyond them); 0: the default
    (vertices 1-3); 64: every vertex."""
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    guide = rt.Guide(scene, seed=5, guide_depth=gdepth, warm_steps=warm)
    p0 = guide.get_params()
    film = rt.Film(cam.width, cam.height)
    stats = rt.rt_stats()
    # 1024 spp: the per-pixel 4-sigma test needs the QMC error past its early
    # transient (the plain tracer fails it at 128 spp just the same)
    rt.rt_render(scene, cam, 1024, 8, film, rt.make_opts(guide=guide, stats=stats, max_paths=pool))
    torch.cuda.synchronize()
    # a warm-up set, then at least one trained set (16 spp each with pool 65536)
    assert stats.waves >= 2
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


def test_guided_render_consistent_on_room_lit_through_the_ceiling():
    """The emitter faces the ceiling: every pixel is lit through a bright
    patch that BSDF sampling finds rarely, the case the proposal changes
    most. The estimator is heavy-tailed there (the plain tracer exceeds the
    per-pixel 4-sigma bound on ~3% of the channels at 1024 spp), so at 4096
    spp the guided image must agree with the oracle reference at least as
    well as the plain tracer does, and in the image mean within 4 sigma."""
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box(light="up")
    scene = rt.Scene(sd)
    mr, vr = reference("up")
    res = {}
    for name, guide in (("plain", None), ("guided", rt.Guide(scene, seed=5))):
        film = rt.Film(cam.width, cam.height)
        rt.rt_render(scene, cam, 4096, 8, film, rt.make_opts(guide=guide))
        torch.cuda.synchronize()
        mg, vg = oracle.resolve(*film.download())
        sig = np.sqrt(vg + vr)
        out = int((np.abs(mg - mr) > 4 * sig + 1e-6).sum())
        d = abs(mg.mean() - mr.mean())
        s_tot = np.sqrt(vg.sum() + vr.sum()) / mg.size
        res[name] = (out, d, s_tot)
        assert d <= 4 * s_tot + 1e-4 * mr.mean(), (name, d, s_tot)
    assert res["guided"][0] <= max(allowed_4sigma(mr.size), 2 * res["plain"][0]), res


def test_guided_render_consistent_in_the_room_lit_through_a_door():
    """The room lit from a closed side chamber through a door: both tracers
    at 4096 spp against the stored oracle reference (2^17 spp) — every pixel
    but the few the per-pixel 4-sigma rule allows (the guided image at most
    twice the plain tracer's count) and the image mean within 4 sigma."""
    from paper_1705_01263_gb300 import rt
    if not os.path.exists(GOLDEN["door"]):
        pytest.skip("stored reference missing")
    sd, cam = scenes.door_room()
    scene = rt.Scene(sd)
    d = np.load(GOLDEN["door"])
    mr, vr = d["mean"], d["var"]
    res = {}
    for name, guide in (("plain", None), ("guided", rt.Guide(scene, seed=5))):
        film = rt.Film(cam.width, cam.height)
        rt.rt_render(scene, cam, 4096, 8, film, rt.make_opts(guide=guide))
        torch.cuda.synchronize()
        mg, vg = oracle.resolve(*film.download())
        sig = np.sqrt(vg + vr)
        out = int((np.abs(mg - mr) > 4 * sig + 1e-6).sum())
        dm = abs(mg.mean() - mr.mean())
        s_tot = np.sqrt(vg.sum() + vr.sum()) / mg.size
        res[name] = (out, dm, s_tot)
        assert dm <= 4 * s_tot + 1e-4 * mr.mean(), (name, dm, s_tot)
    assert res["guided"][0] <= max(allowed_4sigma(mr.size), 2 * res["plain"][0]), res


@pytest.mark.parametrize("wsb", [1, 4])
def test_warm_up_schedules_train_and_stay_consistent(wsb):
    """Warm-up sets of `wsb` training batches (1: a step after each set of
    2^16 paths): the network takes its warm-up steps and the image agrees in
    mean with the plain tracer's."""
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box(light="up")
    scene = rt.Scene(sd)
    guide = rt.Guide(scene, seed=9, warm_set_batches=wsb, warm_steps=8)
    p0 = guide.get_params()
    a = rt.Film(cam.width, cam.height)
    b = rt.Film(cam.width, cam.height)
    stats = rt.rt_stats()
    rt.rt_render(scene, cam, 512, 8, a, rt.make_opts(guide=guide, stats=stats))
    rt.rt_render(scene, cam, 512, 8, b)
    torch.cuda.synchronize()
    assert not np.array_equal(p0, guide.get_params())
    assert stats.waves >= 2
    ma, va = oracle.resolve(*a.download())
    mb, vb = oracle.resolve(*b.download())
    d = abs(ma.mean() - mb.mean())
    s_tot = np.sqrt(va.sum() + vb.sum()) / ma.size
    assert d <= 4 * s_tot + 1e-4 * mb.mean(), (d, s_tot)


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


def test_trained_guide_reduces_error_per_sample():
    """What the network gains: on the room lit through the ceiling, after
    online training, a guided render of the same number of samples is closer
    to the oracle reference than the plain tracer's (per-sample efficiency;
    wall-clock time to equal error is measured by bench.py)."""
    from paper_1705_01263_gb300 import rt
    if not os.path.exists(GOLDEN["up"]):
        pytest.skip("stored reference missing")
    sd, cam = scenes.cornell_box(light="up")
    scene = rt.Scene(sd)
    ref = np.load(GOLDEN["up"])["mean"]
    guide = rt.Guide(scene, seed=5, train_steps=4)
    warm = rt.Film(cam.width, cam.height)
    warm.seek(1 << 20)       # training samples from another part of the sequence
    rt.rt_render(scene, cam, 2048, 8, warm, rt.make_opts(guide=guide, max_paths=65536))
    rmse = {}
    for name, g in (("plain", None), ("guided", guide)):
        f = rt.Film(cam.width, cam.height)
        rt.rt_render(scene, cam, 1024, 8, f, rt.make_opts(guide=g))
        torch.cuda.synchronize()
        m, _ = oracle.resolve(*f.download())
        rmse[name] = float(np.sqrt(np.mean((m - ref) ** 2)))
    assert rmse["guided"] < 0.8 * rmse["plain"], rmse
