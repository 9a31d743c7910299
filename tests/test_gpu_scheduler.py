"""The regeneration scheduler (Sec. 3.1.3: ended paths are replaced by new
ones once more than half the pool has ended) and the device-side timeout
(Appendix A.4: the kernels stop starting paths when the host-mapped abort
word is set or the device clock passes the deadline). Its films equal the
iteration-set scheduler's bit for bit (the same per-path arithmetic, each
pixel's samples added in sample order) whatever the pool size and refill
fraction; a render stopped by the abort flag or the time budget holds a
contiguous range of completed tasks and resumes to the uninterrupted
film."""
import dataclasses
import threading
import time

import numpy as np
import pytest

from paper_1705_01263_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def field():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.sphere_field()
    return sd, cam, rt.Scene(sd)


def render(scene, cam, spp, depth, film=None, **kw):
    from paper_1705_01263_gb300 import rt
    film = film or rt.Film(cam.width, cam.height)
    stats = rt.rt_stats()
    allow = kw.pop("allow_timeout", False)
    st = rt.rt_render(scene, cam, spp, depth, film, rt.make_opts(stats=stats, **kw), allow_timeout=allow)
    torch.cuda.synchronize()
    return film, stats, st


def small(cam, w, h):
    return dataclasses.replace(cam, width=w, height=h)


@pytest.mark.parametrize("pool,frac", [(65536, 0.0), (65536, 0.25), (200_000, 1.0), (1 << 20, 0.5)])
def test_regeneration_equals_iteration_sets_bit_for_bit(field, pool, frac):
    """Without the megakernel tail (whose FP32 operation order differs) the
    two schedulers give identical sums, sums of squares and counts."""
    sd, cam, scene = field
    cam = small(cam, 320, 180)
    a, sa, _ = render(scene, cam, 16, 16, scheduler=1, tail_threshold=1)
    b, sb, _ = render(scene, cam, 16, 16, max_paths=pool, regen_fraction=frac, tail_threshold=1)
    A, B = a.download(), b.download()
    for x, y in zip(A, B):
        assert np.array_equal(x, y)
    assert sb.paths == 16 * 320 * 180 and sb.waves == 1
    if pool < 16 * 320 * 180:
        assert sb.regen_sets > 0
    assert sa.extension_rays == sb.extension_rays and sa.shadow_rays == sb.shadow_rays


@pytest.mark.parametrize("pool,frac", [(1 << 21, 0.5), (3 << 20, 0.0)])
def test_two_half_pools_equal_iteration_sets_bit_for_bit(field, pool, frac):
    """A pool of at least 2^21 slots that refills runs as two half-pools on
    two streams, each with half of the window's tasks; the film, the ray
    counts and the sample counts are those of the iteration-set scheduler."""
    sd, cam, scene = field
    cam = small(cam, 640, 360)
    a, sa, _ = render(scene, cam, 16, 16, scheduler=1, tail_threshold=1)
    b, sb, _ = render(scene, cam, 16, 16, max_paths=pool, regen_fraction=frac, tail_threshold=1)
    A, B = a.download(), b.download()
    for x, y in zip(A, B):
        assert np.array_equal(x, y)
    assert sb.paths == 16 * 640 * 360 and sb.regen_sets > 0
    assert sa.extension_rays == sb.extension_rays and sa.shadow_rays == sb.shadow_rays
    # and with the megakernel tail (default threshold) every task is still done once
    c, sc, _ = render(scene, cam, 16, 16, max_paths=pool, regen_fraction=frac)
    assert np.all(c.download()[2] == 16) and sc.paths == 16 * 640 * 360


def test_regeneration_with_tail_and_sorting_matches(field):
    """With the megakernel tail and the sorted-queue options the film is the
    same up to FP32 operation order."""
    sd, cam, scene = field
    cam = small(cam, 256, 144)
    a, _, _ = render(scene, cam, 8, 12, scheduler=1)
    for kw in ({}, {"sort_by_material": True}, {"sort_rays": True}, {"trace_kernel": 3}):
        b, st, _ = render(scene, cam, 8, 12, max_paths=50_000, **kw)
        A, B = a.download(), b.download()
        assert np.array_equal(A[2], B[2]), kw
        assert np.allclose(A[0], B[0], rtol=1e-5, atol=1e-9), kw
        assert st.tail_launches >= 1 and st.regen_sets > 0


def test_abort_during_a_default_call_then_resume(field):
    """A second host thread raises the abort flag while a default call (the
    full 1080p sphere field, 64 spp) runs: the call returns RT_TIMEOUT with a
    contiguous range of completed tasks in the film, and a second call
    completes the request with the film equal to an uninterrupted render."""
    from paper_1705_01263_gb300 import rt
    sd, cam, scene = field
    ref, sref, _ = render(scene, cam, 64, 16)
    assert sref.paths == 64 * cam.width * cam.height
    flag = np.zeros(1, np.int32)
    film = rt.Film(cam.width, cam.height)
    out = {}

    def run():
        out["r"] = render(scene, cam, 64, 16, film=film, abort_flag=flag.ctypes.data, allow_timeout=True)

    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.03)
    flag[0] = 1
    th.join()
    _, st1, status = out["r"]
    WH = cam.width * cam.height
    assert status == rt.RT_TIMEOUT
    assert 0 < st1.paths < 64 * WH
    # the film holds exactly tasks [0, paths): sample counts per pixel
    _, _, c_mid = film.download()
    full, rem = divmod(st1.paths, WH)
    want = np.full(WH, full, np.uint32)
    want[:rem] += 1
    assert np.array_equal(c_mid.reshape(-1), want)
    assert film.next_iteration() == full
    flag[0] = 0
    _, st2, status = render(scene, cam, 64 - full, 16, film=film)
    assert status == rt.RT_OK and film.next_iteration() == 64
    assert st1.paths + st2.paths == 64 * WH
    A, B = ref.download(), film.download()
    assert np.array_equal(A[2], B[2])
    assert np.allclose(A[0], B[0], rtol=1e-5, atol=1e-9)
    assert np.allclose(A[1], B[1], rtol=1e-5, atol=1e-9)


def test_abort_flag_already_set_runs_one_pool_load(field):
    """Set before the call: the first pool load finishes, nothing more starts."""
    from paper_1705_01263_gb300 import rt
    sd, cam, scene = field
    cam = small(cam, 320, 180)
    flag = np.ones(1, np.int32)
    f, st, status = render(scene, cam, 16, 16, max_paths=100_000, abort_flag=flag.ctypes.data, allow_timeout=True)
    assert status == rt.RT_TIMEOUT and st.paths == 100_000


def test_time_budget_stops_on_the_device(field):
    """A 20 ms budget on a ~250 ms render stops it early, the film holds the
    completed task range, and the call returned soon after the budget (the
    paths in flight drain)."""
    from paper_1705_01263_gb300 import rt
    sd, cam, scene = field
    render(scene, small(cam, 64, 64), 1, 4)   # warm up
    t0 = time.perf_counter()
    f, st, status = render(scene, cam, 64, 16, time_budget_ms=20.0, allow_timeout=True)
    dt = time.perf_counter() - t0
    WH = cam.width * cam.height
    assert status == rt.RT_TIMEOUT and 0 < st.paths < 64 * WH
    assert dt < 0.2, dt
    _, _, c = f.download()
    full, rem = divmod(st.paths, WH)
    assert c.reshape(-1)[:rem].min() == full + 1 and c.reshape(-1)[rem:].max() == full


@pytest.mark.parametrize("scene_name", ["cornell", "field"])
def test_compressed_state_matches_the_oracle(scene_name):
    """State compression (Sec. 3.1.1, an A/B option of the regeneration
    scheduler: octahedral 16:16 directions, BF16 throughput and shadow
    contributions) against the FP64 oracle on the same samples: the same
    per-pixel 4 sigma and mean relative L1 bars as the uncompressed tracer,
    and within the same 1% mean relative L1 of the uncompressed render
    (quantised directions and throughputs move a few paths)."""
    import oracle
    from helpers import allowed_4sigma, image_parity
    from paper_1705_01263_gb300 import rt
    if scene_name == "cornell":
        sd, cam = scenes.cornell_box()
        spp, depth = 16, 8
    else:
        sd, cam = scenes.sphere_field(n_spheres=40, plane_res=(120, 60), env_size=(512, 256), width=160, height=90)
        spp, depth = 32, 8
    scene = rt.Scene(sd)
    a, _, _ = render(scene, cam, spp, depth, max_paths=20_000, state_compression=True)
    b, _, _ = render(scene, cam, spp, depth, max_paths=20_000)
    sa, s2a, ca = a.download()
    sb, s2b, cb = b.download()
    assert np.array_equal(ca, cb)
    S, S2, C, _ = oracle.Scene(sd).render(cam, spp, depth)
    mo, vo = oracle.resolve(S, S2, C)
    ma, va = oracle.resolve(sa, s2a, ca)
    l1, out, n = image_parity(ma, va, mo, vo)
    assert l1 <= 0.01 and out <= allowed_4sigma(n), (l1, out, n)
    mb, _ = oracle.resolve(sb, s2b, cb)
    assert np.abs(ma - mb).sum() / np.abs(mb).sum() < 1e-2


def test_compressed_state_is_rejected_where_unsupported():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    for kw in ({"scheduler": 1}, {"megakernel_only": True}):
        with pytest.raises(rt.RtError) as e:
            rt.rt_render(scene, cam, 1, 4, film, rt.make_opts(state_compression=True, **kw))
        assert e.value.status == 7
