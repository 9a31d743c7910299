"""The allocation-free render entry point (rt_render_static) must give what
rt_render gives, on two calls in a row through the C ABI. It exists for
callers that cannot allocate device memory (a framework that owns all device
allocations, a fixed start-up memory budget, threads where an allocation
would stall the device); it renders with a fixed device array instead.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1705_01263_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_render_matches_rt_render_on_two_calls():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    spp, depth = 8, 8
    ref = rt.Film(cam.width, cam.height)
    rt.rt_render(scene, cam, spp, depth, ref)
    s_ref, s2_ref, c_ref = ref.download()
    for call in range(2):
        s = torch.zeros((cam.height, cam.width, 3), dtype=torch.float64, device="cuda")
        s2 = torch.zeros_like(s)
        c = torch.zeros((cam.height, cam.width), dtype=torch.int32, device="cuda")
        rt.rt_render_static(scene, cam, spp, depth, 0, s, s2, c)
        torch.cuda.synchronize()
        assert np.array_equal(c.cpu().numpy().view(np.uint32), c_ref), call
        # same samples and kernels; only the path pool size differs, which can
        # move a path between the wavefront kernels and the megakernel
        assert np.allclose(s.cpu().numpy(), s_ref, rtol=1e-5, atol=1e-9), call
        assert np.allclose(s2.cpu().numpy(), s2_ref, rtol=1e-5, atol=1e-9), call


def test_static_render_rejects_oversized_pool():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    s = torch.zeros((cam.height, cam.width, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros((cam.height, cam.width), dtype=torch.int32, device="cuda")
    with pytest.raises(rt.RtError) as e:
        rt.rt_render_static(scene, cam, 1, 4, 0, s, s.clone(), c, rt.make_opts(max_paths=65537))
    assert e.value.status == 1


def test_static_render_partial_iterations_resume_and_seed_change():
    """An image above the 65,536-path pool (each iteration is split over
    several calls' worth of sets), rendered as iterations [0, 2) then [2, 4)
    with a call of another seed in between (which rewrites the shared
    sampling table and leaves the pool dirty), equals rt_render of 4
    iterations with the first seed."""
    import dataclasses
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    cam = dataclasses.replace(cam, width=320, height=240)
    scene = rt.Scene(sd)
    depth = 6
    ref = rt.Film(cam.width, cam.height)
    rt.rt_render(scene, cam, 4, depth, ref, rt.make_opts(seed=5))
    s_ref, s2_ref, c_ref = ref.download()
    s = torch.zeros((cam.height, cam.width, 3), dtype=torch.float64, device="cuda")
    s2 = torch.zeros_like(s)
    c = torch.zeros((cam.height, cam.width), dtype=torch.int32, device="cuda")
    rt.rt_render_static(scene, cam, 2, depth, 0, s, s2, c, rt.make_opts(seed=5))
    o = torch.zeros_like(s)
    rt.rt_render_static(scene, cam, 1, depth, 7, o, o.clone(), torch.zeros_like(c), rt.make_opts(seed=77))
    rt.rt_render_static(scene, cam, 2, depth, 2, s, s2, c, rt.make_opts(seed=5))
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy().view(np.uint32), c_ref)
    assert np.allclose(s.cpu().numpy(), s_ref, rtol=1e-5, atol=1e-9)
    assert np.allclose(s2.cpu().numpy(), s2_ref, rtol=1e-5, atol=1e-9)
    # the other seed's samples are not the same image
    assert not np.allclose(o.cpu().numpy(), s_ref / 4, rtol=1e-3)


def test_static_render_rejects_sorted_queues():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    s = torch.zeros((cam.height, cam.width, 3), dtype=torch.float64, device="cuda")
    c = torch.zeros((cam.height, cam.width), dtype=torch.int32, device="cuda")
    for field in ("sort_by_material", "sort_rays"):
        o = rt.make_opts()
        setattr(o, field, 1)
        with pytest.raises(rt.RtError) as e:
            rt.rt_render_static(scene, cam, 1, 4, 0, s, s.clone(), c, o)
        assert e.value.status == 7
