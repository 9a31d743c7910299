"""Batched rendering of many scenes in one wavefront replayed as a CUDA graph
(row A14, not in the paper), and the autotuner: every film equals what
rt_render gives for that job alone."""
import numpy as np
import pytest

import oracle
from paper_1705_01263_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_jobs():
    from paper_1705_01263_gb300 import rt
    out = []
    sd, cam = scenes.cornell_box()
    out.append((rt.Scene(sd), cam, 8, 8))
    sd, cam = scenes.sphere_field(n_spheres=20, plane_res=(60, 30), env_size=(256, 128), width=120, height=68)
    out.append((rt.Scene(sd), cam, 4, 12))
    sd, cam = scenes.furnace_sphere(res=32)
    out.append((rt.Scene(sd), cam, 16, 4))
    sd, cam = scenes.instanced_field(n_meshes=5, n_instances=40, total_tris=50_000, n_emissive=500, width=64,
                                     height=36, min_tris=500, max_tris=3000)
    out.append((rt.Scene(sd), cam, 6, 6))
    return out


def individual(jobs):
    from paper_1705_01263_gb300 import rt
    res = []
    for s, cam, spp, d in jobs:
        f = rt.Film(cam.width, cam.height)
        rt.rt_render(s, cam, spp, d, f)
        res.append(f.download())
    return res


@pytest.mark.parametrize("cap", [0, 5000])
def test_batch_equals_individual_renders(cap):
    from paper_1705_01263_gb300 import rt
    jobs = make_jobs()
    ref = individual(jobs)
    films = [rt.Film(cam.width, cam.height) for _, cam, _, _ in jobs]
    stats = rt.rt_stats()
    rt.rt_render_batch([(s, cam, spp, d, f) for (s, cam, spp, d), f in zip(jobs, films)],
                       rt.make_opts(max_paths=cap, stats=stats))
    torch.cuda.synchronize()
    total = sum(cam.width * cam.height * spp for _, cam, spp, _ in jobs)
    assert stats.paths == total
    for (s_ref, s2_ref, c_ref), f, (_, _, spp, _) in zip(ref, films, jobs):
        s, s2, c = f.download()
        assert np.array_equal(c, c_ref) and np.all(c == spp)
        assert np.allclose(s, s_ref, rtol=1e-5, atol=1e-9)
        assert f.next_iteration() == spp


def test_batch_abort_and_resume():
    from paper_1705_01263_gb300 import rt
    jobs = make_jobs()
    ref = individual(jobs)
    films = [rt.Film(cam.width, cam.height) for _, cam, _, _ in jobs]
    flag = np.ones(1, np.int32)
    spec = [(s, cam, spp, d, f) for (s, cam, spp, d), f in zip(jobs, films)]
    st = rt.rt_render_batch(spec, rt.make_opts(max_paths=20000, abort_flag=flag.ctypes.data), allow_timeout=True)
    assert st == rt.RT_TIMEOUT
    # resume: each film continues from its own next iteration
    done = [f.next_iteration() for f in films]
    assert min(done) < max(s for _, _, s, _ in jobs)
    rest = []
    for (s, cam, spp, d), f in zip(jobs, films):
        # a job interrupted inside a pass resumes at its next task: render the
        # remaining passes one job at a time
        rt.rt_render(s, cam, spp - f.next_iteration(), d, f)
    torch.cuda.synchronize()
    for (s_ref, s2_ref, c_ref), f in zip(ref, films):
        s, s2, c = f.download()
        assert np.array_equal(c, c_ref)
        assert np.allclose(s, s_ref, rtol=1e-5, atol=1e-9)


def test_autotune_picks_a_candidate_and_renders():
    from paper_1705_01263_gb300 import rt
    jobs = make_jobs()
    films = [rt.Film(cam.width, cam.height) for _, cam, _, _ in jobs]
    spec = [(s, cam, spp, d, f) for (s, cam, spp, d), f in zip(jobs, films)]
    o = rt.rt_autotune(spec, 1)
    assert o.max_paths_in_flight in (1 << 20, 1 << 21, 1 << 22, 1 << 23)
    assert o.block_size in (0, 64, 96, 128)   # 0: none beat the first stage (128)
    o1 = rt.rt_autotune(spec[:1], 1)
    assert o1.trace_kernel in (0, 1) and o1.tail_threshold in (1, 8192, 65536)
    for f in films:
        f.clear()
    rt.rt_render_batch(spec, o)
    torch.cuda.synchronize()
    for f, (_, _, spp, _) in zip(films, jobs):
        assert np.all(f.download()[2] == spp)


def test_batch_with_per_job_guides():
    """Jobs carrying their own guiding network: each is rendered with its
    network (which trains during the call) and converges to the oracle's
    reference; the jobs without one equal their individual renders."""
    from paper_1705_01263_gb300 import rt
    from helpers import allowed_4sigma
    jobs = make_jobs()
    ref = individual(jobs)
    sd, cam = scenes.cornell_box()
    cscene = rt.Scene(sd)
    guides = [rt.Guide(cscene, seed=5), rt.Guide(cscene, seed=6)]
    p0 = [g.get_params() for g in guides]
    gfilms = [rt.Film(cam.width, cam.height) for _ in guides]
    films = [rt.Film(c.width, c.height) for _, c, _, _ in jobs]
    spec = [(s, c, spp, d, f) for (s, c, spp, d), f in zip(jobs, films)]
    spec += [(cscene, cam, 1024, 8, f, g) for f, g in zip(gfilms, guides)]
    stats = rt.rt_stats()
    rt.rt_render_batch(spec, rt.make_opts(stats=stats))
    torch.cuda.synchronize()
    total = sum(c.width * c.height * spp for _, c, spp, _ in jobs) + 2 * cam.width * cam.height * 1024
    assert stats.paths == total
    for (s_ref, s2_ref, c_ref), f in zip(ref, films):
        s, s2, c = f.download()
        assert np.array_equal(c, c_ref)
        assert np.allclose(s, s_ref, rtol=1e-5, atol=1e-9)
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "cornell_64_depth8_ref.npz"))
    mr, vr = d["mean"], d["var"]   # FP64 oracle, 2^15 spp from iteration 2^20
    for g, q0, f in zip(guides, p0, gfilms):
        assert not np.array_equal(q0, g.get_params())
        s, s2, c = f.download()
        assert np.all(c == 1024)
        mg, vg = oracle.resolve(s, s2, c)
        out = int((np.abs(mg - mr) > 4 * np.sqrt(vg + vr) + 1e-6).sum())
        assert out <= allowed_4sigma(mg.size), out
    with pytest.raises(rt.RtError):
        rt.rt_autotune(spec, 1)


def test_block_size_changes_nothing_but_speed():
    """rt_render_opts.block_size (64, 96 or 128 threads per block of the
    state kernels) gives bit-identical films; other sizes are rejected."""
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.cornell_box()
    s = rt.Scene(sd)
    out = []
    for b in (0, 64, 96):
        f = rt.Film(cam.width, cam.height)
        rt.rt_render(s, cam, 8, 8, f, rt.make_opts(block_size=b))
        out.append(f.download())
    for o in out[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(o, out[0]))
    for bad in (48, 256):
        with pytest.raises(rt.RtError):
            rt.rt_render(s, cam, 1, 4, rt.Film(cam.width, cam.height), rt.make_opts(block_size=bad))


def test_sixty_four_guided_jobs_in_one_wavefront():
    """64 jobs, each with its own guiding network, in one rt_render_batch
    call: one shared wavefront over the jobs' interleaved tasks, every
    network trained during the call on its own paths' samples; every job's
    film converges to the FP64 oracle's reference (per pixel within 4
    sigma, up to the Gaussian allowance)."""
    import os
    from paper_1705_01263_gb300 import rt
    from helpers import allowed_4sigma
    sd, cam = scenes.cornell_box()
    scene = rt.Scene(sd)
    guides = [rt.Guide(scene, seed=100 + k, train_every=4) for k in range(64)]
    p0 = [g.get_params() for g in guides]
    films = [rt.Film(cam.width, cam.height) for _ in guides]
    # 1024 spp, as the other guided parity tests: at a few hundred samples
    # the per-pixel spread of this scene's QMC estimate (plain or guided)
    # still leaves more than the Gaussian allowance of pixels beyond 4 sigma
    spp = 1024
    stats = rt.rt_stats()
    rt.rt_render_batch([(scene, cam, spp, 8, f, g) for f, g in zip(films, guides)], rt.make_opts(stats=stats))
    torch.cuda.synchronize()
    assert stats.paths == 64 * cam.width * cam.height * spp and stats.waves > 1
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "cornell_64_depth8_ref.npz"))
    mr, vr = d["mean"], d["var"]
    trained = 0
    for g, q0, f in zip(guides, p0, films):
        trained += not np.array_equal(q0, g.get_params())
        s, s2, c = f.download()
        assert np.all(c == spp)
        mg, vg = oracle.resolve(s, s2, c)
        out = int((np.abs(mg - mr) > 4 * np.sqrt(vg + vr) + 1e-6).sum())
        assert out <= allowed_4sigma(mg.size), out
    assert trained == 64
