"""Two-level (instanced) scenes with many textured emitters: GPU hits equal
the oracle's on the flattened scene ((instance, triangle) mapped to the
flattened index), images agree, and the full-size 10M-triangle scene builds
and renders."""
import numpy as np
import pytest

import oracle
from helpers import MISS, allowed_4sigma, image_parity
from paper_1705_01263_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def field():
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.instanced_field(n_meshes=10, n_instances=100, total_tris=200_000, n_emissive=2000, width=96,
                                     height=54, min_tris=500, max_tris=5000)
    flat = sd.flattened()
    return sd, flat, cam, rt.Scene(sd), oracle.Scene(flat)


def flat_index(sd, inst, prim):
    counts = np.diff(sd.mesh_tri_offset)[sd.instance_mesh]
    base = np.concatenate([[0], np.cumsum(counts)[:-1]])
    return base[inst] + (prim.astype(np.int64) - sd.mesh_tri_offset[sd.instance_mesh[inst]])


@pytest.mark.parametrize("kind", ["primary", "incoherent"])
def test_instanced_hits_match_flattened_oracle(field, kind):
    from paper_1705_01263_gb300 import rt
    sd, flat, cam, s, o = field
    rays = scenes.random_rays(flat, 1 << 18, seed=5, kind=kind, cam=cam)
    (prim, inst, t, u, v), _ = rt.rt_trace(s, torch.from_numpy(rays).cuda())
    torch.cuda.synchronize()
    p = prim.cpu().numpy().view(np.uint32)
    i = inst.cpu().numpy().view(np.uint32)
    t = t.cpu().numpy()
    hit = p != MISS
    fp = np.where(hit, flat_index(sd, np.where(hit, i, 0), np.where(hit, p, 0)), MISS).astype(np.uint32)
    # the GPU intersects FP32 object-space triangles with the ray mapped to
    # object space, the oracle the FP32 world-space copy of each instance: the
    # two geometries differ by the rounding of the transform (about 1e-7 of
    # the coordinates), so distances agree to 1e-4 of max(t, |o|, 1), grazing
    # hits included, and near edges both answers can be right; every
    # disagreement must be a valid alternative hit
    from test_gpu_trace import check_closest
    check_closest(flat, rays, (fp, t, u.cpu().numpy(), v.cpu().numpy()), o.trace(rays), min_agree=0.99995,
                  t_rel=1e-4)


def test_instanced_render_parity(field):
    """Converged comparison (8192 spp on a 48 x 27 crop of the camera): the
    emitter fluxes of textured triangles are integrated exactly by the oracle
    and by 16 x 16 supersampling in the GPU preprocess, so the two alias
    tables differ and paths pick different lights; the images then agree only
    statistically."""
    from paper_1705_01263_gb300 import rt
    sd, flat, cam, s, o = field
    cam = scenes.Camera(cam.eye, cam.look_at, cam.up, cam.vfov_deg, 48, 27)
    film = rt.Film(cam.width, cam.height)
    rt.rt_render(s, cam, 8192, 6, film)
    torch.cuda.synchronize()
    mg, vg = oracle.resolve(*film.download())
    S, S2, C, _ = o.render(cam, 8192, 6)
    mo, vo = oracle.resolve(S, S2, C)
    l1, out, n = image_parity(mg, vg, mo, vo)
    assert l1 <= 0.01, l1
    assert out <= allowed_4sigma(n), (out, n)


def test_full_size_many_light_scene_renders():
    """1000 instances of 100 meshes, 10,000,000 instanced triangles, 100k
    textured emitters; one pass at 1920 x 1080, depth 12."""
    from paper_1705_01263_gb300 import rt
    sd, cam = scenes.instanced_field()
    counts = np.diff(sd.mesh_tri_offset)[sd.instance_mesh]
    assert abs(int(counts.sum()) - 10_000_000) < 200_000
    s = rt.Scene(sd)
    film = rt.Film(cam.width, cam.height)
    stats = rt.rt_stats()
    rt.rt_render(s, cam, 1, 12, film, rt.make_opts(stats=stats))
    torch.cuda.synchronize()
    m, v = oracle.resolve(*film.download())
    assert np.isfinite(m).all() and m.mean() > 0
    assert stats.paths == cam.width * cam.height
