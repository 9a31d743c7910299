"""Several devices on one image (Sec. 3.2.2): ranks render disjoint
iteration ranges and their FP64 films are summed once. Here the host side of
that path runs as two gloo ranks on CPU, each rendering its range with the
oracle, and the reduction of the package (paper_1705_01263_gb300.multi) must
give exactly the single-process render of the whole range (counts equal, sums
equal up to FP64 addition order)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, first, spp, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1705_01263_gb300 import multi, scenes
        sd, cam = scenes.cornell_box()
        cam.width = cam.height = 16
        start, n = multi.rank_iterations(rank, world, first, spp)
        S, S2, C, _ = oracle.Scene(sd).render(cam, n, 4, iter0=start)
        ts, ts2 = torch.from_numpy(S), torch.from_numpy(S2)
        tc = torch.from_numpy(C.astype(np.int32))
        multi.reduce_film(ts, ts2, tc)
        q.put((rank, start, n, ts.numpy(), ts2.numpy(), tc.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_rank_iterations_tile_the_range():
    from paper_1705_01263_gb300 import multi
    for world in (1, 2, 3, 8):
        for spp in (0, 1, 7, 64, 1000):
            parts = [multi.rank_iterations(r, world, 5, spp) for r in range(world)]
            assert sum(n for _, n in parts) == spp
            pos = 5
            for s, n in parts:
                assert s == pos and n >= 0
                pos += n
            assert max(n for _, n in parts) - min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        multi.rank_iterations(2, 2, 0, 4)


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_sum_to_the_single_render(world):
    import multiprocessing as pymp
    import oracle
    from paper_1705_01263_gb300 import scenes
    ctx = pymp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    first, spp = 3, 9
    procs = [ctx.Process(target=_worker, args=(r, world, port, first, spp, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    assert [r[2] for r in res] == [5, 4] and res[0][1] == first and res[1][1] == first + 5
    sd, cam = scenes.cornell_box()
    cam.width = cam.height = 16
    S, S2, C, _ = oracle.Scene(sd).render(cam, spp, 4, iter0=first)
    for _, _, _, s, s2, c in res:      # every rank holds the sum
        assert np.array_equal(c.astype(np.uint32), C)
        assert np.allclose(s, S, rtol=1e-13, atol=1e-13)
        assert np.allclose(s2, S2, rtol=1e-13, atol=1e-13)
