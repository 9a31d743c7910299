"""GPU parity of the QMC sampling (Appendix A.2): the device's Halton bits
equal the oracle's exactly, over 2^24 consecutive indices and random 64-bit
indices, and the full-screen enumeration gives the same sequence indices."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_halton_bits_exact_first_2p24_indices():
    from paper_1705_01263_gb300 import rt
    n = 1 << 24
    idx = torch.arange(n, dtype=torch.int64, device="cuda")
    out = rt.rt_halton(1920, 1080, 17050126, idx, 12).cpu().numpy().view(np.uint32)
    # the oracle on a strided sample of the range plus the whole first 2^16
    pick = np.concatenate([np.arange(1 << 16), np.arange(1 << 16, n, 997)]).astype(np.uint64)
    ref = oracle.sample_dims_u32(pick, 12, 1920, 1080, 17050126)
    assert np.array_equal(out[pick.astype(np.int64)], ref)
    # base 2 (dimension 0 after the 2^11 shift) is a bit reversal of i >> 11
    i = np.arange(n, dtype=np.uint64) >> np.uint64(11)
    rev = np.zeros(n, np.uint64)
    x = i.copy()
    for b in range(32):
        rev |= ((x >> np.uint64(b)) & np.uint64(1)) << np.uint64(31 - b)
    assert np.array_equal(out[:, 0].astype(np.uint64), rev)


def test_halton_bits_exact_64bit_indices_all_dims():
    from paper_1705_01263_gb300 import rt
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.integers(0, 2**63, 20000, dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1),
                          np.array([2**64 - 1, 2**63, 2**32 - 1, 2**32, 0], np.uint64)])
    t = torch.from_numpy(idx.view(np.int64)).cuda()
    for seed in (0, 123456789):
        out = rt.rt_halton(64, 64, seed, t, 114).cpu().numpy().view(np.uint32)
        assert np.array_equal(out, oracle.sample_dims_u32(idx, 114, 64, 64, seed))


def test_sample_index_enumeration():
    from paper_1705_01263_gb300 import rt
    for W, H in [(64, 64), (1920, 1080), (5, 3)]:
        rng = np.random.default_rng(W)
        n = 5000
        px, py, j = rng.integers(0, W, n), rng.integers(0, H, n), rng.integers(0, 1 << 20, n)
        out = rt.rt_sample_index(W, H, torch.tensor(px, dtype=torch.int32, device="cuda"),
                                 torch.tensor(py, dtype=torch.int32, device="cuda"),
                                 torch.tensor(j, dtype=torch.int32, device="cuda")).cpu().numpy().view(np.uint64)
        k = max(0, (W - 1).bit_length())
        l = 0
        while 3**l < H:
            l += 1
        P = 2**k * 3**l
        for r in range(0, n, 50):
            assert int(out[r]) == oracle.pixel_base_index(W, H, int(px[r]), int(py[r])) + int(j[r]) * P


def test_halton_empty_and_invalid():
    from paper_1705_01263_gb300 import rt
    idx = torch.zeros(0, dtype=torch.int64, device="cuda")
    assert rt.rt_halton(8, 8, 0, idx, 4).numel() == 0
    with pytest.raises(rt.RtError):
        rt.rt_halton(0, 8, 0, torch.zeros(4, dtype=torch.int64, device="cuda"), 4)
