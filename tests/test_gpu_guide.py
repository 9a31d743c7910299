"""GPU parity of the guiding network (not in the paper; pinned to the FP64
oracle's textbook definitions): the tcgen05 BF16 GEMM against float64
products of the same BF16 values, the network forward pass and the gradient
of the training loss against the oracle, Adam training lowering the loss,
and checkpoint round trips."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 64, 224), (256, 64, 64), (300, 48, 64), (130, 16, 16),
                                   (48, 64, 4096), (64, 224, 65536), (1000, 256, 96), (7, 40, 8)])
def test_gemm_bf16_matches_float64(M, N, K):
    from paper_1705_01263_gb300 import rt
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = rt.rt_gemm_bf16(A.cuda(), B.cuda())
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    got = C.cpu().double()
    err = (got - ref).abs().max().item()
    scale = (A.double().abs() @ B.double().abs().T).max().item()
    assert err <= 1e-5 * scale + 1e-6, (err, scale)


def test_gemm_accumulate_and_strides():
    from paper_1705_01263_gb300 import rt
    g = torch.Generator().manual_seed(3)
    A = torch.randn(256, 80, generator=g).to(torch.bfloat16).cuda()[:, :64]   # row stride 80
    B = torch.randn(32, 64, generator=g).to(torch.bfloat16).cuda()
    C = torch.ones(256, 32, device="cuda")
    rt.rt_gemm_bf16(A, B, C, accumulate=True)
    torch.cuda.synchronize()
    ref = 1.0 + A.double().cpu() @ B.double().cpu().T
    assert torch.allclose(C.cpu().double(), ref, rtol=1e-5, atol=1e-4)


def features(n, seed):
    rng = np.random.default_rng(seed)
    f = rng.random((n, 7))
    return f


def oracle_inputs(f):
    return np.stack([oracle.oneblob(r) for r in f])


def bf16_round(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).double().numpy()


def test_forward_matches_oracle():
    from paper_1705_01263_gb300 import rt
    guide = rt.Guide(seed=11)
    p = guide.get_params().astype(np.float64)
    f = features(2048, 1)
    raw = guide.infer(torch.tensor(f, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = oracle.mlp_forward(bf16_round(p), bf16_round(oracle_inputs(f)))
    rel = np.linalg.norm(raw - want) / np.linalg.norm(want)
    assert rel < 3e-2, rel
    # the mixture the outputs define is a density: oracle pdf integrates to 1
    assert np.isfinite(raw).all()


@pytest.mark.parametrize("n", [1, 127, 128, 129, 5000, 70000])
def test_fused_inference_equals_layer_by_layer(n):
    """The fused kernel (one launch, weights and activations in shared and
    tensor memory) and the GEMM path of the training forward pass take the
    same BF16 operands and accumulate in the same K order, for ragged tiles
    and for more tiles than SMs."""
    from paper_1705_01263_gb300 import rt
    guide = rt.Guide(seed=12)
    x = torch.tensor(features(n, 2), dtype=torch.float32, device="cuda")
    a = guide.infer(x).cpu().numpy()
    b = guide.infer_layers(x).cpu().numpy()
    assert np.isfinite(a).all()
    assert np.abs(a - b).max() <= 1e-5 * max(1.0, np.abs(b).max()), np.abs(a - b).max()
    # after training steps the weights the fused kernel stages change too
    wi = torch.nn.functional.normalize(torch.randn(n, 3, device="cuda"), dim=1)
    w = torch.rand(n, device="cuda")
    guide.train_step(x, wi, w)
    a2 = guide.infer(x).cpu().numpy()
    b2 = guide.infer_layers(x).cpu().numpy()
    assert np.abs(a2 - b2).max() <= 1e-5 * max(1.0, np.abs(b2).max())
    assert np.abs(a2 - a).max() > 0


def test_gradients_match_oracle():
    from paper_1705_01263_gb300 import rt
    guide = rt.Guide(seed=12)
    p = guide.get_params().astype(np.float64)
    n = 4096
    f = features(n, 2)
    rng = np.random.default_rng(3)
    wi = rng.normal(size=(n, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    w = rng.uniform(0.1, 2.0, n)
    loss, g = guide.loss_grad(torch.tensor(f, dtype=torch.float32, device="cuda"),
                              torch.tensor(wi, dtype=torch.float32, device="cuda"),
                              torch.tensor(w, dtype=torch.float32, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    lo, go = oracle.guide_loss_grad(bf16_round(p), bf16_round(oracle_inputs(f)), wi, w)
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    rel = float(np.linalg.norm(g - go) / np.linalg.norm(go))
    assert abs(loss - lo) <= 2e-2 * abs(lo), (loss, lo)
    assert cos >= 0.999, cos
    assert rel <= 2e-2, rel


def test_training_lowers_loss_and_checkpoint_roundtrip():
    from paper_1705_01263_gb300 import rt
    guide = rt.Guide(seed=13, lr=1e-2)
    n = 1 << 14
    f = torch.tensor(features(n, 4), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(5)
    wi = np.array([0.0, 1.0, 0.0]) + 0.3 * rng.normal(size=(n, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wi = torch.tensor(wi, dtype=torch.float32, device="cuda")
    w = torch.ones(n, dtype=torch.float32, device="cuda")
    l0, _ = guide.loss_grad(f, wi, w)
    for _ in range(30):
        guide.train_step(f, wi, w)
    l1, _ = guide.loss_grad(f, wi, w)
    assert l1 < l0 - 0.5, (l0, l1)
    blob = guide.state()
    out_a = guide.infer(f[:256]).cpu().numpy()
    other = rt.Guide(seed=99)
    other.load(blob)
    out_b = other.infer(f[:256]).cpu().numpy()
    assert np.array_equal(out_a, out_b)


def test_gemm_split_k_accumulate_into_strided_c():
    """K long enough to be split across CTAs (partial products summed in a
    second pass), accumulating into a column slice of a wider C."""
    from paper_1705_01263_gb300 import rt
    g = torch.Generator().manual_seed(5)
    A = torch.randn(64, 8192, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(48, 8192, generator=g).to(torch.bfloat16).cuda()
    big = torch.full((64, 80), 2.0, device="cuda")
    C = big[:, 16:64]
    rt.rt_gemm_bf16(A, B, C, accumulate=True)
    torch.cuda.synchronize()
    ref = 2.0 + A.double().cpu() @ B.double().cpu().T
    scale = (A.double().cpu().abs() @ B.double().cpu().abs().T).max().item()
    assert (C.cpu().double() - ref).abs().max().item() <= 1e-5 * scale + 1e-4
    assert torch.all(big[:, :16] == 2.0) and torch.all(big[:, 64:] == 2.0)
