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
    # the asynchronous entry point runs the same kernel
    raw = torch.full((n, 40), float("nan"), device="cuda")
    guide.infer_async(x, raw)
    guide.check()
    assert np.array_equal(raw.cpu().numpy(), a)
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


# ---------------------------------------------------------------------------
# Element-wise parity with the oracle

U_BF16 = 2.0 ** -8   # unit roundoff of BF16 (8 significant bits, round to nearest)
G_ACC = 2.0 ** -24   # unit roundoff of the FP32 accumulation


def _layers(p):
    """Oracle parameter vector -> [W1..W5] ([out][in]) in float64."""
    dims = [224, 64, 64, 64, 64, 40]
    Ws, o = [], 0
    for l in range(5):
        n = dims[l] * dims[l + 1]
        Ws.append(p[o:o + n].reshape(dims[l + 1], dims[l]))
        o += n
    return Ws


def forward_error_sigma(p, x0, acts):
    """Per-element standard deviation of the raw outputs' rounding error when
    both sides take the same BF16 weights and inputs and the GPU rounds every
    hidden activation to BF16 (round to nearest: an error uniform within
    +-u_bf16 |h|, variance (u |h|)^2 / 3), to first order: each layer's
    rounding errors reach the outputs through the Jacobian W5 D4 W4 ... D(l+1)
    W(l+1), with D the ReLU masks of the oracle's activations. The inputs are
    counted the same way (the GPU builds the one-blob bins in FP32, which can
    round to a neighbouring BF16 value); the FP32 accumulation adds K u_acc
    |W||h| at most per product."""
    Ws = _layers(p)
    n = x0.shape[0]
    hs = [x0] + [acts[:, l, :] for l in range(4)]     # h0 = inputs, h1..h4 hidden
    var = np.zeros((n, 40))
    J = np.broadcast_to(Ws[4], (n,) + Ws[4].shape).copy()   # d out / d h4, per row
    for l in range(4, -1, -1):
        var += (J ** 2 * (U_BF16 * hs[l][:, None, :]) ** 2 / 3.0).sum(axis=2)
        if l > 0:
            mask = (hs[l] > 0).astype(np.float64)            # D_l
            J = (J * mask[:, None, :]) @ Ws[l - 1]           # d out / d h(l-1)
    acc = 224 * G_ACC * (np.abs(hs[4]) @ np.abs(Ws[4]).T)
    return np.sqrt(var), acc


@pytest.mark.parametrize("trained", [False, True])
def test_forward_matches_oracle_per_element(trained):
    """Every raw output of the fused inference kernel within 6 standard
    deviations of its first-order BF16 rounding error (plus the FP32
    accumulation bound) of the FP64 oracle on the same BF16 weights and
    inputs, all but one in a thousand within 4; an untrained network and one
    after 20 Adam steps."""
    from paper_1705_01263_gb300 import rt
    guide = rt.Guide(seed=21)
    f = features(3000, 6)
    x = torch.tensor(f, dtype=torch.float32, device="cuda")
    if trained:
        rng = np.random.default_rng(8)
        wi = rng.normal(size=(3000, 3)) + np.array([0.0, 2.0, 0.0])
        wi /= np.linalg.norm(wi, axis=1, keepdims=True)
        for _ in range(20):
            guide.train_step(x, torch.tensor(wi, dtype=torch.float32, device="cuda"),
                             torch.ones(3000, device="cuda"))
    raw = guide.infer(x).cpu().numpy().astype(np.float64)
    p = bf16_round(guide.get_params())
    x0 = bf16_round(oracle_inputs(f))
    want, acts = oracle.mlp_forward_acts(p, x0)
    sig, acc = forward_error_sigma(p, x0, acts)
    err = np.abs(raw - want)
    assert np.all(err <= 6 * sig + acc + 1e-7), np.max((err - acc) / (sig + 1e-30))
    assert np.mean(err > 4 * sig + acc + 1e-7) <= 1e-3
    # the tolerance is tight: far below the outputs' own scale
    assert np.median(6 * sig + acc) < 0.1 * np.median(np.abs(want))


def test_adam_update_matches_oracle_element_wise():
    """Two GPU training steps against the oracle's Adam (first steps of the
    textbook update, beta1 0.9, beta2 0.999, eps 1e-8, lr 1e-2) fed with the
    GPU's gradient at the same weights: parameters and both moments element
    by element at FP32 rounding."""
    from paper_1705_01263_gb300 import rt
    n = 4096
    guide = rt.Guide(seed=31, lr=1e-2)
    f = torch.tensor(features(n, 9), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(10)
    wi = rng.normal(size=(n, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wi = torch.tensor(wi, dtype=torch.float32, device="cuda")
    w = torch.tensor(rng.uniform(0.2, 3.0, n), dtype=torch.float32, device="cuda")
    npar = guide.num_params()

    def unpack(blob):
        a = np.frombuffer(blob, np.uint8)
        P = a[: 4 * npar].view(np.float32).astype(np.float64)
        M = a[4 * npar: 8 * npar].view(np.float32).astype(np.float64)
        V = a[8 * npar: 12 * npar].view(np.float32).astype(np.float64)
        step = int(a[12 * npar: 12 * npar + 8].view(np.int64)[0])
        return P, M, V, step

    P, M, V, step = unpack(guide.state())
    assert step == 0 and not M.any() and not V.any()
    for t in (1, 2):
        _, g = guide.loss_grad(f, wi, w)
        g = g.cpu().numpy().astype(np.float64)
        guide.train_step(f, wi, w)
        Pg, Mg, Vg, step = unpack(guide.state())
        assert step == t
        Po, Mo, Vo = P.copy(), M.copy(), V.copy()
        oracle.adam_step(Po, g, Mo, Vo, t)
        # FP32 rounding of b M + (1 - b) g (a few units in the last place of
        # the larger term; the sum itself may cancel)
        u = 2.0 ** -24
        assert np.all(np.abs(Mg - Mo) <= 4 * u * (0.9 * np.abs(M) + 0.1 * np.abs(g)) + 1e-38)
        assert np.all(np.abs(Vg - Vo) <= 4 * u * (0.999 * V + 0.001 * g * g) + 1e-38)
        step_size = np.abs(Po - P)
        assert np.all(np.abs(Pg - Po) <= 4e-6 * step_size + 2 * np.spacing(np.abs(P).astype(np.float32))), \
            np.abs(Pg - Po).max()
        assert np.abs(Pg - P).max() > 0
        P, M, V = Pg, Mg, Vg


def test_device_mixture_pdf_and_sampler_match_oracle():
    """The von Mises-Fisher mixture code that guided shading runs (decode of
    the raw outputs, density, lobe choice and Jakob's sampling) against the
    oracle's on the same raw outputs and uniforms, sample by sample, from
    broad to sharp lobes (kappa 1e-2 .. 1e3)."""
    from paper_1705_01263_gb300 import rt
    rng = np.random.default_rng(12)
    n = 20000
    raw = rng.normal(size=(n, 40))
    sharp = rng.random(n) < 0.3
    for k in range(8):
        raw[:, 5 * k + 3] = np.where(sharp, rng.uniform(5.0, 1000.0, n), rng.uniform(-6.0, 4.0, n))
        raw[:, 5 * k + 4] *= 2.0
    raw = raw.astype(np.float32).astype(np.float64)
    wi = rng.normal(size=(n, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wi = wi.astype(np.float32).astype(np.float64)
    u = rng.random((n, 3)).astype(np.float32).astype(np.float64)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    pdf_wi, ws, pdf_ws = rt.debug_guide_mixture(t(raw), t(wi), t(u))
    pdf_wi, ws, pdf_ws = (x.cpu().numpy().astype(np.float64) for x in (pdf_wi, ws, pdf_ws))
    kmax = np.log1p(np.exp(np.minimum(raw[:, 3::5], 700.0))).clip(1e-2, 1e4).max(axis=1)
    # density: FP32 exponent kappa (mu.w - 1) carries ~kappa 2^-22 absolute error
    po = np.array([oracle.mixture_pdf(raw[i], wi[i]) for i in range(n)])
    tol = po * (2e-5 + 4.0 * kmax * 2.0 ** -23) + 1e-30
    assert np.all(np.abs(pdf_wi - po) <= tol), np.max(np.abs(pdf_wi - po) / tol)
    # sampling: the same lobe (away from the FP32/FP64 boundary of the
    # cumulative weights) and the same direction
    z = np.exp(raw[:, 4::5] - raw[:, 4::5].max(axis=1, keepdims=True))
    cw = np.cumsum(z / z.sum(axis=1, keepdims=True), axis=1)
    clear = np.min(np.abs(cw[:, :7] - u[:, :1]), axis=1) > 1e-5
    wo = np.array([oracle.mixture_sample(raw[i], *u[i]) for i in range(n)])
    d = np.linalg.norm(ws - wo, axis=1)
    assert clear.mean() > 0.99
    assert np.all(d[clear] <= 2e-4), d[clear].max()
    assert np.all(np.abs(np.linalg.norm(ws, axis=1) - 1) < 1e-5)
    # the density at the sampled direction agrees too
    pos = np.array([oracle.mixture_pdf(raw[i], ws[i]) for i in range(n)])
    tol = pos * (2e-5 + 4.0 * kmax * 2.0 ** -23) + 1e-30
    assert np.all(np.abs(pdf_ws - pos) <= tol), np.max(np.abs(pdf_ws - pos) / tol)
