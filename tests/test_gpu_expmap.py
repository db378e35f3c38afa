"""The learned exponential map on the GPU: its tcgen05 GEMM, its gradients against the
FP64 oracle's back-propagation, the integrator-generated training segments against the
oracle's RK4, training, and checkpoints.

Tolerances.  Every output and every gradient element is held to its own bound
(tests/mlp_bounds.py): the FP64 oracle network at the operands the kernels read (W2 and
W3 as their BF16 copies), and a probabilistic rounding-error bound of 8 standard
deviations carried through the BF16 roundings (unit roundoff 2^-8) and FP32 sums of each
layer.  The parameters are drawn on the CPU and uploaded.  The GEMM itself is compared
with an FP32 product of the same BF16 operands, where only the summation order differs.
"""
import numpy as np
import pytest

import oracle
from mlp_bounds import gradient_bounds, output_bound, violations
from oracle import mlp
from paper_2005_05386_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    return rg


def _bf16(shape, gen, scale=1.0):
    import torch
    return (torch.rand(shape, generator=gen, device="cuda") * 2 - 1).mul_(scale).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 256, 256), (300, 48, 64), (1000, 16, 1024), (129, 256, 512),
                                   (4096, 256, 256)])
def test_gemm_mode0_matches_fp32_product(rg, M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A, B = _bf16((M, K), g), _bf16((N, K), g)
    bias = torch.rand(N, generator=g, device="cuda")
    C = torch.full((M, N), float("nan"), device="cuda")
    rg.rgeo_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, 1, bias.data_ptr(), 0, C.data_ptr(), N, None, 0)
    rg.rgeo_sync()
    ref = A.float() @ B.float().T + bias
    torch.testing.assert_close(C, ref, rtol=1e-5, atol=1e-4 * K ** 0.5)


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (200, 64, 128)])
def test_gemm_mode1_relu_bf16_and_transpose(rg, M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(11 + M)
    A, B = _bf16((M, K), g), _bf16((N, K), g)
    bias = torch.rand(N, generator=g, device="cuda") - 0.5
    C = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    Ct = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
    rg.rgeo_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, 1, bias.data_ptr(), 1, C.data_ptr(), N, Ct.data_ptr(), M)
    rg.rgeo_sync()
    ref = torch.relu(A.float() @ B.float().T + bias)
    torch.testing.assert_close(C.float(), ref, rtol=2 ** -8, atol=1e-5)
    assert torch.equal(Ct, C.T.contiguous())
    assert (C.float() >= 0).all()


@pytest.mark.parametrize("splits", [1, 4, 16])
def test_gemm_mode2_split_k_accumulates(rg, splits):
    import torch
    g = torch.Generator(device="cuda").manual_seed(5 + splits)
    M, N, K = 256, 256, 2048
    A, B = _bf16((M, K), g), _bf16((N, K), g)
    C0 = torch.rand((M, N), generator=g, device="cuda")
    C = C0.clone()
    rg.rgeo_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, splits, None, 2, C.data_ptr(), N, None, 0)
    rg.rgeo_sync()
    torch.testing.assert_close(C, C0 + A.float() @ B.float().T, rtol=1e-5, atol=2e-3)


def test_gemm_rejects_bad_shapes(rg):
    import torch
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 256, device="cuda")
    for M, N, K in [(128, 8, 64), (128, 24, 64), (128, 272, 64), (128, 16, 48), (0, 16, 64)]:
        with pytest.raises(rg.RgeoError):
            rg.rgeo_gemm_bf16(A.data_ptr(), A.data_ptr(), M, N, K, 1, None, 0, C.data_ptr(), 256, None, 0)
    with pytest.raises(rg.RgeoError):  # operand not 16-byte aligned
        rg.rgeo_gemm_bf16(A.data_ptr() + 2, A.data_ptr(), 64, 16, 64, 1, None, 0, C.data_ptr(), 256, None, 0)
    with pytest.raises(rg.RgeoError):  # split-K needs the accumulate epilogue
        rg.rgeo_gemm_bf16(A.data_ptr(), A.data_ptr(), 128, 16, 64, 2, None, 0, C.data_ptr(), 256, None, 0)


def _field_metric(seed=1):
    c, a, s = scenes.random_bumps(seed, 64)
    return scenes.Metric(center=c, amplitude=a, sigma=s)


def _blocks(v):
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    return [(name, v[offs[i]:offs[i + 1]]) for i, (name, _) in enumerate(mlp.SHAPES)]


def test_generator_matches_oracle_rk4(rg):
    """Targets from the device integrator against the oracle's FP64 RK4 of the same segments."""
    m = _field_metric()
    dm = rg.Metric(m)
    box, s_max, h = 4.0, 0.5, 0.005
    X, T = rg.Expmap.generate(dm, 256, seed=17, box=box, s_max=s_max, h=h)
    rg.rgeo_sync()
    X, T = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    # inputs: positions in [-1, 1], unit directions, arc lengths k h / s_max with k in 1..100
    assert np.abs(X[:, :3]).max() <= 1.0
    np.testing.assert_allclose(np.linalg.norm(X[:, 3:6], axis=1), 1.0, atol=1e-6)
    kf = X[:, 6] * s_max / h
    k = np.round(kf)
    np.testing.assert_allclose(kf, k, atol=1e-3)
    assert k.min() >= 1 and k.max() <= 100 and len(np.unique(k)) > 50
    R = mlp.segment_residuals(oracle.Metric.from_desc(m), X, box, s_max, h)
    s = k * h
    # compare unscaled residuals (x_s - x - s v, v_s - v): FP32 integration error lives there
    Ug = np.concatenate([T[:, :3] * s[:, None] ** 2, T[:, 3:] * s[:, None]], axis=1)
    Ur = np.concatenate([R[:, :3] * s[:, None] ** 2, R[:, 3:] * s[:, None]], axis=1)
    err = np.abs(Ug - Ur)
    ok = (err <= 2e-6 + 1e-4 * np.abs(Ur)).all(axis=1)
    assert ok.mean() >= 0.99, (ok.mean(), err.max())
    assert err.max() < 1e-3
    assert np.abs(Ur).max() > 1e-3


def _cpu_params(seed):
    """He-uniform weights and small random biases, drawn on the CPU (float32 values)."""
    r = np.random.default_rng(seed)
    d = {}
    for name, shape in mlp.SHAPES:
        lim = np.sqrt(6.0 / shape[1]) if name.startswith("W") else 0.1
        d[name] = r.uniform(-lim, lim, shape)
    return mlp.pack(d).astype(np.float32)


def _net(rg, seed, max_batch):
    x = rg.Expmap(max_batch=max_batch, seed=seed)
    P = _cpu_params(seed)
    x.set_params(P)
    return x, P.astype(np.float64)


def _inputs(r, n):
    X = np.concatenate([r.uniform(-1, 1, (n, 3)), r.normal(size=(n, 3)), r.uniform(0, 1, (n, 1))], axis=1)
    X[:, 3:6] /= np.linalg.norm(X[:, 3:6], axis=1, keepdims=True)
    return X.astype(np.float32)


def test_forward_matches_oracle_element_by_element(rg):
    import torch
    x, params = _net(rg, 3, 128)
    Xh = _inputs(np.random.default_rng(0), 300)
    Y = x.forward(torch.tensor(Xh, device="cuda"))  # 300 rows: three tiles, ragged tail
    rg.rgeo_sync()
    Yr, bound = output_bound(params, Xh.astype(np.float64), "infer")
    bad = violations(Y.cpu().numpy(), Yr, bound)
    assert not bad.any(), (bad.sum(), np.argwhere(bad)[:5])
    assert x.forward(torch.empty(0, 7, device="cuda")).shape == (0, 7)


def test_forward_rows_independent_of_tile_and_slot(rg):
    """The persistent inference kernel walks several 128-row tiles per CTA, two in flight.
    A row's output must not depend on which tile, CTA or slot it lands in: the full batch
    (5-6 tiles per CTA, ragged tail), a row permutation of it and short slices at odd
    offsets must agree bit for bit, and a sample must match the FP64 oracle element by
    element."""
    import torch
    x, params = _net(rg, 4, 128)
    n = 152 * 128 * 5 + 77
    r = np.random.default_rng(1)
    Xh = _inputs(r, n)
    X = torch.tensor(Xh, device="cuda")
    Y = x.forward(X)
    perm = torch.from_numpy(r.permutation(n)).cuda()
    Yp = x.forward(X[perm].contiguous())
    rg.rgeo_sync()
    assert torch.equal(Yp, Y[perm])
    for a, b in [(0, 1), (5, 300), (n - 200, n), (12345, 12345 + 129), (70000, 97000)]:
        Ys = x.forward(X[a:b].contiguous())
        rg.rgeo_sync()
        assert torch.equal(Ys, Y[a:b]), (a, b)
    px = r.choice(n, 3000, replace=False)
    Yr, bound = output_bound(params, Xh[px].astype(np.float64), "infer")
    bad = violations(Y.cpu().numpy()[px], Yr, bound)
    assert not bad.any(), (bad.sum(), np.argwhere(bad)[:5])


@pytest.mark.parametrize("batch", [256, 2048, 20480])
def test_gradients_match_oracle_element_by_element(rg, batch):
    """Back-propagation on the tensor cores (one persistent kernel over 128-row tiles)
    against the oracle's FP64 back-propagation, every gradient element within its bound;
    at batch 20480 (160 tiles) some CTAs take two tiles.  The same comparison with one W2
    gradient entry or one bias gradient entry planted wrong in a copy of the GPU result
    must fail at exactly that element."""
    dm = rg.Metric(_field_metric())
    X, T = rg.Expmap.generate(dm, batch, seed=23)
    x, params = _net(rg, 9, max(batch, 2048))
    G, L = x.gradients(X, T)
    rg.rgeo_sync()
    Xn, Tn = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    Lr, Gr, DL, DG = gradient_bounds(params, Xn, Tn)
    assert abs(L.item() - Lr) <= DL, (L.item(), Lr, DL)
    G = G.cpu().numpy().astype(np.float64)
    bad = violations(G, Gr, DG)
    assert not bad.any(), [(name, int(v.sum())) for (name, v) in _blocks(bad)]
    offs = dict(zip([nm for nm, _ in mlp.SHAPES], np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])))
    for name, n_el in (("W2", 256 * 256), ("b2", 256)):
        sl = slice(offs[name], offs[name] + n_el)
        ratio = np.where(Gr[sl] != 0, DG[sl] / np.maximum(np.abs(Gr[sl]), 1e-300), np.inf)
        k = offs[name] + int(np.argmin(ratio))
        planted = G.copy()
        planted[k] = -planted[k]
        v = violations(planted, Gr, DG)
        assert v.sum() == 1 and v[k], (name, int(v.sum()))


def test_gradients_reject_bad_batches(rg):
    import torch
    x = rg.Expmap(max_batch=256, seed=1)
    X = torch.zeros(512, 7, device="cuda")
    T = torch.zeros(512, 6, device="cuda")
    for b in (0, 100, 512):
        with pytest.raises(rg.RgeoError):
            x.gradients(X[:b], T[:b])


def test_training_reduces_loss_and_checkpoint_roundtrip(rg, tmp_path):
    import torch
    dm = rg.Metric(_field_metric())
    X, T = rg.Expmap.generate(dm, 1 << 17, seed=31)
    Xv, Tv = rg.Expmap.generate(dm, 4096, seed=32)
    x = rg.Expmap(max_batch=4096, seed=2)

    def holdout():
        _, L = x.gradients(Xv, Tv)
        return L.item()

    l0 = holdout()
    loss = torch.zeros(1, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(0)
    for it in range(400):
        idx = torch.randint(0, X.shape[0], (4096,), generator=g, device="cuda")
        x.train_step(X[idx].contiguous(), T[idx].contiguous(), 1e-3, loss)
    rg.rgeo_sync()
    l1 = holdout()
    assert np.isfinite(l1) and l1 < 0.5 * l0, (l0, l1)
    path = str(tmp_path / "expmap.ckpt")
    x.save(path)
    y = rg.Expmap(max_batch=4096, seed=99)
    assert not np.array_equal(y.get_params(), x.get_params())
    y.load(path)
    assert np.array_equal(y.get_params(), x.get_params())
    Yx, Yy = x.forward(Xv), y.forward(Xv)
    rg.rgeo_sync()
    assert torch.equal(Yx, Yy)
    # The Adam moments and step count travel too: one more step on the same batch moves both
    # copies to the same parameters, bit for bit (the gradient sums have a fixed order; with
    # fresh moments every coordinate would instead move by about lr).
    x.train_step(X[:4096], T[:4096], 1e-3)
    y.train_step(X[:4096], T[:4096], 1e-3)
    rg.rgeo_sync()
    assert np.array_equal(x.get_params(), y.get_params())
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"not a checkpoint")
    with pytest.raises(rg.RgeoError):
        y.load(str(bad))


def test_gradients_and_training_are_deterministic(rg):
    """Each CTA of the training kernel sums its tiles in order and the CTAs' partials are summed
    in CTA order: the same batch gives the same gradient bits on every call, also when CTAs
    take several tiles, and training from the same start on the same batches reaches the same
    parameters bit for bit."""
    import torch
    dm = rg.Metric(_field_metric())
    X, T = rg.Expmap.generate(dm, 40960, seed=41)
    x, _ = _net(rg, 3, 40960)
    for b in (128, 40960):
        G1, L1 = x.gradients(X[:b], T[:b])
        G2, L2 = x.gradients(X[:b], T[:b])
        rg.rgeo_sync()
        assert torch.equal(G1, G2) and torch.equal(L1, L2), b
    nets = [_net(rg, 4, 8192)[0] for _ in range(2)]
    for net in nets:
        for i in range(5):
            net.train_step(X[i * 8192:(i + 1) * 8192], T[i * 8192:(i + 1) * 8192], 1e-3)
    rg.rgeo_sync()
    assert np.array_equal(nets[0].get_params(), nets[1].get_params())
    assert not np.array_equal(nets[0].get_params(), _cpu_params(4))


def test_train_in_one_call(rg):
    """rgeo_expmap_train: integrator-generated segments, device-sampled batches, cosine schedule."""
    import torch
    dm = rg.Metric(_field_metric())
    Xv, Tv = rg.Expmap.generate(dm, 4096, seed=77)
    x = rg.Expmap(max_batch=4096, seed=5)
    _, L0 = x.gradients(Xv, Tv)
    l0 = L0.item()
    tail = x.train(dm, n_segments=1 << 17, steps=400, batch=4096, lr_max=2e-3, lr_min=1e-4, seed=31)
    _, L1 = x.gradients(Xv, Tv)
    rg.rgeo_sync()
    assert np.isfinite(tail) and tail > 0
    assert L1.item() < 0.5 * l0, (l0, L1.item())
    with pytest.raises(rg.RgeoError):   # batch above max_batch
        x.train(dm, n_segments=1 << 14, steps=2, batch=8192)
    with pytest.raises(rg.RgeoError):   # batch not a multiple of 128
        x.train(dm, n_segments=1 << 14, steps=2, batch=1000)
