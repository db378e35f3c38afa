"""The per-element tolerance of the network's GPU arithmetic (tests/mlp_bounds.py), pinned on
the CPU: an emulation of that arithmetic (float32 with BF16 roundings, written apart from the
bound) stays inside the bound on every element, the bound is tight enough to fix most
elements to a few percent, and planted mistakes in the emulation break it."""
import numpy as np
import pytest

from mlp_bounds import (emulate_forward, emulate_gradients, gradient_bounds, output_bound, violations)
from oracle import mlp


def _params(seed):
    r = np.random.default_rng(seed)
    d = {}
    for name, shape in mlp.SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[1])
            d[name] = r.uniform(-lim, lim, shape)
        else:
            d[name] = r.uniform(-0.1, 0.1, shape)
    return mlp.pack(d).astype(np.float32).astype(np.float64)


def _inputs(seed, n):
    r = np.random.default_rng(seed)
    X = np.concatenate([r.uniform(-1, 1, (n, 3)), r.normal(size=(n, 3)), r.uniform(0, 1, (n, 1))], axis=1)
    X[:, 3:6] /= np.linalg.norm(X[:, 3:6], axis=1, keepdims=True)
    T = 0.3 * r.normal(size=(n, 6))
    return X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("mode", ["train", "infer"])
def test_emulated_forward_within_bound_and_bound_is_tight(mode):
    P = _params(1)
    X, _ = _inputs(2, 384)
    Yr, bnd = output_bound(P, X, mode)
    Y, _ = emulate_forward(P, X, mode)
    bad = violations(Y, Yr, bnd)
    assert not bad.any(), np.argwhere(bad)[:5]
    rel = bnd / np.maximum(np.abs(Yr), 1e-30)
    assert np.median(rel) < 0.1, np.median(rel)


def test_emulated_gradients_within_bound_and_bound_is_tight():
    P = _params(3)
    X, T = _inputs(4, 512)
    L, G, DL, DG = gradient_bounds(P, X, T)
    Le, Ge = emulate_gradients(P, X, T)
    assert abs(Le - L) <= DL
    bad = violations(Ge, G, DG)
    assert not bad.any(), np.argwhere(bad)[:5]
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    for i, (name, _) in enumerate(mlp.SHAPES):
        g, b = G[offs[i]:offs[i + 1]], DG[offs[i]:offs[i + 1]]
        fixed = (b <= 0.25 * np.abs(g)).mean()   # elements whose value the bound fixes to 25 %
        assert fixed >= 0.45, (name, fixed)


def _w2_entry():
    o = dict(zip([n for n, _ in mlp.SHAPES], np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])))
    return o["W2"], o["b2"]


def test_planted_single_element_errors_are_caught():
    """One W2 gradient entry 20 % off, or one b2 gradient entry with its sign flipped, fails the
    element-wise check at exactly that element (a normwise check would pass both)."""
    P = _params(5)
    X, T = _inputs(6, 512)
    _, G, _, DG = gradient_bounds(P, X, T)
    _, Ge = emulate_gradients(P, X, T)
    oW2, ob2 = _w2_entry()
    n2 = 256 * 256
    w2 = slice(oW2, oW2 + n2)
    ratio = np.where(G[w2] != 0, DG[w2] / np.maximum(np.abs(G[w2]), 1e-300), np.inf)
    k = oW2 + int(np.argmin(ratio))
    assert DG[k] < 0.05 * abs(G[k])
    bad = Ge.copy()
    bad[k] *= 1.2
    v = violations(bad, G, DG)
    assert v.sum() == 1 and v[k]
    b2 = slice(ob2, ob2 + 256)
    j = ob2 + int(np.argmax(np.abs(G[b2]) / np.maximum(DG[b2], 1e-30)))
    bad = Ge.copy()
    bad[j] = -bad[j]
    v = violations(bad, G, DG)
    assert v.sum() == 1 and v[j]
    rel = np.linalg.norm(bad - G) / np.linalg.norm(G)
    assert rel < 3e-2   # what the former normwise check would have accepted


def test_planted_arithmetic_mistakes_break_the_bound():
    """Mistakes a kernel could make (a dropped ReLU mask in the backward pass, W3 transposed,
    layer 3 using W2) fall outside the bound."""
    P = _params(7)
    X, T = _inputs(8, 256)
    _, G, _, DG = gradient_bounds(P, X, T)
    p = mlp.unpack(P)

    def grads_with(mut):
        import mlp_bounds as mb
        saved = mb.bf16
        try:
            return mut()
        finally:
            mb.bf16 = saved

    # W3 transposed in the forward pass: the forward bound must fail
    q = dict(p)
    q["W3"] = p["W3"].T.copy()
    Yt, _ = emulate_forward(mlp.pack(q), X, "train")
    Yr, bnd = output_bound(P, X, "train")
    assert violations(Yt, Yr, bnd).mean() > 0.5
    # layer 3 with W2's weights
    q = dict(p)
    q["W3"] = p["W2"].copy()
    Yw, _ = emulate_forward(mlp.pack(q), X, "train")
    assert violations(Yw, Yr, bnd).mean() > 0.5
    # the backward pass without the layer-3 ReLU mask
    import mlp_bounds as mb

    def no_mask():
        f32 = np.float32
        pp = {k: np.asarray(v, np.float32) for k, v in p.items()}
        Y, (X32, Z1, H1, Z2, H2, Z3, H3) = mb.emulate_forward(P, X, "train")
        B = X.shape[0]
        Tt = np.asarray(T, np.float32)
        d = Y[:, :6] - Tt
        se = (d * d).sum(axis=1, dtype=f32)
        lg = np.log(se + f32(1e-6)).astype(f32)
        dY = np.zeros_like(Y)
        dY[:, :6] = f32(2) * d / f32(6 * B)
        dY[:, 6] = f32(0.2) * (Y[:, 6] - lg) / f32(B)
        dZ3 = mb.bf16(dY @ pp["W4"])     # mask dropped
        return (dZ3.T @ H2).reshape(-1)

    oW3 = dict(zip([n for n, _ in mlp.SHAPES], np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])))["W3"]
    gw3 = grads_with(no_mask)
    v = violations(gw3, G[oW3:oW3 + 256 * 256], DG[oW3:oW3 + 256 * 256])
    assert v.mean() > 0.2, v.mean()
