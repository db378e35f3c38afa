"""Per-element error bounds of the learned map's GPU arithmetic against the FP64 oracle.

The GPU network rounds some operands to BF16 (8 significant bits, unit roundoff
u = 2^-8) and accumulates in FP32 (unit roundoff e = 2^-24).  The paper fixes no
precision for it (the network is this build's addition), so the tolerance is derived
from that arithmetic.  A worst-case bound carried through three 256-wide layers grows
by the layer width each time and says nothing by layer 3, so the bound is the
probabilistic one of Higham and Mary ("A New Approach to Probabilistic Rounding Error
Analysis", SIAM J. Sci. Comput. 41(5), 2019): every rounding x -> x (1 + d) has an
independent mean-zero error, |d| <= u, hence variance at most u^2 |x|^2 / 3, and
variances propagate through the linear maps (sum over inputs of weight^2 times the
input's variance).  An element is accepted within LAMBDA standard deviations (a
deviation beyond 8 sigma has probability below 1e-10 for any distribution of bounded
variance that is close to Gaussian, as the sums of many independent roundings are).

The reference is the oracle network evaluated in FP64 at the operands the kernels read:
the FP32 master parameters, with W2 and W3 as their BF16 copies (the tensor-core
products take BF16 weights by design), so the systematic weight rounding is part of the
function and only the per-element roundings are statistics.  ReLU passes errors where
the mask is certain; where a pre-activation lies within LAMBDA sigma of zero the GPU's
mask may differ, and the whole masked value joins the variance.  A product of two
perturbed factors (a weight gradient dZ^T H) takes twice the sum of both first-order
variances, which covers any correlation of the two.

Arithmetic modelled (the kernels of paper_2005_05386_gb300/csrc/rgeo_mlp.cu):
  training forward  Z1 = W1 x + b1 in FP32; H_l = bf16(relu(Z_l)); Z2, Z3 = BF16 W x BF16 H
                    products with FP32 accumulation plus the FP32 bias; Y = W4 H3 + b4 in FP32
  fused inference   layers 1 and 4 with each FP32 factor split into two BF16 halves
                    (16 significant bits: products within 3 * 2^-16 relative), biases of
                    layers 2 and 3 split the same way; otherwise as the training forward
  back-propagation  dY in FP32; dZ3 = bf16(mask3 (dY W4)); dZ2 = bf16(mask2 (dZ3 W3b));
                    dZ1 = mask1 (dZ2 W2b) in FP32; weight gradients dZ^T H with the same
                    operands; bias gradients FP32 sums (of the BF16 dZ3 for layer 3, of the
                    FP32 values before rounding for layers 2 and 1)
"""
from __future__ import annotations

import numpy as np

U_BF16 = 2.0 ** -8
E_F32 = 2.0 ** -24
U_SPLIT = 3 * 2.0 ** -16
LAMBDA = 8.0


def _p(params):
    from oracle import mlp
    return mlp.unpack(params)


def gpu_operands(params):
    """The parameters as the kernels read them: W2 and W3 rounded to BF16 (their tensor-core
    copies), everything else FP32.  The FP64 reference is evaluated at these values."""
    from oracle import mlp
    d = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in _p(params).items()}
    d["W2"] = bf16(d["W2"]).astype(np.float64)
    d["W3"] = bf16(d["W3"]).astype(np.float64)
    return mlp.pack(d)


def _rnd(v, u):
    """Variance of one rounding of the values v with unit roundoff u."""
    return (u * u / 3.0) * v * v


def _acc(n, absterms):
    """Variance bound of an FP32 sum of n terms whose magnitudes sum to absterms."""
    return n * (E_F32 * E_F32 / 3.0) * absterms * absterms


def _relu(Z, vZ, vG, G):
    """Error variance of mask(Z > 0) * G given Z's and G's error variances: the term's own
    error where the GPU keeps the oracle's mask, plus the whole term G times the chance that
    Z's error crosses zero (a mask that differs), at most erfc(|Z| / (sigma sqrt 2))."""
    from scipy.special import erfc
    sd = np.sqrt(vZ)
    flip = erfc(np.abs(Z) / np.maximum(sd * np.sqrt(2.0), 1e-300))
    flip = np.where(sd > 0, flip, 0.0)
    return np.where(Z > 0, vG, 0.0) + flip * (G * G + vG)


def forward_bounds(params, X, mode: str = "train"):
    """FP64 activations of the oracle network at the GPU's operands and, per element, the
    error variances of Z1..Z3, H1..H3 and Y.  mode: "train" (training forward) or "infer"
    (fused inference)."""
    from oracle import mlp
    P = gpu_operands(params)
    p = mlp.unpack(P)
    X = np.asarray(X, np.float64)
    Y, (X, Z1, H1, Z2, H2, Z3, H3) = mlp.forward(P, X)
    u = U_BF16
    W1, W2, W3, W4 = (p[k] for k in ("W1", "W2", "W3", "W4"))
    b1, b2, b3, b4 = (p[k] for k in ("b1", "b2", "b3", "b4"))
    m1 = np.abs(X) @ np.abs(W1).T + np.abs(b1)
    if mode == "train":
        vZ1 = _acc(8, m1)
    else:
        vZ1 = (X * X) @ (W1 * W1).T * (U_SPLIT ** 2 / 3) + _rnd(b1, U_SPLIT) + _acc(32, m1)
    vH1 = _relu(Z1, vZ1, vZ1, Z1) + _rnd(H1, u)

    def hidden(vHp, Hp, W, b, Z):
        v = vHp @ (W * W).T + _acc(272, np.abs(Hp) @ np.abs(W).T + np.abs(b)) + _rnd(Z, E_F32)
        if mode == "infer":
            v = v + _rnd(b, U_SPLIT)
        return v

    vZ2 = hidden(vH1, H1, W2, b2, Z2)
    vH2 = _relu(Z2, vZ2, vZ2, Z2) + _rnd(H2, u)
    vZ3 = hidden(vH2, H2, W3, b3, Z3)
    vH3 = _relu(Z3, vZ3, vZ3, Z3) + _rnd(H3, u)
    m4 = H3 @ np.abs(W4).T + np.abs(b4)
    vY = vH3 @ (W4 * W4).T + _acc(258, m4)
    if mode == "infer":
        vY = vY + (H3 * H3) @ (W4 * W4).T * (U_SPLIT ** 2 / 3)
    acts = dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3, Y=Y)
    var = dict(Z1=vZ1, H1=vH1, Z2=vZ2, H2=vH2, Z3=vZ3, H3=vH3, Y=vY)
    return acts, var


def output_bound(params, X, mode: str = "train"):
    """(FP64 outputs at the GPU's operands, per-element bound LAMBDA * sigma)."""
    acts, var = forward_bounds(params, X, mode)
    return acts["Y"], LAMBDA * np.sqrt(var["Y"])


def gradient_bounds(params, X, T, lam: float = 0.1):
    """(loss, flat gradient, loss bound, flat per-element gradient bound) of the training path
    at the GPU's operands, in the parameter order of oracle.mlp.SHAPES."""
    from oracle import mlp
    P = gpu_operands(params)
    p = mlp.unpack(P)
    L, G = mlp.loss_and_grads(P, X, T, lam)
    a, v = forward_bounds(params, X, "train")
    T = np.asarray(T, np.float64)
    u = U_BF16
    B = X.shape[0]
    Y, H1, H2, H3, Z1, Z2, Z3, X = a["Y"], a["H1"], a["H2"], a["H3"], a["Z1"], a["Z2"], a["Z3"], a["X"]
    W2, W3, W4 = p["W2"], p["W3"], p["W4"]
    # loss gradient dY (FP32)
    d = Y[:, :6] - T
    vd = v["Y"][:, :6] + _rnd(d, E_F32)
    se = (d * d).sum(axis=1)
    vse = (4 * d * d * vd).sum(axis=1) + _rnd(se, E_F32) * 6
    lg = np.log(se + 1e-6)
    vlg = vse / (se + 1e-6) ** 2 + _rnd(lg, 4 * E_F32)
    d6 = Y[:, 6] - lg
    vd6 = 2 * (v["Y"][:, 6] + vlg) + _rnd(d6, E_F32)
    dY = np.zeros_like(Y)
    dY[:, :6] = 2 * d / (6 * B)
    dY[:, 6] = 2 * lam * d6 / B
    vdY = np.zeros_like(Y)
    vdY[:, :6] = (2 / (6 * B)) ** 2 * vd + _rnd(dY[:, :6], 3 * E_F32)
    vdY[:, 6] = (2 * lam / B) ** 2 * vd6 + _rnd(dY[:, 6], 3 * E_F32)
    vL = (vse.sum() / (6 * B) ** 2 + (lam / B) ** 2 * (4 * d6 * d6 * vd6).sum() + _acc(B, abs(L)))
    g = {}

    def wgrad(dZ, vdZ, H, vH):
        return 2 * (vdZ.T @ (H * H) + (dZ * dZ).T @ vH) + _acc(B, np.abs(dZ).T @ np.abs(H))

    # layer 4 (FP32)
    g["W4"] = wgrad(dY, vdY, H3, v["H3"])
    g["b4"] = vdY.sum(axis=0) + _acc(B, np.abs(dY).sum(axis=0))
    dH3 = dY @ W4
    vdH3 = vdY @ (W4 * W4) + _acc(7, np.abs(dY) @ np.abs(W4))
    # layer 3: dZ3 = bf16(mask3 dH3)
    dZ3 = dH3 * (Z3 > 0)
    vdZ3 = _relu(Z3, v["Z3"], vdH3, dH3) + _rnd(dZ3, u)
    g["b3"] = vdZ3.sum(axis=0) + _acc(B, np.abs(dZ3).sum(axis=0))
    g["W3"] = wgrad(dZ3, vdZ3, H2, v["H2"])
    dH2 = dZ3 @ W3
    vdH2 = vdZ3 @ (W3 * W3) + _acc(256, np.abs(dZ3) @ np.abs(W3))
    # layer 2: the FP32 values sum into db2, then dZ2 = bf16(...)
    dZ2 = dH2 * (Z2 > 0)
    vpre2 = _relu(Z2, v["Z2"], vdH2, dH2)
    g["b2"] = vpre2.sum(axis=0) + _acc(B, np.abs(dZ2).sum(axis=0))
    vdZ2 = vpre2 + _rnd(dZ2, u)
    g["W2"] = wgrad(dZ2, vdZ2, H1, v["H1"])
    dH1 = dZ2 @ W2
    vdH1 = vdZ2 @ (W2 * W2) + _acc(256, np.abs(dZ2) @ np.abs(W2))
    # layer 1 (FP32)
    dZ1 = dH1 * (Z1 > 0)
    vdZ1 = _relu(Z1, v["Z1"], vdH1, dH1)
    g["b1"] = vdZ1.sum(axis=0) + _acc(B, np.abs(dZ1).sum(axis=0))
    g["W1"] = vdZ1.T @ (X * X) + _acc(B, np.abs(dZ1).T @ np.abs(X))
    return L, G, LAMBDA * np.sqrt(vL), LAMBDA * np.sqrt(mlp.pack(g))


def violations(got, ref, bound):
    """Boolean mask of the elements farther from ref than bound (NaN counts as outside); a
    floor of 2^-40 times the largest reference value covers exact zeros on both sides."""
    got, ref, bound = (np.asarray(v, np.float64) for v in (got, ref, bound))
    err = np.abs(got - ref)
    floor = 2.0 ** -40 * np.abs(ref).max() if ref.size else 0.0
    return ~(err <= bound + floor)


# ---------------------------------------------------------------- CPU emulation (pins)
def bf16(a):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    a = np.ascontiguousarray(a, np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    r = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _split(a):
    hi = bf16(a)
    lo = bf16(np.asarray(a, np.float32) - hi)
    return hi, lo


def emulate_forward(params, X, mode: str = "train"):
    """The GPU network's arithmetic in numpy float32 with BF16 roundings (test emulation)."""
    p = {k: np.asarray(v, np.float32) for k, v in _p(params).items()}
    X = np.asarray(X, np.float32)
    f32 = np.float32
    if mode == "train":
        Z1 = (X @ p["W1"].T + p["b1"]).astype(f32)
    else:
        xh, xl = _split(X)
        wh, wl = _split(p["W1"])
        bh, bl = _split(p["b1"])
        Z1 = (xh @ wh.T + xh @ wl.T + xl @ wh.T + xl @ wl.T + bh + bl).astype(f32)
    H1 = bf16(np.maximum(Z1, 0))

    def hidden(H, W, bb):
        if mode == "train":
            return (H @ bf16(W).T).astype(f32) + bb
        bh, bl = _split(bb)
        return (H @ bf16(W).T + bh + bl).astype(f32)

    Z2 = hidden(H1, p["W2"], p["b2"])
    H2 = bf16(np.maximum(Z2, 0))
    Z3 = hidden(H2, p["W3"], p["b3"])
    H3 = bf16(np.maximum(Z3, 0))
    if mode == "train":
        Y = (H3 @ p["W4"].T + p["b4"]).astype(f32)
    else:
        wh, wl = _split(p["W4"])
        Y = ((H3 @ wh.T).astype(f32) + (H3 @ wl.T).astype(f32)) + p["b4"]
    return Y, (X, Z1, H1, Z2, H2, Z3, H3)


def emulate_gradients(params, X, T, lam: float = 0.1):
    """(loss, flat gradient) of the GPU training path, emulated in float32 with BF16 roundings."""
    from oracle import mlp
    f32 = np.float32
    p = {k: np.asarray(v, np.float32) for k, v in _p(params).items()}
    Y, (X, Z1, H1, Z2, H2, Z3, H3) = emulate_forward(params, X, "train")
    T = np.asarray(T, np.float32)
    B = X.shape[0]
    d = Y[:, :6] - T
    se = (d * d).sum(axis=1, dtype=f32)
    lg = np.log(se + f32(1e-6)).astype(f32)
    d6 = Y[:, 6] - lg
    dY = np.zeros_like(Y)
    dY[:, :6] = f32(2) * d / f32(6 * B)
    dY[:, 6] = f32(2 * lam) * d6 / f32(B)
    L = float((se / f32(6 * B) + f32(lam) * d6 * d6 / f32(B)).sum(dtype=f32))
    g = {}
    g["W4"] = dY.T @ H3
    g["b4"] = dY.sum(axis=0, dtype=f32)
    dZ3 = bf16((dY @ p["W4"]) * (H3 > 0))
    g["b3"] = dZ3.sum(axis=0, dtype=f32)
    g["W3"] = dZ3.T @ H2
    pre2 = ((dZ3 @ bf16(p["W3"])) * (H2 > 0)).astype(f32)
    g["b2"] = pre2.sum(axis=0, dtype=f32)
    dZ2 = bf16(pre2)
    g["W2"] = dZ2.T @ H1
    dZ1 = ((dZ2 @ bf16(p["W2"])) * (H1 > 0)).astype(f32)
    g["b1"] = dZ1.sum(axis=0, dtype=f32)
    g["W1"] = dZ1.T @ X
    return L, mlp.pack(g)
