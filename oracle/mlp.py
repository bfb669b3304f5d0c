"""FP64 reference of the 4-64-64-4 network that warm-starts the energy Newton
solve (test infrastructure only).

Parameter vector (FP32 on the GPU side, float64 here), in this order:
  W1[64][4], b1[64], W2[64][64], b2[64], W3[4][64], b3[4],
  mean[4], inv_std[4]   (input standardisation),
  out_scale[4]          (output scale).
Inputs are the moments' features (rho, u_x, u_y, theta = 2E/rho - |u|^2);
outputs are (mu - mu0) / out_scale with mu the four Lagrange multipliers of
ln(f*_i / W_i) = mu . (1, v_x, v_y, |v|^2) and mu0 = (ln rho - 3/2 u^2,
3 u_x, 3 u_y, 0) the polynomial start point.

Numerics mirrored from the GPU kernels (round=True): the standardisation
(f - mean) * inv_std and the targets dmu / out_scale are evaluated in FP32
(one correctly rounded operation at a time, as the kernels do); standardised
inputs, weights and hidden activations are rounded to BF16 (round to nearest
even); products and sums are exact here (FP64).  Gradients pass straight
through the BF16 roundings (they are taken with respect to the master
weights).  Loss: mean over the batch and the four outputs of the squared
error.

The kernels accumulate the hidden pre-activations z in FP32 in an order of
their own, so where an FP64 z lies within a hair of a BF16 rounding
boundary (or of 0, for the ReLU) the two sides may round it differently.
forward(..., band=b) flags every sample holding such a z (|z - boundary| <
b x the sum of the absolute values of z's terms): the outputs of unflagged
samples are fixed by the arithmetic above up to FP32 accumulation error.

This module is test infrastructure: only the tests and the benchmark's CPU
baseline use it.
"""
import numpy as np

N_IN, N_HID, N_OUT = 4, 64, 4
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,)), ("mean", (N_IN,)), ("inv_std", (N_IN,)),
         ("out_scale", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    r = r.astype(np.uint32)
    nan = np.isnan(f)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def features(rho, jx, jy, e2):
    rho = np.asarray(rho, np.float64)
    ux, uy = jx / rho, jy / rho
    return np.stack([rho, ux, uy, e2 / rho - ux * ux - uy * uy], axis=-1)


def mu0(rho, jx, jy):
    ux, uy = jx / rho, jy / rho
    return np.stack([np.log(rho) - 1.5 * (ux * ux + uy * uy), 3 * ux, 3 * uy, np.zeros_like(ux)],
                    axis=-1)


def standardise(p, feat, round=True):
    d = unpack(p)
    if not round:
        return (np.asarray(feat, np.float64) - d["mean"]) * d["inv_std"]
    f32 = np.float32
    x = (np.asarray(feat, f32) - d["mean"].astype(f32)).astype(f32) * d["inv_std"].astype(f32)
    return bf16(x.astype(f32))


def targets(p, dmu, round=True):
    d = unpack(p)
    if not round:
        return np.asarray(dmu, np.float64) / d["out_scale"]
    f32 = np.float32
    return (np.asarray(dmu, f32) / d["out_scale"].astype(f32)).astype(np.float64)


def _near_boundary(z, mag, band):
    """z within band * mag of a BF16 rounding boundary (a midpoint between
    adjacent BF16 values) or of 0."""
    z = np.asarray(z, np.float64)
    az = np.abs(z).astype(np.float32)
    e = np.floor(np.log2(np.maximum(az, np.float32(2.0 ** -126)))).astype(np.float64)
    ulp = np.exp2(e - 7.0)                              # BF16 spacing at |z|
    mid = (np.floor(np.abs(z) / ulp) + 0.5) * ulp       # the nearest boundary above
    dist = np.minimum(np.abs(np.abs(z) - mid), np.abs(np.abs(z) - (mid - ulp)))
    dist = np.minimum(dist, np.abs(z))
    return dist < band * mag


def forward(p, feat, round=True, band=0.0):
    """Outputs y (scaled multiplier corrections), the cached activations and,
    when band > 0, the per-sample flags of near-boundary roundings."""
    d = unpack(p)
    r = bf16 if round else (lambda a: np.asarray(a, np.float64))
    x = standardise(p, feat, round)
    W1, W2, W3 = r(d["W1"]), r(d["W2"]), r(d["W3"])
    z1 = x @ W1.T + d["b1"]
    h1 = r(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + d["b2"]
    h2 = r(np.maximum(z2, 0.0))
    y = h2 @ W3.T + d["b3"]
    cache = dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, W3=W3)
    if band > 0:
        m1 = np.abs(x) @ np.abs(W1).T + np.abs(d["b1"])
        m2 = h1 @ np.abs(W2).T + np.abs(d["b2"])
        cache["ambiguous"] = (_near_boundary(z1, m1, band).any(axis=1) |
                              _near_boundary(z2, m2, band).any(axis=1))
    return y, cache


def forward_bounds(p, feat, band):
    """Bounds [y_lo, y_hi] of the outputs of every evaluation of the rounded
    network whose hidden pre-activations z stray from their exact values by
    at most band x the sum of the absolute values of z's terms (the FP32
    accumulation of the kernels, in any order).  Rounding to BF16 and the
    ReLU are monotone, so a hidden value lies between the roundings of the
    ends of its z interval; hidden values are >= 0, so the next layer's
    interval takes the positive weights at the same end and the negative
    ones at the other.  The output layer's own accumulation error is left to
    the caller's tolerance.  With band = 0 both bounds are forward's y (up to
    the order of the FP64 sums)."""
    d = unpack(p)
    x = standardise(p, feat, True)
    W1, W2, W3 = bf16(d["W1"]), bf16(d["W2"]), bf16(d["W3"])
    z1 = x @ W1.T + d["b1"]
    m1 = np.abs(x) @ np.abs(W1).T + np.abs(d["b1"])
    h1lo = bf16(np.maximum(z1 - band * m1, 0.0))
    h1hi = bf16(np.maximum(z1 + band * m1, 0.0))
    W2p, W2n = np.maximum(W2, 0.0), np.minimum(W2, 0.0)
    z2lo = h1lo @ W2p.T + h1hi @ W2n.T + d["b2"]
    z2hi = h1hi @ W2p.T + h1lo @ W2n.T + d["b2"]
    m2 = h1hi @ np.abs(W2).T + np.abs(d["b2"])
    h2lo = bf16(np.maximum(z2lo - band * m2, 0.0))
    h2hi = bf16(np.maximum(z2hi + band * m2, 0.0))
    W3p, W3n = np.maximum(W3, 0.0), np.minimum(W3, 0.0)
    ylo = h2lo @ W3p.T + h2hi @ W3n.T + d["b3"]
    yhi = h2hi @ W3p.T + h2lo @ W3n.T + d["b3"]
    return ylo, yhi


def loss_and_grad(p, feat, dmu, round=True):
    """Mean squared error against dmu / out_scale and its gradient with
    respect to the parameters (the standardisation and output-scale entries
    get zero gradient)."""
    y, c = forward(p, feat, round)
    B = y.shape[0]
    diff = y - targets(p, dmu, round)
    loss = float((diff * diff).sum() / (B * N_OUT))
    dy = 2.0 * diff / (B * N_OUT)
    g = {name: np.zeros(shape) for name, shape in SIZES}
    g["W3"] = dy.T @ c["h2"]
    g["b3"] = dy.sum(0)
    dz2 = (dy @ c["W3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ c["W2"]) * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["x"]
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def adam_step(p, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) of the trainable entries."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    trainable = np.zeros_like(p, bool)
    o = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        if name in ("W1", "b1", "W2", "b2", "W3", "b3"):
            trainable[o:o + n] = True
        o += n
    p = p.copy()
    p[trainable] -= lr * mh[trainable] / (np.sqrt(vh[trainable]) + eps)
    return p, m, v


def init_params(seed_uniform, mean, inv_std, out_scale):
    """He-uniform weights from the given uniform [-1, 1) draws, zero biases."""
    u = np.asarray(seed_uniform, np.float64)
    d, o = {}, 0
    for name, shape in SIZES[:6]:
        n = int(np.prod(shape))
        if name.startswith("W"):
            fan_in = shape[1]
            d[name] = (u[o:o + n] * np.sqrt(6.0 / fan_in)).reshape(shape)
        else:
            d[name] = np.zeros(shape)
        o += n
    d["mean"], d["inv_std"], d["out_scale"] = mean, inv_std, out_scale
    return pack(d)
