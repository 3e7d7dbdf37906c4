"""Oracle for the warm-start convolutional net (test infrastructure only: tests, smoke and the bench's
CPU leg use it; the library never does).

Plain FP64 numpy restatement of what lbm_net_* computes:
  forward   Z_l = b_l + sum_o W_l[o] X_l[v + o]  (3x3x3 taps, zero padding), X_{l+1} = relu(Z_l),
            no activation after the last layer; prediction = skip + Z_last[..., :cout]
  loss      mean over marked voxels and output channels of (prediction - target)^2
  backward  written out by hand: dW_l[o] = sum_v dZ_l[v] (x) X_l[v + o], db_l = sum_v dZ_l[v],
            dX_l[u] = sum_o W_l[o]^T dZ_l[u - o], dZ_{l-1} = dX_l * [X_l > 0]
Parameters use the library's flat layout: per layer W[27][16 out][16 in] (tap o = (dz+1)*9 +
(dy+1)*3 + (dx+1)) followed by b[16].  With `bf16_round=True` the oracle rounds to BF16 (round to nearest
even) where the GPU does: the input, the weights, each layer's output and each dZ before it enters a
product; sums stay FP64.

Pins (tests/test_net.py, CPU): the convolution against a brute-force loop, an identity tap, and the
hand-written gradients against central finite differences of the loss.
"""
import numpy as np

CH = 16
TAPS = 27
PER_LAYER = TAPS * CH * CH + CH


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, layers):
    p = np.asarray(params, dtype=np.float64)
    out = []
    for l in range(layers):
        base = l * PER_LAYER
        W = p[base:base + TAPS * CH * CH].reshape(TAPS, CH, CH)
        b = p[base + TAPS * CH * CH:base + PER_LAYER]
        out.append((W, b))
    return out


def tap(o):
    return o // 9 - 1, (o // 3) % 3 - 1, o % 3 - 1   # dz, dy, dx


def shift(x, dz, dy, dx):
    """s[v] = x[v + (dz, dy, dx)] with zeros outside the volume; x is [nvol, D, H, W, C]."""
    n, D, H, W, C = x.shape
    xp = np.zeros((n, D + 2, H + 2, W + 2, C))
    xp[:, 1:D + 1, 1:H + 1, 1:W + 1] = x
    return xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv3d(x, W, b=None):
    """Z[v][m] = b[m] + sum_o sum_k W[o][m][k] x[v + o][k]."""
    z = np.zeros(x.shape[:-1] + (W.shape[1],))
    for o in range(TAPS):
        z += shift(x, *tap(o)) @ W[o].T
    if b is not None:
        z += b
    return z


def forward(params, x, layers, bf16_round=False):
    """Returns [X_0, ..., X_{L-1}, Z_{L-1}] (X_0 = x)."""
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    acts = [r(x)]
    for l, (W, b) in enumerate(unpack(params, layers)):
        z = conv3d(acts[-1], r(W), b)
        if l + 1 < layers:
            z = np.maximum(z, 0.0)
        acts.append(r(z))
    return acts


def loss_and_grads(params, x, target, layers, cout, skip=None, weight=None, bf16_round=False):
    """MSE of skip + Z_last[..., :cout] against target over voxels marked by weight, and the
    gradient of every parameter (flat layout)."""
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    acts = forward(params, x, layers, bf16_round)
    pred = acts[-1][..., :cout] + (0.0 if skip is None else skip)
    w = np.ones(x.shape[:-1]) if weight is None else np.asarray(weight, dtype=np.float64)
    count = w.sum() * cout
    err = pred - target
    loss = float((w[..., None] * err * err).sum() / count)
    dz = np.zeros(acts[-1].shape)
    dz[..., :cout] = 2.0 * w[..., None] * err / count
    dz = r(dz)
    grads = np.zeros(layers * PER_LAYER)
    wl = unpack(params, layers)
    for l in range(layers - 1, -1, -1):
        X = acts[l]
        W = r(wl[l][0])
        gW = np.zeros((TAPS, CH, CH))
        for o in range(TAPS):
            gW[o] = dz.reshape(-1, CH).T @ shift(X, *tap(o)).reshape(-1, CH)
        base = l * PER_LAYER
        grads[base:base + TAPS * CH * CH] = gW.ravel()
        grads[base + TAPS * CH * CH:base + PER_LAYER] = dz.reshape(-1, CH).sum(axis=0)
        if l > 0:
            dx = np.zeros(X.shape)
            for o in range(TAPS):
                dzz, dyy, dxx = tap(o)
                dx += shift(dz, -dzz, -dyy, -dxx) @ W[o]
            dz = r(dx * (X > 0))
    return loss, grads, pred
