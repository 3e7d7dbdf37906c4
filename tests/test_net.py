"""The warm-start convolutional net: the FP64 oracle pinned on the CPU, the tensor-core kernels
(lbm_net_*) against it on the GPU.

GPU tolerances: the kernels round every layer's output and every gradient entering a product to
BF16 (8 significant bits), as the oracle does in its bf16 mode; the sums differ (FP32 on the GPU,
FP64 in the oracle), so a rounding can land one BF16 step apart.  Forward outputs must agree to
4 BF16 steps of the largest value (2^-6), parameter gradients to 2 % of the largest gradient.
"""
import numpy as np
import pytest

from oracle import conv_net as O


def _rng(seed=1):
    return np.random.default_rng(seed)


def _params(rng, layers, cin, cout, scale=1.0):
    p = np.zeros(layers * O.PER_LAYER)
    for l in range(layers):
        ci = cin if l == 0 else O.CH
        co = cout if l + 1 == layers else O.CH
        W = np.zeros((O.TAPS, O.CH, O.CH))
        W[:, :co, :ci] = rng.normal(0.0, scale * np.sqrt(2.0 / (O.TAPS * ci)), (O.TAPS, co, ci))
        b = np.zeros(O.CH)
        b[:co] = rng.normal(0.0, 0.1, co)
        p[l * O.PER_LAYER:(l + 1) * O.PER_LAYER] = np.concatenate([W.ravel(), b])
    return p


def _input(rng, shape, cin):
    x = np.zeros(shape + (O.CH,))
    x[..., :cin] = rng.normal(0.0, 1.0, shape + (cin,))
    return x


# ---------------------------------------------------------------- oracle pins (CPU)

def test_conv3d_matches_a_brute_force_loop():
    rng = _rng(2)
    x = rng.normal(size=(2, 3, 4, 5, O.CH))
    W = rng.normal(size=(O.TAPS, O.CH, O.CH))
    b = rng.normal(size=O.CH)
    z = O.conv3d(x, W, b)
    n, D, H, Wd, _ = x.shape
    ref = np.zeros_like(z)
    for v in range(n):
        for k in range(D):
            for j in range(H):
                for i in range(Wd):
                    s = b.copy()
                    for o in range(O.TAPS):
                        dz, dy, dx = o // 9 - 1, (o // 3) % 3 - 1, o % 3 - 1
                        kk, jj, ii = k + dz, j + dy, i + dx
                        if 0 <= kk < D and 0 <= jj < H and 0 <= ii < Wd:
                            s = s + W[o] @ x[v, kk, jj, ii]
                    ref[v, k, j, i] = s
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


def test_centre_tap_identity_returns_the_input():
    x = _rng(3).normal(size=(1, 4, 3, 5, O.CH))
    W = np.zeros((O.TAPS, O.CH, O.CH))
    W[13] = np.eye(O.CH)
    assert np.array_equal(O.conv3d(x, W), x)
    W[13] = 0.0
    W[14] = np.eye(O.CH)           # tap (0, 0, +1): z[x] = x[x + 1], zero at the last column
    z = O.conv3d(x, W)
    assert np.array_equal(z[..., :-1, :], x[..., 1:, :]) and not z[..., -1, :].any()


def test_gradients_match_central_differences():
    rng = _rng(4)
    layers, cin, cout = 3, 3, 2
    p = _params(rng, layers, cin, cout)
    for l in range(layers - 1):          # positive hidden pre-activations: no ReLU kink nearby
        p[l * O.PER_LAYER + O.TAPS * O.CH * O.CH:(l + 1) * O.PER_LAYER] = 5.0
    x = _input(rng, (1, 3, 3, 4), cin)
    target = rng.normal(size=(1, 3, 3, 4, cout))
    weight = (rng.random((1, 3, 3, 4)) < 0.7).astype(float)
    skip = rng.normal(size=(1, 3, 3, 4, cout))
    loss, g, _ = O.loss_and_grads(p, x, target, layers, cout, skip, weight)
    nz = np.flatnonzero(p)
    pick = np.concatenate([rng.choice(nz, 40, replace=False), [O.PER_LAYER - 1, 2 * O.PER_LAYER - 3]])
    eps = 1e-6
    for i in pick:
        q = p.copy()
        q[i] += eps
        lp = O.loss_and_grads(q, x, target, layers, cout, skip, weight)[0]
        q[i] -= 2 * eps
        lm = O.loss_and_grads(q, x, target, layers, cout, skip, weight)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])


def test_relu_blocks_gradients_of_dead_units():
    rng = _rng(5)
    layers, cin, cout = 2, 2, 2
    p = _params(rng, layers, cin, cout)
    p[O.TAPS * O.CH * O.CH:O.PER_LAYER] = -1e3      # every hidden unit of layer 0 is off
    x = _input(rng, (1, 2, 3, 3), cin)
    _, g, _ = O.loss_and_grads(p, x, rng.normal(size=(1, 2, 3, 3, cout)), layers, cout)
    assert not g[:O.PER_LAYER].any()


def test_bf16_rounding_is_round_to_nearest_even():
    one = 1.0
    ulp = 2.0 ** -7
    assert O.bf16(one + ulp / 2) == one             # tie, even neighbour is 1.0
    assert O.bf16(one + 1.5 * ulp) == one + 2 * ulp  # tie, even neighbour above
    assert O.bf16(one + 0.51 * ulp) == one + ulp
    assert O.bf16(-3.0) == -3.0


# ---------------------------------------------------------------- GPU against the oracle

@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07982_gb300 import build, lbm as mod
    build.build()
    return mod


def _dev(a, dtype):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.gpu
@pytest.mark.parametrize("backend", ["tcgen05", "mma.sync"])
def test_net_forward_matches_the_oracle(lbm, backend):
    import torch
    rng = _rng(6)
    layers, cin, cout = 5, 6, 4
    net = lbm.Net(layers, cin, cout, seed=1)
    net.set_backend(backend)
    p = _params(rng, layers, cin, cout)
    p_b = p.copy()
    for l in range(layers):                       # BF16-representable weights
        s = slice(l * O.PER_LAYER, l * O.PER_LAYER + O.TAPS * O.CH * O.CH)
        p_b[s] = O.bf16(p[s])
    net.set_params(p_b)
    x = O.bf16(_input(rng, (2, 5, 6, 7), cin))     # 420 voxels: not a multiple of 16
    z = net.forward(_dev(x, torch.bfloat16)).float().cpu().numpy()
    ref = O.forward(p_b, x, layers, bf16_round=True)[-1]
    assert np.abs(z - ref).max() <= 2.0 ** -6 * np.abs(ref).max()
    assert np.abs(z[..., cout:]).max() == 0.0
    net.close()


@pytest.mark.gpu
@pytest.mark.parametrize("backend", ["tcgen05", "mma.sync"])
def test_net_gradients_match_the_oracle(lbm, backend):
    import torch
    rng = _rng(7)
    layers, cin, cout = 5, 6, 4
    shape = (3, 6, 5, 9)
    net = lbm.Net(layers, cin, cout, seed=2)
    net.set_backend(backend)
    p = _params(rng, layers, cin, cout)
    for l in range(layers):
        s = slice(l * O.PER_LAYER, l * O.PER_LAYER + O.TAPS * O.CH * O.CH)
        p[s] = O.bf16(p[s])
    net.set_params(p)
    x = O.bf16(_input(rng, shape, cin))
    target = rng.normal(size=shape + (cout,))
    skip = rng.normal(size=shape + (cout,))
    weight = np.zeros(shape)
    weight[:, 1:-1, 1:-1, 1:-1] = 1.0              # interior voxels only, as for a block and its halo
    pred = net.predict(_dev(x, torch.bfloat16), _dev(skip, torch.float32)).cpu().numpy()
    loss = net.gradient(_dev(target, torch.float32), _dev(skip, torch.float32), _dev(weight, torch.float32))
    g = net.grads()
    rl, rg, rp = O.loss_and_grads(p, x, target, layers, cout, skip, weight, bf16_round=True)
    assert np.abs(pred - rp).max() <= 2.0 ** -6 * np.abs(rp).max()
    assert abs(loss - rl) <= 1e-2 * rl
    assert np.abs(g - rg).max() <= 2e-2 * np.abs(rg).max()
    net.close()


@pytest.mark.gpu
def test_tensor_core_paths_agree_on_a_block_volume(lbm):
    """The tcgen05 and mma.sync products on an 18^3 volume (a block of 8^3 with its halo of 5):
    several tiles per plane, and planes at the volume's z faces."""
    import torch
    rng = _rng(9)
    layers, cin, cout = 5, 6, 4
    p = _params(rng, layers, cin, cout)
    x = _dev(O.bf16(_input(rng, (3, 18, 18, 18), cin)), torch.bfloat16)
    out = {}
    for backend in ("tcgen05", "mma.sync"):
        net = lbm.Net(layers, cin, cout, seed=4)
        net.set_backend(backend)
        net.set_params(p)
        out[backend] = net.forward(x).float().cpu().numpy()
        net.close()
    a, b = out["tcgen05"], out["mma.sync"]
    assert np.abs(a - b).max() <= 2.0 ** -6 * np.abs(b).max()


@pytest.mark.gpu
def test_net_training_reduces_the_loss(lbm):
    import torch
    rng = _rng(8)
    layers, cin, cout = 5, 6, 4
    shape = (4, 10, 10, 10)
    x = O.bf16(_input(rng, shape, cin))
    # target: a smooth function of the input that the net can represent
    teacher = _params(rng, 2, cin, cout, scale=0.5)
    target = O.forward(teacher, x, 2)[-1][..., :cout]
    net = lbm.Net(layers, cin, cout, seed=3)
    xd, td = _dev(x, torch.bfloat16), _dev(target, torch.float32)
    first = net.train_step(xd, td, lr=2e-3)
    for _ in range(150):
        last = net.train_step(xd, td, lr=2e-3)
    assert last < 0.2 * first
    net.close()


@pytest.mark.gpu
def test_a_tensor_core_wait_that_runs_out_is_reported(lbm):
    """Failure detection without a GPU fault: in its wait test the tcgen05 convolution issues no
    products, so its bounded mbarrier wait runs out with nothing asynchronous in flight.  The kernel
    flags it and returns; the forward pass returns LBM_ETIMEOUT.  Switched off, the same net on the
    same input matches the mma.sync path again (the context stays usable)."""
    import torch
    rng = _rng(11)
    layers, cin, cout = 5, 6, 4
    p = _params(rng, layers, cin, cout)
    x = _dev(O.bf16(_input(rng, (2, 18, 18, 18), cin)), torch.bfloat16)
    net = lbm.Net(layers, cin, cout, seed=4)
    net.set_params(p)
    net.set_wait_test(True)
    with pytest.raises(lbm.LBMError) as ei:
        net.forward(x)
    assert ei.value.status == lbm.LBM_ETIMEOUT
    net.set_wait_test(False)
    a = net.forward(x).float().cpu().numpy()
    ref = lbm.Net(layers, cin, cout, seed=4)
    ref.set_backend("mma.sync")
    ref.set_params(p)
    b = ref.forward(x).float().cpu().numpy()
    assert np.abs(a - b).max() <= 2.0 ** -6 * np.abs(b).max()
    net.close()
    ref.close()
