"""Tensor-core MLP kernels against the CPU reference: forward values and the
loss gradient against the reference run with the kernels' BF16 rounding
points (only the FP32 summation order differs), and within BF16 accuracy of
the plain FP32 reference; training progress and bit-reproducible training."""
import numpy as np
import pytest

from oracle import mlp_ref

pytestmark = pytest.mark.gpu

DIMS = [13, 128, 128, 128, 3]


def data(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, DIMS[0])).astype(np.float32)
    t = (0.5 * np.tanh(x[:, :3]) + 0.1 * x[:, 3:6] * x[:, 6:9]).astype(np.float32)
    return x, t, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()


def test_forward_matches_reference():
    from paper_2311_05945_b300.zema import Mlp
    net = Mlp(DIMS, seed=1)
    x, t, xd, td = data(1000, 0)   # 1000 rows: 15 full 64-row tiles and a ragged one
    y = net.forward(xd).cpu().numpy()
    yb, _ = mlp_ref.forward(net.get_params(), DIMS, x, bf16=True)
    yr, _ = mlp_ref.forward(net.get_params(), DIMS, x)
    assert np.abs(y - yb).max() < 2e-3 * np.abs(yb).max()
    assert np.abs(y - yr).max() < 3e-2 * np.abs(yr).max()


@pytest.mark.parametrize("n", [1, 77, 4096])
def test_gradient_matches_reference(n):
    from paper_2311_05945_b300.zema import Mlp
    net = Mlp(DIMS, seed=2)
    x, t, xd, td = data(n, 1)
    loss, g = net.gradient(xd, td)
    lb, gb = mlp_ref.loss_and_grad(net.get_params(), DIMS, x, t, bf16=True)
    lr, gr = mlp_ref.loss_and_grad(net.get_params(), DIMS, x, t)
    assert abs(loss - lb) <= 1e-3 * lb
    assert abs(loss - lr) <= 3e-2 * lr
    # element by element against the reference with the same rounding
    # points: the kernels differ from it only in FP32 summation order, whose
    # effect on an entry is bounded by a few units of bfloat16 rounding (a
    # tie that flips the rounding of an intermediate activation or gradient,
    # 2^-8 relative) times the entry's sum of absolute products
    scale = mlp_ref.grad_abs_scale(net.get_params(), DIMS, x, t, bf16=True)
    err = np.abs(g - gb)
    bound = 2.0 ** -6 * scale + 1e-6 * np.abs(gb).max()
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), (worst, err[worst], bound[worst], float((err / bound).max()))
    # per layer, relative to that layer's gradient norm: against the reference
    # with the same rounding points and against plain FP32 (bfloat16 accuracy
    # through three back-propagated layers)
    o = 0
    for l in range(len(DIMS) - 1):
        k = DIMS[l] * DIMS[l + 1] + DIMS[l + 1]
        a, b, c = g[o:o + k], gb[o:o + k], gr[o:o + k]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-9, (l, np.linalg.norm(a - b), np.linalg.norm(b))
        assert np.linalg.norm(a - c) <= 1e-1 * np.linalg.norm(c) + 1e-9, (l, np.linalg.norm(a - c), np.linalg.norm(c))
        o += k


def test_training_reduces_loss_and_is_reproducible():
    from paper_2311_05945_b300.zema import Mlp
    x, t, xd, td = data(8192, 2)
    runs = []
    for _ in range(2):
        net = Mlp(DIMS, seed=3)
        first = None
        for it in range(300):
            l = net.train_step(xd, td, lr=2e-3)
            first = l if first is None else first
        runs.append((first, l, net.get_params()))
    (f0, l0, p0), (f1, l1, p1) = runs
    assert l0 < 0.2 * f0, (f0, l0)
    assert np.array_equal(p0, p1)


@pytest.mark.parametrize("n", [1, 200, 5000])
def test_tcgen05_forward_matches_warp_mma(n):
    # the fifth-generation tensor-core forward (accumulators in tensor memory)
    # against the warp-level mma.sync kernel on the same BF16 operands
    from paper_2311_05945_b300.zema import Mlp
    net = Mlp(DIMS, seed=4)
    x, t, xd, td = data(n, 3)
    y_tc = net.forward(xd).cpu().numpy()
    net.set_kernel(1)
    y_mma = net.forward(xd).cpu().numpy()
    assert np.abs(y_tc - y_mma).max() <= 2e-3 * max(1e-6, np.abs(y_mma).max())
    yb, _ = mlp_ref.forward(net.get_params(), DIMS, x, bf16=True)
    assert np.abs(y_tc - yb).max() <= 2e-3 * max(1e-6, np.abs(yb).max())
