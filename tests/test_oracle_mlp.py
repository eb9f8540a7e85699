"""Pins of the CPU reference MLP (warm-start network): central finite
differences of the loss, the vanishing gradient at the least-squares
optimum of a single linear layer, and bfloat16 rounding against a library
conversion."""
import numpy as np

from oracle import mlp_ref


def test_reference_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    dims = [5, 7, 6, 2]
    n_par = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))
    theta = rng.normal(size=n_par) * 0.7
    x = rng.normal(size=(9, dims[0]))
    t = rng.normal(size=(9, dims[-1]))
    loss, g = mlp_ref.loss_and_grad(theta, dims, x, t)
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(n_par):
        e = np.zeros_like(theta)
        e[i] = h
        fd[i] = (mlp_ref.loss_and_grad(theta + e, dims, x, t)[0] - mlp_ref.loss_and_grad(theta - e, dims, x, t)[0]) / (2 * h)
    assert np.abs(fd - g).max() < 1e-6 * max(1.0, np.abs(g).max())
    assert loss > 0


def test_reference_gradient_vanishes_at_least_squares_optimum():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(40, 3))
    t = rng.normal(size=(40, 2))
    xa = np.hstack([x, np.ones((40, 1))])
    sol, *_ = np.linalg.lstsq(xa, t, rcond=None)
    theta = np.concatenate([sol[:3].ravel(), sol[3]])
    _, g = mlp_ref.loss_and_grad(theta, [3, 2], x, t)
    assert np.abs(g).max() < 1e-12
    # and away from it the loss is larger
    l0 = mlp_ref.loss_and_grad(theta, [3, 2], x, t)[0]
    assert mlp_ref.loss_and_grad(theta + 1e-3, [3, 2], x, t)[0] > l0


def test_bf16_rounding_matches_a_library_conversion():
    # the reference's bfloat16 rounding (nearest, ties to even) against
    # torch's float32 -> bfloat16 conversion on random and tie values
    import torch
    rng = np.random.default_rng(5)
    a = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 3.0 + 2 ** -7], dtype=np.float32)
    a = np.concatenate([a, ties, np.float32([0.0, -0.0, 1e-40, 3.4e38])])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    out = mlp_ref.round_bf16(a)
    assert np.array_equal(out.view(np.uint32), ref.view(np.uint32))
    assert out[-8] == 1.0 and out[-7] == np.float32(1 + 2 ** -6)  # ties go to the even significand


def test_abs_scale_bounds_the_gradient_and_is_tight_without_cancellation():
    # |g| <= scale always (triangle inequality); with non-negative inputs,
    # weights and output errors nothing cancels and the two are equal
    rng = np.random.default_rng(6)
    dims = [4, 6, 3]
    n_par = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))
    theta = np.abs(rng.normal(size=n_par))
    x = np.abs(rng.normal(size=(11, dims[0])))
    t = -np.ones((11, dims[-1]))  # below every output: all output errors positive
    _, g = mlp_ref.loss_and_grad(theta, dims, x, t)
    s = mlp_ref.grad_abs_scale(theta, dims, x, t)
    assert np.allclose(np.abs(g), s, rtol=1e-12, atol=0)
    theta2 = rng.normal(size=n_par)
    x2 = rng.normal(size=(11, dims[0]))
    t2 = rng.normal(size=(11, dims[-1]))
    _, g2 = mlp_ref.loss_and_grad(theta2, dims, x2, t2)
    s2 = mlp_ref.grad_abs_scale(theta2, dims, x2, t2)
    assert np.all(np.abs(g2) <= s2 * (1 + 1e-12))
    assert np.any(np.abs(g2) < 0.9 * s2)  # signs mixed: some entries cancel
