"""GPU local kernels against the oracle on the same seeded inputs: distances
and closest-point weights, barrier energy / gradient / projected Hessian
(Eq. 5-8), Neo-Hookean density / stress / projected F-space Hessian, ACCD."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _stencils(seed, n, scale=1.0, near=False):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 12)) * scale
    if near:  # many point-near-triangle and crossing-edge configurations
        x[::3, 0:3] = (x[::3, 3:6] + x[::3, 6:9] + x[::3, 9:12]) / 3 + 0.05 * scale * rng.standard_normal((len(x[::3]), 3))
    return x


@pytest.mark.parametrize("is_ee", [0, 1])
def test_distance_matches_oracle(is_ee):
    from paper_2311_05945_b300 import zema as Z
    x = _stencils(11 + is_ee, 3000, near=True)
    d2, w = Z.local_distance(x, is_ee)
    for i in range(len(x)):
        r, kind, wr, _, _ = O.stencil_d2(x[i], is_ee)
        assert abs(d2[i] - r) <= 1e-12 * max(1.0, r), (i, d2[i], r)
        # weights give the same closest-point difference vector
        a = (w[i][:, None] * x[i].reshape(4, 3)).sum(0)
        b = (wr[:, None] * x[i].reshape(4, 3)).sum(0)
        assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("is_ee", [0, 1])
def test_barrier_matches_oracle(is_ee):
    from paper_2311_05945_b300 import zema as Z
    rng = np.random.default_rng(21 + is_ee)
    dhat = 1.0
    xs = []
    while len(xs) < 400:
        x = rng.standard_normal(12) * 0.6
        d2 = O.stencil_d2(x, is_ee)[0]
        if 1e-4 < d2 < 0.95:
            xs.append(x)
    xs = np.array(xs)
    eps = np.where(np.arange(len(xs)) % 2 == 0, 1e-3, 10.0) if is_ee else np.zeros(len(xs))
    E, g, H = Z.local_barrier(xs, is_ee, eps, dhat)
    for i in range(len(xs)):
        b, gr, Hr = O.pair_barrier(xs[i], is_ee, dhat, eps[i] if is_ee else 1.0, project=True)
        assert abs(E[i] - b) <= 1e-9 * max(1e-12, abs(b)), (i, E[i], b)
        assert np.abs(g[i] - gr).max() <= 1e-8 * max(1e-12, np.abs(gr).max()), i
        assert np.abs(H[i] - Hr).max() <= 1e-7 * max(1e-12, np.abs(Hr).max()), i


def test_barrier_inactive_is_zero():
    from paper_2311_05945_b300 import zema as Z
    x = np.array([[0.2, 0.2, 2.0, 0, 0, 0, 1, 0, 0, 0, 1, 0]], dtype=float)
    E, g, H = Z.local_barrier(x, 0, 0.0, 1.0)
    assert E[0] == 0 and not g.any() and not H.any()


def test_neo_hookean_matches_oracle():
    from paper_2311_05945_b300 import zema as Z
    rng = np.random.default_rng(5)
    Fs = np.eye(3)[None] + 0.35 * rng.standard_normal((600, 3, 3))
    Fs = Fs[np.linalg.det(Fs) > 0.05]
    mu, lam = 3.4e4, 3.1e5
    psi, P, H = Z.local_neo_hookean(Fs, mu, lam)
    for i in range(len(Fs)):
        v, g, Hr = O.nh(Fs[i], mu, lam, project=True)
        assert abs(psi[i] - v) <= 1e-10 * max(1.0, abs(v))
        assert np.abs(P[i] - g).max() <= 1e-9 * max(1.0, np.abs(g).max())
        assert np.abs(H[i] - Hr).max() <= 1e-8 * max(1.0, np.abs(Hr).max())


@pytest.mark.parametrize("model", [1, 2])
def test_other_materials_match_oracle(model):
    # St. Venant-Kirchhoff (1) and fixed corotated (2): density, stress and
    # PSD-projected F-space Hessian against the oracle's forward-mode
    # derivatives (for 2 through the polar iteration, on the GPU the closed
    # differential of the polar rotation)
    from paper_2311_05945_b300 import zema as Z
    rng = np.random.default_rng(7 + model)
    Fs = np.eye(3)[None] + 0.35 * rng.standard_normal((400, 3, 3))
    Fs = Fs[np.linalg.det(Fs) > 0.05]
    mu, lam = 3.4e4, 3.1e5
    psi, P, H = Z.local_elastic(Fs, mu, lam, model)
    ref = O.stvk if model == 1 else O.fcr
    for i in range(len(Fs)):
        v, g, Hr = ref(Fs[i], mu, lam, project=True)
        assert abs(psi[i] - v) <= 1e-10 * max(1.0, abs(v))
        assert np.abs(P[i] - g).max() <= 1e-9 * max(1.0, np.abs(g).max())
        assert np.abs(H[i] - Hr).max() <= 1e-7 * max(1.0, np.abs(Hr).max()), i
    if model == 2:
        Fi = Fs[0].copy()
        Fi[:, 0] *= -1
        assert Z.local_elastic(Fi[None], mu, lam, 2)[0][0] == np.inf


@pytest.mark.parametrize("is_ee", [0, 1])
def test_accd_matches_oracle(is_ee):
    from paper_2311_05945_b300 import zema as Z
    rng = np.random.default_rng(77 + is_ee)
    n = 500
    x = rng.standard_normal((n, 12))
    p = rng.standard_normal((n, 12)) * 1.5
    t = Z.local_accd(x, p, is_ee)
    ref = np.array([O.accd(x[i], p[i], is_ee)[0] for i in range(n)])
    # identical arithmetic up to rounding; a rounding difference at the stop
    # test can move t by at most one sub-step, so compare with a tolerance and
    # count exact agreements
    close = np.abs(t - ref) <= 1e-9 * np.maximum(ref, 1e-12)
    assert close.mean() > 0.98
    assert np.all(t > 0) and np.all(t <= 1.0)
    # closed form head-on
    x0 = np.array([[0.2, 0.2, 0.01, 0, 0, 0, 1, 0, 0, 0, 1, 0]], dtype=float)
    p0 = np.zeros((1, 12))
    p0[0, 2] = -0.05
    assert abs(Z.local_accd(x0, p0, 0)[0] - 0.9 * 0.01 / 0.05) < 1e-14
