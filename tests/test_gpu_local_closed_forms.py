"""Closed forms checked directly on the CUDA local entry points, independently
of the oracle: plane and crossed-edge distances, the edge-edge mollifier,
Neo-Hookean energy and stress, and the head-on additive-CCD bound."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def Z():
    from paper_2311_05945_b300 import zema
    return zema


def barrier(d, dhat):
    # Eq. 5 written out: -(d - dhat)^2 ln(d / dhat) for d < dhat
    return -(d - dhat) ** 2 * np.log(d / dhat) if d < dhat else 0.0


def test_gpu_distance_closed_forms():
    h = np.array([0.3, 1e-3, 2.5e-6])
    # point above a triangle's interior: d = h
    pt = np.stack([np.concatenate([[0.2, 0.2, t], [0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]]) for t in h])
    d2, _ = Z().local_distance(pt, 0)
    assert np.allclose(d2, h * h, rtol=1e-12, atol=0)
    # perpendicular crossing edges at separation h: d = h
    ee = np.stack([np.concatenate([[-1.0, 0, 0], [1.0, 0, 0], [0, -1.0, t], [0, 1.0, t]]) for t in h])
    d2, _ = Z().local_distance(ee, 1)
    assert np.allclose(d2, h * h, rtol=1e-12, atol=0)


@pytest.mark.parametrize("phi", [0.02, 0.3, 1.2])
def test_gpu_ee_mollifier_closed_form(phi):
    dh, h = 1.0, 0.3
    u = np.array([np.cos(phi), np.sin(phi), 0.0])
    x = np.concatenate([[-1.0, 0, 0], [1.0, 0, 0], [0, 0, h] - u, [0, 0, h] + u])
    c = 16.0 * np.sin(phi) ** 2
    for eps_x in (0.5, 2.0, 8.0):
        r = c / eps_x
        e = r * (2.0 - r) if r < 1.0 else 1.0
        E, _, _ = Z().local_barrier(x[None], 1, eps_x, dh)
        assert abs(E[0] - e * barrier(h, dh)) <= 1e-12 * barrier(h, dh), (phi, eps_x, E[0], e)


@pytest.mark.parametrize("s", [0.7, 1.3])
def test_gpu_neo_hookean_closed_forms(s):
    for mu, lam in ((3.5e4, 0.0), (0.0, 3.1e5), (3.5e4, 3.1e5)):
        psi, g, _ = Z().local_neo_hookean(np.diag([s, 1.0, 1.0])[None], mu, lam)
        ref = mu / 2 * (s * s - 1) - mu * np.log(s) + lam / 2 * np.log(s) ** 2
        assert abs(psi[0] - ref) <= 1e-12 * max(1.0, abs(ref))
        P = np.diag([mu * (s - 1 / s) + lam * np.log(s) / s, lam * np.log(s), lam * np.log(s)])
        assert np.abs(g[0].reshape(3, 3) - P).max() <= 1e-9 * max(1.0, np.abs(P).max())
        psi_s, _, _ = Z().local_neo_hookean((s * np.eye(3))[None], mu, lam)
        ref_s = 1.5 * mu * (s * s - 1) - 3 * mu * np.log(s) + 4.5 * lam * np.log(s) ** 2
        assert abs(psi_s[0] - ref_s) <= 1e-12 * max(1.0, abs(ref_s))


def test_gpu_accd_head_on_closed_form():
    # a point at height d0 over a fixed triangle's interior moving straight
    # down by P: t = (1 - s) d0 / P with s = 0.1; no approach: t = 1
    cases = ((1e-2, 0.05), (3e-4, 1.0), (0.2, 0.21))
    x = np.stack([np.array([0.2, 0.2, d0, 0, 0, 0, 1, 0, 0, 0, 1, 0], dtype=float) for d0, _ in cases])
    p = np.zeros((len(cases), 12))
    for i, (_, P) in enumerate(cases):
        p[i, 2] = -P
    t = Z().local_accd(x, p, 0)
    ref = np.array([0.9 * d0 / P for d0, P in cases])
    assert np.allclose(t, ref, rtol=1e-10, atol=0), (t, ref)
    far = np.array([[0.2, 0.2, 1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0]], dtype=float)
    pf = np.zeros((1, 12))
    pf[0, 2] = -0.1
    assert Z().local_accd(far, pf, 0)[0] == 1.0
