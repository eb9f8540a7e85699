"""The barrier-stiffness rules on the CUDA path: the initial gradient balance
against the oracle (clamped and unclamped), and the doubling rule with its cap
along a weak-barrier trajectory, in both precisions."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def gpu_scene(sc, **kw):
    from paper_2311_05945_b300.zema import Scene
    return Scene(sc, **kw)


@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_gpu_initial_kappa_matches_oracle(name):
    s = S.scene_tiny_contact(mu=0.5) if name == "tiny" else S.scene_c1()
    states = None
    if name == "c1":
        o0 = Oracle(s)
        o0.step(12)  # in contact: the balance lies above kappa_min
        states = [o0.get_state(b) for b in range(len(s.body_order()))]
    o = Oracle(s)
    g = gpu_scene(s)
    if states:
        for b, x in enumerate(states):
            o.set_state(b, x)
            g.set_state(b, x)
    o.prepare(0, friction=True)
    E, _ = g.eval_energy_grad(apply_predictor=True)  # the GPU sets kappa here
    assert abs(g.kappa() - o.kappa()) <= 1e-9 * o.kappa(), (g.kappa(), o.kappa(), o.kappa_min())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kmin", [0.05, 7.5e-6])
def test_gpu_kappa_doubling_rule(kmin, precision):
    s = S.scene_tiny_contact(mu=0.5)
    g = gpu_scene(s, precision=precision)
    g.set_kappa(0, 0.05, kmin)
    dhat = s.params.dhat
    d_prev, k_prev, doubled = np.inf, 0.05, 0
    for _ in range(12):
        st = g.step(1)
        dk, kk = st["dmin"], st["kappa"]
        assert dk > 0
        if dk < 0.1 * dhat and dk < d_prev:
            expect = min(2 * k_prev, 1e4 * kmin)
            doubled += 1
        else:
            expect = k_prev
        assert kk == expect, (dk / dhat, kk, expect)
        d_prev, k_prev = dk, kk
    assert doubled >= 1
