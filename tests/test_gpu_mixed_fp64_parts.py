"""Mixed precision keeps FP64 where the method is sensitive: on identical
inputs the mixed-precision scene's energy (distances below dhat, the barrier
log term, friction, elasticity, inertia) and gradient equal the plain FP64
scene's, bit for bit.  The energy runs the same kernels in both modes (as do
the active set and the ACCD); the gradient comes out of the Hessian kernels,
which are instantiated once per Hessian precision but compute the gradient in
FP64, in the same order, in both."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def gpu_scene(sc, **kw):
    from paper_2311_05945_b300.zema import Scene
    return Scene(sc, **kw)


@pytest.mark.parametrize("name,steps", [("tiny", 6), ("c1", 12)])
def test_fp64_parts_identical_across_precisions(name, steps):
    sc = S.scene_tiny_contact(mu=0.5) if name == "tiny" else S.scene_c1()
    orc = Oracle(sc)
    orc.step(steps)  # in contact
    res = []
    for precision in (0, 1):
        g = gpu_scene(sc, precision=precision)
        for b in range(len(sc.body_order())):
            g.set_state(b, orc.get_state(b))
        g.set_kappa(0, orc.kappa(), orc.kappa_min())
        E, grad = g.eval_energy_grad(apply_predictor=True)
        res.append((E, grad))
    (E0, g0), (E1, g1) = res
    assert np.array_equal(E0, E1), (E0, E1)
    assert np.array_equal(g0, g1), np.abs(g0 - g1).max() / np.abs(g0).max()

