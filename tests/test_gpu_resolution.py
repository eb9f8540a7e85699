"""Runtime over rigid-mesh resolution: the scene's DOF do not depend on the
affine mesh (one body, 12 DOF), and the coarsest scene follows the oracle.
The timing sweep itself is `python -m paper_2311_05945_b300.resolution`."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def test_dof_independent_of_affine_resolution():
    from paper_2311_05945_b300.zema import Scene
    counts = []
    for n in (26, 105):
        g = Scene(S.scene_resolution(n, n_steps=4))
        st = g.step(4)
        assert st["dmin"] > 0
        counts.append(g.counts())
        g.close()
    assert counts[0]["n_nodes"] == counts[1]["n_nodes"]
    # only the sphere's triangles differ: 2 n (n - 1) of them
    assert counts[1]["n_tris"] - counts[0]["n_tris"] == 2 * 105 * 104 - 2 * 26 * 25


def test_coarse_resolution_matches_oracle():
    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_resolution(26, n_steps=8, precision=0, spacing=0.02)
    orc = Oracle(sc, tol_scale=1e-2)
    gpu = Scene(sc, tol_scale=1e-2)
    diag = orc.diag()
    for k in range(8):
        orc.step(1)
        st = gpu.step(1)
        err = max(np.abs(orc.tet_positions(0) - gpu.tet_positions(0)).max(),
                  np.abs(orc.affine_q(1) - gpu.affine_q(1)).max())
        assert err < 1e-5 * diag, (k, err / diag)
    assert st["max_active"] > 0
