"""Per-body learned warm start of the affine bodies on the GPU.

Pins: in free fall (no contact) the recorded features and targets have
closed forms.  After k steps from rest:
- the body's A is the identity;
- h qdot / s of the centre is k (0, -1, 0), and (qhat - q) / s is (k + 1) (0, -1, 0);
- the target, the change of q beyond h qdot in units of s = h^2 |g|, is (0, -1, 0) with zero A part.
A network whose parameters are all zero proposes no correction, so the
learned start must reproduce the constant-velocity run bit for bit.  Wrongly
shaped networks are rejected."""
import numpy as np
import pytest

from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu


def test_free_fall_features_and_targets():
    import torch

    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_free_fall(n_steps=4)
    sc.params.pcg_rel_tol = 1e-13
    g = Scene(sc)
    fb = torch.full((1, 40), float("nan"), dtype=torch.float32, device="cuda")
    tb = torch.full((1, 12), float("nan"), dtype=torch.float32, device="cuda")
    g.record_warmstart_affine(fb, tb)
    down = np.array([0.0, -1.0, 0.0])
    for k in range(4):
        g.step(1)
        f = fb.cpu().numpy()[0].astype(np.float64)
        t = tb.cpu().numpy()[0].astype(np.float64)
        assert np.abs(f[0:9] - np.eye(3).reshape(-1)).max() < 1e-6
        assert np.abs(f[12:15] - k * down).max() < 1e-5
        assert np.abs(f[15:24]).max() < 1e-6
        assert np.abs(f[24:27] - (k + 1) * down).max() < 1e-5
        assert np.abs(f[27:36]).max() < 1e-6
        assert f[36] == 1.0 and np.abs(f[37:40]).max() == 0.0
        assert np.abs(t[0:3] - down).max() < 1e-5
        assert np.abs(t[3:12]).max() < 1e-5
    g.record_warmstart_affine(None)
    g.close()


def pile():
    return S.scene_c5(n_steps=12, tets_per_body=300, n_soft=2, n_convex=2, n_nonconvex=2, n_seg=8,
                      bin_subdiv=1, gap=0.5e-3, precision=1)


def test_zero_network_reproduces_constant_velocity_run():
    from paper_2311_05945_b300.zema import Scene
    sc = pile()
    dims = [40, 128, 128, 128, 12]
    n = sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(4))
    a = Scene(sc)
    b = Scene(sc, warm_start=1)
    b.load_warmstart(dims, np.zeros(n, dtype=np.float32))
    for _ in range(10):
        sa = a.step(1)
        sb = b.step(1)
        assert sa["newton_iters"] == sb["newton_iters"]
        assert sb["warm_learned"] == 0
    for i in range(len(sc.affines)):
        assert np.array_equal(a.affine_q(i), b.affine_q(i))
    for i in range(len(sc.tets)):
        assert np.array_equal(a.tet_positions(i), b.tet_positions(i))
    assert sa["max_active"] > 0
    a.close()
    b.close()


def test_wrong_network_shapes_are_rejected():
    from paper_2311_05945_b300.zema import Scene, ZemaError
    g = Scene(pile())
    for dims in ([40, 16, 3], [13, 16, 12], [12, 16, 12]):
        n = sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))
        with pytest.raises(ZemaError):
            g.load_warmstart(dims, np.zeros(n, dtype=np.float32))
    g.close()
