"""Learned Newton warm start: the recorded features and targets against
numpy restatements from the bodies' states, the learned path converging to
the same tolerance with the committed network, and the network's prediction
gain over the constant-velocity proposal on held-out environments."""
import os

import numpy as np
import pytest

from paper_2311_05945_b300 import scenes as S

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2311_05945_b300",
                       "weights", "warmstart.bin")


def soft_state(g, sc):
    xs, vs = [], []
    for i, b in enumerate(sc.tets):
        st = g.get_state(i)
        n = len(b.X)
        xs.append(st[:3 * n].reshape(n, 3))
        vs.append(st[3 * n:6 * n].reshape(n, 3))
    return xs, vs


def test_recorded_features_and_targets_match_states():
    import torch

    from paper_2311_05945_b300.zema import Scene
    sc = S.scene_tiny_contact(mu=0.5)
    g = Scene(sc)
    g.step(10)  # the cube has landed on the floor
    rows = g.counts()["n_verts"]
    fb = torch.zeros((rows, 13), dtype=torch.float32, device="cuda")
    tb = torch.zeros((rows, 3), dtype=torch.float32, device="cuda")
    x0, v0 = soft_state(g, sc)
    g.record_warmstart(fb, tb)
    g.step(1)
    g.record_warmstart(None)
    x1, _ = soft_state(g, sc)
    f, t = fb.cpu().numpy(), tb.cpu().numpy()
    h, gr = sc.params.dt, np.array(sc.params.gravity)
    s = h * h * np.linalg.norm(gr)
    o = 0
    for bi, b in enumerate(sc.tets):
        n = len(b.X)
        X, x, v = np.asarray(b.X), x0[bi], v0[bi]
        R = 0.5 * np.linalg.norm(X.max(0) - X.min(0))
        c = x.mean(0)
        assert np.allclose(f[o:o + n, 0:3], (x - c) / R, atol=1e-5)
        assert np.allclose(f[o:o + n, 3:6], v * h / s, atol=1e-4 * max(1.0, np.abs(v * h / s).max()))
        assert np.allclose(f[o:o + n, 6:9], (h * v + h * h * gr) / s, atol=1e-4 * max(1.0, np.abs(v * h / s).max()))
        # contact features: distance fraction in [0, 1]; unit normals where in contact, else 0
        d, nn = f[o:o + n, 9], f[o:o + n, 10:13]
        assert ((d >= 0) & (d <= 1)).all()
        norms = np.linalg.norm(nn, axis=1)
        assert np.allclose(norms[d < 1], 1.0, atol=1e-5) and np.allclose(norms[d == 1], 0.0)
        assert (d < 1).any()  # the cube rests on the floor
        assert np.allclose(t[o:o + n], (x1[bi] - x - h * v) / s, atol=1e-3 * max(1.0, np.abs(t).max()))
        o += n


def test_learned_start_converges_and_follows_the_plain_run():
    # at 1e-2 of the Newton tolerance both starts converge to the same
    # minimiser step after step: positions within the parity bound
    from paper_2311_05945_b300.zema import Scene, read_warmstart_blob
    dims, theta = read_warmstart_blob(open(WEIGHTS, "rb").read())
    sc = S.scene_c3(n_envs=2, n_steps=40, min_tets=2000, max_tets=6000, seed0=100100)
    a = Scene(sc, warm_start=0, tol_scale=1e-2)
    b = Scene(sc, warm_start=1, tol_scale=1e-2)
    b.load_warmstart(dims, theta)
    na = nb = 0
    for k in range(30):
        sa, sb = a.step(1), b.step(1)
        na += sa["newton_iters"]
        nb += sb["newton_iters"]
        assert sb["dmin"] > 0
    for i, bd in enumerate(sc.tets):
        pa = a.tet_positions(i)
        diag = float(np.linalg.norm(pa.max(0) - pa.min(0)))
        err = np.abs(pa - b.tet_positions(i)).max()
        assert err < 1e-5 * diag, (i, err / diag)
    print(f"Newton iterations over 30 steps: constant-velocity {na}, learned {nb}")


def test_measured_iteration_ratio_on_held_out_envs():
    # the learned start at the scale it was trained and evaluated at (the
    # committed report: 51,500 env-steps of training, 64 held-out envs x 120
    # steps) costs Newton iterations instead of saving them; a live sample of
    # 8 held-out envs through first contact measures the same: a ratio above
    # 1 and bounded, since the plain start and the energy checks keep every
    # step converging to the same tolerance
    import json

    from paper_2311_05945_b300.zema import Scene, read_warmstart_blob
    rep = json.load(open(os.path.join(os.path.dirname(WEIGHTS), "warmstart_eval.json")))
    assert rep["envs"] == 64 and rep["steps"] == 120 and rep["seed0"] == 100000
    assert 1.0 <= rep["newton_ratio"] <= 1.25
    dims, theta = read_warmstart_blob(open(WEIGHTS, "rb").read())
    sc = S.scene_c3(n_envs=8, n_steps=40, seed0=100000)
    its = []
    for ws in (0, 1):
        g = Scene(sc, warm_start=ws)
        if ws:
            g.load_warmstart(dims, theta)
        st = g.step(36)
        its.append(st["newton_iters"])
        g.close()
    ratio = its[1] / its[0]
    print(f"Newton iterations, 8 held-out envs x 36 steps: constant-velocity {its[0]}, learned {its[1]} "
          f"(ratio {ratio:.3f})")
    assert 0.95 <= ratio <= 1.25


def test_network_predicts_held_out_steps_better_than_constant_velocity():
    import torch

    from paper_2311_05945_b300.zema import Mlp, Scene, read_warmstart_blob
    dims, theta = read_warmstart_blob(open(WEIGHTS, "rb").read())
    net = Mlp(dims)
    net.set_params(theta)
    sc = S.scene_c3(n_envs=2, n_steps=40, min_tets=2000, max_tets=6000, seed0=100200)
    g = Scene(sc)
    rows = g.counts()["n_verts"]
    fb = torch.zeros((rows, 13), dtype=torch.float32, device="cuda")
    tb = torch.zeros((rows, 3), dtype=torch.float32, device="cuda")
    g.record_warmstart(fb, tb)
    e_net = e_cv = 0.0
    for k in range(30):
        g.step(1)
        y = net.forward(fb)
        e_net += float(((y - tb) ** 2).mean())
        e_cv += float((tb ** 2).mean())
    print(f"held-out mean squared error: network {e_net / 30:.5f}, constant velocity {e_cv / 30:.5f}")
    assert e_net < e_cv
