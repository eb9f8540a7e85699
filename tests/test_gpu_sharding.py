"""Env sharding on the GPU path: a batch split into contiguous env ranges
(the partition of the multi-GPU runs, balanced by tet count) steps every env
bit for bit as the whole batch does.  Environments never interact, and with
the schedule pinned (hash cell size and cluster size, which only order the
sums) nothing about one env depends on the others.  Stepped here on one GPU,
one range after the other."""
import numpy as np
import pytest

from paper_2311_05945_b300 import scenes as S
from paper_2311_05945_b300.sharding import shard_envs

pytestmark = pytest.mark.gpu

N_ENVS, STEPS = 4, 24  # through first contact of the fingers (step 20)
PIN = dict(cell_size=0.004, pcg_cluster_size=4)


def env_positions(g, sc):
    out = {}
    for i, b in enumerate(sc.tets):
        out.setdefault(b.env, []).append(g.tet_positions(i))
    return {e: np.concatenate(v) for e, v in out.items()}


@pytest.mark.parametrize("precision", [0, 1])
def test_sharded_envs_step_bit_identically(precision):
    from paper_2311_05945_b300 import zema as Z
    mk = lambda n, a: S.scene_c3(n_envs=n, n_steps=STEPS + 1, min_tets=2000, max_tets=5000, seed0=1000 + a,
                                 slot0=a)
    whole = mk(N_ENVS, 0)
    w = [0] * N_ENVS
    for b in whole.tets:
        w[b.env] += len(b.tets)
    ranges = shard_envs(w, 2)
    assert len(ranges) == 2 and ranges[0][0] == 0 and ranges[-1][1] == N_ENVS
    g = Z.Scene(whole, precision=precision, **PIN)
    g.step(STEPS)
    ref = env_positions(g, whole)
    g.close()
    for a, b in ranges:
        part = mk(b - a, a)
        gp = Z.Scene(part, precision=precision, **PIN)
        st = gp.step(STEPS)
        assert st["max_active"] > 0
        got = env_positions(gp, part)
        for e in range(b - a):
            assert np.array_equal(got[e], ref[a + e]), (a + e, np.abs(got[e] - ref[a + e]).max())
        gp.close()


def test_pinned_cluster_size_is_checked():
    from paper_2311_05945_b300 import zema as Z
    sc = S.scene_tiny_contact()
    with pytest.raises(Z.ZemaError) as ei:
        Z.Scene(sc, pcg_cluster_size=3)
    assert ei.value.status == 1
    g = Z.Scene(sc, pcg_cluster_size=2)
    g.step(1)
    assert g.tuning()[0] == 2
    g.autotune()  # a pinned size is kept
    g.step(1)
    assert g.tuning()[0] == 2
    g.close()
