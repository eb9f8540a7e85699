"""Pins of the oracle's linear solves and of its OpenMP build.

The stepper solves each Newton system H p = -g by dense Cholesky up to 2,500
DOF and otherwise by block-Jacobi CG to a relative residual of 1e-12 (the
plain solve of the method's linear phase, paper Table I "Linear").  The
larger grasp environments only ever take the CG branch, so it is pinned
here on real Newton systems of 2.6k and 3.4k DOF against LAPACK (numpy's
dense solve, an independent library routine) and against the oracle's own
Cholesky with its size limit lifted.  A CG that stopped early, or a wrong
preconditioner block, fails the residual check.  The OpenMP build must
reproduce the serial trajectory bit for bit.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import Oracle
from paper_2311_05945_b300 import scenes as S


@pytest.fixture
def threads():
    n = O.set_threads(os.cpu_count() or 1)
    yield n
    O.set_threads(1)


@pytest.mark.parametrize("seed", [1001, 1002])
def test_cg_solve_of_grasp_newton_systems(seed, threads):
    # a grasp env of the batched workload two steps in (object on the floor,
    # barrier pairs active): the Newton system at the start of step 2
    o = Oracle(S.scene_c3(n_envs=1, n_steps=4, seed0=seed))
    o.step(2)
    o.prepare(0)
    y = o.dofs(0)
    n = len(y)
    assert n > 2500  # the stepper takes the CG branch here
    _, g, H, n_act = o.eval(y, grad=True, hess=True)
    assert n_act > 0
    p_step = o.newton_direction(y, which=0)  # the stepper's own choice
    p_cg = o.newton_direction(y, which=2)
    assert np.array_equal(p_step, p_cg)
    # residual of the CG direction, recomputed on the dense matrix: at most
    # the solve's 1e-12 target plus the rounding of the re-evaluation
    gn = np.linalg.norm(g)
    res = np.linalg.norm(H @ p_cg + g)
    slack = 64 * np.finfo(float).eps * np.linalg.norm(np.abs(H) @ np.abs(p_cg))
    assert res <= 1e-12 * gn + slack, (res / gn, slack / gn)
    # against LAPACK and against the oracle's dense Cholesky
    p_ref = np.linalg.solve(H, -g)
    p_chol = o.newton_direction(y, which=1)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(p_chol, p_ref) < 1e-12
    # a relative residual r bounds the relative error by cond(H) r (2-norm
    # condition number; here 2e5 to 1e6)
    ev = np.linalg.eigvalsh(H)
    assert ev[0] > 0
    bound = (ev[-1] / ev[0]) * (res + slack) / gn
    assert rel(p_cg, p_ref) <= bound, (rel(p_cg, p_ref), bound)
    assert rel(p_cg, p_chol) <= bound
    # a descent direction of the potential
    assert g @ p_cg < 0


def test_dense_solve_against_lapack():
    # the small-system branch on C1's Newton system in contact (387 DOF)
    o = Oracle(S.scene_c1(n_steps=12))
    o.step(10)
    o.prepare(0)
    y = o.dofs(0)
    _, g, H, n_act = o.eval(y, grad=True, hess=True)
    assert n_act > 0 and len(y) <= 2500
    p = o.newton_direction(y, which=0)
    p_ref = np.linalg.solve(H, -g)
    assert np.linalg.norm(p - p_ref) <= 1e-12 * np.linalg.norm(p_ref)
    assert np.linalg.norm(H @ p + g) <= 1e-13 * np.linalg.norm(g)


def test_openmp_build_is_bit_identical_to_serial():
    # parallel loops write their own slots and every sum stays serial in
    # index order, so the thread count cannot change a single bit
    def run(nth):
        O.set_threads(nth)
        try:
            o = Oracle(S.scene_c3(n_envs=1, n_steps=4, seed0=1001))
            o.step(3)
            return np.concatenate([o.get_state(b) for b in range(3)]), np.array(o.energy_log())
        finally:
            O.set_threads(1)

    xs, es = run(1)
    xp, ep = run(max(2, os.cpu_count() or 2))
    assert np.array_equal(xs, xp)
    assert np.array_equal(es, ep)
