"""The values the paper prints that the controller and the scenes take over,
read from tests/golden/paper_printed_values.json (each entry cites its
section or table).

- The grasp controller's defaults: the decay rate k of the closing factor
  (Controller), the stop force and the lift height (AutoGrasp, Lift).
- The resolution sweep (Table IV): each synthetic sphere is the largest UV
  sphere with no more vertices than the paper's mesh at that resolution.  A
  closed genus-0 triangle mesh has 2V - 4 triangles, so the paper's triangle
  counts (2.1 to 2.6 per vertex, from decimating a scanned mesh) are not
  matched as well; the test states that bound instead.
"""
import json
import math
import os

import numpy as np

from paper_2311_05945_b300 import grasp
from paper_2311_05945_b300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_grasp_controller_defaults_are_the_papers():
    g = _golden()
    assert grasp.K_PHI == g["controller"]["k_per_newton"]
    assert grasp.F_STOP == g["autograsp_and_lift"]["stop_force_newton"]
    sc = S.scene_c2(n_steps=1)
    ctl = grasp.AutoGrasp(object(), sc)
    assert ctl.k == g["controller"]["k_per_newton"]
    assert ctl.f_star == g["autograsp_and_lift"]["stop_force_newton"]
    assert ctl.lift_height == g["autograsp_and_lift"]["lift_height_m"]
    # the paper's example desired force: phi at half of it, from the closed form
    fs, k = g["controller"]["f_star_example_newton"], g["controller"]["k_per_newton"]
    expect = (math.exp(-k * fs / 2) - math.exp(-k * fs)) / (1.0 - math.exp(-k * fs))
    assert abs(grasp.phi(fs / 2, fs, k) - expect) < 1e-15


def test_resolution_spheres_follow_the_papers_vertex_counts():
    g = _golden()["runtime_over_resolution"]
    assert len(S.RESOLUTION_SEGMENTS) == len(g["vertices"])
    for n, nv_paper, nf_paper in zip(S.RESOLUTION_SEGMENTS, g["vertices"], g["triangles"]):
        sc = S.scene_resolution(n, n_steps=1)
        V, F = sc.affines[-1].V, sc.affines[-1].F
        nv, nf = len(V), len(F)
        # the largest n x n UV sphere not above the paper's vertex count
        assert nv == n * (n - 1) + 2 and nv <= nv_paper < (n + 1) * n + 2, (n, nv, nv_paper)
        assert nv_paper - nv < 0.05 * nv_paper
        # closed genus-0 surface: every edge in two triangles, Euler characteristic 2
        assert nf == 2 * nv - 4
        E = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
        _, counts = np.unique(E, axis=0, return_counts=True)
        assert np.all(counts == 2) and nv - len(counts) + nf == 2
        assert nf < nf_paper < 1.4 * nf, (nf, nf_paper)
