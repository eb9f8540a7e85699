"""The force-feedback closing factor phi of the grasp controller against its
closed form: 1 at zero force, 0 at and above the desired force f*, strictly
decreasing in between, and the paper's example values (k = 20 1/N,
f* = 0.5 N)."""
import math

from paper_2311_05945_b300.grasp import phi


def test_phi_end_points_and_cutoff():
    for k, fs in ((20.0, 0.5), (20.0, 1.0), (4.0, 1.0)):
        assert abs(phi(0.0, fs, k) - 1.0) < 1e-15
        assert phi(fs, fs, k) == 0.0
        assert phi(2.0 * fs, fs, k) == 0.0
    assert phi(0.3, 0.0, 20.0) == 0.0


def test_phi_closed_form_and_monotone():
    k, fs = 20.0, 0.5
    f = 0.25
    expect = (math.exp(-5.0) - math.exp(-10.0)) / (1.0 - math.exp(-10.0))
    assert abs(phi(f, fs, k) - expect) < 1e-15
    vals = [phi(0.01 * i, fs, k) for i in range(51)]
    assert all(vals[i] > vals[i + 1] for i in range(50))


def test_phi_small_force_decay():
    # far below f* the factor decays like exp(-k f)
    k, fs = 20.0, 1.0
    for f in (0.05, 0.1, 0.2):
        assert abs(phi(f, fs, k) - math.exp(-k * f)) < 1e-8
