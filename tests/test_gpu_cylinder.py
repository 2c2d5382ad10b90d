"""Section III.B at the paper's size: a perfect Janus droplet on a cylinder (200 x 200, cylinder
radius 40, droplet radius 45) for the six contact angles of Fig.7, GPU FP32.  The droplet starts
at the analytical equilibrium of Eq.(23) (tests/physics.py: janus_cylinder_e5) and runs 40,000
steps; a circle is fitted to its outer interface and the contact angle recovered with the law of
cosines of Eq.(23).  The shape counts as steady when the angle moved by less than 0.5 degree over
the last 10,000 steps.  Fig.7 compares shapes, and the paper prints no number for it: the arc's
centre must lie within 2.5 lu of the Eq.(23) distance for its measured radius, the radius within
1.5 lu of 45, and the angle within 5 degrees of the prescribed one (8 at 30 degrees, where the
paper itself shows the shape departing, too few nodes near the contact lines).  The cylinder is a
staircase: its Eq.(19) normals are off the radial direction by up to 11 degrees node by node.
"""
import pytest

from tests import physics as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_04709_gb300 import build, lbm3
    build.build()
    lbm3.load()
    return lbm3


@pytest.mark.parametrize("theta", [30.0, 45.0, 60.0, 90.0, 120.0, 150.0])
def test_janus_droplet_on_cylinder(gpu, theta):
    w = P.janus_cylinder_e5(theta)
    sim = gpu.Lbm3.from_workload(w)
    sim.step(30000)
    R1, D1, t1 = P.e5_arc(sim.fields()[0], w.solid)
    sim.step(10000)
    R, D, t = P.e5_arc(sim.fields()[0], w.solid)
    assert sim.diag()[7] == 0
    sim.close()
    D_eq23 = P.eq23_distance(P.E5_SURFACE, R, theta)
    print(f"\ntheta {theta:5.1f}: measured {t:6.2f} (at 30k steps {t1:6.2f}), arc radius {R:.2f}, "
          f"centre distance {D:.2f} (Eq.23 with that radius {D_eq23:.2f})")
    assert abs(t - t1) < 0.5
    assert abs(D - D_eq23) <= 2.5
    assert abs(R - P.E5_RJ) <= 1.5
    assert abs(t - theta) <= (8.0 if theta < 45.0 else 5.0)
