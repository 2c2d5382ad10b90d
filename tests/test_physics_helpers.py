"""The measurement helpers of tests/physics.py on shapes whose answer is known exactly.  The
physics checks against the paper (Table I, Eq.23, Eq.25) pass or fail on these helpers, so each
is pinned here on smooth synthetic fields (a tanh profile across every interface, like the
simulated diffuse interfaces) and, for Eq.(25), against a direct integration of Eq.(24)."""
import numpy as np
import pytest

from tests import physics as P

W_INT = 2.0   # interface half-width of the synthetic profiles


def smooth(sd):
    """Phase fraction across an interface at signed distance sd (positive outside)."""
    return 0.5 * (1.0 - np.tanh(sd / W_INT))


@pytest.mark.parametrize("theta", [30.0, 45.0, 60.0, 90.0, 120.0, 150.0])
def test_meniscus_angle_of_a_circular_meniscus(theta):
    """Fluid 0 left of a circular meniscus that meets the walls of a 29-wide channel at theta
    inside fluid 1 (cos theta = H / (2 R), centre on the fluid-0 side for theta < 90)."""
    nx, ny, H, x0 = 200, 31, 29.0, 100.0
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    c = np.cos(np.radians(theta))
    if abs(c) < 1e-12:
        sd = x - x0
    else:
        R = H / (2.0 * c)                 # negative: centre on the fluid-1 side
        xc, yc = x0 - R, 15.0
        d = np.hypot(x - xc, y - yc)
        sd = np.where(x < xc, -1e3, d - R) if R > 0 else np.where(x > xc, 1e3, -R - d)
    C0 = smooth(sd)
    rho = np.stack([C0, 1.0 - C0, np.zeros_like(C0)])
    rho[:, solid.astype(bool)] = 0.0
    assert abs(P.meniscus_angle(rho, solid, 0, 1, 0.5, 29.5) - theta) < 0.2


@pytest.mark.parametrize("theta", [45.0, 90.0, 135.0])
def test_e5_arc_of_the_analytical_droplet(theta):
    """A droplet that is exactly the Eq.(23) arc: radius, centre distance and angle back."""
    w = P.janus_cylinder_e5(theta)
    x, y = np.meshgrid(np.arange(w.nx, dtype=float), np.arange(w.ny, dtype=float))
    D = P.eq23_distance(P.E5_SURFACE, P.E5_RJ, theta)
    sd = np.hypot(x - P.E5_XC, y - (P.E5_YC + D)) - P.E5_RJ
    drop = smooth(sd) * (w.solid == 0)
    rho = np.stack([drop, (1.0 - drop) * (w.solid == 0), np.zeros_like(drop)])
    R, Dm, t = P.e5_arc(rho, w.solid)
    assert abs(R - P.E5_RJ) < 0.1 and abs(Dm - D) < 0.1 and abs(t - theta) < 0.3


@pytest.mark.parametrize("cap,alpha", [(90.0, 90.0), (60.0, 75.0), (120.0, 100.0), (100.0, 60.0)])
def test_janus_angles_of_a_synthetic_janus_cap(cap, alpha):
    """One circular cap of contact angle `cap` on the wall y = 1/2, split by a straight line
    through its base point x = xs at angle alpha from the +x direction: fluid 0 left of the
    line, fluid 2 right, fluid 1 outside.  Expected (theta_01, theta_20, theta_12) =
    (cap, alpha, 180 - cap)."""
    nx, ny, Rc = 240, 120, 50.0
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    xc, yc = nx / 2.0, 0.5 - Rc * np.cos(np.radians(cap))
    inside = smooth(np.hypot(x - xc, y - yc) - Rc)
    xs = xc + 4.0
    a = np.radians(alpha)
    side = smooth(-((x - xs) * np.sin(a) - (y - 0.5) * np.cos(a)))   # 1 right of the line
    rho = np.stack([inside * (1.0 - side), 1.0 - inside, inside * side])
    rho[:, solid.astype(bool)] = 0.0
    t01, t20, t12 = P.janus_angles(rho, solid)
    assert abs(t01 - cap) < 0.5 and abs(t12 - (180.0 - cap)) < 0.5 and abs(t20 - alpha) < 0.5


@pytest.mark.parametrize("mu", [(0.35, 0.35, 0.35), (0.35, 0.0035, 0.35), (0.35, 0.0035, 0.0035),
                                (0.1, 0.3, 0.5)])
def test_washburn_ternary_solves_eq24(mu):
    """Eq.(25)-(26) against a fourth-order Runge-Kutta integration of Eq.(24)."""
    H, L, Lg, s0 = 29.0, 450.0, 90.0, 90.0
    args = (0.01, 30.0, 0.01, 60.0)
    A = H * (0.01 * np.cos(np.radians(30.0)) - 0.01 * np.cos(np.radians(60.0))) / 6.0

    def rate(s):
        return A / (mu[0] * s + mu[1] * Lg + mu[2] * (L - Lg - s))

    s, dt = s0, 50.0
    for _ in range(6000):                      # 300,000 time units
        k1 = rate(s)
        k2 = rate(s + 0.5 * dt * k1)
        k3 = rate(s + 0.5 * dt * k2)
        k4 = rate(s + dt * k3)
        s += dt * (k1 + 2 * k2 + 2 * k3 + k4) / 6.0
    closed = float(P.washburn_ternary(np.array([300000.0]), s0, H, L, Lg, *args, *mu)[0])
    assert abs(closed - s) < 1e-9 * s
