"""Measurement helpers shared by the oracle pins and the GPU physics checks: interface
contours, circle fits and contact angles.  No step of the method lives here."""
import numpy as np


def contour_points(C, solid, level=0.5):
    """Points where the field C crosses `level` along grid rows and columns (linear
    interpolation between two fluid nodes)."""
    C = np.asarray(C)
    s = np.asarray(solid).astype(bool)
    pts = []
    a = C[:, :-1] - level
    b = C[:, 1:] - level
    ok = (a * b < 0) & ~s[:, :-1] & ~s[:, 1:]
    ys, xs = np.nonzero(ok)
    for y, x in zip(ys, xs):
        pts.append((x + a[y, x] / (a[y, x] - b[y, x]), y))
    a = C[:-1, :] - level
    b = C[1:, :] - level
    ok = (a * b < 0) & ~s[:-1, :] & ~s[1:, :]
    ys, xs = np.nonzero(ok)
    for y, x in zip(ys, xs):
        pts.append((x, y + a[y, x] / (a[y, x] - b[y, x])))
    return np.array(pts, dtype=np.float64).reshape(-1, 2)


def fit_circle(p):
    """Least-squares circle (xc, yc, R) through points p[:, 2]."""
    A = np.c_[2 * p[:, 0], 2 * p[:, 1], np.ones(len(p))]
    b = (p ** 2).sum(1)
    c = np.linalg.lstsq(A, b, rcond=None)[0]
    xc, yc = c[0], c[1]
    return xc, yc, float(np.sqrt(c[2] + xc * xc + yc * yc))


def cap_angle_bottom(C, solid, wall_y=0.5, y_min=2.5, x_range=None):
    """Contact angle (deg, measured inside the phase where C > 1/2) of a circular cap
    resting on a horizontal wall at height wall_y: cos(theta) = -(yc - wall_y) / R."""
    p = contour_points(C, solid)
    p = p[p[:, 1] > y_min]
    if x_range is not None:
        p = p[(p[:, 0] >= x_range[0]) & (p[:, 0] <= x_range[1])]
    xc, yc, R = fit_circle(p)
    return float(np.degrees(np.arccos(np.clip(-(yc - wall_y) / R, -1, 1)))), (xc, yc, R)


def cap_workload(theta, Rc=12.0, nx=80, ny=40, nu=1.0 / 6.0):
    """Two-phase cap of fluid 0 in fluid 2 on the bottom wall, initialised at the circular
    shape of contact angle theta; the wall triple gives fluid 0 the angle theta against
    fluid 2 (theta_rb = theta, i.e. theta_br = 180 - theta)."""
    from paper_2102_04709_gb300.workloads import Workload, BC_PERIODIC
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = 1
    solid[-1] = 1
    yc = 0.5 - Rc * np.cos(np.radians(theta))
    lab = np.full((ny, nx), 2)
    lab[((x - nx / 2) ** 2 + (y - yc) ** 2 < Rc * Rc) & (y > 0)] = 0
    rho = np.zeros((3, ny, nx))
    for k in range(3):
        rho[k][lab == k] = 1.0
    rho[:, solid.astype(bool)] = 0.0
    ang = np.zeros((ny, nx, 3))
    ang[..., 0] = 90.0
    ang[..., 1] = 180.0 - theta
    ang[..., 2] = 90.0
    return Workload(f"cap{theta}", nx, ny, 0, BC_PERIODIC, solid, rho, ang, (0.01,) * 3,
                    (nu,) * 3, steps=0)
