"""Measurement helpers shared by the oracle pins and the GPU physics checks: interface
contours, circle fits and contact angles.  No step of the method lives here."""
import numpy as np


def contour_points(C, solid, level=0.5):
    """Points where the field C crosses `level` along grid rows and columns (linear
    interpolation between two fluid nodes).  A crossing is a sign change of C - level counted
    half-open (a >= 0 > b or a < 0 <= b), so a node exactly at the level gives one point;
    non-finite values (masked regions) never cross."""
    C = np.asarray(C)
    s = np.asarray(solid).astype(bool)
    pts = []
    a = C[:, :-1] - level
    b = C[:, 1:] - level
    ok = ((a >= 0) != (b >= 0)) & np.isfinite(a) & np.isfinite(b) & ~s[:, :-1] & ~s[:, 1:]
    ys, xs = np.nonzero(ok)
    for y, x in zip(ys, xs):
        pts.append((x + a[y, x] / (a[y, x] - b[y, x]), y))
    a = C[:-1, :] - level
    b = C[1:, :] - level
    ok = ((a >= 0) != (b >= 0)) & np.isfinite(a) & np.isfinite(b) & ~s[:-1, :] & ~s[1:, :]
    ys, xs = np.nonzero(ok)
    for y, x in zip(ys, xs):
        pts.append((x, y + a[y, x] / (a[y, x] - b[y, x])))
    return np.array(pts, dtype=np.float64).reshape(-1, 2)


def fit_circle(p):
    """Least-squares circle (xc, yc, R) through points p[:, 2] (at least three)."""
    if len(p) < 3:
        raise ValueError(f"a circle needs at least 3 points, got {len(p)}")
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



def _cap_angle_inside(p, wall_y):
    """Angle (deg) at the wall, measured inside the phase enclosed by a circle fitted to the
    arc p[:, 2] of a cap on a horizontal wall at wall_y: cos(theta) = -(yc - wall_y) / R."""
    xc, yc, R = fit_circle(p)
    return float(np.degrees(np.arccos(np.clip(-(yc - wall_y) / R, -1.0, 1.0))))


def janus_angles(rho, solid, wall_y=0.5, y_min=0.5, frac=0.7):
    """The three contact angles (deg) of a Janus droplet (fluid 0 on the left, fluid 2 on the
    right, both in fluid 1) resting on the bottom wall, as (theta_01, theta_20, theta_12),
    theta_kl measured inside fluid k:

    * theta_01 at the left contact line: circle fitted to the left arc of the C_1 = 1/2
      contour (a cap enclosing fluid 0);
    * theta_12 at the right contact line: 180 deg minus the angle inside fluid 2 of the
      circle fitted to the right arc;
    * theta_20 where the internal interface, the C_0 / (C_0 + C_2) = 1/2 contour inside the
      droplet, meets the wall: fitted by x = a + b y + c y^2, its tangent (b, 1) at the wall
      makes the angle with the +x direction, the wall on the fluid-2 side.

    Each arc is fitted between wall_y + y_min and wall_y + frac * H, H the height of the triple
    junction (the top of the internal interface), so that the rounded junction region, where
    the three interfaces meet at the Neumann angles, stays out of the fits."""
    rho = np.asarray(rho, dtype=np.float64)
    C = rho / np.maximum(rho.sum(0), 1e-30)
    s = np.asarray(solid).astype(bool)
    with np.errstate(invalid="ignore", divide="ignore"):
        phi = np.where(C[1] < 0.5, C[0] / (C[0] + C[2]), np.nan)
    inner = contour_points(phi, s)
    H = inner[:, 1].max() - wall_y
    band = lambda p: p[(p[:, 1] > wall_y + y_min) & (p[:, 1] < wall_y + frac * H)]
    inner = band(inner)
    outer = band(contour_points(C[1], s))
    xm = inner[:, 0].mean()
    t01 = _cap_angle_inside(outer[outer[:, 0] < xm], wall_y)
    t12 = 180.0 - _cap_angle_inside(outer[outer[:, 0] > xm], wall_y)
    yy = inner[:, 1] - wall_y
    b = np.linalg.lstsq(np.c_[np.ones_like(yy), yy, yy * yy], inner[:, 0], rcond=None)[0][1]
    t20 = float(np.degrees(np.arctan2(1.0, b)))
    return t01, t20, t12


def table1():
    """The six angle sets of Table I: [(label, analytical (rg, br, gb), simulated (rg, br, gb))]."""
    import os
    rows = []
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "table1_janus_flat.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            t = line.split()
            rows.append((t[0], tuple(map(float, t[1:4])), tuple(map(float, t[4:7]))))
    return rows


# ---- Section III.B: a perfect Janus droplet on a cylinder, Eq.(23) ----
E5_NX, E5_NY, E5_XC, E5_YC, E5_RS, E5_RJ = 200, 200, 100.0, 60.0, 40.0, 45.0
E5_SURFACE = E5_RS + 0.5   # halfway bounce-back: the wall lies half a link outside the solid nodes


def eq23_distance(rs, rj, theta):
    """Eq.(23) with its square restored: the distance between the centres of the cylinder
    (radius rs) and of the droplet's circular arc (radius rj) at contact angle theta (deg)."""
    return float(np.sqrt(rs * rs + rj * rj - 2.0 * rs * rj * np.cos(np.radians(theta))))


def janus_cylinder_e5(theta, scale=1.0):
    """Section III.B: 200 x 200, periodic in x, solid rows at the bottom and top, a cylinder of
    radius 40 (solid nodes within 40 of (100, 60)); the droplet starts as its analytical
    equilibrium: a disc of radius 45 whose centre lies eq23_distance(40.5, 45, theta) above the
    cylinder's, fluid 0 left of x = 100 and fluid 2 right of it, in fluid 1.  Wall triple
    (theta_rg, theta_br, theta_gb) = (theta, 90, 180 - theta): fluids 0 and 2 wet alike;
    sigma_01 = sigma_12 = 0.01 and sigma_02 = 1e-4 (the paper's negligible red-blue tension);
    every viscosity 0.1.  ``scale`` multiplies every length (the box, centres and radii)."""
    from paper_2102_04709_gb300.workloads import Workload, BC_PERIODIC
    nx = ny = int(round(E5_NX * scale))
    xc, yc, rs, rj = E5_XC * scale, E5_YC * scale, E5_RS * scale, E5_RJ * scale
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    solid = ((x - xc) ** 2 + (y - yc) ** 2 <= rs ** 2).astype(np.uint8)
    solid[0] = 1
    solid[-1] = 1
    yd = yc + eq23_distance(rs + 0.5, rj, theta)
    drop = ((x - xc) ** 2 + (y - yd) ** 2 < rj ** 2) & (solid == 0)
    lab = np.full((ny, nx), 1)
    lab[drop & (x < xc)] = 0
    lab[drop & (x >= xc)] = 2
    rho = np.zeros((3, ny, nx))
    for k in range(3):
        rho[k][(lab == k) & (solid == 0)] = 1.0
    ang = np.tile(np.array([theta, 90.0, 180.0 - theta]), (ny, nx, 1))
    return Workload(f"janus_cylinder_e5_{theta:g}_{nx}", nx, ny, 0, BC_PERIODIC, solid, rho, ang,
                    (0.01, 1e-4, 0.01), (0.1, 0.1, 0.1), steps=0)


def e5_arc(rho, solid, gap=3.0, scale=1.0):
    """Circle fitted to the droplet's outer interface (C_1 = 1/2), points more than gap from
    the cylinder's wall (radius 40 scale + 1/2); returns (radius, distance of its centre from
    the cylinder's centre, contact angle from the law of cosines of Eq.(23))."""
    xc0, yc0, surf = E5_XC * scale, E5_YC * scale, E5_RS * scale + 0.5
    C1 = rho[1] / np.maximum(rho.sum(0), 1e-30)
    p = contour_points(C1, solid)
    p = p[np.hypot(p[:, 0] - xc0, p[:, 1] - yc0) > surf + gap]
    xc, yc, R = fit_circle(p)
    D = float(np.hypot(xc - xc0, yc - yc0))
    c = (surf ** 2 + R * R - D * D) / (2.0 * surf * R)
    return R, D, float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


# ---- Section III.C: capillary intrusion, Eq.(24)-(26) ----
def meniscus_angle(rho, solid, k, l, y_wall_lo, y_wall_hi):
    """Contact angle (deg) inside fluid l of the meniscus between fluid k (left) and fluid l
    (right) in a channel whose walls lie at y_wall_lo and y_wall_hi: a circle is fitted to the
    C_k / (C_k + C_l) = 1/2 contour where the third fluid is absent, and the angle between the
    wall (pointing into fluid l) and the circle's tangent at the wall is averaged over both
    walls."""
    rho = np.asarray(rho, dtype=np.float64)
    C = rho / np.maximum(rho.sum(0), 1e-30)
    with np.errstate(invalid="ignore", divide="ignore"):
        phi = np.where(C[k] + C[l] > 0.9, C[k] / (C[k] + C[l]), np.nan)
    p = contour_points(phi, solid)
    p = p[(p[:, 1] > y_wall_lo + 1.0) & (p[:, 1] < y_wall_hi - 1.0)]
    sv = np.linalg.svd(p - p.mean(0), compute_uv=False)
    if sv[-1] <= 1e-9 * sv[0]:
        # a straight meniscus (collinear points): x = a + b y, slope b at both walls, the
        # tangent into the fluid mirrored at the upper wall as below
        b = np.polyfit(p[:, 1], p[:, 0], 1)[0]
        return 0.5 * (float(np.degrees(np.arctan2(1.0, b))) + float(np.degrees(np.arctan2(1.0, -b))))
    xc, yc, R = fit_circle(p)
    xm = p[:, 0].mean()
    out = []
    for yw, sgn in ((y_wall_lo, 1.0), (y_wall_hi, -1.0)):
        h = np.sqrt(max(R * R - (yw - yc) ** 2, 0.0))
        xw = xc + h if abs(xc + h - xm) < abs(xc - h - xm) else xc - h
        dxdy = -(yw - yc) / (xw - xc)
        out.append(float(np.degrees(np.arctan2(1.0, sgn * dxdy))))
    return 0.5 * (out[0] + out[1])


def washburn_ternary(t, s0, H, L, Lg, sig_gb, th_gb, sig_gr, th_gr, mu_r, mu_g, mu_b):
    """Eq.(25)-(26): intrusion length s(t) of the red fluid (angles in degrees)."""
    A = H * (sig_gb * np.cos(np.radians(th_gb)) - sig_gr * np.cos(np.radians(th_gr))) / 6.0
    B = mu_g * Lg + mu_b * (L - Lg)
    C = mu_r - mu_b
    t = np.asarray(t, dtype=np.float64)
    if C == 0.0:
        return A / B * t + s0
    f = -0.5 * C * s0 * s0 - B * s0 - A * t
    return (-B + np.sqrt(B * B - 2.0 * C * f)) / C


# ---- Section II.A: a free lens of fluid 1 on a flat interface between fluids 0 and 2 ----
def neumann_angles(sigma):
    """Angles (gamma_0, gamma_1, gamma_2) in degrees, gamma_k inside fluid k, at a triple
    junction where three interfaces with tensions sigma = (sigma_01, sigma_02, sigma_12) meet in
    equilibrium: the tensions balance as the sides of a triangle, sigma_12 / sin gamma_0 =
    sigma_02 / sin gamma_1 = sigma_01 / sin gamma_2, so 180 - gamma_k is the triangle's angle
    opposite the side sigma_lm of the two other fluids (law of cosines)."""
    s01, s02, s12 = sigma
    g0 = 180.0 - np.degrees(np.arccos((s01 ** 2 + s02 ** 2 - s12 ** 2) / (2 * s01 * s02)))
    g1 = 180.0 - np.degrees(np.arccos((s01 ** 2 + s12 ** 2 - s02 ** 2) / (2 * s01 * s12)))
    g2 = 180.0 - np.degrees(np.arccos((s02 ** 2 + s12 ** 2 - s01 ** 2) / (2 * s02 * s12)))
    return g0, g1, g2


def lens_workload(sigma, nx=96, ny=64, c=12.0, nu=1.0 / 6.0):
    """Fully periodic box: fluid 0 in the band 12 <= y < 44, fluid 2 elsewhere, and a lens of
    fluid 1 on the upper 0-2 interface (y0 = 43.5) centred at x = nx / 2: two circular caps
    on the chord of half-length c, the upper one (in fluid 2) and the lower one (in fluid 0)
    each meeting the interface at the angles of Neumann's triangle for sigma, so that the run
    starts near equilibrium."""
    from paper_2102_04709_gb300.workloads import Workload, BC_PERIODIC
    g0, g1, g2 = neumann_angles(sigma)
    au, al = np.radians(180.0 - g2), np.radians(180.0 - g0)   # cap angles inside fluid 1
    y0, xc = 43.5, nx / 2.0
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    lab = np.where((y >= 12) & (y < 44), 0, 2)
    Ru, Rl = c / np.sin(au), c / np.sin(al)
    yu, yl = y0 - Ru * np.cos(au), y0 + Rl * np.cos(al)     # centres of the two arcs
    up = (y >= y0) & ((x - xc) ** 2 + (y - yu) ** 2 < Ru * Ru)
    lo = (y < y0) & ((x - xc) ** 2 + (y - yl) ** 2 < Rl * Rl)
    lab[up | lo] = 1
    rho = np.zeros((3, ny, nx))
    for k in range(3):
        rho[k][lab == k] = 1.0
    solid = np.zeros((ny, nx), np.uint8)
    return Workload(f"lens_{nx}x{ny}", nx, ny, 1, BC_PERIODIC, solid, rho,
                    np.full((ny, nx, 3), 90.0), tuple(sigma), (nu,) * 3, steps=0)


def lens_angles(rho, gap=2.5):
    """Angles (gamma_0, gamma_1, gamma_2) in degrees of a lens of fluid 1 on the 0-2 interface,
    measured from the final fields: the 0-2 interface height y0 is the mean of the
    C_0 / (C_0 + C_2) = 1/2 crossings along the columns more than 12 nodes beyond the lens;
    circles are fitted to the C_1 = 1/2 contour above y0 + gap (the 1-2 interface) and below
    y0 - gap (the 0-1 interface), away from the junctions; each arc meets the line y = y0 at
    the angle alpha of a cap on that line, measured inside fluid 1; gamma_1 = alpha_up +
    alpha_low, gamma_2 = 180 - alpha_up, gamma_0 = 180 - alpha_low."""
    rho = np.asarray(rho, dtype=np.float64)
    C = rho / np.maximum(rho.sum(0), 1e-30)
    ny, nx = C[0].shape
    none = np.zeros((ny, nx), bool)
    p1 = contour_points(C[1], none)
    lx0, lx1 = p1[:, 0].min(), p1[:, 0].max()
    with np.errstate(invalid="ignore", divide="ignore"):
        phi = np.where(C[1] < 0.5, C[0] / (C[0] + C[2]), np.nan)
    p02 = contour_points(phi, none)
    far = (p02[:, 0] < lx0 - 12) | (p02[:, 0] > lx1 + 12)
    top = p02[:, 1] > ny / 2          # the interface that carries the lens (upper one)
    y0 = float(p02[far & top, 1].mean())
    xu, yu, Ru = fit_circle(p1[p1[:, 1] > y0 + gap])
    xl, yl, Rl = fit_circle(p1[p1[:, 1] < y0 - gap])
    au = float(np.degrees(np.arccos(np.clip(-(yu - y0) / Ru, -1.0, 1.0))))
    al = float(np.degrees(np.arccos(np.clip((yl - y0) / Rl, -1.0, 1.0))))
    return 180.0 - al, au + al, 180.0 - au


def line_crossings(rho, solid, lines, k, level=0.5):
    """Crossings of C_k = level along grid lines: lines = [("row", y) | ("col", x)], segments
    touching a solid node skipped; returns [(kind, index, position)] in scan order."""
    rho = np.asarray(rho, dtype=np.float64)
    c = rho[k] / np.maximum(rho.sum(0), 1e-30)
    s = np.asarray(solid).astype(bool)
    out = []
    for kind, idx in lines:
        v, sl = (c[idx], s[idx]) if kind == "row" else (c[:, idx], s[:, idx])
        for j in range(len(v) - 1):
            if not sl[j] and not sl[j + 1] and (v[j] - level) * (v[j + 1] - level) < 0:
                out.append((kind, idx, j + (v[j] - level) / (v[j] - v[j + 1])))
    return out


def cylinder_contact_angles(rho, solid, xc0, yc0, surf, gap=3.0):
    """Contact angles (deg, inside the droplet) of a Janus droplet (fluid 0 left, fluid 2 right,
    in fluid 1) sitting on a cylinder of wall radius surf centred at (xc0, yc0): a circle is
    fitted to each side's outer interface (the C_1 = 1/2 contour left and right of the internal
    interface, points more than gap from the wall), and the angle between that circle and the
    wall at their intersection follows from the law of cosines (Eq.23's triangle of the two
    centres and a contact point)."""
    rho = np.asarray(rho, dtype=np.float64)
    C = rho / np.maximum(rho.sum(0), 1e-30)
    s = np.asarray(solid).astype(bool)
    with np.errstate(invalid="ignore", divide="ignore"):
        phi = np.where(C[1] < 0.5, C[0] / (C[0] + C[2]), np.nan)
    xm = contour_points(phi, s)[:, 0].mean()
    p = contour_points(C[1], s)
    p = p[np.hypot(p[:, 0] - xc0, p[:, 1] - yc0) > surf + gap]
    out = []
    for side in (p[p[:, 0] < xm], p[p[:, 0] > xm]):
        xc, yc, R = fit_circle(side)
        D = float(np.hypot(xc - xc0, yc - yc0))
        c = (surf ** 2 + R * R - D * D) / (2.0 * surf * R)
        out.append(float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))))
    return out[0], out[1]
