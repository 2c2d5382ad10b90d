"""Longer runs, GPU (FP32) against the FP64 oracle on what the method is for: the contact angle
and the interface position.  Tolerances: 0.5 degree on the angle, 0.5 lattice units on every
position (the interface is the C_k = 1/2 contour, located by linear interpolation between nodes).

* A droplet of fluid 0 in fluid 2 on a flat wall, started as a half-disc (90 degrees) with the
  wall angle 60 degrees in fluid 0 (triple (90, 120, 60), Eq.18 holds for equal tensions), 5000
  steps.  Its base half-width a along the first fluid row, its height h on the centre column and
  the cap angle 2 atan(h / a).  The oracle itself relaxes towards the prescribed angle (76 deg at
  1000 steps, 65 deg at 5000), which is checked loosely as physics, not as parity.
* The Janus droplet on the staircased cylinder, 3000 steps: every crossing of C_0 = 1/2 and
  C_2 = 1/2 along rows and columns through the droplet (segments touching a solid node skipped).
"""
import numpy as np
import pytest

from paper_2102_04709_gb300 import workloads as W

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


def both(gpu, oracle_mod, w, steps):
    g = gpu.Lbm3.from_workload(w)
    g.step(steps)
    rg, _ = g.fields()
    o = oracle_mod.Oracle.from_workload(w)
    o.step(steps)
    ro, _ = o.fields()
    return rg, ro


def fraction(rho, k):
    return rho[k] / np.maximum(rho.sum(0), 1e-30)


def crossing(v, start, step):
    """Position where v falls through 1/2 walking from index start in direction step."""
    i = start
    while 0 <= i + step < len(v) and not (v[i] >= 0.5 > v[i + step]):
        i += step
    assert 0 <= i + step < len(v), "no interface on this line"
    return i + step * (v[i] - 0.5) / (v[i] - v[i + step])


def cap(rho, nx):
    c = fraction(rho, 0)
    xc = nx // 2
    xl, xr = crossing(c[1], xc, -1), crossing(c[1], xc, 1)
    h = crossing(c[:, xc], 1, 1) - 0.5      # the halfway wall lies at y = 1/2
    a = (xr - xl) / 2
    return 2.0 * np.degrees(np.arctan(h / a)), a, h


def test_sessile_contact_angle_5000_steps(gpu, oracle_mod):
    nx, ny, R = 96, 48, 14.0
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = 1
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    drop = ((x - nx / 2 + 0.5) ** 2 + (y - 0.5) ** 2 <= R * R) & (solid == 0)
    rho = np.zeros((3, ny, nx))
    rho[0][drop] = 1.0
    rho[2][~drop & (solid == 0)] = 1.0
    w = W.Workload("sessile_60", nx, ny, 0, W.BC_PERIODIC, solid, rho,
                   np.tile(np.array([90.0, 120.0, 60.0]), (ny, nx, 1)), (0.01, 0.01, 0.01),
                   (0.1, 0.1, 0.1))
    rg, ro = both(gpu, oracle_mod, w, 5000)
    tg, ag, hg = cap(rg, nx)
    to, ao, ho = cap(ro, nx)
    print(f"GPU theta {tg:.3f} a {ag:.3f} h {hg:.3f} | oracle theta {to:.3f} a {ao:.3f} h {ho:.3f}")
    assert abs(tg - to) <= 0.5
    assert abs(ag - ao) <= 0.5 and abs(hg - ho) <= 0.5
    assert abs(to - 60.0) < 8.0      # relaxing towards the prescribed angle


def line_crossings(rho, solid, lines, k):
    c = fraction(rho, k)
    out = []
    for kind, idx in lines:
        v, s = (c[idx], solid[idx]) if kind == "row" else (c[:, idx], solid[:, idx])
        for j in range(len(v) - 1):
            if not s[j] and not s[j + 1] and (v[j] - 0.5) * (v[j + 1] - 0.5) < 0:
                out.append((kind, idx, j + (v[j] - 0.5) / (v[j] - v[j + 1])))
    return out


def test_cylinder_interface_positions_3000_steps(gpu, oracle_mod):
    w = W.janus_cylinder(nx=96, ny=90, Rs=16.0, Rj=14.0)
    rg, ro = both(gpu, oracle_mod, w, 3000)
    ys, xs = np.nonzero(w.rho[0] + w.rho[2])
    cy, cx = int(round(ys.mean())), int(round(xs.mean()))
    lines = [("row", cy), ("row", cy + 5), ("row", cy - 5), ("col", cx - 7), ("col", cx),
             ("col", cx + 7)]
    for k in (0, 2):
        cg, co = line_crossings(rg, w.solid, lines, k), line_crossings(ro, w.solid, lines, k)
        assert len(co) >= 4 and [c[:2] for c in cg] == [c[:2] for c in co]
        d = max(abs(a[2] - b[2]) for a, b in zip(cg, co))
        print(f"fluid {k}: {len(co)} crossings, max |d position| = {d:.2e}")
        assert d <= 0.5
