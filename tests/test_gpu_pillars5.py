"""Section III.D at the paper's size (800 x 375, five pillars, compound droplet, Re = 0.75,
Ca = 0.04), GPU FP32, run to t* = U t / R_o = 37.81, the last snapshot of Fig.15.

The paper describes these runs by their snapshots only.  Over 770,000 steps of a flow around
pillars the path a droplet takes depends on every rounding, so the test holds the outcomes that
the paper states and that do not hinge on the path: each droplet keeps its mass (to 1e-3; the
carrier's changes through the open sides) and stays in one piece, and at t* = 37.81 each hangs
from a pillar (C_k > 1/2 within 2.5 lu of a pillar's surface).  Cases (wall triple (theta_rg,
theta_br, theta_gb)):

* the paper's (theta_bg, theta_br, theta_gr) = (135, 45, 40), i.e. (140, 45, 45): the green
  droplet hangs from the leftmost pillar (Fig.13f); this triple violates Eq.(18) as printed and
  runs with the library's Young warning;
* neutral (90, 90, 90) (Fig.15f): both droplets end adhered to pillars.
"""
import numpy as np
import pytest

from paper_2102_04709_gb300 import workloads as W

pytestmark = pytest.mark.gpu

R = 50.0
PILLARS = ((6.9, 3.75), (7.3, 6.2), (7.5, 1.6), (9.5, 5.14), (9.8, 2.54))


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_04709_gb300 import build, lbm3
    build.build()
    lbm3.load()
    return lbm3


def pieces(mask):
    """Connected components of a periodic-in-y mask (8-neighbour), by flood fill."""
    ny, nx = mask.shape
    seen = np.zeros_like(mask, dtype=bool)
    n = 0
    for y0, x0 in zip(*np.nonzero(mask)):
        if seen[y0, x0]:
            continue
        n += 1
        stack = [(y0, x0)]
        seen[y0, x0] = True
        while stack:
            y, x = stack.pop()
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yy, xx = (y + dy) % ny, x + dx
                    if 0 <= xx < nx and mask[yy, xx] and not seen[yy, xx]:
                        seen[yy, xx] = True
                        stack.append((yy, xx))
    return n


def touched_pillars(Ck, w):
    y, x = np.meshgrid(np.arange(w.ny), np.arange(w.nx), indexing="ij")
    out = []
    for j, (cx, cy) in enumerate(PILLARS):
        dy = np.abs(y - cy * R)
        d = np.sqrt((x - cx * R) ** 2 + np.minimum(dy, w.ny - dy) ** 2)
        if np.any((Ck > 0.5) & (d <= 0.8 * R + 2.5) & (w.solid == 0)):
            out.append(j)
    return out


@pytest.mark.parametrize("case", ["green-wetting", "neutral"])
def test_compound_droplet_hangs_from_pillars(gpu, case):
    triple = (140.0, 45.0, 45.0) if case == "green-wetting" else (90.0, 90.0, 90.0)
    w = W.five_pillars(triple)
    sim = gpu.Lbm3.from_workload(w)
    m0 = sim.diag()[:3].copy()
    sim.step(int(round(37.81 * R / w.u_in)))
    r, _ = sim.fields()
    d = sim.diag(check=False)
    sim.close()
    assert d[7] == 0
    C = r / np.maximum(r.sum(0), 1e-30)
    t0, t1 = touched_pillars(C[0], w), touched_pillars(C[1], w)
    n0, n1 = pieces(C[0] > 0.5), pieces(C[1] > 0.5)
    dm = (d[:3] - m0) / m0
    print(f"\n{case}: red touches pillars {t0} in {n0} piece(s), green {t1} in {n1}; relative "
          f"mass change {dm[0]:+.2e} {dm[1]:+.2e}")
    assert np.all(np.abs(dm[:2]) <= 1e-3)
    assert n0 == 1 and n1 == 1
    assert t0 and t1
    if case == "green-wetting":
        assert 0 in t1
