"""The two larger standard configurations at their stated sizes, GPU against the FP64 oracle at
a checkpoint the oracle reaches in about a minute on the host's cores (3000 steps), on what the
method is for: contact angles within 0.5 degree and interface positions within 0.5 lattice
units (the C_k = 1/2 contour, located by linear interpolation between nodes along grid lines).
The largest pointwise density difference is printed and bounded as well (after 3000 steps it
is the density change of a fraction of a lattice unit's interface shift).

* Perfect Janus droplet on a cylinder (Section III.B): 512 x 512 periodic box, solid disc of
  radius 60, droplet of radius 50 of fluids 0 and 2 in fluid 1, sigma_02 = 0.005, angles
  (90, 90, 135).  Both contact angles on the cylinder and the interface crossings on rows and
  columns through the droplet.
* Ternary capillary intrusion (Section III.C): 2048 x 128, channel rows 24..103, modified
  periodic seam, angles (90, 135, 45); equal viscosities with FP32 and with FP16 offset storage,
  and the viscosity contrast (1.0, 0.01, 0.01) with FP32.  The menisci's crossings on five rows
  and the intruded length (fluid-0 mass per channel row).
"""
import numpy as np
import pytest

from paper_2102_04709_gb300 import workloads as W
from tests import physics as P

pytestmark = pytest.mark.gpu

STEPS = 3000


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_04709_gb300 import build, lbm3
    build.build()
    lbm3.load()
    return lbm3


def gpu_fields(gpu, w, precision=0):
    g = gpu.Lbm3.from_workload(w, precision=precision)
    g.step(STEPS)
    r, _ = g.fields()
    g.diag()
    g.close()
    return r


def oracle_fields(oracle_mod, w):
    o = oracle_mod.Oracle.from_workload(w, threads=0)
    o.step(STEPS)
    return o.fields()[0]


def compare_crossings(rg, ro, solid, lines, k, tol=0.5):
    cg, co = P.line_crossings(rg, solid, lines, k), P.line_crossings(ro, solid, lines, k)
    assert len(co) >= 4, "the interfaces must cross the sampled lines"
    assert [c[:2] for c in cg] == [c[:2] for c in co], "the same crossings on both sides"
    d = max(abs(a[2] - b[2]) for a, b in zip(cg, co))
    assert d <= tol, f"fluid {k}: max |d position| = {d:.3e}"
    return d, len(co)


def test_config2_janus_cylinder_512(gpu, oracle_mod):
    w = W.config2()
    rg = gpu_fields(gpu, w)
    ro = oracle_fields(oracle_mod, w)
    err = np.abs(rg - ro).max()
    ag = P.cylinder_contact_angles(rg, w.solid, 256.0, 256.0, 60.5)
    ao = P.cylinder_contact_angles(ro, w.solid, 256.0, 256.0, 60.5)
    # rows above the cylinder's top (y = 316) and columns through each half of the droplet, clear
    # of the vertical internal interface at x = 256
    lines = [("row", 326), ("row", 346), ("row", 356), ("col", 231), ("col", 241), ("col", 271),
             ("col", 281)]
    d0, n0 = compare_crossings(rg, ro, w.solid, lines, 0)
    d2, n2 = compare_crossings(rg, ro, w.solid, lines, 2)
    print(f"{w.name} after {STEPS} steps: max |d rho_k| {err:.3e}; angles GPU {ag[0]:.3f} "
          f"{ag[1]:.3f} oracle {ao[0]:.3f} {ao[1]:.3f}; crossings fluid 0: {n0} within {d0:.2e}, "
          f"fluid 2: {n2} within {d2:.2e}")
    assert abs(ag[0] - ao[0]) <= 0.5 and abs(ag[1] - ao[1]) <= 0.5
    assert err <= 1e-3


def capillary_lines():
    return [("row", y) for y in (26, 40, 64, 88, 101)]


def intrusion(rho, H=80):
    return float(rho[0].sum()) / H


@pytest.mark.parametrize("nu", [(0.1, 0.1, 0.1), (1.0, 0.01, 0.01)], ids=["equal", "contrast"])
def test_config3_capillary_2048(gpu, oracle_mod, nu):
    w = W.config3(nu=nu)
    ro = oracle_fields(oracle_mod, w)
    precisions = (0, 1) if nu[0] == nu[1] else (0,)
    for prec in precisions:
        rg = gpu_fields(gpu, w, prec)
        err = np.abs(rg - ro).max()
        d0, n0 = compare_crossings(rg, ro, w.solid, capillary_lines(), 0)
        d2, n2 = compare_crossings(rg, ro, w.solid, capillary_lines(), 2)
        ds = abs(intrusion(rg) - intrusion(ro))
        name = {0: "fp32", 1: "fp16"}[prec]
        print(f"{w.name} nu={nu} {name} after {STEPS} steps: max |d rho_k| {err:.3e}; menisci "
              f"crossings within {max(d0, d2):.2e} lu ({n0 + n2}); intrusion {intrusion(rg):.4f} vs "
              f"{intrusion(ro):.4f} (|d| {ds:.2e} lu)")
        assert ds <= 0.5
        # pointwise, the densities differ where a meniscus sits a little elsewhere: a shift d of
        # an interface whose fraction profile has slope at most beta0 / 2 = 0.35 per lu moves
        # rho_k by at most 0.35 d; FP32 holds its crossings within 1e-3 lu here (measured
        # 3.5e-4), so within 3.5e-4 + 1e-5 pointwise; the 16-bit offsets carry their stated error
        if prec == 0:
            assert max(d0, d2) <= 1e-3
            assert err <= 0.35 * 1e-3 + 1e-5
        else:
            # 16-bit offsets: their error is stated (printed above); the positions hold the
            # 0.5 lu of the longer runs (checked above), the densities move with them
            assert err <= 0.35 * max(d0, d2) + 1e-3
