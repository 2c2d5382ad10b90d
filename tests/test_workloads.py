"""The synthetic inputs: the seeded generator, the pillar layouts and the paper's set-ups match
the recipe the design states, and the Table I fixture is consistent with Eq.(18)."""
import math

import numpy as np

from paper_2102_04709_gb300 import workloads as W
from tests import physics as P


def test_splitmix64_published_vector():
    """SplitMix64 from state 0 gives the published first outputs of the generator."""
    g = W.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                 0x06C45D188009454F]
    u = W.SplitMix64(7)
    vals = [u.uniform(2.0, 5.0) for _ in range(1000)]
    assert min(vals) >= 2.0 and max(vals) < 5.0


def test_pillar_layout_of_the_4096x2048_workload():
    """60 discs, radius in [40, 80], centre x in [900, 3900], at least 8 lattice units apart
    across the periodic y direction; the same layout on every call (seed 2102); the compound
    droplet (core 120, shell 200 at (400, 1024)) clear of every solid node."""
    pl, _ = W.place_pillars(4096, 2048, 60, 40.0, 80.0, 900.0, 3900.0, 8.0, 2102)
    pl2, _ = W.place_pillars(4096, 2048, 60, 40.0, 80.0, 900.0, 3900.0, 8.0, 2102)
    assert pl == pl2 and len(pl) == 60
    for i, (x, y, r) in enumerate(pl):
        assert 40.0 <= r <= 80.0 and 900.0 <= x <= 3900.0 and 0.0 <= y < 2048.0
        for (x2, y2, r2) in pl[:i]:
            dy = abs(y - y2)
            assert math.hypot(x - x2, min(dy, 2048 - dy)) >= r + r2 + 8.0
    w = W.config4()
    assert w.solid.shape == (2048, 4096) and w.bc_x == W.BC_ZOUHE and w.periodic_y == 1
    assert w.rho[:2].sum() > 0 and not np.any(w.rho[:, w.solid.astype(bool)])
    yy, xx = np.nonzero(w.solid)
    assert np.hypot(xx - 400.0, yy - 1024.0).min() > 200.0


def test_five_pillar_setup_of_section_3d():
    """Re = 0.75 and Ca = 0.04 from the chosen viscosity and inflow; five pillar discs of radius
    40 at the printed centres; core and shell areas of the compound droplet."""
    w = W.five_pillars()
    R = 50.0
    assert (w.nx, w.ny) == (800, 375)
    assert abs(w.u_in * R / w.nu[0] - 0.75) < 1e-12 and abs(w.u_in * w.nu[0] / 0.01 - 0.04) < 1e-12
    assert abs(w.solid.sum() / (5 * math.pi * 40.0 ** 2) - 1.0) < 0.01
    for cx, cy in ((6.9, 3.75), (7.3, 6.2), (7.5, 1.6), (9.5, 5.14), (9.8, 2.54)):
        assert w.solid[int(round(cy * R)), int(round(cx * R))] == 1
    assert abs(w.rho[0].sum() / (math.pi * 30.0 ** 2) - 1.0) < 0.01
    assert abs(w.rho[1].sum() / (math.pi * (50.0 ** 2 - 30.0 ** 2)) - 1.0) < 0.01


def test_table1_fixture_satisfies_young():
    """Every analytical triple of Table I satisfies Eq.(18) for equal tensions, and each
    simulated value the paper prints lies within its stated 3.0 % of the analytical one."""
    rows = P.table1()
    assert [r[0] for r in rows] == list("abcdef")
    for _, ana, sim in rows:
        assert abs(sum(math.cos(math.radians(t)) for t in ana)) < 1e-12
        for a, s in zip(ana, sim):
            assert abs(s - a) <= 0.0301 * a
