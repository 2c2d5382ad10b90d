"""The oracle's reference tape (oracle/lbm3_oracle_tape.cpp): the oracle's own step recorded
with a reverse-mode scalar type and swept backwards, for the gradient of J = x-centroid of
fluid 0 with respect to the wall angles of every C_SB node and the Zou-He inflow velocity.
Pinned against central finite differences of the FP64 oracle (a different method: two forward
runs per derivative), on a small case whose droplet shell wets a pillar under inflow."""
import numpy as np

from paper_2102_04709_gb300 import workloads as W


def tape_case():
    """48 x 24, one pillar wetted by the shell of a compound droplet, Zou-He inflow, per-node
    angles in [60, 120], initial densities perturbed by a seeded 1e-6 (a generic point where J
    is smooth in the angles)."""
    w = W.pillars(nx=48, ny=24, count=1, r_lo=4.0, r_hi=5.0, x_lo=24.0, x_hi=28.0, gap=4.0,
                  seed=3, drop=(14.0, 12.0), r_core=3.0, r_shell=7.0,
                  theta_range=(60.0, 120.0), u_in=0.02)
    rng = np.random.default_rng(2)
    w.rho = w.rho * (1.0 + 1e-6 * rng.standard_normal(w.rho.shape))
    return w


def oracle_J(O, w, steps, angles, u_in):
    o = O.Oracle(w.nx, w.ny, w.periodic_y, w.bc_x, w.solid, angles, w.sigma, w.nu, w.beta0, u_in,
                 w.rho_out)
    o.set_fields(w.rho)
    o.step(steps)
    d = o.diag()
    return d[3] / d[0]


def test_tape_matches_central_differences(oracle_mod):
    O = oracle_mod
    w = tape_case()
    steps = 60
    J, g, du = O.tape_centroid_gradient(w, steps)
    assert J == oracle_J(O, w, steps, w.angles, w.u_in)      # the same forward operations
    solid = w.solid.astype(bool)
    assert np.all(g[~solid] == 0.0)                          # angles act at C_SB nodes only
    # dJ/du_in
    h = 1e-6
    fdu = (oracle_J(O, w, steps, w.angles, w.u_in + h) -
           oracle_J(O, w, steps, w.angles, w.u_in - h)) / (2 * h)
    assert abs(du - fdu) <= 1e-6 * abs(fdu), (du, fdu)
    # the three largest angle components and a random direction over all of them
    scale = np.abs(g).max()
    assert scale > 1e-7
    flat = np.argsort(-np.abs(g).reshape(-1))[:3]
    for j in flat:
        y, x, c = np.unravel_index(j, g.shape)
        ap, am = w.angles.copy(), w.angles.copy()
        ap[y, x, c] += 1e-3
        am[y, x, c] -= 1e-3
        fd = (oracle_J(O, w, steps, ap, w.u_in) - oracle_J(O, w, steps, am, w.u_in)) / 2e-3
        assert abs(g[y, x, c] - fd) <= 1e-4 * scale, (y, x, c, g[y, x, c], fd)
    v = np.random.default_rng(7).standard_normal(g.shape) * solid[..., None]
    fd = (oracle_J(O, w, steps, w.angles + 1e-3 * v, w.u_in) -
          oracle_J(O, w, steps, w.angles - 1e-3 * v, w.u_in)) / 2e-3
    ad = float((g * v).sum())
    assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)
