"""Planted mistakes: each case copies the oracle to a temporary directory, changes one line the
way a plausible slip would (a dropped term, a wrong sign, a wrong index or weight), builds the
copy and runs one of the pins of test_oracle_pins.py on it, which must fail.  The oracle itself is
never modified; this shows that the pins, not only the parity with the CUDA path, would catch
such a mistake in the oracle."""
import importlib.util
import os
import shutil

import pytest

from tests import test_oracle_pins as PINS

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")

# (what the slip is, text in lbm3_oracle.c, replacement, pin, pin arguments after the module)
MUTATIONS = [
    ("a diagonal weight 1/18 instead of 1/36",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 18.0};",
     "test_lattice_isotropy", ()),
    ("the forcing term of Eq.9 with the wrong sign",
     "Ft[a] = WQ[a] * (cx * Fs[0] + cy * Fs[1]);",
     "Ft[a] = -WQ[a] * (cx * Fs[0] + cy * Fs[1]);",
     "test_collision_conserves_mass_and_adds_force", ()),
    ("the 1/2 of the relaxation time dropped",
     "return mu / (rho * CS2) + 0.5;",
     "return mu / (rho * CS2) + 1.0;",
     "test_shear_wave_decay", ()),
    ("s_4 = s_1 instead of Eq.6's 8(2 - s_1)/(8 - s_1)",
     "real s4 = 8.0 * (2.0 - s1) / (8.0 - s1);",
     "real s4 = s1;",
     "test_halfway_walls_in_poiseuille_flow", ()),
    ("an arithmetic instead of a harmonic mixture viscosity in Eq.7",
     "for (int k = 0; k < NF; k++) inv += rk[k] / (o->rho0[k] * o->nu[k]);\n    real mu = rho / inv;",
     "for (int k = 0; k < NF; k++) inv += rk[k] * (o->rho0[k] * o->nu[k]);\n    real mu = inv / rho;",
     "test_mixture_viscosity_is_harmonic", ()),
    ("the Eq.12 stencil without its 1/c_s^2",
     "g[0] += WQ[a] * v[a] * EX[a] / CS2;\n        g[1] += WQ[a] * v[a] * EY[a] / CS2;",
     "g[0] += WQ[a] * v[a] * EX[a];\n        g[1] += WQ[a] * v[a] * EY[a];",
     "test_gradient_symbol", ()),
    ("I + nn instead of I - nn in the Eq.10 stress",
     "T[0] += s * (1.0 - nx * nx);",
     "T[0] += s * (1.0 + nx * nx);",
     "test_laplace_law", ()),
    ("A_kl of Eq.10 without its factor 1e6",
     "real A = fmin(1e6 * rk[k] * rk[l] / (o->rho0[k] * o->rho0[l]), 1.0);",
     "real A = fmin(1.0 * rk[k] * rk[l] / (o->rho0[k] * o->rho0[l]), 1.0);",
     "test_laplace_law", ()),
    ("halfway bounce-back that does not reverse the population",
     "o->fnew[((size_t)k * Q + o->opp[a]) * n + i] = v;",
     "o->fnew[((size_t)k * Q + a) * n + i] = v;",
     "test_uniform_fluid_at_rest_stays_at_rest", ()),
    ("the triple-point term of Eq.14 with 3.5 for 35",
     "real trip = fmin(35.0 * rk[0] * rk[1] * rk[2] / (rho * rho * rho), 1.0);",
     "real trip = fmin(3.5 * rk[0] * rk[1] * rk[2] / (rho * rho * rho), 1.0);",
     "test_beta_table", ()),
    ("the X > 0 branch of g(X) in Eq.15 with the wrong sign",
     "    if (X <= 1.0) return sin(acos(X)) - 1.0;",
     "    if (X <= 1.0) return 1.0 - sin(acos(X));",
     "test_gfun_values", ()),
    ("the recolouring term of Eq.13 with the wrong sign",
     "v += beta * WQ[a] * rk[k] * rk[l] / rho * ne;",
     "v -= beta * WQ[a] * rk[k] * rk[l] / rho * ne;",
     "test_flat_interface_segregation_balance", ()),
    ("the Zou-He inlet population with the wrong sign of U",
     "real g1 = f[3] + 2.0 / 3.0 * rho * U;",
     "real g1 = f[3] - 2.0 / 3.0 * rho * U;",
     "test_zou_he_uniform_inflow", ()),
    ("the Zou-He outlet population with the wrong sign of u",
     "real h3 = f[1] - 2.0 / 3.0 * ro * ux;",
     "real h3 = f[1] + 2.0 / 3.0 * ro * ux;",
     "test_zou_he_uniform_inflow", ()),
    ("Eq.21 for fluid 1 weighted by the wrong fluid",
     "        th[1] = t_gr + Cb / (Cb + Cr) * (t_gb - t_gr);",
     "        th[1] = t_gr + Cr / (Cb + Cr) * (t_gb - t_gr);",
     "test_weighted_contact_angle", ()),
    ("no fluid swap across the modified periodic seam",
     "int kk = sw ? swapk(k) : k;",
     "int kk = k;",
     "test_mass_modified_periodic", ()),
    ("a row of the transformation matrix M of Eq.4 with one wrong sign",
     "{0, 1, 0, -1, 0, 1, -1, -1, 1},",
     "{0, 1, 0, -1, 0, 1, 1, -1, 1},",
     "test_transform_matrix", ()),
    ("the Eq.19 normal left pointing into the solid",
     "            o->ns[2 * (size_t)i] = -sx / nrm;\n            o->ns[2 * (size_t)i + 1] = -sy / nrm;",
     "            o->ns[2 * (size_t)i] = sx / nrm;\n            o->ns[2 * (size_t)i + 1] = sy / nrm;",
     "test_normals_flat_and_curved", ()),
    ("the Eq.20 weights of the first two shells exchanged",
     "        case 1: return 4.0 / 21.0;\n        case 2: return 4.0 / 45.0;",
     "        case 1: return 4.0 / 45.0;\n        case 2: return 4.0 / 21.0;",
     "test_normals_flat_and_curved", ()),
    ("interpolation along a horizontal grid line from the wrong end",
     "*CD = Clef + fr * (Crig - Clef);",
     "*CD = Crig + fr * (Clef - Crig);",
     "test_rays_flat_wall_hand_worked", ()),
    ("interpolation along a vertical grid line from the wrong end",
     "*CD = Clow + fr * (Cup - Clow);",
     "*CD = Cup + fr * (Clow - Cup);",
     "test_rays_vertical_wall_hand_worked", ()),
    ("an unweighted instead of a w-weighted neighbour mean",
     "            s += WQ[a] * c_at(o, idx, sw, k);\n            ws += WQ[a];",
     "            s += c_at(o, idx, sw, k);\n            ws += 1.0;",
     "test_initial_wall_values_weighted_mean", ()),
    ("the third wall value without C_1 in 1 - C_0 - C_1",
     "        real cb = fmax(0.0, 1.0 - cr - cg);",
     "        real cb = fmax(0.0, 1.0 - cr);",
     "test_wall_values_close_to_one", ()),
    ("Eq.22's max and min exchanged",
     "return theta_k <= 90.0 ? fmax(c1, c2) : fmin(c1, c2);",
     "return theta_k <= 90.0 ? fmin(c1, c2) : fmax(c1, c2);",
     "test_contact_angle_flat_wall", (45.0,)),
    ("the tensions sigma_02 and sigma_12 assigned to each other's pair",
     "    o->sigma[0][2] = o->sigma[2][0] = sigma[1];\n    o->sigma[1][2] = o->sigma[2][1] = sigma[2];",
     "    o->sigma[0][2] = o->sigma[2][0] = sigma[2];\n    o->sigma[1][2] = o->sigma[2][1] = sigma[1];",
     "test_neumann_lens", ((0.010, 0.012, 0.008),)),
    ("the Eq.10 stress of a pair weighted by the tension of another pair",
     "real s = 0.5 * o->sigma[k][l] * A * Gn;",
     "real s = 0.5 * o->sigma[k][3 - k - l] * A * Gn;",
     "test_neumann_lens", ((0.010, 0.012, 0.008),)),
    ("X_kl of Eq.15 built around the wrong pair (sigma_kl and sigma_ml exchanged)",
     "            double X = (o->sigma[m][k] * o->sigma[m][k] + o->sigma[m][l] * o->sigma[m][l] -\n                        o->sigma[k][l] * o->sigma[k][l]) /\n                       (2.0 * o->sigma[m][k] * o->sigma[m][l]);",
     "            double X = (o->sigma[m][k] * o->sigma[m][k] + o->sigma[k][l] * o->sigma[k][l] -\n                        o->sigma[m][l] * o->sigma[m][l]) /\n                       (2.0 * o->sigma[m][k] * o->sigma[k][l]);",
     "test_beta_table", ()),
    ("a missing Eq.12 neighbour of a wall node taking the node's own value",
     "                for (int k = 0; k < NF; k++) v[k][a] = 2.0 * c0[k] - c_at(o, idx2, sw2, k);",
     "                for (int k = 0; k < NF; k++) v[k][a] = c0[k];",
     "test_gradient_at_wall_node_linear_field", ()),
    ("Eq.21 weighted by the wrong fluid",
     "th[0] = t_rg + Cb / (Cb + Cg) * (t_rb - t_rg);",
     "th[0] = t_rg + Cg / (Cb + Cg) * (t_rb - t_rg);",
     "test_weighted_contact_angle", ()),
]


def mutant(d, old, new, tag):
    """Build the oracle with `old` replaced by `new` in directory d; return its module."""
    d.mkdir()
    src = open(os.path.join(ORACLE, "lbm3_oracle.c")).read()
    assert src.count(old) == 1, "the planted text must occur exactly once"
    (d / "lbm3_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE, "oracle.py"), d / "oracle.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{tag}", d / "oracle.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return mod


def test_every_planted_mistake_is_caught(tmp_path):
    """All cases at once on threads (each mutant is its own library; the oracle's C calls
    release the GIL); the failure message names every slip that no pin caught."""
    from concurrent.futures import ThreadPoolExecutor

    def run(j):
        what, old, new, pin, args = MUTATIONS[j]
        mod = mutant(tmp_path / f"m{j}", old, new, j)
        try:
            getattr(PINS, pin)(mod, *args)
        except AssertionError:
            return None
        return f"{what} (pin {pin})"

    with ThreadPoolExecutor(8) as ex:
        missed = [m for m in ex.map(run, range(len(MUTATIONS))) if m]
    assert not missed, "not caught: " + "; ".join(missed)
