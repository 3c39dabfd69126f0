"""The pins are strong enough: plant one plausible mistake at a time in a copy of
the oracle's C source (on the CPU), rebuild it, and check that at least one pin of
test_oracle_pins fails. The product code is never touched."""
import functools
import os
import sys
import subprocess
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import test_oracle_pins as pins  # noqa: E402

# (name, text in rti_oracle.c, replacement): each one a mistake a port could make
MUTANTS = [
    ("mass: flux sum instead of difference", "dtdx * (Me - Mw)", "dtdx * (Me + Mw)"),
    ("mass: N faces swapped", "dtdx * (Nn - Ns)", "dtdx * (Ns - Nn)"),
    ("pressure: wrong sign", "grad = eR - eL;", "grad = eL - eR;"),
    ("pressure: still-water depth only", "Df = 0.5 * (hL + hR) + 0.5 * (eL + eR);",
     "Df = 0.5 * (hL + hR);"),
    ("pressure: y uses the x stencil", "grad = eN - eS;", "grad = eN - eN;"),
    ("friction: n instead of n^2", "p->g * nf * nf *", "p->g * nf *"),
    ("friction: D^(4/3) instead of D^(7/3)", "(Df * Df * orc_cube_root(Df))",
     "(Df * orc_cube_root(Df))"),
    ("friction: cube root with two Newton steps", "for (int k = 0; k < 3; ++k) {",
     "for (int k = 0; k < 2; ++k) {"),
    ("friction: cube root start not scaled by 2^(-r/3)",
     "double s = r == 0 ? 1.0 : (r == 1 ? 0.7937005259840998 : 0.6299605249474366);",
     "double s = 1.0;"),
    ("advection: downwind on the x term", "if (w > 0) return okm ? phi0 - phim : 0.0;",
     "if (w > 0) return okp ? phip - phi0 : 0.0;"),
    ("advection: Nbar from the wrong row",
     "(b->N[FY(b, f - 1, j + 1)] + b->N[FY(b, f, j + 1)])",
     "(b->N[FY(b, f - 1, j)] + b->N[FY(b, f, j)])"),
    ("flood: dry cell's ground sign", "} else if (wL && !wR && eL > -hR) {",
     "} else if (wL && !wR && eL > hR) {"),
    ("radiation: inward", "return sign * (sqrt(", "return -sign * (sqrt("),
    ("nesting: fine faces not interpolated", "return (2.0 * v[k] + v[kn]) / 3.0;",
     "return v[kn];"),
    ("nesting: ring mean without the 1/count",
     "out[(size_t)J * a + I] = sum * (1.0 / (double)wet);",
     "out[(size_t)J * a + I] = sum * (1.0 / 8.0);"),
    ("nesting: full feedback still only on the ring",
     "if (p->nest_feedback == ORC_NEST_FULL) return 1;",
     "if (p->nest_feedback == -1) return 1;"),
    ("nesting: constant flux still interpolated", "if (sub == 1 || constant) return v[k];",
     "if (sub == 1) return v[k];"),
    ("nesting: chained exchange (each level receives before its parent packs)",
     "    if (buf[k]) unpack_child(s, k, buf[k]);",
     "    if (buf[k]) { pack_child(s, k, buf[k]); unpack_child(s, k, buf[k]); }"),
    ("nesting: full feedback patch one child row off",
     "for (int y = 3 * J; y < 3 * J + 3; ++y) { /* inner",
     "for (int y = 3 * J + 1; y < 3 * J + 4 && y < c->ny; ++y) { /* inner"),
    ("front: outflow limit of half a cell", "double cap = (m > 0 ? Dlo : Dhi) * dx / (4.0 * dt);",
     "double cap = (m > 0 ? Dlo : Dhi) * dx / (2.0 * dt);"),
    ("front: velocity limit on the still-water depth",
     "    double vc = vel_limit * Df;", "    double vc = vel_limit * (0.5 * (Dlo + Dhi));"),
    ("front: velocity limit ignored", "    if (vc < cap) cap = vc;", "    (void)vc;"),
    ("front: outflow limit on the downwind cell", "double cap = (m > 0 ? Dlo : Dhi) * dx / (4.0 * dt);",
     "double cap = (m > 0 ? Dhi : Dlo) * dx / (4.0 * dt);"),
    ("initial: no floor at the ground", "      if (e < -h) e = -h;\n    } else {",
     "    } else {"),
    ("initial: uplift on land too", "    } else {\n      e = -h;\n    }",
     "    } else {\n      e = dz ? dz[c] : -h;\n    }"),
    ("friction: the smoother neighbour (x)", "double nf = b->n[L] > b->n[R] ? b->n[L] : b->n[R];",
     "double nf = b->n[L] < b->n[R] ? b->n[L] : b->n[R];"),
    ("friction: the cell's own roughness (y)", "double nf = b->n[S] > b->n[Nc] ? b->n[S] : b->n[Nc];",
     "double nf = b->n[S];"),
    ("nesting: mean not floored at the parent's ground",
     "      if (avg < -P->h[pc]) avg = -P->h[pc];\n", ""),
    ("mass: pressure from the old level", "double eL = b->eta1[L], eR = b->eta1[R]",
     "double eL = b->eta[L], eR = b->eta[R]"),
    ("advection: face depth from the old level (x)",
     "return 0.5 * (b->h[L] + b->h[R]) + 0.5 * (b->eta1[L] + b->eta1[R]);",
     "return 0.5 * (b->h[L] + b->h[R]) + 0.5 * (b->eta[L] + b->eta[R]);"),
    ("advection: face depth from the old level (y)",
     "return 0.5 * (b->h[S] + b->h[Nc]) + 0.5 * (b->eta1[S] + b->eta1[Nc]);",
     "return 0.5 * (b->h[S] + b->h[Nc]) + 0.5 * (b->eta[S] + b->eta[Nc]);"),
    ("advection: faces of dry depth still used",
     "return f >= 1 && f <= b->nx - 1 && j >= 0 && j <= b->ny - 1 && dep_x(b, f, j) > eps;",
     "return f >= 1 && f <= b->nx - 1 && j >= 0 && j <= b->ny - 1;"),
    ("radiation: also from a dry edge cell", "  if (!(h + e > p->dry_eps)) return 0.0;\n  return sign",
     "  return sign"),
    ("outputs: strict arrival threshold", "e >= p->arrival_thr", "e > p->arrival_thr"),
    ("outputs: max tracked on dry cells", "if (b->h[c] + e > p->dry_eps && e > b->emax[c])",
     "if (e > b->emax[c])"),
    ("velocity: west face only",
     "double u = 0.5 * (face_velocity(M[FX(b, i, j)], Dw, eps) + face_velocity(M[FX(b, i + 1, j)], De, eps));",
     "double u = face_velocity(M[FX(b, i, j)], Dw, eps);"),
    ("velocity: speed without the depth", "return D > eps ? q / D : 0.0;",
     "return D > eps ? q : 0.0;"),
    ("velocity: y faces of the wrong row", "face_velocity(N[FY(b, i, j + 1)], Dn, eps)",
     "face_velocity(N[FY(b, i, j)], Dn, eps)"),
    ("velocity: the cell's depth for every face",
     "double Dw = face_depth(b, eta, i > 0 ? C(b, i - 1, j) : c, c);",
     "double Dw = D;"),
    ("velocity: not a running maximum", "if (s2 > b->vmax2[C(b, i, j)]) b->vmax2[C(b, i, j)] = s2;",
     "b->vmax2[C(b, i, j)] = s2 > 0 ? s2 : 0.0;"),
]

# cheapest first; each takes the oracle module as its only argument
BATTERY = [
    pins.test_cfl_and_nesting_rejected,
    pins.test_cube_root_is_within_four_ulp,
    pins.test_max_velocity_averages_the_two_faces_of_a_cell,
    pins.test_max_velocity_of_uniform_flow_is_exact,
    pins.test_max_velocity_takes_each_face_over_its_own_depth,
    pins.test_max_velocity_is_zero_at_rest_and_on_dry_land_and_grows_monotonically,
    pins.test_max_and_arrival_are_functions_of_history,
    pins.test_outflow_limit_on_a_puddle,
    pins.test_velocity_limit_on_a_puddle,
    pins.test_advective_depth_is_the_new_level,
    pins.test_initial_condition_r10,
    pins.test_nest_constant_field_ring_average,
    pins.test_nest_edge_flux_reproduces_linear_profile,
    pins.test_constant_flux_gives_each_fine_face_its_coarse_face,
    pins.test_full_feedback_sets_every_covered_cell_to_the_child_mean,
    pins.test_full_feedback_exchange_is_simultaneous,
    pins.test_mirror_and_transpose_symmetry_bitwise,
    pins.test_friction_matches_manning_ode,
    pins.test_friction_takes_the_rougher_neighbour,
    pins.test_radiation_west_edge_absorbs,
    pins.test_dry_basin_with_open_edges_stays_dry,
    functools.partial(pins.test_standing_wave_discrete_period, cfl=0.7),
    pins.test_budget_closes_with_drying_and_radiation,
    pins.test_nested_budget_closes,
    pins.test_nested_plane_wave_matches_fine_grid,
    pins.test_closed_basin_mass_conservation,
    pins.test_lake_at_rest_nested_bitwise,
    pins.test_thacker_parabolic_bowl,
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(oracle_mod, tmp_path, name, old, new):
    src = open(oracle_mod.SRC).read()
    assert src.count(old) >= 1, f"mutation site missing: {old}"
    csrc = tmp_path / "rti_oracle.c"
    csrc.write_text(src.replace(old, new))
    hdr = os.path.join(os.path.dirname(oracle_mod.SRC), "rti_oracle.h")
    (tmp_path / "rti_oracle.h").write_text(open(hdr).read())
    so = str(tmp_path / "mut.so")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", so, str(csrc), "-lm"])
    fake = types.SimpleNamespace(
        Oracle=functools.partial(oracle_mod.Oracle, lib_path=so),
        OracleError=oracle_mod.OracleError, lib=functools.partial(oracle_mod.lib, so),
        from_scenario=functools.partial(oracle_mod.from_scenario, lib_path=so),
        SRC=oracle_mod.SRC, NEST_RING=oracle_mod.NEST_RING, NEST_FULL=oracle_mod.NEST_FULL,
        FLUX_LINEAR=oracle_mod.FLUX_LINEAR, FLUX_CONSTANT=oracle_mod.FLUX_CONSTANT)
    for pin in BATTERY:
        try:
            pin(fake)
        except (AssertionError, oracle_mod.OracleError, FloatingPointError, ValueError):
            return  # caught
    pytest.fail(f"no pin caught the planted mistake: {name}")
