"""Plant plausible mistakes in copies of the oracle and check the pins catch each.

Every mutant is a one-line textual change of ``oracle/ljoracle.c`` (a dropped
factor, a flipped sign, a wrong index, a transposed operand), compiled to a
temporary library and run against all pins in a child process (a crash or a
hang counts as caught).  CPU only.
"""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "force_dropped_factor_2": ("*f_over_r = 24.0 * eps * (2.0 * s12 - s6) / r2;", "*f_over_r = 24.0 * eps * (s12 - s6) / r2;"),
    "energy_wrong_sign": ("*u = 4.0 * eps * (s12 - s6);", "*u = 4.0 * eps * (s12 + s6);"),
    "sigma_not_squared": ("double s2 = (sig * sig) / r2;", "double s2 = sig / r2;"),
    "image_sign": ("return xi - (xj + (double)k * L);", "return xi - (xj - (double)k * L);"),
    "min_image_wrong_k": ("if (d > 0.5 * L) return 1;", "if (d > 0.5 * L) return -1;"),
    "r2_wrong_index": ("return (a + b) + c;", "return (a + b) + b;"),
    "shift_added": ("U += u - shift_energy(p, type[i], type[j]);", "U += u + shift_energy(p, type[i], type[j]);"),
    "cells_shift_added": ("U += 0.5 * (u - shift_energy(p, type[i], type[j]));", "U += 0.5 * (u + shift_energy(p, type[i], type[j]));"),
    "newton3_sign": ("F[3*j+0] -= f * dx; F[3*j+1] -= f * dy; F[3*j+2] -= f * dz;", "F[3*j+0] += f * dx; F[3*j+1] += f * dy; F[3*j+2] += f * dz;"),
    "cutoff_compares_r2_to_rc": ("if (!(r2 < rc * rc)) continue;\n            double f, u;", "if (!(r2 < rc)) continue;\n            double f, u;"),
    "cells_reach_floor": ("reach[d] = (int64_t)ceil(rcmax / side[d] + 1e-9);", "reach[d] = (int64_t)floor(rcmax / side[d]);"),
    "cells_image_transposed": ("(int)(k[0] + mimg[3*i+0] - mimg[3*j+0])", "(int)(k[0] - mimg[3*i+0] + mimg[3*j+0])"),
    "cells_self_pair": ("if (j == i && k[0] == 0 && k[1] == 0 && k[2] == 0) continue;", "if (0) continue;"),
    "verlet_full_first_kick": ("v[3*i+d] += h * F[3*i+d];\n                x[3*i+d] += dt * v[3*i+d];", "v[3*i+d] += 2.0 * h * F[3*i+d];\n                x[3*i+d] += dt * v[3*i+d];"),
    "verlet_drift_half": ("x[3*i+d] += dt * v[3*i+d];", "x[3*i+d] += 0.5 * dt * v[3*i+d];"),
    "stats_variance_not_rooted": ("out[1] = mean > 0.0 ? sqrt(var) / mean : 0.0;", "out[1] = mean > 0.0 ? var / mean : 0.0;"),
    "stats_median_upper": ("0.5 * ((double)cnt[nb / 2 - 1] + (double)cnt[nb / 2])", "(double)cnt[nb / 2]"),
    "list_newton3_sign": ("F[3*j+d] -= f * r[d];", "F[3*j+d] += f * r[d];"),
    "vjp_dropped_radial_term": ("double w = g * u[d] + 2.0 * dgds * ur * r[d];", "double w = g * u[d] + dgds * ur * r[d];"),
    "vjp_j_sign": ("gx[3*j+d] -= w;", "gx[3*j+d] += w;"),
    "vjp_cotangent_transposed": ("u[d] = c[3*i+d] - c[3*j+d];", "u[d] = c[3*j+d] - c[3*i+d];"),
    "vjp_dgds_power": ("4.0 * sig6 / s5);", "4.0 * sig6 / s4);"),
    "vjp_dgdsig_factor": ("(24.0 * sig11 / s7 - 6.0 * sig5 / s4)", "(12.0 * sig11 / s7 - 6.0 * sig5 / s4)"),
    "vjp_symmetric_entry_missing": ("gsig[b * nt + a] += ur * dgdsig;", "gsig[b * nt + a] += 0.0;"),
    "rollout_drift_half": ("x[3*i+d] += dt * v[3*i+d];\n            }\n    }\n    free(x); free(v); free(F);",
                           "x[3*i+d] += 0.5 * dt * v[3*i+d];\n            }\n    }\n    free(x); free(v); free(F);"),
    "rollout_vjp_drift_coefficient": ("gv0[k] += dt * gx0[k];", "gv0[k] += 0.5 * dt * gx0[k];"),
    "rollout_vjp_kick_levels_swapped": ("xs + (size_t)(t + level) * n3", "xs + (size_t)(t + 1 - level) * n3"),
    "walls_no_velocity_flip": ("if (*x < 0.0) { *x = -*x; *v = -*v; }", "if (*x < 0.0) { *x = -*x; }"),
    "walls_far_face_mirror": ("else if (*x > L) { *x = 2.0 * L - *x; *v = -*v; }", "else if (*x > L) { *x = L - *x; *v = -*v; }"),
    "walls_image_taken": ("return p->walls[d] ? 0 : min_image_k(xi, xj, p->box[d]);", "return min_image_k(xi, xj, p->box[d]);"),
    "walls_cells_image_taken": ("if (p->walls[d] && k[d] != 0) skip = 1;", "if (0) skip = 1;"),
    "thermostat_no_sqrt": ("double f = sqrt((T + dT) / T);", "double f = (T + dT) / T;"),
    "thermostat_dof": ("double dof = walled ? 3.0 * (double)n : 3.0 * (double)n - 3.0;", "double dof = 3.0 * (double)n;"),
    "rollout_vjp_full_kick": ("cot[3*i+d] = 0.5 * dt / mass[type[i]] * gv0[3*i+d];", "cot[3*i+d] = dt / mass[type[i]] * gv0[3*i+d];"),
}

RUNNER = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import oracle, oracle_pins as P
    lib = oracle.load({so!r})
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(lib)
        except Exception as e:
            failed.append(pin.__name__)
            break
    print("FAILED_PINS", failed)
    sys.exit(1 if failed else 0)
""")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "ljoracle.c")).read()
    assert src.count(old) >= 1, "mutation site vanished: " + name
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / "mut.c"
    cpath.write_text(mutated)
    so = str(tmp_path / "libmut.so")
    oracle.build(force=True, src=str(cpath), out=so)
    script = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), so=so)
    try:
        r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=60)
    except subprocess.TimeoutExpired:
        return  # a hang is a detected failure
    assert r.returncode != 0, "mutant %s passed every pin:\n%s%s" % (name, r.stdout, r.stderr)
