"""Plant one mistake at a time in a copy of the FP64 oracle and check that the CPU pins catch it.

Each entry below replaces one expression of the oracle (oracle/oracle.c or oracle/oracle.py) by a
plausible slip: a dropped term, a wrong sign, factor or index, a transposed operand, a wrong sampling
density.  For each, the oracle, the tests and the input generators are copied to a scratch folder, the
replacement is made there, and `pytest -m "not gpu"` runs on the copy; the planting counts as caught
when a pin fails (or the pins do not finish, for a slip that sends the march into a loop).  The
repository itself is never modified.

    python tests/plant_mistakes.py [--scratch DIR] [name ...]

Exits 1 if a planting that changes what the oracle computes is not caught.  CPU only; about ten
minutes for the whole list.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
import time

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C = "oracle/oracle.c"
P = "oracle/oracle.py"
MUTATIONS = [
    ("rayleigh_sampler_printed", C, "double q = 4.0 * z - 2.0;", "double q = 4.0 * z - 1.0;"),
    ("hg_sampler_term", C, "(1.0 - g + 2.0 * g * z)", "(1.0 - g + g * z)"),
    ("rayleigh_phase_mu2", C, "return 0.75 * (1.0 + mu * mu); }", "return 0.75 * (1.0 + mu); }"),
    ("hg_phase_sign", C, "double den = 1.0 + g * g - 2.0 * g * mu;", "double den = 1.0 + g * g + 2.0 * g * mu;"),
    ("theta_norm", C, "(1.0 - pgas) * orc_phase_hg(mu, g)) / (4.0 * ORC_PI);",
     "(1.0 - pgas) * orc_phase_hg(mu, g)) / (2.0 * ORC_PI);"),
    ("theta_kind_norm", C, "(1.0 - pgas) * pc) / (4.0 * ORC_PI);", "(1.0 - pgas) * pc) / (2.0 * ORC_PI);"),
    ("tthg_g2_sign", C, "*g2 = -0.5 * g;", "*g2 = 0.5 * g;"),
    ("tthg_weight", C, "*a = 1.0 - (*g2) * (*g2);", "*a = 1.0 - (*g2);"),
    ("limb_quadratic", C, "case 2: I = 1.0 - c[0] * x - c[1] * x * x; break;",
     "case 2: I = 1.0 - c[0] * x - c[1] * x; break;"),
    ("turn_backwards", C, "out[i] = mu * d[i] + s * (cp * e1[i] + sp * e2[i]);",
     "out[i] = -mu * d[i] + s * (cp * e1[i] + sp * e2[i]);"),
    ("march_entry_root", C, "if (fabs(t[0]) <= fabs(t[1])) t[0] = t[1];", "if (fabs(t[0]) > fabs(t[1])) t[0] = t[1];"),
    ("march_entry_face", C, "case F_LATHI: c[1] += 1; entry = F_LATLO; break;",
     "case F_LATHI: c[1] += 1; entry = F_LATHI; break;"),
    ("albedo_pgas", C, "pgas[i] = sca > 0.0 ? ray / sca : 1.0;", "pgas[i] = sca > 0.0 ? ray / ext : 1.0;"),
    ("albedo_omega", C, "double sca = ray + wcld * ac;", "double sca = ray + ac;"),
    ("planck_power", C, "pow(lam, 5.0)", "pow(lam, 4.0)"),
    ("emission_interp_transposed", C,
     "double lk = (1 - wT) * (1 - wp) * l00 + wT * (1 - wp) * l10 + (1 - wT) * wp * l01 + wT * wp * l11;",
     "double lk = (1 - wT) * (1 - wp) * l00 + wT * (1 - wp) * l01 + (1 - wT) * wp * l10 + wT * wp * l11;"),
    ("emission_L_4pi", C, "L[idx] = 4.0 * ORC_PI * V * alpha[idx] * planck_lambda(lam, T[idx]);",
     "L[idx] = V * alpha[idx] * planck_lambda(lam, T[idx]);"),
    ("emission_weight", C, "w = q > 0.0 ? (L[idx] / Ltot) / q : 0.0;", "w = q > 0.0 ? 1.0 : 0.0;"),
    ("emission_tau_vert_cut", C, "incl[idx] = tau_above < tau_vert_max;", "incl[idx] = 1;"),
    ("emission_volume_lat", C, "(sin(G->lat_edges[j + 1]) - sin(G->lat_edges[j]))",
     "(G->lat_edges[j + 1] - G->lat_edges[j])"),
    ("emission_position_r", C, "double r = cbrt(r1 * r1 * r1 + u[1] * (r2 * r2 * r2 - r1 * r1 * r1));",
     "double r = r1 + u[1] * (r2 - r1);"),
    ("emission_peel_4pi", C, "f_obs[o] += W * e / (4.0 * ORC_PI);", "f_obs[o] += W * e;"),
    ("doppler_sign", C, "double le = lam0 * (1.0 - v / ORC_C_LIGHT);", "double le = lam0 * (1.0 + v / ORC_C_LIGHT);"),
    ("vlos_rotation_sign", C, "                omega_rot * rmid * sin(th) * sin(view_theta) * sin(dph);",
     "                -omega_rot * rmid * sin(th) * sin(view_theta) * sin(dph);"),
    ("albedo_launch_disk", C, "double b = (A->mode == 0) ? Rtoa * sqrt(u[0]) : R0 + u[0] * (Rtoa - R0);",
     "double b = (A->mode == 0) ? Rtoa * u[0] : R0 + u[0] * (Rtoa - R0);"),
    ("chord_missing_b", C, "if (st == END_ESCAPE) contrib = (1.0 - exp(-tau)) * b / Rtoa;",
     "if (st == END_ESCAPE) contrib = (1.0 - exp(-tau));"),
    ("peel_half_tau", C, "if (st == END_ESCAPE) return exp(-tau);", "if (st == END_ESCAPE) return exp(-0.5 * tau);"),
    ("survival_no_reduce", C, "            W *= om;\n", "            ;\n"),
    ("scatterer_choice", C, "double mu = (u[1] < pg) ? orc_sample_rayleigh(u[2])",
     "double mu = (u[1] > pg) ? orc_sample_rayleigh(u[2])"),
    ("peel_angle_sign", C, "orc_theta_kind(dot3(d, od), pg, gg, S->cloud_phase)",
     "orc_theta_kind(-dot3(d, od), pg, gg, S->cloud_phase)"),
    ("surface_cosine", C, "orc_turn(nrm, sqrt(u[2]), 2.0 * ORC_PI * u[3], nd);", "orc_turn(nrm, u[2], 2.0 * ORC_PI * u[3], nd);"),
    ("surface_peel_phase", C, "const double fo = W * As * (mo / ORC_PI) * e;", "const double fo = W * As * (1.0 / ORC_PI) * e;"),
    ("forced_weight", C, "                W *= p;\n", "                ;\n"),
    ("forced_truncation", C, "tau_t = -log1p(-u[0] * p);", "tau_t = -log(u[0]);"),
    ("cont_abs_decay", C, "const double Wn = W * exp(-M.tau2);", "const double Wn = W * exp(-0.5 * M.tau2);"),
    ("stretch_pdf", C, "const double q = 0.5 * (exp(-tau_t) + a * exp(-a * tau_t));",
     "const double q = 0.5 * (exp(-tau_t) + exp(-a * tau_t));"),
    ("hybrid_weight", C, "reweight(acc, &W, ft / (0.5 * ft + 0.5 / tau_m));", "reweight(acc, &W, ft / (0.5 * ft + 0.5 * tau_m));"),
    ("gsample_weight", C, "Wg = C->g_w[g];", "Wg = 1.0;"),
    ("philox_multiplier", C, "mulhilo(0xD2511F53u, c0, &hi0);", "mulhilo(0xD2511F54u, c0, &hi0);"),
    ("uniform_offset", C, "return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0); }", "return ((double)(w >> 8) + 0.25) * (1.0 / 16777216.0); }"),
    ("g_table_composite", P, "q = (1.0 - beta) * p + beta / ng", "q = (1.0 - beta) * p + beta"),
    ("postscale_ag_r0", P, '"A_g_R0": math.pi * S * (g.R_toa / g.R0) ** 2', '"A_g_R0": math.pi * S * (g.R0 / g.R_toa) ** 2'),
    ("postscale_ip_pi", P, "Ip = Lp / (math.pi * g.R_toa ** 2)", "Ip = Lp / (g.R_toa ** 2)"),
    ("postscale_area", P, '"area_over_pi": g.R0 ** 2 + 2.0 * Ip}', '"area_over_pi": g.R0 ** 2 + Ip}'),
    ("transit_omega_star", P, "omega_star = 2.0 * math.pi * (1.0 - math.sqrt(1.0 - (Rs / a) ** 2))",
     "omega_star = 4.0 * math.pi * (1.0 - math.sqrt(1.0 - (Rs / a) ** 2))"),
    ("cone_nappe", C, "if ((theta > 0 && z > 0) || (theta < 0 && z < 0)) t[n++] = cand[i];",
     "if ((theta > 0 && z > 0) || (theta < 0 && z > 0)) t[n++] = cand[i];"),
    ("cone_B_term", C, "double B = x[2] * d[2] - s2 * dot3(x, d);", "double B = x[2] * d[2] - s * dot3(x, d);"),
    ("lon_halfplane", C, "if (!(along > 0.0)) return 0;", "if (!(along > -1e300)) return 0;"),
    ("locate_lat", C, "double lat = atan2(x[2], sqrt(x[0] * x[0] + x[1] * x[1]));",
     "double lat = atan2(x[2], fabs(x[0]) + fabs(x[1]));"),
    ("roulette_gain", C, "            if (W < S->w_rr * W0) {\n                double v[4];\n                draw(A->seed, n, ev | 0x80000000u, A->job_key, v);\n                if (v[1] < S->p_surv) {\n                    double Wn = W / S->p_surv;\n                    kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - W);\n                    W = Wn;\n                } else {\n                    kahan(&acc->ledger[5], &acc->ledger_c[5], W);\n                    break;\n                }\n            }\n        } else {\n            double v[4];\n            draw(A->seed, n, ev | 0x80000000u, A->job_key, v);\n            if (!(v[0] < om))",
     "            if (W < S->w_rr * W0) {\n                double v[4];\n                draw(A->seed, n, ev | 0x80000000u, A->job_key, v);\n                if (v[1] < S->p_surv) {\n                    double Wn = W;\n                    kahan(&acc->ledger[4], &acc->ledger_c[4], Wn - W);\n                    W = Wn;\n                } else {\n                    kahan(&acc->ledger[5], &acc->ledger_c[5], W);\n                    break;\n                }\n            }\n        } else {\n            double v[4];\n            draw(A->seed, n, ev | 0x80000000u, A->job_key, v);\n            if (!(v[0] < om))"),
    ("analog_absorb", C, "if (!(v[0] < om)) { kahan(&acc->ledger[2], &acc->ledger_c[2], W); break; }",
     "if (!(v[0] < 0.5 * om)) { kahan(&acc->ledger[2], &acc->ledger_c[2], W); break; }"),
    ("emission_stratified_target", C, "double target = ((double)n + u[0]) * (C->cdf_total / (double)A->n_packets);",
     "double target = u[0] * C->cdf_total;"),
    ("emission_cdf_search", C, "if (cdf[mid] > target) hi = mid; else lo = mid + 1;",
     "if (cdf[mid] >= target) hi = mid + 1; else lo = mid + 1;"),
    ("trans_launch_b", C, ": R0 + u[0] * (Rtoa - R0);", ": R0 + sqrt(u[0]) * (Rtoa - R0);"),
    ("limb_mu", C, "W = W0 = q < 1.0 ? orc_limb(S->ld_law, S->ld_coef, sqrt(1.0 - q)) : 0.0;",
     "W = W0 = q < 1.0 ? orc_limb(S->ld_law, S->ld_coef, 1.0 - q) : 0.0;"),
    ("chord_cutoff_contrib", C, "else if (st == END_CUTOFF || st == END_BOTTOM) contrib = b / Rtoa;",
     "else if (st == END_CUTOFF || st == END_BOTTOM) contrib = 0.0;"),
    ("scattered_peel_scale", C, "peel_scale = b / Rtoa;", "peel_scale = 1.0;"),
    ("surface_survival", C, "                W *= As;\n", "                ;\n"),
    ("cf_kind", C, "if (A->cf) cf_put(acc, idx, 1, o, fo);", "if (A->cf) cf_put(acc, idx, 0, o, fo);"),
    ("tthg_term_choice", C, "return orc_sample_hg(zc < a ? g1 : g2, z, eps);", "return orc_sample_hg(zc < a ? g2 : g1, z, eps);"),
    ("hg_iso_threshold", C, "if (fabs(g) < eps) return 2.0 * z - 1.0;", "if (fabs(g) < 0.7) return 2.0 * z - 1.0;"),
    ("interp_linear_T", C, "*w = (log(v) - log(grid[lo])) / (log(grid[lo + 1]) - log(grid[lo]));",
     "*w = (v - grid[lo]) / (grid[lo + 1] - grid[lo]);"),
    ("xsec_lambda_weight", C, "alpha[idx] = rho[idx] * exp((1.0 - wl) * ls[0] + wl * ls[1]);",
     "alpha[idx] = rho[idx] * exp(wl * ls[0] + (1.0 - wl) * ls[1]);"),
    ("vlos_view_theta", C, "v = u * sin(view_theta) * sin(dph)", "v = u * cos(view_theta) * sin(dph)"),
    ("gsample_target", C, "target = u[0] * C->g_cdftot[g];", "target = u[0];"),
    ("emission_launch_lat", C, "double sl = s1 + u[2] * (s2 - s1);",
     "double sl = sin(G->lat_edges[c[1]] + u[2] * (G->lat_edges[c[1] + 1] - G->lat_edges[c[1]]));"),
    ("forced_remainder", C, "const double rem = W * exp(-tau_m);", "const double rem = W * exp(-0.5 * tau_m);"),
    ("g_table_weight", P, "W = np.where(q > 0, p / np.where(q > 0, q, 1.0), 0.0)", "W = np.where(q > 0, 1.0, 0.0)"),
    ("prep_band_lband", P, "out.update(per_g=per, gtab=gt, L_tot=gt[\"L_band\"],", "out.update(per_g=per, gtab=gt, L_tot=per[0][\"L_tot\"],"),
    ("transit_core_mu", P, "w_core = limb(law, coef, math.sqrt(1.0 - q)) if q < 1.0 else 0.0",
     "w_core = limb(law, coef, 1.0 - q) if q < 1.0 else 0.0"),
    ("transit_area_core", P, "area = w_core * g.R0 ** 2 + 2.0 * I_p", "area = g.R0 ** 2 + 2.0 * I_p"),
    ("transit_scattered_sign", P, "I_p = I_dir - omega_star * I_sca", "I_p = I_dir + omega_star * I_sca"),
    ("emission_capped_booking", C, "} else if (capped || (S->scatter_emission && M.steps >= M.max_steps)) {",
     "} else if (M.steps >= M.max_steps) {"),
]

# plantings that do not change what the oracle computes, with the reason
EQUIVALENT = {
    "gsample_target": "each g-ordinate's cumulative pdf sums to 1 by construction, so scaling the launch "
                      "uniform by its total changes nothing",
}


def fresh_copy(scratch):
    if os.path.isdir(scratch):
        shutil.rmtree(scratch)
    os.makedirs(scratch)
    for d in ("oracle", "tests", "paper_2110_15640_gb300"):
        shutil.copytree(os.path.join(REPO, d), os.path.join(scratch, d),
                        ignore=shutil.ignore_patterns("__pycache__", "*.so", "_build", "*.o"))


def run(scratch, name, path, old, new):
    """(status, message): status is 'caught', 'missed' or 'skipped'."""
    fresh_copy(scratch)
    fn = os.path.join(scratch, path)
    with open(fn) as f:
        src = f.read()
    n = src.count(old)
    if n != 1:
        return "skipped", f"{name}: SKIPPED (pattern found {n} times)"
    with open(fn, "w") as f:
        f.write(src.replace(old, new))
    t0 = time.time()
    cmd = [sys.executable, "-m", "pytest", "tests", "-m", "not gpu", "-x", "-q", "-p", "no:cacheprovider",
           "--ignore=tests/test_abi.py", "--ignore=tests/test_multirank.py", "--ignore=tests/test_host_logic.py",
           "--ignore=tests/test_inputs.py", "--ignore=tests/test_bench_host.py", "--ignore=tests/test_plant_mistakes.py"]
    try:
        r = subprocess.run(cmd, cwd=scratch, capture_output=True, text=True, timeout=180)
    except subprocess.TimeoutExpired:
        return "caught", f"{name}: caught (the pins did not finish in 180 s)"
    out = r.stdout + r.stderr
    dt = time.time() - t0
    if r.returncode == 0:
        return "missed", f"{name}: NOT CAUGHT ({dt:.0f} s)"
    failed = [l for l in out.splitlines() if l.startswith(("FAILED", "ERROR"))]
    last = out.splitlines()[-1] if out.strip() else f"exit {r.returncode}"
    return "caught", f"{name}: caught by {(failed[0] if failed else last).split(' - ')[0]} ({dt:.0f} s)"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scratch", default=None, help="scratch folder (default: a new temporary folder)")
    ap.add_argument("names", nargs="*")
    a = ap.parse_args()
    scratch = a.scratch or tempfile.mkdtemp(prefix="plant_mistakes_")
    missed = []
    try:
        for m in MUTATIONS:
            if a.names and m[0] not in a.names:
                continue
            status, msg = run(scratch, *m)
            if status == "missed" and m[0] in EQUIVALENT:
                msg += f" -- equivalent: {EQUIVALENT[m[0]]}"
            elif status != "caught":
                missed.append(m[0])
            print(msg, flush=True)
    finally:
        shutil.rmtree(scratch, ignore_errors=True)
    if missed:
        print("not caught:", ", ".join(missed))
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
