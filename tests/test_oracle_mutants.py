"""The oracle's pins catch plausible mistakes.

Each mutant is a copy of oracle/arc_oracle.c with one planted mistake (a
dropped term, a wrong sign or index, a transposed operand, a wrong factor),
compiled on the CPU and swapped in for the real oracle; at least one pin of
tests/test_oracle_*.py must then fail.  Mistakes are planted only in the
oracle, never in the CUDA path.
"""
import tempfile

import pytest

import oracle
import test_oracle_chem as CH
import test_oracle_correction as GC
import test_oracle_healpix as HP
import test_oracle_rates as RT
import test_oracle_thin as TH
import test_oracle_trace as TR

# (name, original text, mutated text)
MUTANTS = [
    ("pix2vec swaps cos/sin", "v[0] = st * cos(phi);\n    v[1] = st * sin(phi);",
     "v[0] = st * sin(phi);\n    v[1] = st * cos(phi);"),
    ("pix2vec belt shift parity", "kshift = (int)((jr - ns) & 1);", "kshift = (int)((jr - ns + 1) & 1);"),
    ("pix2vec south cap sign", "z = one_minus_z_or_plus - 1.0;", "z = 1.0 - one_minus_z_or_plus;"),
    ("split radius without sqrt", "return 1.0 / sqrt(p->phi * omega);", "return 1.0 / (p->phi * omega);"),
    ("ray keeps absorbed photons", "                N[b] -= A;\n", "\n"),
    ("linearised absorption", "const double A = N[b] * (-expm1(-dtau));", "const double A = N[b] * dtau;"),
    ("rate without cell length", "const double rate = A * p->sigma[s][b] * c->dx / (kappa_b * c->V);",
     "const double rate = A * p->sigma[s][b] / (kappa_b * c->V);"),
    ("transposed cell index", "idx = ((int64_t)cell[0] * n + cell[1]) * n + cell[2];",
     "idx = ((int64_t)cell[2] * n + cell[1]) * n + cell[0];"),
    ("always steps forward", "cell[ax] += (u[ax] > 0.0) ? 1 : -1;", "cell[ax] += 1;"),
    ("children get half", "Nc[b] = N[b] / 4.0;", "Nc[b] = N[b] / 2.0;"),
    ("residual dropped", "                    c->absorbed += N[b];\n                    if (kap[b] > 0.0) deposit(c, idx, b, N[b], kap[b]);\n",
     "\n"),
    ("threshold not scaled by level", "const double thr = c->thr_base / pow(4.0, level - p->l_base);",
     "const double thr = c->thr_base;"),
    ("heating sign of edge", "rate * (p->E_group_eV[b] - E_S[s]) * EVERG", "rate * (p->E_group_eV[b] + E_S[s]) * EVERG"),
    ("escape not booked",
     "for (int b = 0; b < G; b++) c->escaped += N[b];\n            if (tau0 < THIN_TAU) c->rthin = fmin(c->rthin, r);",
     "if (tau0 < THIN_TAU) c->rthin = fmin(c->rthin, r);"),
    ("recombination on HI", "const double DH = r[0] * ne * nH;", "const double DH = r[0] * ne * nHI;"),
    ("HeI source from HeI", "const double C1 = G1 + r[4] * ne, D1 = r[1] * ne * nHeII;",
     "const double C1 = G1 + r[4] * ne, D1 = r[1] * ne * nHeI;"),
    ("electrons miss HeIII", "const double ne = (nH - nHI) + nHeII + 2.0 * (nHe - nHeI - nHeII);",
     "const double ne = (nH - nHI) + nHeII + (nHe - nHeI - nHeII);"),
    ("energy factor", "E = 1.5 * KB * T * (nH + nHe + ne);", "E = 2.5 * KB * T * (nH + nHe + ne);"),
    ("Compton sign", "Tg * Tg * Tg * Tg * (T - Tg) * ne", "Tg * Tg * Tg * Tg * (Tg - T) * ne"),
    ("collisional sink dropped", "const double CH = G0 + (r[3] + r[0]) * ne;", "const double CH = G0 + r[0] * ne;"),
    ("case-B exponent", "return 2.753e-14 * pow(lam, 1.5)", "return 2.753e-14 * pow(lam, 1.4)"),
    ("limiter ignores n_HII", "const double lim = eps * fmax(fmin(nHI, nH - nHI), p->x_fp64 * nH);",
     "const double lim = eps * fmax(nHI, p->x_fp64 * nH);"),
    ("negative-direction plane one cell off", "else if (u[a] < 0.0) tn[a] = ((double)cell[a] - o[a]) / u[a];",
     "else if (u[a] < 0.0) tn[a] = ((double)cell[a] - 1.0 - o[a]) / u[a];"),
    ("nearest plane picks the largest", "if (tn[2] < tn[ax]) ax = 2;", "if (tn[2] > tn[ax]) ax = 2;"),
    ("segment from the cell start", "double ds = r1 - r;", "double ds = r1 - r0;"),
    # optically thin approximation (Sec. 2.6) and emission masks (Sec. 2.2)
    ("thin depth 0.2", "#define THIN_TAU 0.1 ", "#define THIN_TAU 0.2 "),
    ("crossing without cell length", "r + (THIN_TAU - tau0) / (ks * c->dx)", "r + (THIN_TAU - tau0) / ks"),
    ("softest group is the hardest", "if (p->E_group_eV[b] < p->E_group_eV[c.soft]) c.soft = b;",
     "if (p->E_group_eV[b] > p->E_group_eV[c.soft]) c.soft = b;"),
    ("children restart the depth", "trace_ray(c, level + 1, 4 * pix + (uint64_t)k, r, Nc, tau0);",
     "trace_ray(c, level + 1, 4 * pix + (uint64_t)k, r, Nc, 0.0);"),
    ("fill without 4 pi", "const double A = S[b] * kap / (4.0 * PI * rr);", "const double A = S[b] * kap / rr;"),
    ("fill falls as 1/r", "const double rr = r2 > 0.25 ? r2 : 0.25;", "const double rr = sqrt(r2 > 0.25 ? r2 : 0.25);"),
    ("rays start at the source", "trace_ray(&c, p->l_base, q, R, N0, 0.0);", "trace_ray(&c, p->l_base, q, 0.0, N0, 0.0);"),
    ("no split at the start", "if (r0 >= r_stop) {", "if (r0 > 1e30) {"),
    ("mask ignores the source", "opt->open[(int64_t)s * (int64_t)nrays + (int64_t)q]", "opt->open[(int64_t)q]"),
    ("blocked rays still emit", "c.nrec++;\n                continue;", "c.nrec++;"),
    ("fill photons not booked", "                        tot += A;\n", "\n"),
    # rate coefficients and cooling (Sec. 2.8): one planted typo per coefficient family
    ("HeII radiative coefficient", "out[1] = 1.26e-14 * pow(lHeI, 0.750) +", "out[1] = 1.62e-14 * pow(lHeI, 0.750) +"),
    ("dielectronic threshold", "1.90e-3 * pow(T, -1.5) * exp(-4.7e5 / T)", "1.90e-3 * pow(T, -1.5) * exp(-7.4e5 / T)"),
    ("dielectronic prefactor", "1.90e-3 * pow(T, -1.5)", "1.09e-3 * pow(T, -1.5)"),
    ("HeIII alpha not doubled", "out[2] = 2.0 * hg_alpha_b(lHeII);", "out[2] = hg_alpha_b(lHeII);"),
    ("HI collisional exponent", "pow(1.0 + pow(lHI / 0.354, 0.874), 1.101)", "pow(1.0 + pow(lHI / 0.354, 0.874), 1.01)"),
    ("HeI collisional coefficient", "32.38 * t32", "23.38 * t32"),
    ("HeII collisional scale", "lHeII / 0.553", "lHeII / 5.53"),
    ("HII recombination cooling exponent", "3.435e-30 * T * pow(lam, 1.970)", "3.435e-30 * T * pow(lam, 1.907)"),
    ("HeII recombination cooling without kT", "L[4] = ne * 1.26e-14 * pow(lHeI, 0.750) * KB * T * nHeII;",
     "L[4] = ne * 1.26e-14 * pow(lHeI, 0.750) * KB * 1e4 * nHeII;"),
    ("HeIII recombination cooling unscaled", "hg_recool_b(T * (T_HI / T_HEII), lHeII)", "hg_recool_b(T, lHeII)"),
    ("dielectronic cooling coefficient", "L[6] = ne * 1.24e-13", "L[6] = ne * 1.42e-13"),
    ("HI excitation ten times", "L[7] = ne * 7.5e-19", "L[7] = ne * 7.5e-18"),
    ("HI excitation energy", "exp(-118348.0 / T)", "exp(-183480.0 / T)"),
    ("HeII excitation power sign", "5.54e-17 * pow(T, -0.397)", "5.54e-17 * pow(T, 0.397)"),
    ("free-free HeIII charge", "(nHII + nHeII + 4.0 * nHeIII)", "(nHII + nHeII + 2.0 * nHeIII)"),
    ("free-free coefficient", "L[9] = 1.42e-27", "L[9] = 1.42e-26"),
    ("HeI ionisation energy in cooling", "L[1] = ne * r[4] * nHeI * KB * T_HEI;", "L[1] = ne * r[4] * nHeI * KB * T_HI;"),
    ("helium sub-step limit dropped", "            if (nHe > 0.0) {\n                const double nHeIII = nHe - nHeI - nHeII;",
     "            if (0) {\n                const double nHeIII = nHe - nHeI - nHeII;"),
    # Sec. 3.6 correction variants
    ("squared variant not squared", "if (p->geo_corr == 3) fc = fc * fc;", "if (p->geo_corr == 3) fc = fc;"),
]

# fast pins first; a mutant is killed at the first failure
PINS = [
    RT.test_case_b_hii_against_table,
    RT.test_radiative_heii_recombination_against_table,
    RT.test_heiii_recombination_is_hydrogenic,
    RT.test_collisional_ionisation_against_independent_fit,
    RT.test_collisional_ionisation_cooling_is_the_ionisation_energy,
    RT.test_recombination_cooling_energy_per_recombination,
    RT.test_dielectronic_recombination_energy_and_threshold,
    RT.test_collisional_excitation_threshold_and_strength,
    RT.test_free_free_coefficient_gaunt_and_charge,
    lambda: HP.test_roundtrip(2),
    lambda: HP.test_ring_latitudes_and_sizes(2),
    lambda: HP.test_children_nest_inside_parent(1),
    lambda: TR.test_uniform_medium_escape_closed_form((3.25, 10.5, 7.75)),
    TR.test_budget_and_cell_sum_identity,
    TR.test_clump_casts_sharp_shadow,
    TR.test_energy_budget_of_heating,
    lambda: TR.test_visit_counts_closed_form(0),
    lambda: TR.test_cells_and_segments_against_plane_crossing_bruteforce((1.37, 2.11, 1.73)),
    CH.test_case_b_alpha_matches_paper_test1,
    lambda: CH.test_pure_h_equilibrium_quadratic(1e-3),
    lambda: CH.test_pure_h_equilibrium_quadratic(0.3),
    CH.test_h_he_photoionisation_equilibrium,
    CH.test_recombination_decay,
    CH.test_photoheating_of_neutral_gas_is_linear,
    CH.test_compton_coefficient,
    CH.test_collisional_ionisation_equilibrium,
    lambda: CH.test_helium_photoionisation_follows_the_exponential(1.0),
    TR.test_termination_distance_in_uniform_medium,
    TR.test_rays_per_face_at_split_equals_phi,
    TR.test_optically_thin_shells,
    lambda: TH.test_thin_radius_uniform_closed_form((10.25, 19.5, 14.75), 0.02),
    TH.test_thin_radius_uses_softest_group,
    lambda: TH.test_thin_start_tree_and_escape_radius((9.25, 20.5, 13.75), 3.1),
    lambda: TH.test_thin_trace_beyond_radius_is_the_plain_one_unattenuated(7.5),
    TH.test_thin_fill_matches_traced_small_tau_limit,
    TH.test_complementary_masks_add_up,
    lambda: TH.test_single_open_pixel_lights_its_cone(22),
    TH.test_thin_ledger_matches_the_cell_rates_with_helium,
    GC.test_only_the_secondary_variant_conserves_photons,
]


def killed(path):
    with oracle.use_library(path):
        for pin in PINS:
            try:
                pin()
            except Exception:
                return True
    return False


def test_every_mutant_is_killed():
    src = oracle.source_text()
    survivors = []
    with tempfile.TemporaryDirectory() as d:
        for name, old, new in MUTANTS:
            assert src.count(old) == 1, f"mutation site not unique or missing: {name}"
            sub = tempfile.mkdtemp(dir=d)
            path = oracle.build_variant(src.replace(old, new), sub)
            if not killed(path):
                survivors.append(name)
    assert not survivors, survivors


def test_unmutated_oracle_passes_the_battery():
    with tempfile.TemporaryDirectory() as d:
        path = oracle.build_variant(oracle.source_text(), d)
        assert not killed(path)
