"""Mutation testing of the oracle: evidence that its pins are specific.

Each entry below is a single-site change to `oracle/ldpm_oracle.cpp`: a plausible slip against the
passage named in its group (a dropped term, a wrong sign, an index or operand swapped, a clamp or
a guard removed).  The runner compiles every mutant with the oracle's own build (`oracle.build`,
pointed at the mutated source) and runs the oracle's CPU pins (`tests/test_oracle_*.py`) against
it in a child process.  A mutant is caught when some pin fails; a survivor means the oracle has
behaviour no pin fixes, and the run exits non-zero.

    python tests/oracle_mutants.py            # all mutants, in parallel, after a control run
    python tests/oracle_mutants.py NAME ...   # selected mutants
    python tests/oracle_mutants.py --list

The control run executes the same child on the unmodified source, which must pass.
`tests/test_oracle_mutants.py` keeps the table in step with the source (every site occurs exactly
once) and runs one mutant end to end.  The oracle is test infrastructure; nothing here is part of
the library.
"""
import concurrent.futures
import glob
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE = os.path.join(ROOT, "oracle", "ldpm_oracle.cpp")
ORDER = ["invariants", "law", "hysteresis", "adjoint", "dynamics", "kinematics"]

# (name, original text, replacement); each original occurs exactly once in the source.
MUTANTS = [
    # App. A.1, fracture
    ('emax_not_max',
     'S emax = emax_old > eeff ? emax_old : eeff;',
     'S emax = eeff;'),
    ('reload_rule_inverted',
     'if (e_tr > e_old) de_eff',
     'if (e_tr < e_old) de_eff'),
    ('effective_traction_alpha',
     'S t_eff_old = sqrt(t_old[0] * t_old[0] + (t_old[1] * t_old[1] + t_old[2] * t_old[2]) / alpha);',
     'S t_eff_old = sqrt(t_old[0] * t_old[0] + (t_old[1] * t_old[1] + t_old[2] * t_old[2]) * alpha);'),
    ('sigma0_r',
     'S sigma0 = 2.0 * sigma_t / (s + sqrt(s * s + 4.0 * alpha * c * c / r2));',
     'S sigma0 = 2.0 * sigma_t / (s + sqrt(s * s + 4.0 * alpha * c * c / p->r_st));'),
    ('Ht_form',
     'S Ht = 2.0 * E0 / (p->l_t / l - 1.0);',
     'S Ht = 2.0 * E0 / (p->l_t / l);'),
    ('over_e0',
     'S over = emax - e0 > 0.0 ? emax - e0 : 0.0;',
     'S over = emax > 0.0 ? emax : 0.0;'),
    ('nt_exponent',
     'pow(2.0 * omega / ORC_PI, p->n_t)',
     'pow(2.0 * omega / ORC_PI, 1.0)'),
    ('traction_map_alpha',
     't_new[1] = alpha * t / eeff * e[1];',
     't_new[1] = t / eeff * e[1];'),
    ('Hs_over_alpha',
     'S H0 = Hs / alpha + (Ht - Hs / alpha) * pow',
     'S H0 = Hs + (Ht - Hs) * pow'),
    ('etr_no_sigma_bt',
     'S e_tr = p->k_t * (emax - sigma_bt / E0);',
     'S e_tr = p->k_t * emax;'),
    ('etr_no_guard',
     'if (e_tr > e_old) de_eff = eeff > e_tr ? eeff - e_tr : S(0.0);',
     'de_eff = eeff > e_tr ? eeff - e_tr : S(0.0);'),
    ('eeff_no_alpha',
     'S eeff = sqrt(e[0] * e[0] + alpha * eT2);',
     'S eeff = sqrt(e[0] * e[0] + eT2);'),
    ('omega_no_alpha',
     'S omega = atan2(e[0], sqrt(alpha * eT2));',
     'S omega = atan2(e[0], sqrt(eT2));'),
    ('eold_no_alpha',
     'S e_old = sqrt(e_prev[0] * e_prev[0] + alpha * (e_prev[1] * e_prev[1] + e_prev[2] * e_prev[2]));',
     'S e_old = sqrt(e_prev[0] * e_prev[0] + (e_prev[1] * e_prev[1] + e_prev[2] * e_prev[2]));'),
    ('tiny_emax',
     '*emax_new = emax_old > eeff ? emax_old : eeff;\n            return;',
     '*emax_new = emax_old;\n            return;'),
    # App. A.2, compression
    ('stiffness_regimes_swapped',
     'S ENc = (-t_old[0] <= p->sigma_c0) ? E0 : Ed;',
     'S ENc = (-t_old[0] <= p->sigma_c0) ? Ed : E0;'),
    ('compression_clamp_sign',
     'if (tN < -sigma_bc) tN = -sigma_bc;',
     'if (tN < -sigma_bc) tN = sigma_bc;'),
    ('eDV_beta',
     'S eDV = eV + p->beta * eD;',
     'S eDV = eV + eD;'),
    ('Hc_kc2',
     'S Hc = (Hc0 - Hc1) / (1.0 + p->kc2 * mac) + Hc1;',
     'S Hc = (Hc0 - Hc1) / (1.0 + mac) + Hc1;'),
    ('rDV_sign',
     'S rDV = (eV <= 0.0) ? -fabs(eD) / (eV - eV0) : fabs(eD) / eV0;',
     'S rDV = (eV <= 0.0) ? fabs(eD) / (eV - eV0) : fabs(eD) / eV0;'),
    ('eV0_no_E0',
     'S eV0 = p->kc3 * p->sigma_c0 / E0;',
     'S eV0 = p->kc3 * p->sigma_c0;'),
    ('sigma_c1_no_ec0',
     'S sigma_c1 = p->sigma_c0 + (ec1 - ec0) * Hc;',
     'S sigma_c1 = p->sigma_c0 + ec1 * Hc;'),
    ('exp_no_sigma_c1',
     'sigma_bc = sigma_c1 * exp((-eDV - ec1) * Hc / sigma_c1);',
     'sigma_bc = sigma_c1 * exp((-eDV - ec1) * Hc);'),
    ('mac_no_kc1',
     'S mac = rDV - p->kc1 > 0.0 ? rDV - p->kc1 : 0.0;',
     'S mac = rDV > 0.0 ? rDV : 0.0;'),
    ('Hc_no_Hc1',
     'S Hc = (Hc0 - Hc1) / (1.0 + p->kc2 * mac) + Hc1;',
     'S Hc = Hc0 / (1.0 + p->kc2 * mac);'),
    ('tN_no_upper_clamp',
     'if (tN > 0.0) tN = 0.0;',
     ';'),
    ('eDV_minus',
     'S eDV = eV + p->beta * eD;',
     'S eDV = eV - p->beta * eD;'),
    ('sigma_bc_case1',
     '        sigma_bc = p->sigma_c0;\n    } else if',
     '        sigma_bc = 0.5 * p->sigma_c0;\n    } else if'),
    # App. A.3, friction
    ('friction_return_one_component',
     '        tL *= sigma_bs / tau;\n',
     ''),
    ('shear_total_not_incremental',
     'S tM = t_old[1] + alpha * E0 * de[1];',
     'S tM = alpha * E0 * e[1];'),
    ('mu_inf_sign',
     'S sigma_bs = sigma_s + dmu * p->sigma_N0 - p->mu_inf * tN - dmu * p->sigma_N0 * exp(tN / p->sigma_N0);',
     'S sigma_bs = sigma_s + dmu * p->sigma_N0 + p->mu_inf * tN - dmu * p->sigma_N0 * exp(tN / p->sigma_N0);'),
    ('sigma_s_no_rst',
     'S sigma_s = p->r_st * sigma_t;',
     'S sigma_s = sigma_t;'),
    # Sec. 2, kinematics and facet geometry
    ('rotation_sign_I',
     'jump[a] = uJ[a] + rJ - uI[a] - rI;',
     'jump[a] = uJ[a] + rJ - uI[a] + rI;'),
    ('cross_order_J',
     'const S rJ = uJ[3 + b] * cJ[c] - uJ[3 + c] * cJ[b];',
     'const S rJ = uJ[3 + c] * cJ[b] - uJ[3 + b] * cJ[c];'),
    ('strain_no_l',
     'e[0] = (n[0] * jump[0] + n[1] * jump[1] + n[2] * jump[2]) / l;',
     'e[0] = (n[0] * jump[0] + n[1] * jump[1] + n[2] * jump[2]);'),
    ('eV_factor',
     '    return dv / 3.0;\n}',
     '    return dv / 2.0;\n}'),
    ('gradN0_sign',
     'g[a] = -(g[3 + a] + g[6 + a] + g[9 + a]);',
     'g[a] = (g[3 + a] + g[6 + a] + g[9 + a]);'),
    ('centroid',
     'xc[a] = (p0[a] + p1[a] + p2[a]) / 3.0;',
     'xc[a] = (p0[a] + p1[a]) / 2.0;'),
    ('area_unprojected',
     'double A = 0.5 * twoA0 * fabs(dot3(nn, nc) / twoA0);',
     'double A = 0.5 * twoA0;'),
    # Eq. (2), assembly
    ('moment_J_sign',
     'fJ[3 + a] -= mJ;',
     'fJ[3 + a] += mJ;'),
    ('moment_arm_I_for_J',
     'const S mJ = cJ[b] * Fk[c] - cJ[c] * Fk[b];',
     'const S mJ = cI[b] * Fk[c] - cI[c] * Fk[b];'),
    ('assemble_FJ_sign',
     '            fJ[a] -= Fk[a];',
     '            fJ[a] += Fk[a];'),
    ('elastic_force_alpha',
     't[1] = M->mat.alpha * M->mat.E0 * e[1];\n        t[2] = M->mat.alpha * M->mat.E0 * e[2];\n        facet_force',
     't[1] = M->mat.E0 * e[1];\n        t[2] = M->mat.alpha * M->mat.E0 * e[2];\n        facet_force'),
    # Sec. 3.2.5, lumped mass
    ('mass_split_3',
     'node_mass[v[i]] += mat->rho * vol / 4.0;',
     'node_mass[v[i]] += mat->rho * vol / 3.0;'),
    ('inertia_5',
     'mi * d * d / 10.0;',
     'mi * d * d / 5.0;'),
    ('dpos_min',
     'double d = (diameter && diameter[i] > 0.0) ? diameter[i] : dpos_min;',
     'double d = (diameter && diameter[i] > 0.0) ? diameter[i] : 1.0;'),
    # Sec. 3 and 4, time integration, constraints, reactions, energies
    ('full_kick',
     'vh[i] = T.v[i] + 0.5 * dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i];',
     'vh[i] = T.v[i] + dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i];'),
    ('bc_ramp_time',
     'vh[i] = M->bc_vel[i] * ramp(M, t + 0.5 * dt);',
     'vh[i] = M->bc_vel[i] * ramp(M, t);'),
    ('Wint_sign',
     'W[0] += 0.5 * (fint_old[i] - T.f_asm[i]) * dq[i];',
     'W[0] += 0.5 * (fint_old[i] + T.f_asm[i]) * dq[i];'),
    ('reaction_accel',
     'a = M->bc_vel[i] * (ramp(M, t + 0.5 * M->dt) - ramp(M, t - 0.5 * M->dt)) / M->dt;',
     'a = 0.0;'),
    ('ramp_no_upper',
     '    if (r > 1.0) r = 1.0;',
     ';'),
    ('fext_ignored_kick',
     'vh[i] = T.v[i] + 0.5 * dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i];',
     'vh[i] = T.v[i] + 0.5 * dt * (T.f_asm[i]) / M->mass[i];'),
    ('fext_in_W',
     'if (M->bc_mask[i] == 0) return S(M->f_ext[i]);',
     'if (M->bc_mask[i] == 0) return S(0.0);'),
    ('reaction_split',
     'reaction[(mk == 1 ? 0 : 6) + (int)(i % 6)] += ext_force_on_dof(M, i, t, M->f_asm);',
     'reaction[(mk == 2 ? 0 : 6) + (int)(i % 6)] += ext_force_on_dof(M, i, t, M->f_asm);'),
    ('Wk_half',
     'for (size_t i = 0; i < n6; ++i) Wk += 0.5 * M->mass[i] * M->v[i] * M->v[i];',
     'for (size_t i = 0; i < n6; ++i) Wk += 0.5 * M->mass[i] * M->v[i] * M->v[i] * (i % 6 < 3);'),
    ('Wkin0_dropped',
     'out[3] = den > 0.0 ? 100.0 * fabs(M->W_ext + M->W_kin0 - M->W_int - Wk) / den : 0.0;',
     'out[3] = den > 0.0 ? 100.0 * fabs(M->W_ext - M->W_int - Wk) / den : 0.0;'),
    ('setbc_no_vel',
     '        if (M->bc_mask[i] == 2) M->v[i] = M->bc_vel[i] * ramp(M, t);\n    }\n}',
     '    }\n}'),
    ('lambda_sign',
     '        for (size_t i = 0; i < n6; ++i) xKx -= x[i] * f[i];',
     '        for (size_t i = 0; i < n6; ++i) xKx += x[i] * f[i];'),
    # state exchange
    ('set_state_m_lv_swap',
     'M->t_loc[3 * k + 1] = dot3(h + 1, M->m + 3 * (size_t)k);\n        M->t_loc[3 * k + 2] = dot3(h + 1, M->lv + 3 * (size_t)k);',
     'M->t_loc[3 * k + 1] = dot3(h + 1, M->lv + 3 * (size_t)k);\n        M->t_loc[3 * k + 2] = dot3(h + 1, M->m + 3 * (size_t)k);'),
    ('set_state_Wkin0',
     '    M->W_int = M->W_ext = 0.0;\n    M->W_kin0 = 0.0;\n    for (size_t i = 0; i < n6; ++i) M->W_kin0 += 0.5 * M->mass[i] * M->v[i] * M->v[i];\n}',
     '    M->W_int = M->W_ext = 0.0;\n}'),
    ('set_state_no_forces',
     '    M->step = step;\n    forces_from_history(M);',
     '    M->step = step;'),
    ('get_state_lv_sign',
     'hist5[5 * k + 1 + a] = t[1] * M->m[3 * k + a] + t[2] * M->lv[3 * k + a];',
     'hist5[5 * k + 1 + a] = t[1] * M->m[3 * k + a] - t[2] * M->lv[3 * k + a];'),
    # Sec. 4 crack opening; Sec. 5 perturbations
    ('metrics_wn_clamp',
     '            if (wn < 0.0) wn = 0.0;',
     ';'),
    ('metrics_aE',
     'double wm = e[1] - t[1] / aE, wl = e[2] - t[2] / aE;',
     'double wm = e[1] - t[1] / E0, wl = e[2] - t[2] / E0;'),
    ('perturb_constrained',
     '        if (M->bc_mask[i] == 0) M->q[i] += dq[i];',
     '        M->q[i] += dq[i];'),
    ('perturb_no_eprev',
     '    for (int32_t k = 0; k < M->F; ++k) facet_strain(M, M->q, k, M->e_prev + 3 * (size_t)k);\n}',
     '}'),
    ('perturb_fixed_only',
     '        if (M->bc_mask[i] == 0) M->q[i] += dq[i];',
     '        if (M->bc_mask[i] != 1) M->q[i] += dq[i];'),
    # derivatives (forward-mode dual numbers, objective)
    ('dual_div',
     'r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;',
     'r.d[i] = (a.d[i] + r.v * b.d[i]) / b.v;'),
    ('dual_atan2',
     '(x.v * y.d[i] - y.v * x.d[i]) / den',
     '(x.v * y.d[i] + y.v * x.d[i]) / den'),
    ('dual_pow',
     'const double g = n * pow(a.v, n - 1.0);',
     'const double g = pow(a.v, n - 1.0);'),
    ('dual_cos',
     'for (int i = 0; i < D; ++i) r.d[i] = -s * a.d[i];',
     'for (int i = 0; i < D; ++i) r.d[i] = s * a.d[i];'),
    ('dual_sqrt',
     'r.d[i] = r.v > 0.0 ? a.d[i] / (2.0 * r.v) : 0.0;',
     'r.d[i] = r.v > 0.0 ? a.d[i] / r.v : 0.0;'),
    ('dJ_no_mean',
     'if (dJ) dJ[d0 + w] = Js.d[w] * inv;',
     'if (dJ) dJ[d0 + w] = Js.d[w];'),
    ('dalpha_sign',
     'if (dalpha) al[k].d[w] = dalpha[row];',
     'if (dalpha) al[k].d[w] = -dalpha[row];'),
    ('seed_prescribed_only',
     'if (seed && M->bc_mask[i] != 0) *J += seed[i] * g_new;',
     'if (seed && M->bc_mask[i] == 2) *J += seed[i] * g_new;'),
    ('dir_block_offset',
     'const size_t row = (size_t)(d0 + w) * F + k;',
     'const size_t row = (size_t)w * F + k;'),
    # the derivative rules, the ramp's start, the elastic responses, create and error reporting
    ('dual_exp_rule',
     'for (int i = 0; i < D; ++i) r.d[i] = r.v * a.d[i];',
     'for (int i = 0; i < D; ++i) r.d[i] = a.d[i];'),
    ('dual_sin_rule',
     'for (int i = 0; i < D; ++i) r.d[i] = c * a.d[i];',
     'for (int i = 0; i < D; ++i) r.d[i] = -c * a.d[i];'),
    ('dual_product_rule',
     'r.d[i] = a.d[i] * b.v + a.v * b.d[i];',
     'r.d[i] = a.d[i] * b.v;'),
    ('dual_fabs_no_flip',
     'template <int D> Dual<D> fabs(const Dual<D> &a) { return a.v < 0.0 ? -a : a; }',
     'template <int D> Dual<D> fabs(const Dual<D> &a) { return a; }'),
    ('ramp_no_lower_clamp',
     '    if (r < 0.0) r = 0.0;',
     ';'),
    ('ramp_zero_time_is_zero',
     'if (M->ramp_time <= 0.0) return 1.0;',
     'if (M->ramp_time <= 0.0) return 0.0;'),
    ('elastic_flag_shear_no_alpha',
     '        /* Sec. 2: t = E e with E = E0 diag(1, alpha, alpha). */\n        t_new[0] = E0 * e[0];\n        t_new[1] = alpha * E0 * e[1];',
     '        /* Sec. 2: t = E e with E = E0 diag(1, alpha, alpha). */\n        t_new[0] = E0 * e[0];\n        t_new[1] = E0 * e[1];'),
    ('tiny_strain_shear_no_alpha',
     '             * path is E0, so a vanishing effective strain responds elastically, t = E e. */\n            t_new[0] = E0 * e[0];\n            t_new[1] = alpha * E0 * e[1];',
     '             * path is E0, so a vanishing effective strain responds elastically, t = E e. */\n            t_new[0] = E0 * e[0];\n            t_new[1] = E0 * e[1];'),
    ('tet_volume_signed',
     'double vol = fabs(det) / 6.0;',
     'double vol = det / 6.0;'),
    ('create_Wkin0_dropped',
     '    M->W_kin0 = 0.0;\n    for (size_t i = 0; i < n6; ++i) M->W_kin0 += 0.5 * M->mass[i] * M->v[i] * M->v[i];\n    return M;',
     '    M->W_kin0 = 0.0;\n    return M;'),
    ('facet_pass_no_e_prev_update',
     '            T.e_prev[3 * k + a] = e[a];',
     '            ;'),
    ('march_total_not_increment',
     'double de[3] = {e[0] - e_prev[0], e[1] - e_prev[1], e[2] - e_prev[2]};',
     'double de[3] = {e[0], e[1], e[2]};'),
    ('step_nonfinite_not_reported',
     '        if (!isfinite(M->q[i]) || !isfinite(M->v[i])) return -5;',
     '        ;'),
    ('tangent_nonfinite_not_reported',
     'if (!isfinite(value_of(q[i])) || !isfinite(value_of(v[i]))) rc = -5;',
     ';'),
    ('v0_fixed_not_zeroed',
     '        M->v[i] = v0 ? v0[i] : 0.0;\n        if (M->bc_mask[i] == 1) M->v[i] = 0.0;',
     '        M->v[i] = v0 ? v0[i] : 0.0;'),
    ('kick_uses_mass_of_next_dof',
     'T.v[i] = vh[i] + 0.5 * dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i];',
     'T.v[i] = vh[i] + 0.5 * dt * (M->f_ext[i] + T.f_asm[i]) / M->mass[i - i % 6];'),
    # facet force mapping, frame, power iteration, energy error, set_bc, the march driver, metrics
    ('facet_force_tangents_swapped',
     'F[a] = M->area[k] * (M->n[3 * k + a] * t[0] + M->m[3 * k + a] * t[1] + M->lv[3 * k + a] * t[2]);',
     'F[a] = M->area[k] * (M->n[3 * k + a] * t[0] + M->lv[3 * k + a] * t[1] + M->m[3 * k + a] * t[2]);'),
    ('frame_not_orthogonalised',
     'for (int a = 0; a < 3; ++a) mm[a] -= pr * nn[a];',
     ';'),
    ('power_iteration_unnormalised',
     'for (size_t i = 0; i < n6; ++i) x[i] /= nrm;',
     ';'),
    ('energy_error_denominator',
     'double den = fabs(M->W_ext) + M->W_kin0;',
     'double den = fabs(M->W_ext);'),
    ('set_bc_fixed_keeps_velocity',
     '    for (size_t i = 0; i < n6; ++i) {\n        if (M->bc_mask[i] == 1) M->v[i] = 0.0;\n        if (M->bc_mask[i] == 2) M->v[i] = M->bc_vel[i] * ramp(M, t);',
     '    for (size_t i = 0; i < n6; ++i) {\n        if (M->bc_mask[i] == 2) M->v[i] = M->bc_vel[i] * ramp(M, t);'),
    ('march_emax_not_carried',
     '        em = emn;',
     '        ;'),
    ('march_traction_not_carried',
     '            t[a] = tn[a];',
     '            ;'),
    ('metrics_eV_of_first_tet',
     '        for (int32_t t = 0; t < M->T; ++t) eV[t] = tet_volumetric_strain(M, M->q, t);\n}',
     '        for (int32_t t = 0; t < M->T; ++t) eV[t] = tet_volumetric_strain(M, M->q, 0);\n}'),
    ('sigma_bs_exp_sign',
     'S sigma_bs = sigma_s + dmu * p->sigma_N0 - p->mu_inf * tN - dmu * p->sigma_N0 * exp(tN / p->sigma_N0);',
     'S sigma_bs = sigma_s + dmu * p->sigma_N0 - p->mu_inf * tN - dmu * p->sigma_N0 * exp(-tN / p->sigma_N0);'),
    ('fracture_clamp_below_zero_removed',
     '        if (t < 0.0) t = 0.0;\n        if (t > sigma_bt) t = sigma_bt;',
     '        if (t > sigma_bt) t = sigma_bt;'),
    ('tN_trial_total',
     'S tN = t_old[0] + ENc * de[0];',
     'S tN = ENc * e[0];'),
    # branch selection, the L components, strain projection, per-facet parameter slots, outputs
    ('branch_on_e_N_nonnegative',
     '    if (e[0] > 0.0) {\n        /* App. A.1, fracture.',
     '    if (e[0] >= 0.0) {\n        /* App. A.1, fracture.'),
    ('friction_trial_L_no_alpha',
     'S tL = t_old[2] + alpha * E0 * de[2];',
     'S tL = t_old[2] + E0 * de[2];'),
    ('strain_M_projects_on_n',
     'e[1] = (m[0] * jump[0] + m[1] * jump[1] + m[2] * jump[2]) / l;',
     'e[1] = (n[0] * jump[0] + n[1] * jump[1] + n[2] * jump[2]) / l;'),
    ('strains_output_of_facet_0',
     'for (int32_t k = 0; k < M->F; ++k) facet_strain(M, q, k, e3 + 3 * (size_t)k);',
     'for (int32_t k = 0; k < M->F; ++k) facet_strain(M, q, 0, e3 + 3 * (size_t)k);'),
    ('elastic_operator_L_no_alpha',
     't[2] = M->mat.alpha * M->mat.E0 * e[2];',
     't[2] = M->mat.E0 * e[2];'),
    ('facet_params_alpha_sigma_swapped',
     'double **dst[3] = {&M->pE0, &M->palpha, &M->psig};',
     'double **dst[3] = {&M->pE0, &M->psig, &M->palpha};'),
    ('jacobian_E0_alpha_slots_swapped',
     'facet_law<S>(p, x[11], x[12], x[13], l, x, x + 3, x[6], x + 7, x[10], tn, &em);',
     'facet_law<S>(p, x[12], x[11], x[13], l, x, x + 3, x[6], x + 7, x[10], tn, &em);'),
    ('geometry_area_unreported',
     'if (area) memcpy(area, M->area, sizeof(double) * M->F);',
     ';'),
]


def pin_files():
    """The oracle's CPU pins, cheapest first (the child stops at the first failure)."""
    files = [f for f in glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py"))
             if os.path.basename(f) != "test_oracle_mutants.py"]  # the runner's own test is not a pin
    rank = {n: i for i, n in enumerate(ORDER)}
    return sorted(files, key=lambda f: (rank.get(os.path.basename(f)[12:-3], len(ORDER)), f))


CHILD = """
import sys
sys.path.insert(0, sys.argv[1])
import oracle
oracle._SRC, oracle._LIB = sys.argv[2], sys.argv[3]
import pytest
sys.exit(pytest.main(['-q', '-x', '-m', 'not gpu', '-p', 'no:cacheprovider'] + sys.argv[4:]))
"""


def mutated_source(name):
    src = open(SOURCE).read()
    for n, a, b in MUTANTS:
        if n == name:
            assert src.count(a) == 1, "site of %s occurs %d times" % (name, src.count(a))
            return src.replace(a, b)
    raise KeyError(name)


def run_one(name, timeout=900):
    """Compile the mutant (or the unmodified source for name None) and run the pins against it.
    Returns (caught, first failing test or summary line)."""
    with tempfile.TemporaryDirectory(prefix="oracle_mutant_") as d:
        src = os.path.join(d, "ldpm_oracle.cpp")
        open(src, "w").write(open(SOURCE).read() if name is None else mutated_source(name))
        r = subprocess.run([sys.executable, "-c", CHILD, ROOT, src, os.path.join(d, "liboracle.so")] + pin_files(),
                           cwd=ROOT, capture_output=True, text=True, timeout=timeout)
    lines = r.stdout.splitlines()
    first = next((l for l in lines if l.startswith("FAILED")), None) or next(
        (l for l in reversed(lines) if "passed" in l or "failed" in l or "error" in l), r.stderr[-300:])
    return r.returncode != 0, first


def main(argv):
    if "--list" in argv:
        for n, _, _ in MUTANTS:
            print(n)
        return 0
    names = [a for a in argv if not a.startswith("-")] or [n for n, _, _ in MUTANTS]
    caught, msg = run_one(None)
    print("control (unmodified oracle) ->", "FAILS" if caught else "passes", "|", msg, flush=True)
    if caught:
        return 2
    survivors = []
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        for name, (c, m) in zip(names, ex.map(run_one, names)):
            print(name, "->", "caught" if c else "SURVIVED", "|", m, flush=True)
            if not c:
                survivors.append(name)
    print("%d mutants, %d caught, %d survived%s" % (len(names), len(names) - len(survivors), len(survivors),
                                                    (": " + ", ".join(survivors)) if survivors else ""))
    return 1 if survivors else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
