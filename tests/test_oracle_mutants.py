"""Mutation check of the oracle's pins (CPU only).

Each mutant plants one plausible mistake in a copy of the oracle package (its C++ arithmetic or
its Python composition and binary64 adjoint references): a dropped term, a wrong sign or index, a
transposed operand, a threshold taken with the wrong comparison, a tie broken the other way, a
rounding or clamping rule changed, two stages run in the wrong order. The pins
(`tests/test_oracle_pins.py`, `tests/test_oracle_adjoint.py`) run against the copy, which the
test conftest imports in place of the oracle when TSGM_ORACLE_ROOT names its folder. Every mutant
must fail at least one pin, and the unmodified copy must pass, so that a pin that stopped
checking what it claims is noticed. No mutant writes outside its buffers.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CPP = os.path.join(ROOT, "oracle", "tsgm_oracle.cpp")
PY = os.path.join(ROOT, "oracle", "__init__.py")
WORK = os.path.join(ROOT, "oracle", "_build", "mutants")
PINS = [os.path.join(ROOT, "tests", f) for f in ("test_oracle_pins.py", "test_oracle_adjoint.py")]

# (name, text of tsgm_oracle.cpp, replacement); each text occurs exactly once in the file
CPP_MUTANTS = [
    # Eq. 1-4: disparity-space homography
    ("H_t_sign", "{R[0], R[1], R[2], t[0]}", "{R[0], R[1], R[2], -t[0]}"),
    ("H_R_transposed", "{R[0], R[1], R[2], t[0]},\n                      {R[3], R[4], R[5], t[1]}",
     "{R[0], R[3], R[2], t[0]},\n                      {R[1], R[4], R[5], t[1]}"),
    ("H_baseline_dropped", "{0, 0, 0, f * b}, {0, 0, 1, 0}}", "{0, 0, 0, f}, {0, 0, 1, 0}}"),
    # Sec. 2.2, Eq. 3, 5-6: forward warp, z-buffer and variance prediction
    ("warp_truncates", "std::floor((xp + cx) + 0.5f)", "std::floor((xp + cx))"),
    ("warp_y_about_cx", "const float yt = (float)v - cy;", "const float yt = (float)v - cx;"),
    ("zbuffer_tie_to_last", "if (dp > best[tgt]) {", "if (dp >= best[tgt]) {"),
    ("zbuffer_far_wins", "if (dp > best[tgt]) {", "if (best[tgt] < 0.0f || dp < best[tgt]) {"),
    ("phi_not_squared", "const float phi2 = phi * phi;", "const float phi2 = phi;"),
    ("phi_inverted", "const float phi = dp / Dprev[src[i]];", "const float phi = Dprev[src[i]] / dp;"),
    ("q_dropped", "Ppred[i] = pp + q;", "Ppred[i] = pp;"),
    # Sec. 2.2, Eq. 7-8: gap filling
    ("fill_threshold_le", "if (!(diff < gamma_f)) continue;", "if (!(diff <= gamma_f)) continue;"),
    ("fill_variance_sum", "P[i] = ps * 0.5f;", "P[i] = ps;"),
    ("fill_passes_share_input", "        std::copy(D, D + n, d0.begin());\n        std::copy(P, P + n, p0.begin());\n", ""),
    # Sec. 2.2, disparity refinement: edge rejection
    ("edge_threshold_strict", "if (!(std::fabs(d0[i] - d0[j]) < edge_thr)) edge = true;",
     "if (!(std::fabs(d0[i] - d0[j]) <= edge_thr)) edge = true;"),
    ("edge_holes_are_edges", "                    if (!(finite_nonneg(d0[j]) && finite_nonneg(p0[j]))) continue;\n", ""),
    ("edge_no_upper_row", "            for (int dy = -1; dy <= 1; ++dy)\n                for (int dx = -1; dx <= 1; ++dx) {\n                    if (dx == 0 && dy == 0) continue;",
     "            for (int dy = 0; dy <= 1; ++dy)\n                for (int dx = -1; dx <= 1; ++dx) {\n                    if (dx == 0 && dy == 0) continue;"),
    ("edge_four_neighbours", "if (dx == 0 && dy == 0) continue;\n                    const int xn",
     "if ((dx == 0) == (dy == 0)) continue;\n                    const int xn"),
    # Sec. 2.2, Sec. 3 (Fig. 3(d)): the prediction's left-right check
    ("predlr_truncates", "const float rf = std::floor(d + 0.5f);\n    return", "const float rf = std::floor(d);\n    return"),
    ("predlr_first_surface", "if (r >= 0 && d[x] > R[r]) R[r] = d[x];", "if (r >= 0 && R[r] < 0.0f) R[r] = d[x];"),
    ("predlr_threshold_strict", "std::fabs(d[x] - R[r]) <= tol", "std::fabs(d[x] - R[r]) < tol"),
    # Sec. 2.4: SAD check
    ("sad_area_width_only", "const float lim = sad_thr * (float)(sw * sh);", "const float lim = sad_thr * (float)(sw);"),
    ("sad_shift_sign", "const int xr = clampi(x - dx + u, 0, W - 1);", "const int xr = clampi(x + dx + u, 0, W - 1);"),
    ("sad_threshold_ge", "if ((float)sad > lim) {", "if ((float)sad >= lim) {"),
    ("sad_truncates", "const float rf = std::floor(D[i] + 0.5f);", "const float rf = std::floor(D[i]);"),
    ("sad_one_row", "const int yy = clampi(y + v, 0, Hh - 1);", "const int yy = clampi(y, 0, Hh - 1);"),
    # Sec. 2.3: reduced windows
    ("window_hi_floor", "const float hi_f = std::ceil(d + r);", "const float hi_f = std::floor(d + r);"),
    ("window_lo_ceil", "const float lo_f = std::floor(d - r);", "const float lo_f = std::ceil(d - r);"),
    ("window_variance_not_sigma", "const float r = sigma_mult * s;", "const float r = sigma_mult * p;"),
    # census and Hamming cost
    ("census_le", "if (img[qy * W + qx] < c)", "if (img[qy * W + qx] <= c)"),
    ("census_bits_reversed", "code |= (uint64_t)1 << bit;", "code |= (uint64_t)1 << (cw * ch - 2 - bit);"),
    ("cost_no_shift", "if (x - d >= 0) c = popcount64(cl[i] ^ cr[y * W + x - d]);",
     "if (x - d >= 0) c = popcount64(cl[i] ^ cr[y * W + x + d - d]);"),
    ("cost_border_zero", "                int c = Bc;\n", "                int c = 0;\n"),
    # Sec. 2.3: SGM recursion
    ("sgm_P1_as_P2", "best = std::min(best, (int)L[off[j] + (d - 1 - lo[j])] + P1)",
     "best = std::min(best, (int)L[off[j] + (d - 1 - lo[j])] + P2)"),
    ("sgm_P2_as_P1", "int best = m + P2;", "int best = m + P1;"),
    ("sgm_min_not_subtracted", "L[off[i] + (d - lo[i])] = (uint16_t)(c + best - m);",
     "L[off[i] + (d - lo[i])] = (uint16_t)(c + best);"),
    ("sgm_wrong_predecessor", "const int qx = x - dx, qy = y - dy;", "const int qx = x - dx, qy = y + dy;"),
    # WTA, sub-pixel, matching variance (Eq. 9)
    ("wta_tie_to_high", "if (s[d - a] < s[best - a]) best = d;", "if (s[d - a] <= s[best - a]) best = d;"),
    ("subpixel_half", "const int den = 2 * (sm - 2 * s0 + sp);", "const int den = (sm - 2 * s0 + sp);"),
    ("subpixel_sign", "if (den > 0) delta = (float)(sm - sp) / (float)den;", "if (den > 0) delta = (float)(sp - sm) / (float)den;"),
    ("eq9_threshold_le", "if ((float)run < s_thr) ++nl; else break;", "if ((float)run <= s_thr) ++nl; else break;"),
    ("eq9_not_running_sum", "        for (int d = best - 1; d >= a; --d) {\n            run += s[d - a] - s[best - a];",
     "        for (int d = best - 1; d >= a; --d) {\n            run = s[d - a] - s[best - a];"),
    ("eq9_no_floor", "if (r < r_min) r = r_min;", ""),
    # Sec. 2.4: left-right check
    ("lr_tie_to_high", "if (s < bs) {  // increasing d", "if (s <= bs) {  // increasing d"),
    ("lr_threshold_strict", "ok = dr >= 0 && std::abs(d - dr) <= tol;", "ok = dr >= 0 && std::abs(d - dr) < tol;"),
    ("lr_drops_largest_d", "for (int x = xr; x < W && x - xr < D; ++x) {", "for (int x = xr; x < W && x - xr < D - 1; ++x) {"),
    # Sec. 2.4, Eq. 10-12: Kalman update
    ("kalman_innovation_sign", "const float innov = Dz[i] - Dp[i];", "const float innov = Dp[i] - Dz[i];"),
    ("kalman_gain_swapped", "const float K = Pp[i] / s;", "const float K = rz[i] / s;"),
    ("kalman_variance_K", "const float omk = 1.0f - K;", "const float omk = K;"),
    ("kalman_measurement_only_keeps_p", "            D[i] = Dz[i];\n            P[i] = rz[i];",
     "            D[i] = Dz[i];\n            P[i] = Pp[i];"),
    # window edges and validity tests (each off by one label, one pixel or one condition)
    ("valid_accepts_inf", "return v >= 0.0f && v <= FLT_MAX;", "return v >= 0.0f;"),
    ("warp_drops_last_column", "fx <= (float)(W - 1)", "fx < (float)(W - 1)"),
    ("predlr_drops_column_0", "return rf > (float)x ? -1 : x - (int)rf;", "return rf >= (float)x ? -1 : x - (int)rf;"),
    ("window_top_label_is_a_miss", "if (lo_f <= (float)(D - 1) && hi_f >= 0.0f) {",
     "if (lo_f < (float)(D - 1) && hi_f >= 0.0f) {"),
    ("census_left_clamp_to_1", "int qx = std::min(std::max(x + dx, 0), W - 1);",
     "int qx = std::min(std::max(x + dx, 1), W - 1);"),
    ("sgm_m_misses_top_label", "for (int k = lo[j]; k <= hi[j]; ++k) m = std::min(m, (int)L[off[j] + (k - lo[j])]);",
     "for (int k = lo[j]; k < hi[j]; ++k) m = std::min(m, (int)L[off[j] + (k - lo[j])]);"),
    ("sgm_upper_neighbour_at_edge", "if (d + 1 >= lo[j] && d + 1 <= hi[j]) best",
     "if (d + 1 >= lo[j] && d + 1 < hi[j]) best"),
    ("subpixel_needs_two_above", "if (best - 1 >= a && best + 1 <= b) {", "if (best - 1 >= a && best + 1 < b) {"),
    ("lr_window_top_excluded", "if (d < lo[i] || d > hi[i]) continue;", "if (d < lo[i] || d >= hi[i]) continue;"),
    ("kalman_measurement_ignores_r", "const bool mv = finite_nonneg(Dz[i]) && finite_nonneg(rz[i]);",
     "const bool mv = finite_nonneg(Dz[i]);"),
    ("kalman_prediction_ignores_p", "const bool pv = finite_nonneg(Dp[i]) && finite_nonneg(Pp[i]);",
     "const bool pv = finite_nonneg(Dp[i]);"),
]

# (name, text of __init__.py, replacement): parameters, the per-frame composition (Sec. 2) and
# the binary64 adjoint references
PY_MUTANTS = [
    ("Bc_counts_the_centre", "return self.census_w * self.census_h - 1", "return self.census_w * self.census_h"),
    ("s_thr_not_per_path", "return float(np.float32(self.S_max) * np.float32(self.n_paths))",
     "return float(np.float32(self.S_max))"),
    ("K_cx_cy_swapped", "return float(K[0, 0]), float(K[0, 2]), float(K[1, 2])",
     "return float(K[0, 0]), float(K[1, 2]), float(K[0, 2])"),
    ("tracker_q_dropped", "np.float32(cx), np.float32(cy), prm.q)", "np.float32(cx), np.float32(cy), 0.0)"),
    ("tracker_fill_before_edge",
     "            if prm.edge_reject:\n                Dp, Pp = edge_reject(Dp, Pp, prm.edge_thr)\n"
     "            if prm.fill_gaps:\n                Dp, Pp = fill_gaps(Dp, Pp, prm.gamma_f)\n",
     "            if prm.fill_gaps:\n                Dp, Pp = fill_gaps(Dp, Pp, prm.gamma_f)\n"
     "            if prm.edge_reject:\n                Dp, Pp = edge_reject(Dp, Pp, prm.edge_thr)\n"),
    ("tracker_pred_lr_before_fill",
     "            if prm.fill_gaps:\n                Dp, Pp = fill_gaps(Dp, Pp, prm.gamma_f)\n"
     "            if prm.pred_lr_check:\n                Dp, Pp = pred_lr_check(Dp, Pp, prm.pred_lr_tol)\n",
     "            if prm.pred_lr_check:\n                Dp, Pp = pred_lr_check(Dp, Pp, prm.pred_lr_tol)\n"
     "            if prm.fill_gaps:\n                Dp, Pp = fill_gaps(Dp, Pp, prm.gamma_f)\n"),
    ("tracker_state_keeps_rejected", "meas = _finite_nonneg(m[\"Dz\"]) & _finite_nonneg(m[\"rz\"])",
     "meas = np.ones(D.shape, bool)"),
    ("tracker_full_range_ignored", "        if prm.full_range:\n            lo = np.zeros((Hh, W), np.int16)",
     "        if False:\n            lo = np.zeros((Hh, W), np.int16)"),
    ("tracker_sad_skipped", "            D, P = sad_check(left, right, D, P, prm.sad_w, prm.sad_h, prm.sad_thr)\n",
     "            pass\n"),
    ("rodrigues_sign", "return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * (Kx @ Kx)",
     "return np.eye(3) - np.sin(th) * Kx + (1 - np.cos(th)) * (Kx @ Kx)"),
    ("adj_forward_phi_not_squared", "pp = (dp / d) ** 2 * p + q             # Eq. 5-6",
     "pp = (dp / d) * p + q             # Eq. 5-6"),
    ("adj_forward_gain_swapped", "Kg = Pp[both] / (Pp[both] + r[both])   # Eq. 10",
     "Kg = r[both] / (Pp[both] + r[both])   # Eq. 10"),
    ("adj_forward_measurement_only_unscaled", "D[mo], P[mo] = dz[mo], r[mo]", "D[mo], P[mo] = dz[mo], rr[mo]"),
    ("adj_grad_dP_dpp", "dP_dpp = np.where(mv, (r / den) ** 2, 1.0)", "dP_dpp = np.where(mv, r / den, 1.0)"),
    ("adj_grad_phi_chain", "dL_ddp = gd * dD_ddp + dL_dpp * 2 * p * dp / d ** 2",
     "dL_ddp = gd * dD_ddp + dL_dpp * p * dp / d ** 2"),
    ("adj_grad_t2_baseline", "g_t2 = np.sum(dL_dw3 * d / (f * b))", "g_t2 = np.sum(dL_dw3 * d / f)"),
    ("adj_grad_measurement_only_dropped",
     "g_sr += np.sum(gP.reshape(-1)[mo].astype(np.float64) * rall[mo])", "g_sr += 0.0"),
]


def _run_pins(name: str, cpp: str, py: str) -> tuple[str, int, str]:
    pkg = os.path.join(WORK, name, "oracle")
    os.makedirs(pkg, exist_ok=True)
    for fname, text in (("tsgm_oracle.cpp", cpp), ("__init__.py", py)):
        with open(os.path.join(pkg, fname), "w") as f:
            f.write(text)
    env = dict(os.environ, TSGM_ORACLE_ROOT=os.path.dirname(pkg))
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    lines = r.stdout.strip().splitlines() or [""]
    failed = [ln for ln in lines if ln.startswith(("FAILED", "ERROR"))]
    return name, r.returncode, "; ".join(failed[:1] + lines[-1:])


def test_every_mutant_text_occurs_once():
    names = [m[0] for m in CPP_MUTANTS + PY_MUTANTS]
    assert len(set(names)) == len(names)
    for path, mutants in ((CPP, CPP_MUTANTS), (PY, PY_MUTANTS)):
        orig = open(path).read()
        for name, a, _ in mutants:
            assert orig.count(a) == 1, name


def test_every_planted_mistake_fails_a_pin():
    cpp, py = open(CPP).read(), open(PY).read()
    jobs = ([("unmodified", cpp, py)] +
            [(name, cpp.replace(a, b, 1), py) for name, a, b in CPP_MUTANTS] +
            [(name, cpp, py.replace(a, b, 1)) for name, a, b in PY_MUTANTS])
    workers = max(1, min(8, os.cpu_count() or 1))
    try:
        with cf.ThreadPoolExecutor(workers) as ex:
            results = {name: (rc, tail) for name, rc, tail in ex.map(lambda j: _run_pins(*j), jobs)}
    finally:
        shutil.rmtree(WORK, ignore_errors=True)
    rc, tail = results.pop("unmodified")
    assert rc == 0, f"the unmodified copy fails its pins: {tail}"
    survivors = {name: tail for name, (rc, tail) in results.items() if rc == 0}
    assert not survivors, f"mistakes no pin catches: {survivors}"
