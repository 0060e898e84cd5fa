"""The oracle's pins must catch plausible mistakes (no GPU).

Each case plants one mistake in a temporary copy of ``oracle/cliffs_oracle.cpp`` (a dropped
term, a wrong sign, a wrong index or factor), builds it with the host compiler, points the
oracle module at it, and requires at least one pin of ``test_oracle_pins`` to fail. The
oracle's Python-level functions (quake initialisation, initial-condition interpolation) get
the same treatment on a mutated copy of their source. The committed oracle is never
modified.
"""
import inspect
import os
import subprocess
import tempfile
import textwrap

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "cliffs_oracle.cpp")

# (name, exact text in the oracle source, replacement, pins expected to notice)
MUTATIONS = [
    ("depth term of eq. (eqQ) dropped",
     "return 0.5 * (lam_a + lam_b) * (r_a - r_b) / ds - GRAV * (d_a - d_b) / ds;",
     "return 0.5 * (lam_a + lam_b) * (r_a - r_b) / ds;",
     ["test_lake_at_rest", "test_pulse_closed_form"]),
    ("sign of the averaged flux in eq. (solver2)",
     "pn = pC - Fp + lpC", "pn = pC + Fp + lpC",
     ["test_pulse_closed_form", "test_dalembert_speed_and_second_order"]),
    ("second-order term of eq. (solver2) dropped",
     "pn = pC - Fp + lpC * k2 * (QpR - QpL) - adt + sdt;", "pn = pC - Fp - adt + sdt;",
     ["test_pulse_closed_form"]),
    ("mirror ghost keeps the velocity sign",
     "Node<T> Gh{S.e1[j], -S.w1[j], S.t1[j], d[j]};", "Node<T> Gh{S.e1[j], S.w1[j], S.t1[j], d[j]};",
     ["test_standing_wave_wall_at_half_node", "test_mass_linear_limit"]),
    ("wall on the node instead of half a node out",
     "const double dsR = (j < n - 1) ? ds[j] : ds[n - 2];",
     "const double dsR = (j < n - 1) ? ds[j] : 0.5 * ds[n - 2];",
     ["test_standing_wave_wall_at_half_node"]),
    ("eq. (stateh) with 8g",
     "T hn = (pn - qn) * (pn - qn) / (16.0 * g);", "T hn = (pn - qn) * (pn - qn) / (8.0 * g);",
     ["test_lake_at_rest", "test_pulse_closed_form"]),
    ("friction exponent 3/2 instead of 4/3",
     "inline double pow43(double a) { return a * std::cbrt(a); }",
     "inline double pow43(double a) { return a * std::sqrt(a); }",
     ["test_friction_uniform_flow"]),
    ("flooding test with -d_i",
     "if (!(val(eta[j]) + d[i] > hmin)) continue;", "if (!(val(eta[j]) - d[i] > hmin)) continue;",
     ["test_step_b_flooding_by_hand", "test_step_b_threshold_and_dry_velocity"]),
    ("tie-break picks the smaller eta",
     "if (best < 0 || val(eta[j]) > val(eta[best])) best = j;",
     "if (best < 0 || val(eta[j]) < val(eta[best])) best = j;",
     ["test_step_b_tie_break"]),
    ("cushion sets h_j instead of h_j/2",
     "if (val(hi) > 0.5 * val(hj)) S.e2[i] = 0.5 * hj - d[i];",
     "if (val(hi) > 0.5 * val(hj)) S.e2[i] = hj - d[i];",
     ["test_step_e_cushion_limiter"]),
    ("transverse advection sign",
     "tn = C.t - Ft + C.w * k2 * (QtR - QtL);", "tn = C.t + Ft + C.w * k2 * (QtR - QtL);",
     ["test_transverse_velocity_advected_by_u"]),
    ("cos(phi) missing from the row metric",
     "const double f = sph() ? R_SPHERE * std::cos(y[jy] * DEG) * DEG : 1.0;",
     "const double f = sph() ? R_SPHERE * DEG : 1.0;",
     ["test_spherical_zonal_speed_scales_with_cos_lat"]),
    ("spherical continuity term with the wrong sign",
     "if (src) sdt = dt * cC * C.w * src[j];", "if (src) sdt = -dt * cC * C.w * src[j];",
     ["test_spherical_area_weighted_mass"]),
    ("friction reverses the flow",
     "if (std::fabs(val(adt)) > std::fabs(val(C.w))) adt = C.w;", "",
     ["test_friction_clamp_never_reverses"]),
    ("max-wave counts dry cells",
     "if (!(fl && val(eta[c]) + Gd.d[c] >= Gd.P.h_min)) continue;", "(void)fl;",
     ["test_maxwave_ignores_dry_cells"]),
    ("bilinear weights transposed",
     "w01 = a * (1 - b), w10 = (1 - a) * b", "w01 = (1 - a) * b, w10 = a * (1 - b)",
     ["test_gauges_maxwave_and_bilinear_boundary"]),
    ("eq. (newdw) over 2 instead of 4",
     "nd = s * s / 4.0;", "nd = s * s / 2.0;",
     ["test_depth_filter_by_hand"]),
    ("tangent of a quotient with the wrong sign",
     "return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));",
     "return Dual(a.v / b.v, (a.d * b.v + a.v * b.d) / (b.v * b.v));",
     ["test_tlm_matches_central_differences"]),
    ("open edge as a zero-gradient ghost",
     "    const T p = right ? C.w + 2.0 * c : T(2.0 * c0);\n    const T q = right ? T(-2.0 * c0) : C.w - 2.0 * c;",
     "    const T p = C.w + 2.0 * c;\n    const T q = C.w - 2.0 * c;",
     ["test_open_edges_drain_a_raised_level_toward_still_water"]),
    ("open edge with the ends' invariants swapped",
     "if (j == n - 1 && (open & 2)) R = open_ghost(C, true, g);",
     "if (j == n - 1 && (open & 2)) R = open_ghost(C, false, g);",
     ["test_open_edge_lets_a_simple_wave_leave"]),
    ("incoming invariant of still water with the wrong sign",
     "const T q = right ? T(-2.0 * c0) : C.w - 2.0 * c;",
     "const T q = right ? T(2.0 * c0) : C.w - 2.0 * c;",
     ["test_open_edges_keep_a_lake_at_rest", "test_open_edge_lets_a_simple_wave_leave"]),
    ("eq. (solver1) flux over one interval instead of two",
     "Fp = dt * Q_literal(lpR, lpL, pR, pL, R.d, L.d, dsL + dsR);",
     "Fp = dt * Q_literal(lpR, lpL, pR, pL, R.d, L.d, dsR);",
     ["test_dalembert_speed_and_second_order", "test_literal_and_perturbation_forms_agree"]),
    ("eq. (solver1) speed difference without the depth term",
     "T dcRL = g * ((R.eta - L.eta) + (R.d - L.d)) / (cR + cL);",
     "T dcRL = g * (R.eta - L.eta) / (cR + cL);",
     ["test_literal_and_perturbation_forms_agree"]),
    ("alternating splitting never swaps the order",
     "const bool yfirst = Gd.P.alternate && (k & 1);", "const bool yfirst = false;",
     ["test_alternating_sweeps_take_y_first_on_odd_steps"]),
    ("alternating splitting swaps on even steps",
     "const bool yfirst = Gd.P.alternate && (k & 1);", "const bool yfirst = Gd.P.alternate && !(k & 1);",
     ["test_alternating_sweeps_take_y_first_on_odd_steps"]),
    ("eq. (newdc) over alpha instead of alpha^2",
     "nd = (lw ? line[j - 1] : line[j + 1]) / a2;", "nd = (lw ? line[j - 1] : line[j + 1]) / alpha;",
     ["test_depth_filter_by_hand"]),
    ("gauges recorded every step whatever gout",
     "O->gout > 0 && k % O->gout == 0", "O->gout > 0",
     ["test_gauges_maxwave_and_bilinear_boundary"]),
    ("max-wave taken every step whatever maxout",
     "O->maxout > 0 && k % O->maxout == 0", "O->maxout > 0",
     ["test_gauges_maxwave_and_bilinear_boundary"]),
    ("max-wave without the fold of the final state",
     "    if (fold_final && eta_max) {", "    if (false && eta_max) {",
     ["test_gauges_maxwave_and_bilinear_boundary"]),
    ("gauge records with u and v swapped",
     "r[3 * g + 0] = val(eta[c]); r[3 * g + 1] = val(u[c]); r[3 * g + 2] = val(v[c]);",
     "r[3 * g + 0] = val(eta[c]); r[3 * g + 1] = val(v[c]); r[3 * g + 2] = val(u[c]);",
     ["test_gauges_maxwave_and_bilinear_boundary"]),
    ("boundary series with u and v swapped",
     "r[3 * p + 0] = bil(u); r[3 * p + 1] = bil(v); r[3 * p + 2] = bil(eta);",
     "r[3 * p + 0] = bil(v); r[3 * p + 1] = bil(u); r[3 * p + 2] = bil(eta);",
     ["test_gauges_maxwave_and_bilinear_boundary"]),
    ("second-order coefficient over twice the right spacing",
     "const double k2 = dt * dt / (dsL + dsR);", "const double k2 = dt * dt / (2.0 * dsR);",
     ["test_pulse_closed_form_on_unequal_spacing"]),
    ("left flux of p over the right spacing",
     "T QpL = Q_literal(lpC, lpL, pC, pL, C.d, L.d, dsL);", "T QpL = Q_literal(lpC, lpL, pC, pL, C.d, L.d, dsR);",
     ["test_pulse_closed_form_on_unequal_spacing"]),
    ("boundary input held at the earlier record",
     "val[f] = (1.0 - w) * a + w * b;", "val[f] = a;",
     ["test_boundary_input_is_linear_between_records"]),
    ("boundary input weights reversed",
     "w = (t - times[k]) / (times[k + 1] - times[k]);", "w = (times[k + 1] - t) / (times[k + 1] - times[k]);",
     ["test_boundary_input_is_linear_between_records"]),
]


def _pin_functions(names):
    out = []
    for name in names:
        fn = getattr(pins, name)
        params = getattr(fn, "pytestmark", [])
        combos = [{}]
        for m in params:
            if m.name == "parametrize":
                keys = [k.strip() for k in m.args[0].split(",")]
                vals = m.args[1]
                new = []
                for c in combos:
                    for v in vals:
                        v = v if isinstance(v, tuple) else (v,)
                        cc = dict(c)
                        cc.update(zip(keys, v))
                        new.append(cc)
                combos = new
        for c in combos:
            out.append((name, fn, c))
    return out


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(case, tmp_path):
    name, old, new, targets = case
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must occur exactly once: %r" % old
    path = tmp_path / "mut.cpp"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                    "-ffp-contract=off", "-o", str(so), str(path)], check=True)
    oracle.swap_library(str(so))
    caught = []
    try:
        for pname, fn, kw in _pin_functions(targets):
            try:
                fn(**kw)
            except (AssertionError, ValueError, FloatingPointError):
                caught.append((pname, kw))
    finally:
        oracle.swap_library(None)
    assert caught, "no pin caught: %s" % name


# Mistakes in the oracle's Python-level functions: (name, function, exact text, replacement,
# pins expected to notice). The mutated function replaces the module's for the pins' calls.
PY_MUTATIONS = [
    ("initial-condition weight measured from the far node", "interp_initial",
     "return k, (xp - c[k]) / (c[k + 1] - c[k])", "return k, (c[k + 1] - xp) / (c[k + 1] - c[k])",
     ["test_initial_condition_interpolation_exact_for_linear_fields_and_zero_outside"]),
    ("quake lowers the floor", "quake_init",
     "return depth - zeta, np.where(wet, zeta, 0.0)", "return depth + zeta, np.where(wet, zeta, 0.0)",
     ["test_quake_lifts_the_floor_and_the_water_column_with_it"]),
    ("quake lifts the surface on dry nodes too", "quake_init",
     "return depth - zeta, np.where(wet, zeta, 0.0)", "return depth - zeta, zeta.copy()",
     ["test_quake_lifts_the_floor_and_the_water_column_with_it"]),
    ("quake ignores walls", "quake_init",
     "wet = (depth >= h_min) & ((itopo != 0) | (depth >= dwall))", "wet = depth >= h_min",
     ["test_quake_lifts_the_floor_and_the_water_column_with_it"]),
]


@pytest.mark.parametrize("case", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_pins_catch_planted_mistake_in_python(case, monkeypatch):
    name, fname, old, new, targets = case
    src = textwrap.dedent(inspect.getsource(getattr(oracle, fname)))
    assert src.count(old) == 1, "mutation anchor must occur exactly once: %r" % old
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutant %s>" % fname, "exec"), ns)
    monkeypatch.setattr(oracle, fname, ns[fname])
    caught = []
    for pname, fn, kw in _pin_functions(targets):
        try:
            fn(**kw)
        except (AssertionError, ValueError, FloatingPointError):
            caught.append((pname, kw))
    assert caught, "no pin caught: %s" % name
