"""Plant plausible mistakes in a copy of the oracle source and check that the
pins catch each one (the oracle itself is never modified)."""
import os
import subprocess

import pytest

import oracle as O
from oracle import build as OB
import tests.test_oracle_pins as P

# (name, original text, planted mistake, pins expected to catch it)
MUTATIONS = [
    ("eq7 control sign", "(1.0 - a * xr[i] * xr[i])", "(1.0 + a * xr[i] * xr[i])",
     [lambda: P.test_eq7_product_formula_with_pinned_walls(0.3)]),
    ("eq7 denominator", "* pr[i] / (double)(M - m)", "* pr[i] / (double)(M - m + 1)",
     [P.test_gbsb_a0_is_bsb]),
    ("eq3 coupling sign", "(pr[i] * xr[i] - c * f[i])", "(pr[i] * xr[i] + c * f[i])",
     [P.test_coupling_sign_on_uniform_mode]),
    ("eq3 dropped p x term", "(pr[i] * xr[i] - c * f[i])", "(0.0 * xr[i] - c * f[i])",
     [lambda: P.test_eq10_harmonic_closed_form(1.0, 0.5)]),
    ("eq4 scale", "xr[i] = xr[i] + yr[i] * dt;", "xr[i] = xr[i] + yr[i] * dt * dt;",
     [lambda: P.test_eq10_harmonic_closed_form(0.3, 1.25)]),
    ("eq6 schedule index", "1.0 - (double)(m + 1) / (double)M", "1.0 - (double)(m) / (double)M",
     [lambda: P.test_time_reversal_of_wall_free_step("bsb")]),
    ("eq1 energy factor", "return -0.5 * e;", "return -1.0 * e;",
     [lambda: P.test_energy_cut_identity("pm1")]),
    ("wall keeps momentum", "yr[i] = 0.0;", "yr[i] = yr[i];",
     [lambda: P.test_eq7_product_formula_with_pinned_walls(0.3)]),
    ("dsb coupling uses x", "v[j] = orc_sgn(xr[j]);", "v[j] = xr[j];",
     [lambda: P.test_time_reversal_of_wall_free_step("dsb")]),
    ("jx16 grid scale", "v[j] = rint(u) / 32768.0;", "v[j] = rint(u) / 16384.0;",
     [P.test_jx16_grid_scale_and_rounding_by_hand]),
    ("jx16 rounds half up", "v[j] = rint(u) / 32768.0;", "v[j] = floor(u + 0.5) / 32768.0;",
     [P.test_jx16_grid_scale_and_rounding_by_hand]),
    ("jx16 coupling exact", "v[j] = rint(u) / 32768.0;", "v[j] = xr[j];",
     [P.test_jx16_grid_scale_and_rounding_by_hand]),
    ("best keeps latest tie", "if (e < best_E[r]) {", "if (e <= best_E[r]) {",
     [P.test_walls_and_best_keeping]),
    ("control uses new x", None, None, [lambda: P.test_time_reversal_of_wall_free_step("gbsb")]),
    ("tangent coupling sign", "(dpr[i] * xr[i] + pr[i] * dxr[i] - c * dfi)",
     "(dpr[i] * xr[i] + pr[i] * dxr[i] + c * dfi)",
     [lambda: P.test_tangent_matches_central_differences("gbsb"), P.test_tangent_growth_rate_at_equilibrium]),
    ("tangent drops p' dx", "(dpr[i] * xr[i] + pr[i] * dxr[i] - c * dfi)",
     "(dpr[i] * xr[i] - c * dfi)", [lambda: P.test_tangent_matches_central_differences("bsb")]),
    ("adjoint drops J lf", "for (int32_t i = 0; i < N; ++i) lx[i] += Jlf[i];",
     "for (int32_t i = 0; i < N; ++i) lx[i] += 0.0 * Jlf[i];",
     [lambda: P.test_adjoint_matches_central_differences("gbsb"),
      P.test_adjoint_dot_product_identity_with_tangent]),
    ("adjoint dt term sign", "sdt += -lyt * (pn[i] * x[i] - c * f[i]);",
     "sdt += lyt * (pn[i] * x[i] - c * f[i]);",
     [lambda: P.test_adjoint_matches_central_differences("bsb")]),
    ("adjoint control factor", "lpi = lpn * (1.0 - g / rem);", "lpi = lpn;",
     [lambda: P.test_adjoint_matches_central_differences("gbsb")]),
    ("tangent dp drops 2Ax dx p", "(g * dpr[i] - 2.0 * a * xr[i] * dxr[i] * pr[i])",
     "(g * dpr[i])", [lambda: P.test_tangent_matches_central_differences("gbsb")]),
]


def _mutate_control_new_x(src):
    # move the FP block after the position update: Eq. 7 would then see x(t_{m+1})
    start = src.index("            /* FP: bifurcation parameter(s) at t_{m+1}, from x(t_m) */")
    end = src.index("            /* JX: many-body term")
    fp_block = src[start:end]
    src = src[:start] + src[end:]
    anchor = "            /* Eq. 5: perfectly inelastic walls at |x| = 1 */"
    return src.replace(anchor, fp_block + anchor)


@pytest.mark.parametrize("name,orig,bad,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, orig, bad, pins):
    src = open(OB.SRC).read()
    if orig is None:
        mutated = _mutate_control_new_x(src)
    else:
        assert src.count(orig) >= 1, orig
        mutated = src.replace(orig, bad)
    assert mutated != src
    c_path = tmp_path / "mut.c"
    so_path = tmp_path / "libmut.so"
    c_path.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-shared",
                    "-fPIC", "-o", str(so_path), str(c_path), "-lm"], check=True)
    old = O._load_library_for_tests(str(so_path))
    try:
        caught = 0
        for pin in pins:
            try:
                pin()
            except (AssertionError, ValueError):
                caught += 1
        assert caught == len(pins), f"planted mistake '{name}' not caught"
    finally:
        O._restore_library_for_tests(old)
    # the real oracle still passes the same pins
    for pin in pins:
        pin()
