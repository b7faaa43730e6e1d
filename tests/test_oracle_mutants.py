"""Mutation checks of the oracle's pins: a plausible mistake is planted in a copy of
the oracle's C source (never in the CUDA library), the copy is compiled, and the pin
written for that part of the method must fail against it. Each mutant names the
passage it breaks."""
import pytest

import oracle
import test_oracle_pins as pins

# (name, passage, original text, mistaken text, pin that must fail)
MUTANTS = [
    ("eq1_shear_dropped", "Eq. 1",
     "    F = vsub(F, vscale(vt, P->ksh));\n", "",
     pins.test_simple_model_shear_decays_sliding_exponentially),
    ("eq1_shear_sign", "Eq. 1",
     "    F = vsub(F, vscale(vt, P->ksh));\n", "    F = vadd(F, vscale(vt, P->ksh));\n",
     pins.test_simple_model_shear_decays_sliding_exponentially),
    ("hertz_kt_from_cn", "Eqs. 8-9",
     "        kt = P->ct * s;\n", "        kt = P->cn * s;\n",
     pins.test_hertz_tangential_stiffness_sets_stick_oscillation_period),
    ("hertz_kt_without_sqrt", "Eqs. 8-9",
     "        kt = P->ct * s;\n", "        kt = P->ct;\n",
     pins.test_hertz_tangential_stiffness_sets_stick_oscillation_period),
    ("cap_reset_without_dashpot", "Eq. 5 (spring after slip)",
     "dt = vscale(vadd(Ft, vscale(vt, eta_t)), -1.0 / kt);", "dt = vscale(Ft, -1.0 / kt);",
     pins.test_spring_after_slip_keeps_eq4_an_identity_on_reversal),
    ("cap_without_reset", "Eq. 5 (spring after slip)",
     "        if (kt > 0.0) dt = vscale(vadd(Ft, vscale(vt, eta_t)), -1.0 / kt);\n", "",
     pins.test_spring_after_slip_keeps_eq4_an_identity_on_reversal),
    ("eq7_magnitude_restored", "Eq. 7",
     "    vec3 dt = vadd(vsub(dt_old, vscale(n, vdot(dt_old, n))), vscale(vt, P->dt));\n",
     "    vec3 pr = vsub(dt_old, vscale(n, vdot(dt_old, n)));\n"
     "    if (vnorm(pr) > 0.0) pr = vscale(pr, vnorm(dt_old) / vnorm(pr));\n"
     "    vec3 dt = vadd(pr, vscale(vt, P->dt));\n",
     pins.test_history_projection_shrinks_spring_by_cos_theta),
]


@pytest.mark.parametrize("name,passage,old,new,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_fails_on_planted_mistake(name, passage, old, new, pin, tmp_path):
    src = oracle.source()
    assert src.count(old) == 1, f"mutation site of {name} ({passage}) not found exactly once"
    with oracle.variant(src.replace(old, new), tmp_path):
        with pytest.raises(AssertionError):
            pin()
    # and the same pin passes on the oracle as it stands
    pin()
