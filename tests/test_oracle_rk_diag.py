"""Pins of the oracle's RK(5,4) scheme and the Taylor--Green diagnostics (Sec. 2.4, Sec. 4.2)."""
import math
from fractions import Fraction

import pytest
import torch

from oracle import diagnostics, physics as ph, rk
from oracle.mesh import BoxMesh
from oracle.operator import DGOperator
from paper_1806_03095_gb300 import inputs


def _tableau():
    a, b = rk.butcher_from_2n(rk.LSRK54_A, rk.LSRK54_B)
    c = [sum(row) for row in a]
    return a, b, c


def test_lsrk54_stage_times_match_published_C():
    _, _, c = _tableau()
    for ci, Ci in zip(c, rk.LSRK54_C):
        assert abs(float(ci - Ci)) < 1e-12


def test_lsrk54_order_conditions():
    """All eight conditions of order <= 4 for an explicit Butcher tableau."""
    a, b, c = _tableau()
    s = len(b)
    f = float
    conds = {
        "sum b": (sum(b), Fraction(1)),
        "b c": (sum(b[i] * c[i] for i in range(s)), Fraction(1, 2)),
        "b c^2": (sum(b[i] * c[i] ** 2 for i in range(s)), Fraction(1, 3)),
        "b a c": (sum(b[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), Fraction(1, 6)),
        "b c^3": (sum(b[i] * c[i] ** 3 for i in range(s)), Fraction(1, 4)),
        "b c a c": (sum(b[i] * c[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), Fraction(1, 8)),
        "b a c^2": (sum(b[i] * a[i][j] * c[j] ** 2 for i in range(s) for j in range(s)), Fraction(1, 12)),
        "b a a c": (sum(b[i] * a[i][j] * a[j][l] * c[l] for i in range(s) for j in range(s) for l in range(s)),
                    Fraction(1, 24)),
    }
    for name, (val, want) in conds.items():
        assert abs(f(val - want)) < 1e-11, name


def test_lsrk54_negative_control_typo_breaks_order():
    """A single mistyped digit in one B coefficient violates the order conditions."""
    Bbad = list(rk.LSRK54_B)
    Bbad[2] = Fraction(1720146321549, 2090206949499)
    a, b = rk.butcher_from_2n(rk.LSRK54_A, Bbad)
    assert abs(float(sum(b) - 1)) > 1e-13


def _conditions(a, b, c):
    s = len(b)
    return {
        "sum b": (sum(b), Fraction(1)),
        "b c": (sum(b[i] * c[i] for i in range(s)), Fraction(1, 2)),
        "b c^2": (sum(b[i] * c[i] ** 2 for i in range(s)), Fraction(1, 3)),
        "b a c": (sum(b[i] * a[i][j] * c[j] for i in range(s) for j in range(s)), Fraction(1, 6)),
        "b c^3": (sum(b[i] * c[i] ** 3 for i in range(s)), Fraction(1, 4)),
        "b a a c": (sum(b[i] * a[i][j] * a[j][l] * c[l] for i in range(s) for j in range(s) for l in range(s)),
                    Fraction(1, 24)),
    }


def test_lsrk33_third_order_exactly_and_not_fourth():
    """Williamson's 2N scheme: the Butcher tableau from (A, B) meets the four conditions of order <= 3
    exactly (rational arithmetic), reproduces the stage times C, and misses order 4."""
    a, b = rk.butcher_from_2n(rk.LSRK33_A, rk.LSRK33_B)
    c = [sum(row) for row in a]
    assert c == list(rk.LSRK33_C)
    conds = _conditions(a, b, c)
    for name in ("sum b", "b c", "b c^2", "b a c"):
        assert conds[name][0] == conds[name][1], name
    assert any(conds[n][0] != conds[n][1] for n in ("b c^3", "b a a c"))


def test_lsrk33_negative_control_typo():
    a, b = rk.butcher_from_2n((Fraction(0), Fraction(-5, 9), Fraction(-153, 127)), rk.LSRK33_B)
    c = [sum(row) for row in a]
    conds = _conditions(a, b, c)
    assert any(conds[n][0] != conds[n][1] for n in ("sum b", "b c", "b c^2", "b a c"))


def test_lsrk33_scalar_ode_order_3():
    lam = -1.3
    errs = []
    for nst in (10, 20, 40):
        dt = 1.0 / nst
        y = torch.tensor(1.0, dtype=torch.float64)
        for i in range(nst):
            y = rk.lsrk_step(lambda v, t: lam * v, y, dt, i * dt, rk.LSRK33_A, rk.LSRK33_B, rk.LSRK33_C)
        errs.append(abs(float(y) - math.exp(lam)))
    for e0, e1 in zip(errs, errs[1:]):
        assert abs(math.log2(e0 / e1) - 3.0) < 0.15


def test_lsrk_step_with_rk54_coefficients_is_step():
    op = DGOperator(BoxMesh((2, 2, 2), [-math.pi] * 3, [math.pi] * 3, (1, 1, 1), 2), ph.Physics.from_numbers(1600.0, 0.71, 0.1),
                    4, 3)
    U = inputs.tgv_state(op.xyz)
    Lf = lambda V, t: op.L(V)  # noqa: E731
    a = rk.step(Lf, U, 1e-3, 0.0)
    b = rk.lsrk_step(Lf, U, 1e-3, 0.0, rk.LSRK54_A, rk.LSRK54_B, rk.LSRK54_C)
    assert torch.equal(a, b)


def test_lsrk54_scalar_ode_order_4():
    lam = -1.3
    errs = []
    for nst in (10, 20, 40):
        dt = 1.0 / nst
        y = torch.tensor(1.0, dtype=torch.float64)
        for i in range(nst):
            y = rk.step(lambda v, t: lam * v, y, dt, i * dt)
        errs.append(abs(float(y) - math.exp(lam)))
    assert math.log2(errs[1] / errs[2]) > 3.8, errs


def test_lsrk54_time_dependent_rhs_uses_stage_times():
    """y' = cos t, y(0) = 0 -> sin(1): order 4 needs the published C_i stage times."""
    errs = []
    for nst in (8, 16):
        dt = 1.0 / nst
        y = torch.tensor(0.0, dtype=torch.float64)
        for i in range(nst):
            y = rk.step(lambda v, t: torch.cos(torch.tensor(t, dtype=torch.float64)), y, dt, i * dt)
        errs.append(abs(float(y) - math.sin(1.0)))
    assert math.log2(errs[0] / errs[1]) > 3.7, errs


# -- Taylor--Green closed forms (Sec. 4.2.1, Sec. 4.2.3) --------------------------------------------
PHYS = ph.Physics.from_numbers(1600.0, 0.71, 0.1)


def _tgv(N, k):
    mesh = BoxMesh((N,) * 3, [-math.pi] * 3, [math.pi] * 3, (1, 1, 1), k)
    op = DGOperator(mesh, PHYS, (3 * k) // 2 + 1, k + 1)
    U = inputs.tgv_state(torch.as_tensor(mesh.xyz))
    return op, U


def test_tgv_initial_kinetic_energy_and_dissipation():
    """e_k(0) = U0^2/8 = 0.125 and eps(0) = 3 nu / 4 for the closed-form initial field."""
    d = [diagnostics.diagnostics(*_tgv(N, 3)) for N in (4, 8)]
    for dd, tol_ek, tol_eps in zip(d, (1e-4, 2e-6), (1e-3, 2e-5)):
        assert abs(float(dd[0]) - 0.125) < tol_ek
        assert abs(float(dd[1]) / (0.75 * PHYS.nu) - 1.0) < tol_eps
    assert abs(float(d[1][0]) - 0.125) < abs(float(d[0][0]) - 0.125) / 10  # converging


def test_tgv_initial_dissipation_balance():
    """At t = 0 the (nearly incompressible) flow has -de_k/dt = eps up to the resolution error."""
    op, U = _tgv(8, 3)
    d = diagnostics.diagnostics(op, U, op.L(U))
    assert abs(float(d[2]) / float(d[1]) - 1.0) < 1e-4


def test_conservation_totals_over_rk_steps():
    op, U = _tgv(2, 3)
    U = U + 0.01 * inputs.uniform(U.shape, 9)
    d0 = diagnostics.diagnostics(op, U)
    dt = 5e-3
    for i in range(3):
        U = rk.step(lambda V, t: op.L(V), U, dt, i * dt)
    d1 = diagnostics.diagnostics(op, U)
    # rounding scale of the update: dt * steps * volume * max |F_c row| (the pressure
    # terms of the momentum and energy fluxes cancel between cell and face integrals)
    Fc = ph.conv_flux(U.transpose(1, 2), PHYS.gamma)
    row = Fc.abs().amax(dim=(0, 1, 3))
    vol = (2 * math.pi) ** 3
    for c in (3, 4, 5, 6, 7):
        assert abs(float(d1[c] - d0[c])) <= 1e-13 * 3 * dt * vol * float(row[c - 3])
    assert float(d1[8]) == 0.0


def test_totals_equal_mass_matrix_sum():
    op, U = _tgv(2, 2)
    d = diagnostics.diagnostics(op, U)
    MU = op.mass_apply(U)
    assert torch.allclose(d[3:8], MU.sum((0, 2)), rtol=1e-13)


def test_nonfinite_count():
    op, U = _tgv(2, 2)
    U[0, 0, 0] = float("nan")
    U[1, 4, 3] = float("inf")
    assert float(diagnostics.diagnostics(op, U)[8]) == 2.0


def test_golden_tgv_constants():
    """The oracle's physical constants and closed forms match the paper's Sec. 4.2.1 values."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tgv_constants.json")))
    phys = ph.Physics.from_numbers(g["Re"], g["Pr"], g["Ma"], g["gamma"], g["R"], g["rho0"], g["U0"], g["L"])
    assert abs(phys.T_wall - g["T0"]) < 1e-15
    assert abs(g["rho0"] * g["R"] * phys.T_wall - g["p0"]) < 1e-12
    assert abs(0.75 * phys.nu - g["eps_0"]) < 1e-18
    assert abs(phys.mu * phys.c_p / phys.lam - g["Pr"]) < 1e-14


def test_dissipation_golden_reproduces_from_its_script():
    """The stored oracle history (tests/golden/tgv8_k5_dissipation.json) is what its committed script
    produces: rerun the oracle for the first 8 steps and compare the first two samples exactly."""
    import json
    import math
    import os

    from oracle import diagnostics as odiag
    from oracle import physics as ph
    from oracle import rk as ork
    from oracle.mesh import BoxMesh
    from oracle.operator import DGOperator
    from paper_1806_03095_gb300 import inputs
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    gold = json.load(open(os.path.join(here, "tgv8_k5_dissipation.json")))
    op = DGOperator(BoxMesh((8,) * 3, (-math.pi,) * 3, (math.pi,) * 3, (1, 1, 1), 5),
                    ph.Physics.from_numbers(1600.0, 0.71, 0.1), 8, 6)
    dt, every = gold["dt"], gold["every"]
    U = inputs.tgv_state(op.xyz)
    dU = U * 0.0
    got = []
    for n in range(every + 1):
        LU = op.L(U)
        if n % every == 0:
            got.append([float(v) for v in odiag.diagnostics(op, U, LU)[:3]])
        if n == every:
            break
        for i in range(ork.STAGES):
            dU = ork.A[i] * dU + dt * (LU if i == 0 else op.L(U))
            U = U + ork.B[i] * dU
    # exact on one machine; 1e-12 leaves room for a different reduction order on another host
    for s_got, row in zip(got, gold["samples"][:2]):
        for a, b in zip(s_got, row[2:5]):
            assert abs(a - b) <= 1e-12 * abs(b), (s_got, row)
