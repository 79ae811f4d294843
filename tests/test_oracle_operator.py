"""Pins of the oracle's weak form (Eq. WeakFormulationConservedVariables) against what
the paper and the mathematics fix: exact mass matrices, free-stream preservation,
discrete conservation, SIPG symmetry, closed-form penalty and point fluxes,
order-(k+1) convergence on manufactured and exact solutions.  Some tests plant a
mistake in the oracle (monkeypatch, CPU only) to show that the pin catches it."""
import math

import numpy as np
import pytest
import torch
from torch.func import jvp, vmap

from oracle import mms, physics as ph, rk
from oracle.basis import basis_3d, cell_points, face_points, gauss_legendre_01, lagrange_1d
from oracle.mesh import MAP_AFFINE, MAP_CHANNEL, MAP_SINE, BoxMesh, RotatedBoxMesh
from oracle.operator import WHAT_ALL, WHAT_CONV, WHAT_VISC, DGOperator
from paper_1806_03095_gb300 import inputs

TGV_PHYS = ph.Physics.from_numbers(1600.0, 0.71, 0.1)
PI = math.pi


def tgv_mesh(N, k, mapping=MAP_AFFINE, A=0.0):
    return BoxMesh((N,) * 3, [-PI] * 3, [PI] * 3, (1, 1, 1), k, mapping, A)


def make_op(mesh, phys=TGV_PHYS, nqc=None, nqv=None):
    k = mesh.k
    return DGOperator(mesh, phys, (3 * k) // 2 + 1 if nqc is None else nqc, k + 1 if nqv is None else nqv)


def const_state(Nc, n3):
    U = torch.empty((Nc, 5, n3), dtype=torch.float64)
    for c, v in enumerate((1.1, 0.3, -0.2, 0.1, 180.0)):
        U[:, c] = v
    return U


# -- point physics (Eq. CompressibleNavierStokesFluxes) --------------------------------------
def test_conv_flux_closed_form():
    g = 1.4
    rho, u, p = 2.0, torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64), 3.0
    rhoE = p / (g - 1) + 0.5 * rho * float((u * u).sum())
    U = torch.tensor([rho, *(rho * u).tolist(), rhoE], dtype=torch.float64)
    F = ph.conv_flux(U, g)
    assert torch.allclose(ph.pressure(U, g), torch.tensor(p, dtype=torch.float64))
    assert torch.allclose(F[0], rho * u)
    assert torch.allclose(F[1:4], rho * torch.outer(u, u) + p * torch.eye(3, dtype=torch.float64))
    assert torch.allclose(F[4], (rhoE + p) * u)
    assert torch.allclose(ph.sound_speed(U, g), torch.tensor(math.sqrt(g * p / rho), dtype=torch.float64))


def test_visc_flux_pure_shear_closed_form():
    """rho = 1, u = (s y, 0, 0), uniform T: tau_xy = mu s, energy flux (tau.u)_y = mu s^2 y, no heat flux."""
    phys = TGV_PHYS
    s, y = 0.7, 0.3
    u = torch.tensor([s * y, 0.0, 0.0], dtype=torch.float64)
    T = 2.0
    rhoE = phys.c_v * T + 0.5 * float((u * u).sum())
    U = torch.tensor([1.0, s * y, 0.0, 0.0, rhoE], dtype=torch.float64)
    G = torch.zeros((5, 3), dtype=torch.float64)
    G[1, 1] = s                      # d(rho u)/dy
    G[4, 1] = s * y * s              # d(rho E)/dy = u . du/dy
    F = ph.visc_flux(U, G, phys)
    expect = torch.zeros((5, 3), dtype=torch.float64)
    expect[1, 1] = expect[2, 0] = phys.mu * s
    expect[4, 1] = phys.mu * s * s * y
    assert torch.allclose(F, expect, atol=1e-15, rtol=1e-13)


def test_visc_flux_heat_conduction_closed_form():
    """Fluid at rest with grad T = (a, 0, 0) at constant rho: F_v = (0, 0, 0, 0, lambda grad T)."""
    phys = TGV_PHYS
    a, T = 0.4, 3.0
    U = torch.tensor([1.5, 0.0, 0.0, 0.0, 1.5 * phys.c_v * T], dtype=torch.float64)
    G = torch.zeros((5, 3), dtype=torch.float64)
    G[4, 0] = 1.5 * phys.c_v * a
    F = ph.visc_flux(U, G, phys)
    expect = torch.zeros((5, 3), dtype=torch.float64)
    expect[4, 0] = phys.lam * a
    assert torch.allclose(F, expect, atol=1e-15, rtol=1e-13)


def test_divergence_free_stress_trace():
    """tau is trace-free (zero bulk viscosity) for any velocity gradient."""
    phys = TGV_PHYS
    U = torch.tensor([1.2, 0.3, -0.1, 0.2, 200.0], dtype=torch.float64)
    G = inputs.uniform((5, 3), 3)
    F = ph.visc_flux(U, G, phys)
    assert abs(float(F[1, 0] + F[2, 1] + F[3, 2])) < 1e-15
    assert torch.allclose(F[1:4], F[1:4].T)


# -- mass matrix (Sec. 2.2.3, Sec. 2.3) -------------------------------------------------------
@pytest.mark.parametrize("k", [1, 3, 5])
def test_affine_mass_matrix_is_kron_of_1d(k):
    mesh = BoxMesh((2, 1, 1), [0, 0, 0], [2.0, 0.5, 0.25], (1, 1, 1), k)
    op = make_op(mesh)
    M = op.mass_matrices(torch.arange(1))[0].numpy()
    x, w = gauss_legendre_01(20)
    V, _ = lagrange_1d(mesh.nodes_1d, x)
    M1 = (V * w[:, None]).T @ V
    h = mesh.h
    Mref = np.kron(M1, np.kron(M1, M1)) * h[0] * h[1] * h[2]
    assert np.allclose(M, Mref, rtol=1e-13, atol=1e-16)


def test_mass_solve_inverts_mass_apply_deformed():
    mesh = tgv_mesh(2, 3, MAP_SINE, 0.05)
    op = make_op(mesh)
    U = inputs.random_state(mesh.Nc, mesh.n ** 3, 5)
    assert torch.allclose(op.mass_solve(op.mass_apply(U)), U, rtol=1e-12, atol=0)


# -- free stream (constant U gives F(U) = 0) -----------------------------------------------------
@pytest.mark.parametrize("mapping,A", [(MAP_AFFINE, 0.0), (MAP_SINE, 0.08)])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_free_stream_preservation(mapping, A, k):
    mesh = tgv_mesh(2, k, mapping, A)
    op = make_op(mesh)
    R = op.residual(const_state(mesh.Nc, mesh.n ** 3))
    assert float(R.abs().max()) < 5e-12


def test_free_stream_negative_control_underintegrated():
    """With nq = k+1 the deformed-mesh metric terms (degree 3k-1) are under-integrated: F(U0) != 0."""
    mesh = tgv_mesh(2, 3, MAP_SINE, 0.08)
    op = make_op(mesh, nqc=4)
    assert float(op.residual(const_state(mesh.Nc, mesh.n ** 3)).abs().max()) > 1e-3


def test_free_stream_channel_mesh():
    mesh = BoxMesh((2, 3, 2), [0, -1, 0], [2 * PI, 1, PI], (1, 0, 1), 3, MAP_CHANNEL, 1.8)
    phys = ph.Physics.from_numbers(180.0, 0.71, 0.1, u_mach=18.3)
    op = make_op(mesh, phys)
    U = const_state(mesh.Nc, mesh.n ** 3)
    U[:, 1:4] = 0.0       # at rest: the wall state mirrors to itself only for u = 0 ...
    U[:, 4] = 1.1 * phys.c_v * phys.T_wall  # ... and T = T_wall
    R = op.residual(U)
    assert float(R.abs().max()) < 1e-13 * float(U.abs().max())


# -- conservation (V = 1 lies in the test space) ------------------------------------------------
@pytest.mark.parametrize("mapping,A", [(MAP_AFFINE, 0.0), (MAP_SINE, 0.08)])
def test_discrete_conservation_periodic(mapping, A):
    mesh = tgv_mesh(3, 3, mapping, A)
    op = make_op(mesh)
    U = inputs.random_state(mesh.Nc, mesh.n ** 3, 11)
    R = op.residual(U)
    tot = R.sum((0, 2))
    scale = R.abs().sum((0, 2))
    assert torch.all(tot.abs() <= 1e-13 * scale)


@pytest.mark.parametrize("k,A", [(8, 0.0), (8, 0.05), (11, 0.0)])
def test_free_stream_and_conservation_high_degree(k, A):
    """The degrees of the global-workspace kernels (default rule q_c = floor(3k/2)+1, q_v = k+1): free-stream
    preservation and discrete conservation of a random state on 2^3 periodic cells, affine and deformed."""
    mesh = tgv_mesh(2, k, MAP_SINE if A else MAP_AFFINE, A)
    op = make_op(mesh)
    R = op.residual(const_state(mesh.Nc, mesh.n ** 3))
    assert float(R.abs().max()) < 5e-11
    R = op.residual(inputs.random_state(mesh.Nc, mesh.n ** 3, 12))
    assert torch.all(R.sum((0, 2)).abs() <= 1e-12 * R.abs().sum((0, 2)))


def test_channel_wall_conserves_mass():
    mesh = BoxMesh((2, 2, 2), [0, -1, 0], [2 * PI, 1, PI], (1, 0, 1), 3, MAP_CHANNEL, 1.8)
    phys = ph.Physics.from_numbers(180.0, 0.71, 0.1, u_mach=18.3, body_force=(1.0, 0.0, 0.0))
    op = make_op(mesh, phys)
    U = inputs.channel_state(torch.as_tensor(mesh.xyz), 1806)
    R = op.residual(U)
    assert abs(float(R[:, 0].sum())) <= 1e-13 * float(R[:, 0].abs().sum())
    # body force: sum_i (V_i, F_rhs) = int F_rhs, i.e. f1 * volume for the x-momentum row
    Fr = op.body_force(U)
    assert abs(float(Fr[:, 1].sum()) - mesh.volume()) < 1e-11 * mesh.volume()


def test_conservation_negative_control_one_sided_lambda(monkeypatch):
    """Planted mistake: LLF wave speed from the own side only -> face fluxes no longer single-valued."""
    mesh = tgv_mesh(2, 2)
    op = make_op(mesh)
    U = inputs.random_state(mesh.Nc, mesh.n ** 3, 12)
    monkeypatch.setattr(torch, "maximum", lambda a, b: a)
    R = op.residual(U, WHAT_CONV)
    monkeypatch.undo()
    assert float(R[:, 0].sum().abs()) > 1e-8 * float(R[:, 0].abs().sum())


# -- SIPG symmetry of the viscous bilinear form -------------------------------------------------
def _linearised_visc(op, U0, W):
    return jvp(lambda V: op.residual(V, WHAT_VISC), (U0,), (W,))[1]


def _momentum_only(shape, seed):
    W = inputs.uniform(shape, seed)
    W[:, 0] = 0.0
    W[:, 4] = 0.0
    return W


@pytest.mark.parametrize("mapping,A", [(MAP_AFFINE, 0.0), (MAP_SINE, 0.06)])
def test_sipg_momentum_block_symmetric(mapping, A):
    """At rest (u = 0) the momentum block of the linearised viscous operator is the SIPG
    discretisation of the Lame operator, which is symmetric: <V, A W> = <W, A V>."""
    mesh = tgv_mesh(2, 2, mapping, A)
    op = make_op(mesh)
    U0 = const_state(mesh.Nc, mesh.n ** 3)
    U0[:, 1:4] = 0.0
    V = _momentum_only(U0.shape, 1)
    W = _momentum_only(U0.shape, 2)
    a_vw = float((V * _linearised_visc(op, U0, W)).sum())
    a_wv = float((W * _linearised_visc(op, U0, V)).sum())
    assert abs(a_vw - a_wv) <= 1e-12 * abs(a_vw)


def test_sipg_symmetry_negative_control_dropped_half_term(monkeypatch):
    """Planted mistake: drop the -1/2 (grad V, F_v(U, [[U]])) face term -> form is no longer symmetric."""
    mesh = tgv_mesh(2, 2)
    op = make_op(mesh)
    face_grads = [op.face_tables(op.nq_visc, d, s)[1] for d in range(3) for s in range(2)]
    orig = DGOperator.test_grad

    def patched(grad, Jinv, F, wdet):
        out = orig(grad, Jinv, F, wdet)
        return out * 0.0 if any(grad is g for g in face_grads) else out

    monkeypatch.setattr(DGOperator, "test_grad", staticmethod(patched))
    U0 = const_state(mesh.Nc, mesh.n ** 3)
    U0[:, 1:4] = 0.0
    V = _momentum_only(U0.shape, 1)
    W = _momentum_only(U0.shape, 2)
    a_vw = float((V * _linearised_visc(op, U0, W)).sum())
    a_wv = float((W * _linearised_visc(op, U0, V)).sum())
    assert abs(a_vw - a_wv) > 1e-6 * abs(a_vw)


# -- penalty (Eq. TauIP_Element) -----------------------------------------------------------------
def test_tau_ip_affine_cube():
    mesh = tgv_mesh(4, 3)
    op = make_op(mesh)
    h = 2 * PI / 4
    assert torch.allclose(op.tau_cell, torch.full_like(op.tau_cell, 3 * TGV_PHYS.nu * 16 / h), rtol=1e-13)


def test_tau_ip_channel_wall_cells():
    mesh = BoxMesh((2, 4, 2), [0, -1, 0], [2 * PI, 1, PI], (1, 0, 1), 3, MAP_CHANNEL, 1.8)
    phys = ph.Physics.from_numbers(180.0, 0.71, 0.1, u_mach=18.3)
    op = make_op(mesh, phys)
    hx, hz = PI, PI / 2
    yedges = np.tanh(1.8 * (2 * np.linspace(0, 1, 5) - 1)) / np.tanh(1.8)
    cc = mesh.cell_coords()
    for e in range(mesh.Nc):
        cy = cc[e, 1]
        dy = yedges[cy + 1] - yedges[cy]
        vol = hx * hz * dy
        wall = cy in (0, 3)
        a_int = 2 * hx * dy + 2 * hz * dy + (1 if wall else 2) * hx * hz
        a_bnd = hx * hz if wall else 0.0
        expect = phys.nu * 16 * (0.5 * a_int + a_bnd) / vol
        assert abs(float(op.tau_cell[e]) - expect) < 1e-12 * expect


# -- convergence (order k+1) -----------------------------------------------------------------------
def _l2_error(op, U, exact_fun):
    nq = op.k + 3
    pts, w = cell_points(nq)
    phi, grad = basis_3d(op.mesh.nodes_1d, pts)
    phi, grad, w = torch.as_tensor(phi), torch.as_tensor(grad), torch.as_tensor(w)
    wdet = torch.abs(torch.linalg.det(op.jacobian(op.xyz, grad))) * w
    xq = torch.einsum("pn,ean->epa", phi, op.xyz)
    Uh = torch.einsum("pn,ecn->epc", phi, U)
    return math.sqrt(float(((Uh - exact_fun(xq)) ** 2 * wdet[..., None]).sum()))


MMS_PHYS = ph.Physics(gamma=1.4, R=1.0, mu=0.01, lam=0.01 * 3.5 / 0.71, rho0=1.0)


def _mms_error(N, k, mapping, A, T=0.1, nsteps=10, plant=None):
    """L2 error after integrating the steady manufactured problem; ``plant`` (a context
    manager factory) is entered after the exact source is computed, so a planted
    mistake changes the discrete operator only."""
    mesh = BoxMesh((N,) * 3, [0.0] * 3, [2 * PI] * 3, (1, 1, 1), k, mapping, A)
    op = make_op(mesh, MMS_PHYS)
    U = mms.steady_exact(torch.as_tensor(mesh.xyz), MMS_PHYS.gamma)
    S = op.body_force(U, mms.steady_source(MMS_PHYS))
    dt = T / nsteps
    import contextlib
    with (plant() if plant is not None else contextlib.nullcontext()):
        for i in range(nsteps):
            U = rk.step(lambda V, t: op.mass_solve(-op.residual(V) + S), U, dt, i * dt)
    Uf = vmap(mms.conserved(mms.steady_primitive, MMS_PHYS.gamma))
    return _l2_error(op, U, lambda xq: Uf(xq.reshape(-1, 3)).reshape(xq.shape[:-1] + (5,)))


@pytest.mark.slow
@pytest.mark.parametrize("k,mapping,A", [(2, MAP_AFFINE, 0.0), (3, MAP_SINE, 0.04)])
def test_mms_navier_stokes_order(k, mapping, A):
    e = [_mms_error(N, k, mapping, A) for N in (2, 4, 8)]
    order = math.log2(e[1] / e[2])
    assert order > k + 0.7, (e, order)


def _truncation_error(N, k, mapping, A):
    """|| L(I U_ex) + M^{-1}(V, S) ||_M for the steady manufactured field (one operator evaluation)."""
    mesh = BoxMesh((N,) * 3, [0.0] * 3, [2 * PI] * 3, (1, 1, 1), k, mapping, A)
    op = make_op(mesh, MMS_PHYS)
    U = mms.steady_exact(torch.as_tensor(mesh.xyz), MMS_PHYS.gamma)
    S = op.body_force(U, mms.steady_source(MMS_PHYS))
    D = op.mass_solve(-op.residual(U) + S)
    return math.sqrt(float((D * op.mass_apply(D)).sum()))


@pytest.mark.parametrize("k,mapping,A", [(2, MAP_AFFINE, 0.0), (3, MAP_AFFINE, 0.0), (3, MAP_SINE, 0.04)])
def test_mms_truncation_error_order_k(k, mapping, A):
    """The DG truncation error of the interpolated manufactured solution decays like h^k."""
    e = [_truncation_error(N, k, mapping, A) for N in (2, 4, 8)]
    assert math.log2(e[1] / e[2]) > k - 0.4, e


def test_mms_negative_control_energy_flux_without_pressure(monkeypatch):
    """Planted mistake: energy flux rho E u instead of (rho E + p) u -> truncation error stalls."""
    orig = ph.conv_flux
    src = mms.steady_source(MMS_PHYS)  # exact source from the correct flux

    def bad(U, gamma):
        F = orig(U, gamma)
        p = ph.pressure(U, gamma)
        return torch.cat([F[..., :4, :], (F[..., 4, :] - p[..., None] * U[..., 1:4] / U[..., 0:1])[..., None, :]], -2)

    errs = []
    for N in (4, 8):
        mesh = BoxMesh((N,) * 3, [0.0] * 3, [2 * PI] * 3, (1, 1, 1), 3)
        op = make_op(mesh, MMS_PHYS)
        U = mms.steady_exact(torch.as_tensor(mesh.xyz), MMS_PHYS.gamma)
        S = op.body_force(U, src)
        monkeypatch.setattr(ph, "conv_flux", bad)
        D = op.mass_solve(-op.residual(U) + S)
        monkeypatch.undo()
        errs.append(math.sqrt(float((D * op.mass_apply(D)).sum())))
    assert math.log2(errs[0] / errs[1]) < 1.0, errs


def _entropy_wave_error(N, k, T=0.05, nsteps=5):
    phys = ph.Physics(gamma=1.4, R=1.0, mu=0.0, lam=0.0, rho0=1.0)
    mesh = BoxMesh((N,) * 3, [0.0] * 3, [2 * PI] * 3, (1, 1, 1), k)
    op = make_op(mesh, phys)
    U = mms.entropy_wave_exact(torch.as_tensor(mesh.xyz), 0.0, phys.gamma)
    dt = T / nsteps
    for i in range(nsteps):
        U = rk.step(lambda V, t: op.L(V, WHAT_CONV), U, dt, i * dt)

    def exact(xq):
        return mms.entropy_wave_exact(xq.permute(0, 2, 1), T, phys.gamma).permute(0, 2, 1)

    return _l2_error(op, U, exact)


def test_euler_entropy_wave_order():
    e = [_entropy_wave_error(N, 2) for N in (2, 4, 8)]
    assert math.log2(e[1] / e[2]) > 2.6, e


# -- L(U) assembly -------------------------------------------------------------------------------
def test_L_is_minus_Minv_F_without_forcing():
    mesh = tgv_mesh(2, 2)
    op = make_op(mesh)
    U = inputs.random_state(mesh.Nc, mesh.n ** 3, 4)
    assert torch.allclose(op.mass_apply(op.L(U)), -op.residual(U), rtol=1e-11, atol=1e-11)


def test_what_splits_add_up():
    mesh = tgv_mesh(2, 2)
    op = make_op(mesh)
    U = inputs.random_state(mesh.Nc, mesh.n ** 3, 6)
    assert torch.allclose(op.residual(U, WHAT_CONV) + op.residual(U, WHAT_VISC), op.residual(U), rtol=1e-12, atol=1e-11)


def test_oracle_tangent_linear_model_matches_finite_differences():
    """The oracle's forward-mode derivative of L (used as the adjoint's reference) against central differences."""
    mesh = tgv_mesh(2, 2)
    op = make_op(mesh)
    U = inputs.random_state(mesh.Nc, mesh.n ** 3, 90)
    V = inputs.uniform(U.shape, 91)
    JV = jvp(op.L, (U,), (V,))[1]
    h = 1e-6
    fd = (op.L(U + h * V) - op.L(U - h * V)) / (2 * h)
    assert float(torch.linalg.norm(JV - fd) / torch.linalg.norm(JV)) < 1e-7


# -- body force (Sec. 2.1: F_rhs = (0, f, f.u)) -------------------------------------------------------------
BF_PHYS = ph.Physics.from_numbers(180.0, 0.71, 0.1, u_mach=18.3, body_force=(0.7, -0.4, 1.3))


def _linear_flow(xyz, rho=2.0):
    """rho constant, u = a + B x (degree 1 in x, so degree k in the reference coordinates of a degree-k
    isoparametric cell: the nodal field is exact), p from a constant temperature."""
    a = torch.tensor([0.3, -1.1, 0.8], dtype=torch.float64)
    B = torch.tensor([[0.5, -0.2, 0.1], [0.3, 0.4, -0.6], [-0.7, 0.2, 0.9]], dtype=torch.float64)
    u = a[None, :, None] + torch.einsum("ab,ebn->ean", B, xyz)
    U = torch.empty((xyz.shape[0], 5, xyz.shape[2]), dtype=torch.float64)
    U[:, 0] = rho
    U[:, 1:4] = rho * u
    U[:, 4] = rho * (BF_PHYS.c_v * 300.0 + 0.5 * (u * u).sum(1))
    return U, u, a, B


def _body_force_pins_hold(op, mesh, centroid):
    f = torch.tensor(BF_PHYS.body_force, dtype=torch.float64)
    U, u, a, B = _linear_flow(torch.as_tensor(mesh.xyz))
    Fr = op.body_force(U)
    nodal = op.mass_solve(Fr)
    # M^-1 (V, F_rhs): density row 0, momentum rows f, energy row f . u at every node (f . u lies in the
    # space, and M and the load use the same k+1 point rule)
    ok = bool(torch.allclose(nodal[:, 0], torch.zeros_like(nodal[:, 0]), atol=1e-12))
    for d in range(3):
        ok &= bool(torch.allclose(nodal[:, 1 + d], f[d].expand_as(nodal[:, 1 + d]), rtol=1e-12, atol=1e-12))
    ok &= bool(torch.allclose(nodal[:, 4], torch.einsum("a,ean->en", f, u), rtol=1e-11, atol=1e-11))
    # v = 1: the energy row sums to int f . u = |Omega| f . (a + B x_centroid)
    if centroid is not None:
        exact = mesh.volume() * float(f @ (a + B @ torch.as_tensor(centroid, dtype=torch.float64)))
        ok &= abs(float(Fr[:, 4].sum()) - exact) <= 1e-12 * abs(exact)
    return ok


@pytest.mark.parametrize("mapping,A", [(MAP_AFFINE, 0.0), (MAP_CHANNEL, 1.8)])
def test_body_force_rows(mapping, A):
    """(V, F_rhs) with F_rhs = (0, f, f.u) on a linear flow at constant density 2: every nodal row of
    M^{-1}(V, F_rhs) is its closed form, and on the affine box the energy row integrates to int f.u."""
    mesh = BoxMesh((2, 3, 2), [0.0, -1.0, 0.0], [2.0, 1.0, 1.0], (1, 0, 1), 3, mapping, A)
    op = make_op(mesh, BF_PHYS)
    assert _body_force_pins_hold(op, mesh, (1.0, 0.0, 0.5) if mapping == MAP_AFFINE else None)


@pytest.mark.parametrize("mistake", ["f.m", "sign"])
def test_body_force_negative_control(monkeypatch, mistake):
    """Planted mistakes in the energy row: f.m for f.u (a factor rho = 2 here) and a flipped sign."""
    mesh = BoxMesh((2, 3, 2), [0.0, -1.0, 0.0], [2.0, 1.0, 1.0], (1, 0, 1), 3, MAP_AFFINE, 0.0)
    op = make_op(mesh, BF_PHYS)
    orig = DGOperator.body_force_cells

    def planted(self, U, E, source=None, t=0.0):
        r = orig(self, U, E, source, t)
        r[:, 4] = r[:, 4] * (U[E][:, 0, :1] if mistake == "f.m" else -1.0)
        return r

    monkeypatch.setattr(DGOperator, "body_force_cells", planted)
    assert not _body_force_pins_hold(op, mesh, (1.0, 0.0, 0.5))


# -- isothermal no-slip wall: the mirror reading (Sec. 4.3.1) -----------------------------------------------
def _wall_pins_hold(ghost):
    """For random interior states: rho+ = rho-, the face averages are u = 0 and T = T_wall, and the LLF
    mass flux through the wall, {{m}}.n + Lambda/2 (rho- - rho+), vanishes for any normal."""
    phys = BF_PHYS
    r = inputs.uniform((4096, 5), 31)
    rho = 1.0 + 0.5 * r[:, 0]
    u = 20.0 * r[:, 1:4]
    T = phys.T_wall * (1.0 + 0.3 * r[:, 4])
    Um = torch.cat([rho[:, None], rho[:, None] * u, (rho * (phys.c_v * T + 0.5 * (u * u).sum(1)))[:, None]], 1)
    Up = ghost(Um, phys)
    rp = Up[:, 0]
    up = Up[:, 1:4] / rp[:, None]
    Tp = (Up[:, 4] / rp - 0.5 * (up * up).sum(1)) / phys.c_v
    n = inputs.uniform((4096, 3), 32)
    n = n / torch.linalg.norm(n, dim=1, keepdim=True)
    lam = torch.linalg.norm(u, dim=1) + ph.sound_speed(Um, phys.gamma)
    mass_flux = 0.5 * ((Um[:, 1:4] + Up[:, 1:4]) * n).sum(1) + 0.5 * lam * (Um[:, 0] - rp)
    return (bool(torch.equal(rp, rho)) and float((0.5 * (u + up)).abs().max()) < 1e-12
            and float((0.5 * (T + Tp) - phys.T_wall).abs().max()) < 1e-9 * phys.T_wall
            and float(mass_flux.abs().max()) < 1e-12)


def test_wall_ghost_state_reading():
    assert _wall_pins_hold(ph.wall_ghost_state)


def test_wall_ghost_state_negative_controls():
    """Planted mistakes: T+ = T_wall - T-, and a mirror of the first velocity component only."""
    def state(rho, m, T, phys):
        u = m / rho[:, None]
        return torch.cat([rho[:, None], m, (rho * (phys.c_v * T + 0.5 * (u * u).sum(1)))[:, None]], 1)

    def temperature(U, phys):
        u = U[:, 1:4] / U[:, 0:1]
        return (U[:, 4] / U[:, 0] - 0.5 * (u * u).sum(1)) / phys.c_v

    def half_temperature(U, phys):
        return state(U[:, 0], -U[:, 1:4], phys.T_wall - temperature(U, phys), phys)

    def first_component_only(U, phys):
        m = U[:, 1:4].clone()
        m[:, 0] = -m[:, 0]
        return state(U[:, 0], m, 2.0 * phys.T_wall - temperature(U, phys), phys)

    assert not _wall_pins_hold(half_temperature)
    assert not _wall_pins_hold(first_component_only)


# -- rotated-frame meshes ---------------------------------------------------------------------------------------
ROT_NC, ROT_LO, ROT_HI = (3, 2, 4), (-1.0, 0.0, 0.5), (2.0, 1.5, 2.5)


def _rotated_invariance_gap(mesh_cls=RotatedBoxMesh, op_cls=DGOperator, k=3, qc=5, qv=4, seed=1806, deform=0.0):
    """Max-norm gap, relative to max |L|, between L on a rotated-frame box and L on the same box with aligned
    frames (both moved by the same sine deformation), for a random discontinuous state carried node by node
    into the rotated frames.  Nodes are matched by their physical coordinates.  Q_k and the tensor Gauss rules
    are invariant under the 48 symmetries of the cube, the node set too, so both meshes interpolate the same
    geometry; the weak form is written in physical space, so the two operators agree up to rounding."""
    Nc = int(np.prod(ROT_NC))
    m0 = BoxMesh(ROT_NC, ROT_LO, ROT_HI, (1, 1, 1), k, MAP_SINE, deform)
    mr = mesh_cls(ROT_NC, ROT_LO, ROT_HI, k, inputs.cell_frames(Nc, seed), deform=deform)
    dist = np.linalg.norm(mr.xyz[:, :, :, None] - m0.xyz[:, :, None, :], axis=1)  # [Nc, n^3 (rotated), n^3]
    assert dist.min(2).max() < 1e-14
    perm = torch.as_tensor(dist.argmin(2))
    assert torch.equal(perm.sort(1).values, torch.arange(m0.n ** 3).expand(Nc, -1))
    idx = perm[:, None, :].expand(-1, 5, -1)
    phys = ph.Physics.from_numbers(1600.0, 0.71, 0.1)
    U0 = inputs.random_state(Nc, m0.n ** 3, 3)
    L0 = DGOperator(m0, phys, qc, qv).L(U0)
    Lr = op_cls(mr, phys, qc, qv).L(torch.gather(U0, 2, idx))
    return float((Lr - torch.gather(L0, 2, idx)).abs().max() / L0.abs().max())


def test_rotated_frames_cover_reflections_and_cycles():
    """The seeded frames of a 4096-cell mesh take all 48 values, so the pins below meet odd and even
    permutations, 3-cycles and every reflection pattern."""
    fr = inputs.cell_frames(4096, 1806)
    assert set(fr.tolist()) == set(range(48))
    mr = RotatedBoxMesh(ROT_NC, ROT_LO, ROT_HI, 3, inputs.cell_frames(24, 1806))
    assert len(set((mr.frames // 8).tolist())) >= 4 and mr.flip.any(0).all()


@pytest.mark.parametrize("k,qc,qv,deform", [(3, 5, 4, 0.0), (2, 3, 3, 0.0), (3, 5, 4, 0.05), (2, 4, 3, 0.08),
                                           (1, 2, 2, 0.0), (4, 7, 5, 0.04)])
def test_rotated_frame_operator_invariance(k, qc, qv, deform):
    assert _rotated_invariance_gap(k=k, qc=qc, qv=qv, deform=deform) < 1e-12


def test_rotated_frame_located_points_are_physical_matches():
    """On the deformed rotated-frame mesh, every located neighbour point maps (through the neighbour's own
    degree-k geometry) to the physical position of the face point it stands for (through this cell's)."""
    Nc = int(np.prod(ROT_NC))
    mr = RotatedBoxMesh(ROT_NC, ROT_LO, ROT_HI, 3, inputs.cell_frames(Nc, 1806), deform=0.08)
    E = np.arange(Nc)
    L = mr.hi - mr.lo
    for d in range(3):
        for s in range(2):
            pts, _ = face_points(5, d, s)
            nb = mr.nbr[:, d, s]
            zeta = mr.from_box(nb, mr.to_box(E, pts) - mr.offset[:, d, s][:, None, :])
            x_own = np.einsum("pn,ean->epa", basis_3d(mr.nodes_1d, pts)[0], mr.xyz)
            phi_n = basis_3d(mr.nodes_1d, zeta.reshape(-1, 3))[0].reshape(Nc, len(pts), -1)
            x_nb = np.einsum("epn,ean->epa", phi_n, mr.xyz[nb])
            gap = (x_nb - x_own) / L
            gap -= np.round(gap)  # across the periodic boundary
            assert np.abs(gap).max() < 1e-13, (d, s)


def test_rotated_frame_neighbours_are_geometric():
    """Every local face of every cell has a neighbour whose facing face coincides with it: the six face
    centres of the neighbour contain this face's centre, and the relation is symmetric."""
    Nc = int(np.prod(ROT_NC))
    mr = RotatedBoxMesh(ROT_NC, ROT_LO, ROT_HI, 3, inputs.cell_frames(Nc, 1806))
    E = np.arange(Nc)

    def face_centres(cells):
        out = []
        for d in range(3):
            for s in range(2):
                c = np.full((1, 3), 0.5)
                c[0, d] = float(s)
                eta = mr.to_box(cells, c)[:, 0, :]
                out.append((mr.cell_coords()[cells] + eta) % np.asarray(ROT_NC))
        return np.stack(out, 1)  # [len(cells), 6, 3] box coordinates, wrapped

    own = face_centres(E)
    for d in range(3):
        for s in range(2):
            nb = mr.nbr[:, d, s]
            theirs = face_centres(nb)
            gap = np.abs(theirs - own[:, None, 2 * d + s, :])
            gap = np.minimum(gap, np.asarray(ROT_NC) - gap).max(2)  # periodic distance
            assert (gap.min(1) < 1e-12).all()
            back = np.array([mr.nbr[n].reshape(-1) for n in nb])
            assert (back == E[:, None]).any(1).all()


class _NoReflection(RotatedBoxMesh):
    """Planted mistake: neighbours located without their reflections."""
    def from_box(self, E, eta):
        E = np.asarray(E)
        xi = np.empty_like(eta)
        np.put_along_axis(xi, np.broadcast_to(self.perm[E][:, None, :], eta.shape), eta, axis=2)
        return xi


class _InversePermutation(RotatedBoxMesh):
    """Planted mistake: the neighbour's axis permutation applied instead of its inverse."""
    def from_box(self, E, eta):
        E = np.asarray(E)
        val = np.where(self.flip[E][:, None, :], 1.0 - eta, eta)
        return np.take_along_axis(val, np.broadcast_to(self.perm[E][:, None, :], val.shape), axis=2)


class _AlignedNeighbour(DGOperator):
    """Planted mistake: the neighbour's trace taken on its own face (d, 1 - s) in this face's point order, as
    on a mesh with aligned frames."""
    def _exterior_located(self, U, E, d, s, nq):
        nb = self.nbr[E, d, s]
        phi, grad, _ = self.face_tables(nq, d, 1 - s)
        Jinv = torch.linalg.inv(self.jacobian(self.xyz[nb], grad))
        return self.values(phi, U[nb]), self.gradients(grad, Jinv, U[nb]), torch.ones(len(E), dtype=torch.bool), nb


def test_rotated_frame_negative_controls():
    assert _rotated_invariance_gap(mesh_cls=_NoReflection) > 1e-3
    assert _rotated_invariance_gap(mesh_cls=_NoReflection, deform=0.05) > 1e-3
    assert _rotated_invariance_gap(mesh_cls=_InversePermutation) > 1e-3
    assert _rotated_invariance_gap(op_cls=_AlignedNeighbour) > 1e-3
