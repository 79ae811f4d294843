"""Adjoint of the CUDA operator (through the C ABI) against the oracle's automatic
differentiation: the vector-Jacobian product of L (reverse mode of the oracle), the
RK stage adjoint, the kinetic-energy gradient, and the full discrete adjoint of the
RK(5,4) integration with checkpointing against the oracle's tangent-linear model
(forward mode) and central finite differences."""
import math

import pytest
import torch
from torch.func import jvp

from oracle import physics as ph, rk as ork
from oracle.mesh import BoxMesh
from oracle.operator import DGOperator
from paper_1806_03095_gb300 import inputs

pytestmark = pytest.mark.gpu
PI = math.pi

if torch.cuda.is_available():
    from paper_1806_03095_gb300 import adjoint as adj
    from paper_1806_03095_gb300.api import DGCNS


def rel(a, b):
    a, b = a.detach().double().cpu(), b.detach().double().cpu()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b)), float((a - b).abs().max() / b.abs().max())


def pair(ncells, k, mapping=0, param=0.0, periodic=(1, 1, 1), lo=(-PI,) * 3, hi=(PI,) * 3, precision=0,
         Re=1600.0, u_mach=0.0, kernel=1):
    """kernel 1: element-centric adjoint kernel; kernel 2: face-centric adjoint face kernel + cell kernel."""
    qc, qv = (3 * k) // 2 + 1, k + 1
    g = DGCNS(ncells, lo, hi, periodic, k, qc, qv, Re=Re, u_mach=u_mach, precision=precision, mapping=mapping,
              map_param=param, kernel=kernel)
    mesh = BoxMesh(ncells, lo, hi, periodic, k, mapping, param)
    return g, DGOperator(mesh, ph.Physics.from_numbers(Re, 0.71, 0.1, u_mach=(u_mach or None)), qc, qv)


def oracle_vjp(op, U, W):
    Ur = U.clone().requires_grad_(True)
    return torch.autograd.grad(op.L(Ur), Ur, W)[0]


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("k", [2, 3])
def test_adjoint_apply_matches_oracle_vjp(k, kernel):
    g, op = pair((2, 2, 3), k, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 60 + k)
    W = inputs.uniform(U.shape, 61 + k)
    l2, mx = rel(g.adjoint_apply(U.cuda(), W.cuda()), oracle_vjp(op, U, W))
    assert l2 < 1e-12 and mx < 1e-12, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
def test_adjoint_dot_product_identity_with_oracle_tlm(kernel):
    """<W, J V> (oracle forward mode) = <J^T W, V> (CUDA adjoint)."""
    g, op = pair((2, 2, 2), 3, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 70)
    V = inputs.uniform(U.shape, 71)
    W = inputs.uniform(U.shape, 72)
    JV = jvp(op.L, (U,), (V,))[1]
    lhs = float((W * JV).sum())
    rhs = float((g.adjoint_apply(U.cuda(), W.cuda()).cpu() * V).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("kernel", [1, 2])
def test_adjoint_apply_walls(kernel):
    g, op = pair((2, 3, 2), 3, periodic=(1, 0, 1), lo=(0, -1, 0), hi=(2 * PI, 1, PI), Re=180.0, u_mach=18.3,
                 kernel=kernel)
    U = inputs.channel_state(g.node_coords().cpu(), 5)
    W = inputs.uniform(U.shape, 73)
    l2, mx = rel(g.adjoint_apply(U.cuda(), W.cuda()), oracle_vjp(op, U, W))
    assert l2 < 1e-11 and mx < 1e-11, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
def test_adjoint_apply_walls_on_every_side(kernel):
    """Walls on all six sides of a ragged 3x2x4 box (lower-wall faces of the face-centric kernel)."""
    g, op = pair((3, 2, 4), 2, periodic=(0, 0, 0), lo=(0, 0, 0), hi=(1.5, 1.0, 2.0), Re=180.0, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 78)
    W = inputs.uniform(U.shape, 79)
    l2, mx = rel(g.adjoint_apply(U.cuda(), W.cuda()), oracle_vjp(op, U, W))
    assert l2 < 1e-11 and mx < 1e-11, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
def test_adjoint_apply_deformed_mesh(kernel):
    g, op = pair((2, 2, 2), 3, mapping=2, param=0.05, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 74)
    W = inputs.uniform(U.shape, 75)
    l2, mx = rel(g.adjoint_apply(U.cuda(), W.cuda()), oracle_vjp(op, U, W))
    assert l2 < 1e-12 and mx < 1e-12, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
def test_adjoint_apply_mixed_precision(kernel):
    g, op = pair((2, 2, 2), 3, precision=1, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 76)
    W = inputs.uniform(U.shape, 77)
    l2, mx = rel(g.adjoint_apply(U.cuda(), W.float().cuda()), oracle_vjp(op, U, W))
    assert l2 < 1e-4 and mx < 1e-3, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("stage", [0, 3])
def test_rk_stage_adjoint_matches_oracle(stage, kernel):
    g, op = pair((2, 2, 2), 2, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 80)
    dU = 1e-2 * inputs.uniform(U.shape, 81)
    lamU = inputs.uniform(U.shape, 82)
    lamdU = inputs.uniform(U.shape, 83)
    dt = 1e-3
    Ur = U.clone().requires_grad_(True)
    dUr = dU.clone().requires_grad_(True)
    dUn = ork.A[stage] * dUr + dt * op.L(Ur)
    Un = Ur + ork.B[stage] * dUn
    gU, gdU = torch.autograd.grad((Un, dUn), (Ur, dUr), (lamU, lamdU))
    lu, ld = lamU.cuda(), lamdU.cuda()
    g.rk_stage_adjoint(stage, dt, U.cuda(), lu, ld)
    assert max(rel(lu, gU)) < 1e-12
    if stage == 0:
        assert float(ld.abs().max()) == 0.0
    else:
        assert max(rel(ld, gdU)) < 1e-12


def oracle_ek(op, U):
    phi, _, _ = op.cell_tables(op.nq_conv)
    tot, vol = 0.0, 0.0
    for E in op._chunks():
        _, wdet = op.cell_geometry(E, op.nq_conv)
        Uq = op.values(phi, U[E])
        u = Uq[..., 1:4] / Uq[..., 0:1]
        tot = tot + (0.5 * (u * u).sum(-1) * wdet).sum()
        vol = vol + wdet.sum()
    return tot / vol


@pytest.mark.parametrize("mapping,param", [(0, 0.0), (2, 0.05)])
def test_kinetic_energy_gradient(mapping, param):
    g, op = pair((2, 2, 2), 3, mapping=mapping, param=param)
    U = inputs.tgv_state(op.xyz) + 1e-3 * inputs.uniform((op.mesh.Nc, 5, op.mesh.n ** 3), 84)
    Ur = U.clone().requires_grad_(True)
    ref = torch.autograd.grad(oracle_ek(op, Ur), Ur)[0]
    assert max(rel(g.kinetic_energy_gradient(U.cuda()), ref)) < 1e-12


# -- full discrete adjoint: d e_k(U(T)) / d u0 ---------------------------------------------------------------
def control_to_state(u0, rho, T0, cv):
    """Initial state from the nodal velocity field u0 [Nc, 3, n^3] at fixed density and temperature."""
    m = rho[:, None] * u0
    rhoE = rho * (cv * T0 + 0.5 * (u0 * u0).sum(1))
    return torch.cat([rho[:, None], m, rhoE[:, None]], 1)


def _setup_tgv_adjoint(N=4, k=4, kernel=1):
    g, op = pair((N, N, N), k, kernel=kernel)
    U0 = inputs.tgv_state(op.xyz)
    rho = U0[:, 0].clone()
    u0 = U0[:, 1:4] / rho[:, None]
    cv = op.phys.c_v
    T0 = op.phys.T_wall
    return g, op, rho, u0, T0, cv


_TLM_CACHE = {}


@pytest.mark.parametrize("kernel", [1, 2])
def test_full_adjoint_gradient_vs_oracle_tlm_and_fd(kernel):
    """TGV 4^3, k = 4: 6 RK(5,4) steps with checkpoints every 2 steps; gradient of the final kinetic energy
    with respect to the initial velocity field, along 8 seeded unit directions (the oracle's directional
    derivatives are computed once and reused for both kernel organisations)."""
    g, op, rho, u0, T0, cv = _setup_tgv_adjoint(kernel=kernel)
    dt = 2e-3
    nsteps, every = 6, 2
    rho_g, u0_g = rho.cuda(), u0.cuda().requires_grad_(True)
    UT = adj.integrate(g, control_to_state(u0_g, rho_g, T0, cv).contiguous(), nsteps, dt, every)
    J = adj.kinetic_energy(g, UT)
    J.backward()
    grad = u0_g.grad.detach().cpu()

    def J_oracle(u):
        U = control_to_state(u, rho, T0, cv)
        for i in range(nsteps):
            U = ork.step(lambda V, t: op.L(V), U, dt, i * dt)
        return oracle_ek(op, U)

    def J_gpu(u):
        U = control_to_state(u.cuda(), rho_g, T0, cv).contiguous()
        U = g.rk_steps(nsteps, dt, 0.0, U)
        return float(g.diagnostics(U)[0])

    assert abs(float(J) - float(J_oracle(u0))) < 1e-12 * abs(float(J))
    # tolerances relative to |grad J| (the largest directional derivative over unit directions):
    # a direction nearly orthogonal to the gradient has a tiny derivative known only to FP64 noise
    gnorm = float(torch.linalg.norm(grad))
    h = 1e-6
    for i in range(8):
        v = inputs.random_direction(u0.shape, 1806 + i)
        dJ = float((grad * v).sum())
        if i not in _TLM_CACHE:
            _TLM_CACHE[i] = float(jvp(J_oracle, (u0,), (v,))[1])
        tlm = _TLM_CACHE[i]
        assert abs(dJ - tlm) <= 1e-10 * gnorm, (i, dJ, tlm, gnorm)
        fd = (J_gpu(u0 + h * v) - J_gpu(u0 - h * v)) / (2 * h)
        assert abs(dJ - fd) <= 1e-6 * gnorm, (i, dJ, fd, gnorm)
