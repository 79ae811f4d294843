"""The benchmark workloads at full size, in the launch configurations the benchmark times (face-centric
kernels, seeded random states with independent nodal draws, discontinuous across every face):
  - Taylor--Green vortex meshes on [-pi, pi]^3: 64^3 cells, k = 3, n_q 5 / 4 (FP64 and mixed) and
    40^3 cells, k = 5, n_q 8 / 6 (FP64);
  - the turbulent channel mesh, 2 pi x 2 x pi, 32^3 cells stretched towards the walls, k = 3, n_q 5 / 4,
    isothermal walls and body force (FP64 and mixed);
  - the adjoint on the Taylor--Green mesh of 24^3 cells, k = 4, n_q 7 / 5 (FP64).

Sampled cells.  A cell's L(U) needs only its own values and those of its six face neighbours (M is
block diagonal, a face term couples only the two cells of the face; Sec. 2.2), and the geometry of a
cell of these meshes depends only on its position along the wall-bounded axes.  The oracle therefore
evaluates L of each sampled cell on a patch mesh: 3 cells (centred on the origin) along each periodic
axis and the whole extent, with the full mesh's coordinates, along a wall-bounded axis, filled with the
sampled cell's neighbourhood.  A CPU test checks the reduction against the oracle on a whole mesh.  The
adjoint's (dL/dU)^T W is compared on every cell with the oracle's reverse mode on the whole mesh (30 s of
CPU at 24^3, k = 4).

Every cell.  On a periodic mesh the domain integral of L(U) vanishes in every component: tested with
v = 1, the cell terms carry grad v = 0, the numerical fluxes are single valued and the penalty term
carries [[v]] = 0.  With walls (mirror state: no mass flux through the wall) and a body force (no mass
source) this holds for the density alone.  With the k+1 Gauss rule of the mass matrix,
integral(L) = 1^T M L = 1^T (-F(U) + F_rhs(U)) exactly, so a stage's dU = dt L integrates to zero and an
RK step keeps the integral of U.  The integral of a nodal field X is sum_e sum_n W_{e,n} X_{e,n} with
W_{e,n} the integral of the n-th basis function over cell e, which depends only on the cell's position
along the wall-bounded axes; a CPU test checks it against the oracle's integration.  The adjoint is
also checked by the identity <W, J V> = <J^T W, V>, with J V from central differences of the CUDA
operator, and the discrete adjoint of the whole integration (200 RK steps, checkpoints every 20) by
central differences of the final kinetic energy along 8 smooth seeded directions.
"""
import pytest
import torch

from oracle import physics as ph, rk as ork
from oracle.mesh import BoxMesh
from oracle.operator import DGOperator
from paper_1806_03095_gb300 import configs, inputs

TOL64 = 1e-12
# FP32 arithmetic: the weak-form sums with v = 1 cancel only to the rounding of the FP32 tables and
# fluxes (relative 6e-8 per term, a few tens of terms per node), and the per-cell errors have random
# signs; the bound is set well above that estimate.
TOL_MIXED_CONSERVATION = 1e-5
# Central differences with a relative step of 1e-6: truncation ~1e-12, rounding ~1e-16 / 1e-6 times the
# cancellation of the residual terms (10^2 for these states).
FD_STEP, TOL_FD = 1e-6, 1e-6


def rel_err(a, b):
    a = a.detach().double().cpu()
    b = b.detach().double().cpu()
    return (float(torch.linalg.norm(a - b) / torch.linalg.norm(b)), float((a - b).abs().max() / b.abs().max()))


def physics(cfg):
    return ph.Physics.from_numbers(cfg["Re"], cfg["Pr"], cfg["Ma"], gamma=cfg["gamma"], R=cfg["R"],
                                   u_mach=(cfg["u_mach"] or None), body_force=cfg["body_force"])


def cell_size(cfg):
    return [(hi - lo) / n for lo, hi, n in zip(cfg["lo"], cfg["hi"], cfg["ncells"])]


def oracle_on(cfg, patch=False, periodic_cells=3):
    """The oracle on the configuration's whole mesh, or (patch) on a patch mesh: periodic_cells cells of
    the configuration's size, centred on the origin, along each periodic axis (node coordinates of the
    size of a few cells, so that the Jacobians computed from them carry little rounding), and the whole
    extent with the configuration's coordinates along each wall-bounded axis."""
    if not patch:
        n, lo, hi = cfg["ncells"], cfg["lo"], cfg["hi"]
    else:
        h = cell_size(cfg)
        n, lo, hi = [], [], []
        for d in range(3):
            if cfg["periodic"][d]:
                n.append(periodic_cells)
                lo.append(-0.5 * periodic_cells * h[d])
                hi.append(0.5 * periodic_cells * h[d])
            else:
                n.append(cfg["ncells"][d])
                lo.append(cfg["lo"][d])
                hi.append(cfg["hi"][d])
    mesh = BoxMesh(n, lo, hi, cfg["periodic"], cfg["k"], cfg["mapping"], cfg["map_param"])
    return DGOperator(mesh, physics(cfg), cfg["nq_conv"], cfg["nq_visc"])


def neighbourhood(cfg, op, e):
    """Full-mesh cell of every cell of the patch mesh op when the patch holds cell e's neighbourhood, and
    the patch index of e."""
    nf, npch = cfg["ncells"], op.mesh.ncells
    c = [e % nf[0], (e // nf[0]) % nf[1], e // (nf[0] * nf[1])]
    p = torch.arange(op.mesh.Nc)
    q = [p % npch[0], (p // npch[0]) % npch[1], p // (npch[0] * npch[1])]
    f = [(c[d] + q[d] - 1) % nf[d] if cfg["periodic"][d] else q[d] for d in range(3)]
    centre = [1 if cfg["periodic"][d] else c[d] for d in range(3)]
    return f[0] + nf[0] * (f[1] + nf[1] * f[2]), centre[0] + npch[0] * (centre[1] + npch[1] * centre[2])


def patch_L(cfg, U, E):
    """L(U) of the cells E of the configuration's mesh, by the oracle on the patch mesh."""
    op = oracle_on(cfg, patch=True)
    out = []
    for e in (int(v) for v in E):
        idx, centre = neighbourhood(cfg, op, e)
        out.append(op.L_cells(U[idx], [centre]))
    return torch.cat(out)


def cell_weights(cfg):
    """(W_col, col): W_col[j, n] the integral of the n-th basis function over a cell in position j along
    the wall-bounded axes (one cell per periodic axis), col[e] that position for every cell e."""
    op = oracle_on(cfg, patch=True, periodic_cells=1)
    phi, _, _ = op.cell_tables(op.nq_mass)
    _, wdet = op.cell_geometry(torch.arange(op.mesh.Nc), op.nq_mass)
    nf, npch = cfg["ncells"], op.mesh.ncells
    e = torch.arange(nf[0] * nf[1] * nf[2])
    c = [e % nf[0], (e // nf[0]) % nf[1], e // (nf[0] * nf[1])]
    q = [torch.zeros_like(c[d]) if cfg["periodic"][d] else c[d] for d in range(3)]
    return wdet @ phi, q[0] + npch[0] * (q[1] + npch[1] * q[2])


def conservation_defect(X, weights, components):
    """max over the given components of |integral X| / integral |X| for a nodal field X [cells, 5, nodes]."""
    W_col, col = weights
    X = X.detach().double()
    W_col, col = W_col.to(X.device), col.to(X.device)

    def integral(Y):
        Ycol = torch.zeros((W_col.shape[0],) + tuple(Y.shape[1:]), dtype=Y.dtype, device=Y.device)
        Ycol.index_add_(0, col, Y)
        return (Ycol * W_col[:, None, :]).sum((0, 2))

    tot, scale = integral(X), integral(X.abs())
    return float((tot.abs() / scale)[list(components)].max())


def conserved(cfg):
    return (0, 1, 2, 3, 4) if all(cfg["periodic"]) and not any(cfg["body_force"]) else (0,)


def random_state(cfg, g, seed):
    """Seeded random state about the configuration's reference state: rho in rho0 (1 +- 0.1), momentum in
    +-0.1 u_ref, rho E in rho0 c_v T0 (1 +- 0.1), c0 = u_ref / Ma, T0 = c0^2 / (gamma R)."""
    u_ref = cfg["u_mach"] or 1.0
    c0 = u_ref / cfg["Ma"]
    T0 = c0 * c0 / (cfg["gamma"] * cfg["R"])
    rhoE0 = 1.0 * cfg["R"] / (cfg["gamma"] - 1.0) * T0
    return inputs.random_state(g.n_cells, g.n ** 3, seed, mom=0.1 * u_ref, rhoE0=rhoE0)


def parity_state(cfg, g, seed):
    """inputs.parity_state about the configuration's reference state (as random_state)."""
    u_ref = cfg["u_mach"] or 1.0
    c0 = u_ref / cfg["Ma"]
    T0 = c0 * c0 / (cfg["gamma"] * cfg["R"])
    rhoE0 = 1.0 * cfg["R"] / (cfg["gamma"] - 1.0) * T0
    return inputs.parity_state(cfg["ncells"], g.n ** 3, seed, mom=0.1 * u_ref, rhoE0=rhoE0)


def sample_cells(cfg, count=32):
    """count cells spread over the mesh plus the cells whose neighbours wrap around a periodic boundary
    in x, y and z alone (or that lie on a wall)."""
    nx, ny, nz = cfg["ncells"]
    Nc = nx * ny * nz
    E = set(int(v) for v in torch.linspace(0, Nc - 1, count).round().long())
    E |= {nx - 1, (ny - 1) * nx, (nz - 1) * nx * ny}
    return torch.as_tensor(sorted(E))


# -- the checks, run on the CUDA path at full size and, for the host logic, on the oracle -----------------
def check_fp64(cfg, g, device):
    """One RK stage (stages 0 and 3) on 32+ sampled cells against the oracle, conservation of stage 0's
    dU = dt L over every cell, and of U through one RK step of dg_cns_rk_steps."""
    U = random_state(cfg, g, 41)
    dU = inputs.uniform(U.shape, 42)
    dt = configs.time_step(cfg)
    E = sample_cells(cfg)
    L_E = patch_L(cfg, U, E)
    weights = cell_weights(cfg)
    Ug, Eg = U.to(device), E.to(device)
    for stage in (0, 3):
        dUg, Uo = dU.to(device, copy=True), g.empty_state()
        g.rk_stage(stage, dt, 0.0, Ug, dUg, Uo)
        g.status()
        dU_ref = ork.A[stage] * dU[E] + dt * L_E
        U_ref = U[E] + ork.B[stage] * dU_ref
        assert max(rel_err(dUg[Eg], dU_ref)) < TOL64
        assert max(rel_err(Uo[Eg], U_ref)) < TOL64
        if stage == 0:
            # A_0 = 0: dU = dt L(U) on every cell
            assert conservation_defect(dUg, weights, conserved(cfg)) < TOL64
    U1 = g.rk_steps(1, dt, 0.0, Ug.clone())
    g.status()
    assert conservation_defect(U1 - Ug, weights, conserved(cfg)) < TOL64


def check_mixed(cfg, g, device):
    """The mixed form: FP32 cell and face arithmetic conserves over all cells to FP32 rounding, through a
    single stage and through dg_cns_rk_steps' chained deviation state."""
    U = random_state(cfg, g, 43)
    dt = configs.time_step(cfg)
    weights = cell_weights(cfg)
    Ug = U.to(device)
    dUg, Uo = torch.zeros(g.shape, dtype=g.rdtype, device=device), g.empty_state()
    g.rk_stage(0, dt, 0.0, Ug, dUg, Uo)
    g.status()
    assert torch.isfinite(dUg).all()
    assert conservation_defect(dUg, weights, conserved(cfg)) < TOL_MIXED_CONSERVATION
    U1 = g.rk_steps(1, dt, 0.0, Ug.clone())
    g.status()
    assert conservation_defect(U1 - Ug, weights, conserved(cfg)) < TOL_MIXED_CONSERVATION


def check_adjoint(cfg, g, device):
    """(dL/dU)^T W on every cell against the oracle's reverse mode on the whole mesh, and <W, J V> = <J^T W, V>
    with J V from central differences of the CUDA operator, on a state where the differences are well posed.

    The LLF wave speed Lambda = max(lambda^-, lambda^+) is not differentiable where the two traces' speeds
    tie.  With independent nodal draws about one state, a few face points (8 of 2.2 M at TGV 24^3, k = 4)
    lie within the step's reach of a tie; the central difference there averages the two branches while
    the derivative takes one, and the few cells around them carry a gap of 5.5e-5 in <W, J V> on the
    oracle as on the GPU (the oracle's forward mode closes it to 1e-15).  The identity is therefore taken
    on a state whose energy level alternates between face neighbours (inputs.parity_state), so that the
    two sound speeds of every face point differ by a wide margin that no step can cross; the CPU test
    below checks that margin."""
    U = random_state(cfg, g, 47)
    W = inputs.uniform(U.shape, 48)
    G_ref = OracleContext.vjp(oracle_on(cfg), U, W)
    Ug, Wg = U.to(device), W.to(device)
    G = g.adjoint_apply(Ug, Wg)
    g.status()
    assert max(rel_err(G, G_ref)) < TOL64
    Up = parity_state(cfg, g, 50).to(device)
    Gp = g.adjoint_apply(Up, Wg)
    g.status()
    V = inputs.uniform(U.shape, 49).to(device) * Up
    JV = (g.apply(Up + FD_STEP * V) - g.apply(Up - FD_STEP * V)) / (2 * FD_STEP)
    lhs, rhs = float((Wg * JV).sum()), float((Gp * V).sum())
    assert abs(lhs - rhs) < TOL_FD * abs(rhs), (lhs, rhs)


class OracleContext:
    """The context calls the checks make, answered by the oracle on the CPU (2N stage: dU = A dU + dt L(U),
    U_out = U + B dU, with dU stored in the residual type of the precision; the VJP by reverse mode)."""

    def __init__(self, cfg):
        self.op = oracle_on(cfg)
        self.n_cells, self.n = self.op.mesh.Nc, self.op.mesh.n
        self.shape = (self.n_cells, 5, self.n ** 3)
        self.rdtype = torch.float32 if cfg["precision"] == 1 else torch.float64

    def empty_state(self):
        return torch.empty(self.shape, dtype=torch.float64)

    def status(self):
        pass

    def apply(self, U):
        return self.op.L(U)

    @staticmethod
    def vjp(op, U, W):
        Ur = U.clone().requires_grad_(True)
        return torch.autograd.grad(op.L(Ur), Ur, W)[0]

    def adjoint_apply(self, U, W):
        return self.vjp(self.op, U, W)

    def rk_stage(self, stage, dt, t, U_in, dU, U_out):
        dU.copy_(ork.A[stage] * dU.double() + dt * self.op.L(U_in))
        U_out.copy_(U_in + ork.B[stage] * dU.double())

    def rk_steps(self, nsteps, dt, t0, U):
        dU = torch.zeros(self.shape, dtype=self.rdtype)
        for _ in range(nsteps):
            for stage in range(ork.STAGES):
                U_out = self.empty_state()
                self.rk_stage(stage, dt, t0, U, dU, U_out)
                U.copy_(U_out)
        return U


# -- the harness on small meshes against the oracle on the whole mesh (CPU) ------------------------------
SMALL = {
    "tgv_k3": lambda precision=0: configs.tgv(4, 3, precision=precision),
    "tgv_k5": lambda precision=0: configs.tgv(3, 5, precision=precision),
    "channel_k3": lambda precision=0: configs.channel(4, 3, precision=precision),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_patch_reduction_equals_oracle_on_the_whole_mesh(name):
    cfg = SMALL[name]()
    g = OracleContext(cfg)
    U = random_state(cfg, g, 44)
    E = sample_cells(cfg, 8)
    # the two differ by the rounding of Jacobians computed from node coordinates of different size
    l2, mx = rel_err(patch_L(cfg, U, E), g.op.L_cells(U, E))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("name", ["tgv_k3", "channel_k3"])
def test_cell_weight_integral_equals_oracle_integration(name):
    cfg = SMALL[name]()
    g = OracleContext(cfg)
    X = inputs.uniform(g.shape, 45)
    W_col, col = cell_weights(cfg)
    Xcol = torch.zeros((W_col.shape[0],) + g.shape[1:], dtype=torch.float64).index_add_(0, col, X)
    assert torch.allclose((Xcol * W_col[:, None, :]).sum((0, 2)), g.op.integrate(X), rtol=1e-13, atol=0)
    # the defect of the oracle's own L is at its rounding level; a field with a net integral is not
    assert conservation_defect(g.apply(random_state(cfg, g, 46)), (W_col, col), conserved(cfg)) < TOL64
    assert conservation_defect(X + 0.01, (W_col, col), conserved(cfg)) > 1e-3


@pytest.mark.parametrize("name,precision", [("tgv_k3", 0), ("tgv_k3", 1), ("tgv_k5", 0), ("channel_k3", 0),
                                            ("channel_k3", 1)])
def test_checks_on_the_oracle(name, precision):
    cfg = SMALL[name](precision=precision)
    (check_fp64 if precision == 0 else check_mixed)(cfg, OracleContext(cfg), "cpu")


def test_adjoint_checks_on_the_oracle():
    cfg = configs.tgv(4, 2)
    check_adjoint(cfg, OracleContext(cfg), "cpu")


@pytest.mark.parametrize("k", [2, 4])
def test_parity_state_separates_the_llf_wave_speeds(k):
    """At every convective face point of the parity state the two traces' LLF speeds |u| + c differ by more
    than 10 % (a step of 1e-6 relative cannot reach a tie of max(lambda^-, lambda^+)); the random state
    about one level has near ties."""
    cfg = configs.tgv(4, k)
    g = OracleContext(cfg)
    op = g.op

    def min_gap(U):
        gap = []
        for E in op._chunks():
            for d in range(3):
                phi, _, _ = op.face_tables(op.nq_conv, d, 1)
                Um = op.values(phi, U[E])
                Up, _, _, _ = op._exterior(U, E, d, 1, op.nq_conv, Um)
                lm, lp = [torch.linalg.norm(V[..., 1:4] / V[..., 0:1], dim=-1) + ph.sound_speed(V, op.phys.gamma)
                          for V in (Um, Up)]
                gap.append(((lm - lp).abs() / torch.maximum(lm, lp)).min())
        return float(min(gap))

    assert min_gap(parity_state(cfg, g, 50)) > 0.1
    assert min_gap(random_state(cfg, g, 47)) < 1e-3


# -- the CUDA path at full size ------------------------------------------------------------------------
def full_size(workload, precision):
    cfg = configs.WORKLOADS[workload](precision=precision, kernel=2)
    g = configs.make_context(cfg)
    assert g.n_cells == cfg["ncells"][0] * cfg["ncells"][1] * cfg["ncells"][2] and g.n == cfg["k"] + 1
    return cfg, g


@pytest.mark.gpu
@pytest.mark.full_size
@pytest.mark.parametrize("workload", ["tgv64_k3", "tgv40_k5", "channel32_k3"])
def test_benchmark_workload_fp64_sampled_cells_and_conservation(workload):
    check_fp64(*full_size(workload, 0), "cuda")


@pytest.mark.gpu
@pytest.mark.full_size
@pytest.mark.parametrize("workload", ["tgv64_k3", "channel32_k3"])
def test_benchmark_workload_mixed_conservation(workload):
    check_mixed(*full_size(workload, 1), "cuda")


@pytest.mark.gpu
@pytest.mark.full_size
def test_adjoint_workload_every_cell_vjp_and_dot_product():
    check_adjoint(*full_size("tgv24_k4", 0), "cuda")


def control_to_state(u0, rho, T0, cv):
    """Initial state from the nodal velocity field u0 [Nc, 3, n^3] at fixed density and temperature."""
    m = rho[:, None] * u0
    rhoE = rho * (cv * T0 + 0.5 * (u0 * u0).sum(1))
    return torch.cat([rho[:, None], m, rhoE[:, None]], 1)


@pytest.mark.gpu
@pytest.mark.full_size
def test_adjoint_workload_gradient_vs_central_differences():
    """The adjoint workload: TGV 24^3, k = 4, 200 RK(5,4) steps with checkpoints every 20 steps; the gradient
    of the final kinetic energy with respect to the initial nodal velocity field (discrete adjoint through
    torch.autograd.Function) against central differences of the CUDA forward integration along 8 seeded
    directions of unit root-mean-square (inputs.fd_direction: the initial field plus a smooth random field),
    step 1e-6, in FP64: 1e-6 relative to each directional derivative.  Two 200-step trajectories differ by
    rounding noise of about 3e-10 in the central difference, so the directions keep the derivative O(1);
    with purely random smooth directions one of 8 had a derivative of 2e-4 and missed the bound by that
    noise (1.4e-6).  The state is the smooth Taylor--Green field, whose traces differ across faces only by
    the interpolation error, so a crossing of the LLF max() moves the differences by far less than that."""
    from paper_1806_03095_gb300 import adjoint as adj
    cfg, g = full_size("tgv24_k4", 0)
    dt, nsteps, every, h = configs.time_step(cfg), 200, 20, 1e-6
    xyz = g.node_coords()
    U0 = inputs.tgv_state(xyz)
    rho = U0[:, 0].clone()
    u0 = (U0[:, 1:4] / rho[:, None]).clone()
    phys = physics(cfg)
    T0, cv = phys.T_wall, phys.c_v
    u0g = u0.clone().requires_grad_(True)
    J = adj.kinetic_energy(g, adj.integrate(g, control_to_state(u0g, rho, T0, cv).contiguous(), nsteps, dt, every))
    J.backward()
    grad = u0g.grad.detach()
    g.status()

    def J_fd(u):
        U = g.rk_steps(nsteps, dt, 0.0, control_to_state(u, rho, T0, cv).contiguous())
        return float(g.diagnostics(U)[0])

    res = []
    for i in range(8):
        v = inputs.fd_direction(u0, xyz, 1806 + i).to(grad.device)
        dJ = float((grad * v).sum())
        fd = (J_fd(u0 + h * v) - J_fd(u0 - h * v)) / (2 * h)
        res.append((i, dJ, fd, abs(dJ - fd) / abs(fd)))
    assert all(r[3] <= TOL_FD for r in res), res
