"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 form: every output within 1e-12 relative (2-norm and max-norm over all
5N entries), the tolerance of the operator statement (for smooth states the
larger of 1e-12 and 4x the oracle's own sensitivity to a one-ulp change of U).
Mixed form: a loose bound on the error of FP32 cell/face arithmetic on these
small states (its size at full scale is measured by bench.py's extras).
"""
import math

import numpy as np
import pytest
import torch

from oracle import diagnostics as odiag, physics as ph, rk as ork
from oracle.mesh import BoxMesh, RotatedBoxMesh
from oracle.operator import WHAT_ALL, WHAT_CONV, WHAT_VISC, DGOperator
from paper_1806_03095_gb300 import inputs

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1806_03095_gb300 import api
    from paper_1806_03095_gb300.api import DGCNS

TOL64 = 1e-12
PI = math.pi


def rel_err(a, b):
    a = a.detach().double().cpu()
    b = b.detach().double().cpu()
    l2 = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    mx = float((a - b).abs().max() / b.abs().max())
    return l2, mx


def fp64_tol(fun, U, seed=5):
    """1e-12, or 4x the oracle's own change under a one-ulp relative perturbation of U,
    whichever is larger (smooth states: the weak-form terms cancel by ~10^3, so the
    FP64 result is only determined to ~1e-11 relative by any summation order)."""
    ref = fun(U)
    Up = U * (1.0 + 2.0 ** -52 * inputs.uniform(U.shape, seed))
    l2, mx = rel_err(fun(Up), ref)
    return ref, max(TOL64, 4 * l2), max(TOL64, 4 * mx)


def pair(ncells, k, qc=None, qv=None, precision=0, kernel=1, periodic=(1, 1, 1), lo=(-PI,) * 3, hi=(PI,) * 3,
         Re=1600.0, Ma=0.1, body_force=(0.0, 0.0, 0.0), u_mach=0.0):
    qc = (3 * k) // 2 + 1 if qc is None else qc
    qv = k + 1 if qv is None else qv
    g = DGCNS(ncells, lo, hi, periodic, k, qc, qv, Re=Re, Ma=Ma, body_force=body_force, u_mach=u_mach,
              precision=precision, kernel=kernel)
    mesh = BoxMesh(ncells, lo, hi, periodic, k)
    phys = ph.Physics.from_numbers(Re, 0.71, Ma, u_mach=(u_mach or None), body_force=body_force)
    return g, DGOperator(mesh, phys, qc, qv)


def on_gpu(U):
    return U.to("cuda").contiguous()


# -- geometry -------------------------------------------------------------------------------------
def test_node_coords_match_oracle():
    g, op = pair((3, 2, 4), 3)
    xyz = g.node_coords().cpu()
    assert torch.allclose(xyz, op.xyz, rtol=0, atol=1e-14)


def test_set_initial_tgv_matches_closed_form():
    """dg_cns_set_initial_tgv against the closed-form field of the input module at the same nodes
    (sin/cos of the GPU and of the host may differ in the last bit)."""
    g, op = pair((3, 2, 4), 3)
    U = g.set_initial_tgv().cpu()
    ref = inputs.tgv_state(op.xyz)
    l2, mx = rel_err(U, ref)
    assert l2 < 1e-14 and mx < 1e-14, (l2, mx)


@pytest.mark.parametrize("seed", [1806, (1 << 40) + 7])
def test_set_initial_channel_matches_input_module_bitwise(seed):
    """dg_cns_set_initial_channel and the input module draw the same Philox numbers and evaluate the same
    formula with the same rounding: identical states, on the stretched channel mesh."""
    g, op = pair_mapped((3, 4, 2), 3, 1, 1.8, **CHANNEL)
    U = g.set_initial_channel(seed).cpu()
    ref = inputs.channel_state(g.node_coords().cpu(), seed)
    assert torch.equal(U, ref)


# -- residual F(U), per term and combined ------------------------------------------------------------
CASES = [((2, 2, 2), 1), ((2, 2, 2), 2), ((2, 2, 2), 3), ((3, 2, 4), 3), ((2, 2, 2), 4), ((2, 2, 2), 5),
         ((2, 2, 2), 6)]


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("ncells,k", CASES)
def test_residual_fp64_random_state(ncells, k, kernel):
    g, op = pair(ncells, k, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 100 + k)
    ref = op.residual(U)
    out = g.apply(on_gpu(U), op=api.OP_F)
    l2, mx = rel_err(out, ref)
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("kernel", [0, 2])
@pytest.mark.parametrize("what,op_code", [(WHAT_CONV, 2), (WHAT_VISC, 3)])
def test_residual_terms_fp64(what, op_code, kernel):
    g, op = pair((2, 3, 2), 3, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 7)
    out = g.apply(on_gpu(U), op=op_code)
    l2, mx = rel_err(out, op.residual(U, what))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("k,qc,qv", [(3, 4, 4), (3, 5, 5), (5, 6, 6), (2, 4, 4), (4, 7, 7), (5, 8, 8)])
def test_other_quadrature_rules(k, qc, qv, kernel):
    """The k+1 rule on both terms, and the paper's 3/2 rule on both terms (Sec. 2.2.3)."""
    g, op = pair((2, 2, 2), k, qc, qv, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 8)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("k,qc,qv", [(2, 5, 5), (3, 7, 7), (4, 9, 9), (7, 11, 8)])
def test_over_integration_and_degree_seven(k, qc, qv):
    """The 2k+1 rule on both terms at k = 2, 3, 4 (Sec. 4.1.2, over-integration) and k = 7 with the 3/2 rule
    (the convective cell term formed one direction at a time, 15 n_q^3 values per cell), face-centric
    kernels, FP64: F and L against the oracle at 1e-12 on a ragged box of 2x3x2 cells."""
    g, op = pair((2, 3, 2), k, qc, qv, kernel=2)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 26 + k)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("k,qc,qv,ncells", [(8, 13, 9, (2, 3, 2)), (5, 11, 11, (2, 2, 2)), (7, 15, 15, (2, 1, 2)),
                                            (11, 17, 12, (2, 2, 1)), (15, 23, 16, (2, 1, 1))])
def test_high_degrees_global_workspace(k, qc, qv, ncells):
    """Degrees whose cell working set exceeds shared memory (k = 8, 11, 15 with the default rule, the 2k+1 rule
    at k = 5 and 7): the operator kernels keep it in the global workspace.  Face-centric kernels, FP64, F and
    L against the oracle at 1e-12 on small periodic boxes (one or two cells along an axis); at k = 8 also an
    RK stage."""
    g, op = pair(ncells, k, qc, qv, kernel=2)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 40 + k)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    Lref = op.L(U)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), Lref)
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    if k == 8:
        dU0 = inputs.uniform(U.shape, 41)
        dt = 1e-3
        dUg, Uo = on_gpu(dU0), g.empty_state()
        g.rk_stage(3, dt, 0.0, on_gpu(U), dUg, Uo)
        dU_ref = ork.A[3] * dU0 + dt * Lref
        l2, mx = rel_err(dUg, dU_ref)
        assert l2 < TOL64 and mx < TOL64, (l2, mx)
        l2, mx = rel_err(Uo, U + ork.B[3] * dU_ref)
        assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("k,qc,qv,ncells", [(8, 13, 9, (2, 2, 3)), (11, 17, 12, (2, 1, 1))])
def test_high_degrees_element_centric(k, qc, qv, ncells, kernel):
    """The split and fused (element-centric) kernels from the global workspace: F and L at 1e-12."""
    g, op = pair(ncells, k, qc, qv, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 60 + k)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


def test_high_degree_workspace_chunks():
    """More cells than the global workspace holds (4 CTA slices per SM, so the operator kernel runs in
    chunks): L at k = 8 on 9x9x9 cells, compared with the oracle's per-cell L on the cells at each chunk
    boundary, the first and the last cell."""
    g, op = pair((9, 9, 9), 8, 13, 9, kernel=2)
    chunk = 4 * torch.cuda.get_device_properties(g.device).multi_processor_count
    assert chunk < op.mesh.Nc
    E = sorted({0, chunk - 1, chunk, 2 * chunk - 1, 2 * chunk, op.mesh.Nc - 1} & set(range(op.mesh.Nc)))
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 49)
    n0 = g.dg_cns_launch_count()
    out = g.apply(on_gpu(U), op=api.OP_L).cpu()
    assert g.dg_cns_launch_count() - n0 == 1 + -(-op.mesh.Nc // chunk)  # the face kernel, then the chunks
    l2, mx = rel_err(out[E], op.L_cells(U, E))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
def test_single_cell_periodic_box(kernel):
    """Degenerate mesh: one cell per direction, the cell is its own neighbour on every face."""
    g, op = pair((1, 1, 1), 3, kernel=kernel)
    U = inputs.random_state(1, 64, 9)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_walls_affine_box(kernel):
    """Non-periodic y axis: isothermal no-slip walls (mirror-state reading)."""
    g, op = pair((2, 3, 2), 3, periodic=(1, 0, 1), lo=(0, -1, 0), hi=(2 * PI, 1, PI), Re=180.0, u_mach=18.3,
                 kernel=kernel)
    xyz = g.node_coords().cpu()
    U = inputs.channel_state(xyz, 1806)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("kernel", [1, 2])
def test_walls_on_every_side_ragged_box(kernel):
    """Walls on all six sides of a ragged 3x4x5 box: lower-wall faces in several batches per direction."""
    g, op = pair((3, 4, 5), 2, periodic=(0, 0, 0), lo=(0, 0, 0), hi=(1.5, 2.0, 2.5), Re=180.0, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 15)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


# -- L(U), inverse mass, body force ------------------------------------------------------------------
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_L_fp64(kernel):
    g, op = pair((2, 2, 3), 3, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 10)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_inverse_mass_fp64(k):
    g, op = pair((2, 1, 2), k)
    R = inputs.uniform((op.mesh.Nc, 5, op.mesh.n ** 3), 11)
    l2, mx = rel_err(g.inverse_mass(on_gpu(R)), op.mass_solve(R))
    assert l2 < TOL64 and mx < TOL64


@pytest.mark.parametrize("precision", [0, 1])
def test_inverse_mass_many_batches(precision):
    """7581 cells: the pipelined inverse-mass kernel runs several batches per CTA, with a ragged last batch."""
    g, op = pair((21, 19, 19), 3, precision=precision)
    R = inputs.uniform((op.mesh.Nc, 5, op.mesh.n ** 3), 19)
    out = g.inverse_mass(on_gpu(R).to(g.rdtype))
    ref = op.mass_solve(R)
    l2, mx = rel_err(out.double(), ref)
    tol = TOL64 if precision == 0 else 1e-5
    assert l2 < tol and mx < 10 * tol, (l2, mx)
    g.status()


@pytest.mark.parametrize("stage", [0, 3])
def test_split_rk_stage_many_batches_sampled(stage):
    """Split organisation on 1716 cells (the pipelined M^-1 + update kernel runs several batches per CTA),
    checked on 24 sampled cells whose L the oracle evaluates one by one."""
    g, op = pair((13, 12, 11), 3, kernel=0)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 20)
    dU = inputs.uniform(U.shape, 21)
    dt = 1e-3
    Ug, dUg, Uo = on_gpu(U), on_gpu(dU), g.empty_state()
    g.rk_stage(stage, dt, 0.0, Ug, dUg, Uo)
    g.status()
    E = torch.as_tensor(sorted(set(int(v) for v in torch.linspace(0, op.mesh.Nc - 1, 24).round().long())))
    dU_ref = ork.A[stage] * dU[E] + dt * op.L_cells(U, E)
    U_ref = U[E] + ork.B[stage] * dU_ref
    assert max(rel_err(dUg.cpu()[E], dU_ref)) < TOL64
    assert max(rel_err(Uo.cpu()[E], U_ref)) < TOL64


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_L_with_body_force_and_walls(kernel):
    g, op = pair((2, 2, 2), 3, periodic=(1, 0, 1), lo=(0, -1, 0), hi=(2 * PI, 1, PI), Re=180.0, u_mach=18.3,
                 body_force=(1.0, 0.0, 0.0), kernel=kernel)
    U = inputs.channel_state(g.node_coords().cpu(), 3)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


# -- RK stages ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_rk_stage_fp64(kernel):
    g, op = pair((2, 2, 2), 3, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 12)
    dU = inputs.uniform(U.shape, 13)
    dt = 1e-3
    for stage in (0, 2):
        Uo = g.empty_state()
        dUg = on_gpu(dU)
        g.rk_stage(stage, dt, 0.0, on_gpu(U), dUg, Uo)
        dU_ref = ork.A[stage] * dU + dt * op.L(U)
        U_ref = U + ork.B[stage] * dU_ref
        assert max(rel_err(dUg, dU_ref)) < TOL64
        assert max(rel_err(Uo, U_ref)) < TOL64


def test_rk_stage_split_in_place_allowed_fused_rejected():
    g, op = pair((2, 2, 2), 2, kernel=0)
    U = on_gpu(inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 14))
    dU = g.empty_residual()
    g.rk_stage(0, 1e-3, 0.0, U, dU, U)
    gf, _ = pair((2, 2, 2), 2, kernel=1)
    with pytest.raises(api.DGCNSError) as ei:
        gf.rk_stage(0, 1e-3, 0.0, U, dU, U)
    assert ei.value.code == -1


@pytest.mark.parametrize("kernel", [1, 2])
def test_mixed_rk_steps_chained_deviation_equals_stage_calls(kernel):
    """Inside dg_cns_rk_steps the mixed form's stage kernel writes the next stage's FP32 deviation state
    itself; it is the same rounding of the same FP64 state as the pre-pass of single stage calls, so two
    steps agree bit for bit with ten dg_cns_rk_stage calls."""
    g, op = pair((3, 2, 2), 3, precision=1, kernel=kernel)
    U0 = inputs.tgv_state(op.xyz) + 1e-2 * inputs.uniform((op.mesh.Nc, 5, op.mesh.n ** 3), 22)
    dt = 1e-3
    Us = on_gpu(U0)
    g.rk_steps(2, dt, 0.0, Us)
    a, b, dU = on_gpu(U0), g.empty_state(), g.empty_residual()
    for n in range(2):
        for s in range(5):
            g.rk_stage(s, dt, n * dt, a, dU, b)
            a, b = b, a
    assert torch.equal(Us, a)
    g.status()


def test_rk_stage_face_centric_in_place():
    """The face-centric stage reads neighbours only in the face kernel, so U_out may alias U_in."""
    g, op = pair((2, 3, 2), 3, kernel=2)
    U0 = on_gpu(inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 16))
    dU0 = on_gpu(inputs.uniform(U0.shape, 17))
    Uo, dU1 = g.empty_state(), dU0.clone()
    g.rk_stage(1, 1e-3, 0.0, U0, dU1, Uo)
    Ui, dU2 = U0.clone(), dU0.clone()
    g.rk_stage(1, 1e-3, 0.0, Ui, dU2, Ui)
    assert torch.equal(Ui, Uo) and torch.equal(dU1, dU2)


def test_tgv_dissipation_rate_history_against_oracle():
    """TGV 8^3, k = 5, to t = 2 (783 RK(5,4) steps): -de_k/dt every 8 steps against the oracle's history
    stored in tests/golden (written by the oracle-only script beside it, same dt and sampling)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tgv8_k5_dissipation.json")
    with open(path) as f:
        gold = json.load(f)
    dt, every, nsteps = gold["dt"], gold["every"], gold["nsteps"]
    ref = torch.tensor([r[4] for r in gold["samples"]], dtype=torch.float64)
    g, op = pair((8, 8, 8), 5, kernel=2)
    U = on_gpu(inputs.tgv_state(op.xyz))
    Ut, dU = g.empty_state(), g.empty_residual()
    vals = []
    for n in range(0, nsteps + 1, every):
        vals.append(float(g.diagnostics(U, g.apply(U, op=api.OP_L))[2]))
        if n + every <= nsteps:
            g.rk_steps(every, dt, n * dt, U, Ut, dU)
    got = torch.tensor(vals, dtype=torch.float64)
    assert len(got) == len(ref)
    assert abs(float(got[0] - ref[0])) <= 1e-12 * abs(float(ref[0]))
    l2 = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
    mx = float((got - ref).abs().max() / ref.abs().max())
    assert l2 < 1e-10 and mx < 1e-10, (l2, mx)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_tgv_8cubed_ten_rk_steps_fp64(kernel):
    """Taylor--Green 8^3, k = 3, one operator evaluation plus 10 RK(5,4) steps at CFL 0.4."""
    g, op = pair((8, 8, 8), 3, kernel=kernel)
    U0 = inputs.tgv_state(op.xyz)
    ref, t2, tm = fp64_tol(op.L, U0)
    assert t2 < 1e-10 and tm < 1e-9  # the conditioning itself is pinned
    l2, mx = rel_err(g.apply(on_gpu(U0), op=api.OP_L), ref)
    assert l2 < t2 and mx < tm, (l2, mx, t2, tm)
    dt = api.cfl_dt(3, 2 * PI / 8, 1.0, 0.1, Cr=0.4, nu=1.0 / 1600)
    Ug = on_gpu(U0)
    g.rk_steps(10, dt, 0.0, Ug)
    Ur = U0
    for i in range(10):
        Ur = ork.step(lambda V, t: op.L(V), Ur, dt, i * dt)
    # the change of the state over 10 steps (50 evaluations of L): the per-evaluation
    # rounding noise accumulates, so allow 3x the single-evaluation bound
    l2, mx = rel_err(Ug - on_gpu(U0), Ur - U0)
    assert l2 < 3 * t2 and mx < 3 * tm, (l2, mx)
    l2, mx = rel_err(Ug, Ur)
    assert l2 < TOL64 and mx < TOL64


# -- diagnostics ---------------------------------------------------------------------------------------
def test_diagnostics_fp64():
    g, op = pair((4, 4, 4), 3)
    U = inputs.tgv_state(op.xyz)
    LU = op.L(U)
    ref = odiag.diagnostics(op, U, LU).numpy()
    out = g.diagnostics(on_gpu(U), on_gpu(LU))
    assert np.allclose(out[:8], ref[:8], rtol=1e-12, atol=1e-14)
    assert out[8] == 0


def test_diagnostics_nonfinite_reported():
    g, op = pair((2, 2, 2), 2)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 15)
    U[1, 2, 3] = float("nan")
    with pytest.raises(api.DGCNSError) as ei:
        g.diagnostics(on_gpu(U))
    assert ei.value.code == -5
    assert g.diagnostics(on_gpu(U), check=False)[8] == 1


# -- mixed precision ----------------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_mixed_precision_error_bound(kernel):
    """FP32 cell/face arithmetic: residual error of a few FP32 ulps of the state scale."""
    g, op = pair((4, 4, 4), 3, precision=1, kernel=kernel)
    U = inputs.tgv_state(op.xyz)
    ref = op.L(U)
    out = g.apply(on_gpu(U), op=api.OP_L)
    assert out.dtype == torch.float32
    l2, mx = rel_err(out, ref)
    assert l2 < 2e-3 and mx < 2e-3, (l2, mx)


# -- argument errors -------------------------------------------------------------------------------------
def test_unsupported_configuration():
    with pytest.raises(api.DGCNSError) as ei:
        DGCNS((2, 2, 2), (0, 0, 0), (1, 1, 1), (1, 1, 1), 3, 9, 9)
    assert ei.value.code == -2
    with pytest.raises(api.DGCNSError) as ei:
        DGCNS((2, 2, 2), (0, 0, 0), (1, 1, 1), (1, 1, 1), 3, 3, 3)
    assert ei.value.code == -1


# -- non-affine meshes: stored geometry (channel stretching, sinusoidal deformation) ----------------------
def pair_mapped(ncells, k, mapping, param, periodic, lo, hi, precision=0, kernel=1, Re=1600.0, u_mach=0.0,
                body_force=(0.0, 0.0, 0.0), geometry=0):
    qc, qv = (3 * k) // 2 + 1, k + 1
    g = DGCNS(ncells, lo, hi, periodic, k, qc, qv, Re=Re, u_mach=u_mach, body_force=body_force, precision=precision,
              kernel=kernel, mapping=mapping, map_param=param, geometry=geometry)
    mesh = BoxMesh(ncells, lo, hi, periodic, k, mapping, param)
    phys = ph.Physics.from_numbers(Re, 0.71, 0.1, u_mach=(u_mach or None), body_force=body_force)
    return g, DGOperator(mesh, phys, qc, qv)


CHANNEL = dict(periodic=(1, 0, 1), lo=(0.0, -1.0, 0.0), hi=(2 * PI, 1.0, PI), Re=180.0, u_mach=18.3)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_channel_mesh_residual_and_L_fp64(kernel):
    g, op = pair_mapped((2, 3, 2), 3, 1, 1.8, kernel=kernel, body_force=(1.0, 0.0, 0.0), **CHANNEL)
    xyz = g.node_coords().cpu()
    assert torch.allclose(xyz, op.xyz, rtol=0, atol=1e-14)
    U = inputs.channel_state(xyz, 1806)
    ref, t2, tm = fp64_tol(op.residual, U)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), ref)
    assert l2 < t2 and mx < tm, (l2, mx, t2, tm)
    ref, t2, tm = fp64_tol(op.L, U)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), ref)
    assert l2 < t2 and mx < tm, (l2, mx, t2, tm)


@pytest.mark.parametrize("k", [2, 3, 5])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_deformed_periodic_mesh_fp64(k, kernel):
    g, op = pair_mapped((2, 2, 2), k, 2, 0.05, (1, 1, 1), (-PI,) * 3, (PI,) * 3, kernel=kernel)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 40 + k)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), op.residual(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)


def test_deformed_mesh_free_stream_on_gpu():
    g, op = pair_mapped((3, 2, 2), 3, 2, 0.08, (1, 1, 1), (-PI,) * 3, (PI,) * 3)
    U = torch.empty(g.shape, dtype=torch.float64)
    for c, v in enumerate((1.1, 0.3, -0.2, 0.1, 180.0)):
        U[:, c] = v
    R = g.apply(on_gpu(U), op=api.OP_F).cpu()
    assert float(R.abs().max()) < 1e-13 * 180.0 * 10


def test_deformed_mesh_diagnostics_and_rk_step():
    g, op = pair_mapped((2, 2, 2), 3, 2, 0.05, (1, 1, 1), (-PI,) * 3, (PI,) * 3)
    U = inputs.tgv_state(op.xyz)
    LU = op.L(U)
    ref = odiag.diagnostics(op, U, LU).numpy()
    out = g.diagnostics(on_gpu(U), on_gpu(LU))
    assert np.allclose(out[:8], ref[:8], rtol=1e-11, atol=1e-13), (out, ref)
    dt = 1e-3
    Ug = on_gpu(U)
    g.rk_steps(2, dt, 0.0, Ug)
    Ur = U
    for i in range(2):
        Ur = ork.step(lambda V, t: op.L(V), Ur, dt, i * dt)
    l2, mx = rel_err(Ug - on_gpu(U), Ur - U)
    assert l2 < 1e-9 and mx < 1e-9, (l2, mx)


def test_channel_mixed_precision_error():
    g, op = pair_mapped((2, 4, 2), 3, 1, 1.8, precision=1, body_force=(1.0, 0.0, 0.0), **CHANNEL)
    U = inputs.channel_state(op.xyz, 1806)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < 1e-3 and mx < 1e-2, (l2, mx)


# -- non-affine meshes: Jacobians recomputed in the operator kernels from the node coordinates -------------
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_channel_mesh_geometry_on_the_fly_fp64(kernel):
    g, op = pair_mapped((2, 3, 2), 3, 1, 1.8, kernel=kernel, body_force=(1.0, 0.0, 0.0), geometry=1, **CHANNEL)
    U = inputs.channel_state(op.xyz, 1807)
    ref, t2, tm = fp64_tol(op.residual, U)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_F), ref)
    assert l2 < t2 and mx < tm, (l2, mx, t2, tm)
    ref, t2, tm = fp64_tol(op.L, U)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), ref)
    assert l2 < t2 and mx < tm, (l2, mx, t2, tm)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_deformed_periodic_mesh_geometry_on_the_fly_fp64(kernel):
    g, op = pair_mapped((3, 2, 2), 3, 2, 0.05, (1, 1, 1), (-PI,) * 3, (PI,) * 3, kernel=kernel, geometry=1)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 77)
    for what in (WHAT_CONV, WHAT_VISC):
        l2, mx = rel_err(g.apply(on_gpu(U), op=2 if what == WHAT_CONV else 3), op.residual(U, what))
        assert l2 < TOL64 and mx < TOL64, (what, l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    dt = 1e-3
    Ug = on_gpu(U)
    g.rk_steps(1, dt, 0.0, Ug)
    Ur = ork.step(lambda V, t: op.L(V), U, dt, 0.0)
    l2, mx = rel_err(Ug - on_gpu(U), Ur - U)
    assert l2 < 1e-9 and mx < 1e-9, (l2, mx)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_channel_geometry_on_the_fly_mixed_error(kernel):
    g, op = pair_mapped((2, 4, 2), 3, 1, 1.8, precision=1, kernel=kernel, body_force=(1.0, 0.0, 0.0), geometry=1,
                        **CHANNEL)
    U = inputs.channel_state(op.xyz, 1806)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < 1e-3 and mx < 1e-2, (l2, mx)


# -- rotated-frame meshes: every cell in one of the 48 cube frames, neighbours read through orientation codes --
ROT_LO, ROT_HI = (-1.0, 0.0, 0.5), (2.0, 1.5, 2.5)


def pair_rotated(ncells, seed, precision=0, kernel=1, deform=0.0, geometry=1):
    k, qc, qv = 3, 5, 4
    g = DGCNS(ncells, ROT_LO, ROT_HI, (1, 1, 1), k, qc, qv, precision=precision, kernel=kernel,
              mapping=api.MAP_ROTATED, map_param=float(seed), deform=deform, geometry=geometry)
    mesh = RotatedBoxMesh(ncells, ROT_LO, ROT_HI, k, inputs.cell_frames(int(np.prod(ncells)), seed), deform=deform)
    return g, DGOperator(mesh, ph.Physics.from_numbers(1600.0, 0.71, 0.1), qc, qv)


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("ncells,seed,deform,geometry", [((3, 2, 4), 1806, 0.0, 1), ((4, 3, 3), (1 << 40) + 3, 0.0, 1),
                                                         ((3, 3, 2), 99, 0.06, 1), ((1, 3, 2), 7, 0.04, 1),
                                                         ((3, 2, 4), 1806, 0.0, 0), ((3, 3, 2), 99, 0.06, 0),
                                                         ((1, 3, 2), 7, 0.04, 0)])
def test_rotated_frame_mesh_fp64(ncells, seed, deform, geometry, kernel):
    """Split, fused and face-centric kernels on a periodic box whose cells have random frames, affine or
    moved by the sine deformation (one case with a single cell along x: a cell is its own neighbour), with
    geometry on the fly or stored (the neighbour's stored face Jacobians read through the orientation code):
    node coordinates, the TGV initial state, F_c, F_v, L(U) on a random state (FP64, 1e-12) and one RK(5,4)
    step against the oracle, which locates the neighbour's polynomial at the physical face points."""
    g, op = pair_rotated(ncells, seed, kernel=kernel, deform=deform, geometry=geometry)
    xyz = g.node_coords().cpu()
    assert torch.allclose(xyz, op.xyz, rtol=0, atol=1e-14)
    l2, mx = rel_err(g.set_initial_tgv().cpu(), inputs.tgv_state(op.xyz))
    assert l2 < 1e-14 and mx < 1e-14, (l2, mx)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 91)
    for what, code in ((WHAT_CONV, api.OP_FC), (WHAT_VISC, api.OP_FV)):
        l2, mx = rel_err(g.apply(on_gpu(U), op=code), op.residual(U, what))
        assert l2 < TOL64 and mx < TOL64, (what, l2, mx)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), op.L(U))
    assert l2 < TOL64 and mx < TOL64, (l2, mx)
    dt = 1e-3
    Ug = on_gpu(U)
    g.rk_steps(1, dt, 0.0, Ug)
    Ur = ork.step(lambda V, t: op.L(V), U, dt, 0.0)
    l2, mx = rel_err(Ug - on_gpu(U), Ur - U)
    assert l2 < 1e-9 and mx < 1e-9, (l2, mx)


@pytest.mark.parametrize("geometry", [0, 1])
@pytest.mark.parametrize("deform", [0.0, 0.06])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_rotated_frame_mesh_mixed(kernel, deform, geometry):
    """The mixed form on the rotated-frame box: F and L(U) of a random state to FP32 accuracy."""
    g, op = pair_rotated((3, 4, 3), 7, precision=1, kernel=kernel, deform=deform, geometry=geometry)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 92)
    for code, ref in ((api.OP_F, op.residual(U)), (api.OP_L, op.L(U))):
        l2, mx = rel_err(g.apply(on_gpu(U), op=code), ref)
        assert l2 < 1e-5 and mx < 1e-4, (code, l2, mx)


def test_rotated_frame_mesh_is_not_the_aligned_mesh():
    """The same state on the aligned box gives a different L: the frames are in effect."""
    g, op = pair_rotated((3, 2, 4), 1806)
    g0 = DGCNS((3, 2, 4), ROT_LO, ROT_HI, (1, 1, 1), 3, 5, 4, kernel=1, geometry=1, mapping=api.MAP_SINE,
               map_param=0.0)
    U = on_gpu(inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 91))
    assert float((g.apply(U) - g0.apply(U)).abs().max()) > 1e-3 * float(g0.apply(U).abs().max())


@pytest.mark.parametrize("kernel", [1, 2])
def test_rotated_frame_mesh_refusals(kernel):
    g, _ = pair_rotated((2, 2, 2), 5, kernel=kernel)
    U = g.set_initial_tgv()
    with pytest.raises(api.DGCNSError) as ei:
        g.adjoint_apply(U, U.clone())
    assert ei.value.code == -2


def test_geometry_on_the_fly_unsupported_and_invalid():
    with pytest.raises(api.DGCNSError) as ei:
        pair_mapped((2, 2, 2), 5, 2, 0.05, (1, 1, 1), (-PI,) * 3, (PI,) * 3, geometry=1)
    assert ei.value.code == -2
    with pytest.raises(api.DGCNSError) as ei:
        pair_mapped((2, 2, 2), 3, 2, 0.05, (1, 1, 1), (-PI,) * 3, (PI,) * 3, geometry=7)
    assert ei.value.code == -1


def test_overlapping_arrays_are_rejected_before_any_launch():
    """Arrays of one call must not share memory: views at an offset inside another argument are refused with
    INVALID_ARG before anything runs; adjacent non-overlapping ranges of one buffer are accepted."""
    import ctypes
    g, op = pair((2, 2, 2), 2, kernel=2)
    U = on_gpu(inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 18))
    n = U.numel()
    buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    buf[:n] = U.reshape(-1)
    p = lambda off: ctypes.c_void_p(buf.data_ptr() + 8 * off)  # noqa: E731
    lib = g.lib
    assert lib.dg_cns_apply(g.ctx, p(0), p(8), api.OP_L) == -1
    assert b"overlap" in lib.dg_cns_last_error(g.ctx)
    assert lib.dg_cns_rk_stage(g.ctx, 1, 1e-3, 0.0, p(0), p(n - 8), p(2 * n)) == -1
    assert lib.dg_cns_rk_stage(g.ctx, 1, 1e-3, 0.0, p(0), p(2 * n), p(8)) == -1
    assert lib.dg_cns_rk_steps(g.ctx, 1, 1e-3, 0.0, p(0), p(n // 2), p(2 * n)) == -1
    assert lib.dg_cns_adjoint_apply(g.ctx, p(0), p(n), p(n - 1)) == -1
    assert lib.dg_cns_apply(g.ctx, p(0), p(n), api.OP_L) == 0
    torch.cuda.synchronize()
    assert torch.equal(buf[n:2 * n].reshape(U.shape), g.apply(U))


def test_lsrk_stage_and_steps_general_2n_schemes():
    """dg_cns_lsrk_stage with a stage's RK(5,4) coefficients is dg_cns_rk_stage, dg_cns_lsrk_steps with the
    RK(5,4) table is dg_cns_rk_steps (bit for bit), and Williamson's 3-stage scheme matches the oracle's 2N
    step at 1e-12 (face-centric and fused kernels)."""
    from oracle import rk as ork
    from paper_1806_03095_gb300 import schemes
    for kernel in (1, 2):
        g, op = pair((3, 2, 4), 3, kernel=kernel)
        U0 = on_gpu(inputs.tgv_state(op.xyz) + 1e-3 * inputs.uniform((op.mesh.Nc, 5, op.mesh.n ** 3), 19))
        dU0 = on_gpu(inputs.uniform(U0.shape, 20))
        dt = 2e-3
        Ua, dUa, Ub, dUb = g.empty_state(), dU0.clone(), g.empty_state(), dU0.clone()
        g.rk_stage(2, dt, 0.0, U0, dUa, Ua)
        g.lsrk_stage(schemes.LSRK54[0][2], schemes.LSRK54[1][2], dt, U0, dUb, Ub)
        assert torch.equal(Ua, Ub) and torch.equal(dUa, dUb)
        assert torch.equal(g.rk_steps(2, dt, 0.0, U0.clone()), g.lsrk_steps(schemes.LSRK54, 2, dt, U0.clone()))
        got = g.lsrk_steps(schemes.LSRK33, 3, dt, U0.clone())
        U = U0.cpu()
        for n in range(3):
            U = ork.lsrk_step(lambda V, t: op.L(V), U, dt, n * dt, ork.LSRK33_A, ork.LSRK33_B, ork.LSRK33_C)
        l2, mx = rel_err(got, U)
        assert l2 < TOL64 and mx < TOL64, (kernel, l2, mx)
        with pytest.raises(Exception):
            g.lsrk_steps(((0.0, float("nan")), (0.5, 0.5)), 1, dt, U0.clone())


@pytest.mark.parametrize("what", ["F", "FC", "FV"])
@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
@pytest.mark.parametrize("k", [3, 4, 5])
def test_mixed_face_centric_random_states(k, periodic, what):
    """The mixed form's face-centric kernels (FP32 arithmetic) on random states: independent nodal draws give
    jumps on every face and no cancellation between the weak-form terms, so F, F_c and F_v agree with the
    FP64 oracle to FP32 accuracy (2-norm 1e-5, max 1e-4 relative).  A ragged 3x4x5 box, periodic or with
    walls on all six sides (lower and upper wall faces of every direction); k = 3, 4, 5 (the FP32 task face
    kernel at every degree, the task cell kernel at k = 3)."""
    lo, hi = (-1.0, -1.5, -2.0), (2.0, 1.5, 2.5)
    g, op = pair((3, 4, 5), k, precision=1, kernel=2, periodic=periodic, lo=lo, hi=hi)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 23)
    op_code = {"F": api.OP_F, "FC": api.OP_FC, "FV": api.OP_FV}[what]
    which = {"F": WHAT_ALL, "FC": WHAT_CONV, "FV": WHAT_VISC}[what]
    out = g.apply(on_gpu(U), op=op_code)
    ref = op.residual(U, which)
    l2, mx = rel_err(out, ref)
    assert l2 < 1e-5 and mx < 1e-4, (l2, mx)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 0, 0)])
@pytest.mark.parametrize("k", [3, 4, 5])
def test_mixed_face_centric_L_and_stage_random_states(k, periodic):
    """The mixed form's face-centric cell + inverse-mass + stage kernel on random states against the FP64
    oracle: L(U) to FP32 accuracy (2-norm 1e-5, max 1e-4 relative), and one RK stage (stage 3: dU is read):
    dU to the same bound, and U_out - U = B dU with the FP32 dU accumulated in FP64 (1e-10).  Ragged 3x4x5
    box, periodic or with walls on all six sides."""
    lo, hi = (-1.0, -1.5, -2.0), (2.0, 1.5, 2.5)
    g, op = pair((3, 4, 5), k, precision=1, kernel=2, periodic=periodic, lo=lo, hi=hi)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 24)
    Lref = op.L(U)
    l2, mx = rel_err(g.apply(on_gpu(U), op=api.OP_L), Lref)
    assert l2 < 1e-5 and mx < 1e-4, (l2, mx)
    dU0 = inputs.uniform(U.shape, 25)
    dt = 1e-3
    dUg, Uo = on_gpu(dU0).float().contiguous(), g.empty_state()
    g.rk_stage(3, dt, 0.0, on_gpu(U), dUg, Uo)
    dU_ref = ork.A[3] * dU0.float().double() + dt * Lref
    l2, mx = rel_err(dUg, dU_ref)
    assert l2 < 1e-5 and mx < 1e-4, (l2, mx)
    # the state is accumulated in FP64: U_out - U is B times the FP32 dU, rounded at the ulp of U (~3e-14
    # of 178) against an increment of order B; an FP32 accumulation would miss this by 1e-6
    inc = (Uo.cpu() - U)
    l2, mx = rel_err(inc, ork.B[3] * dUg.double().cpu())
    assert l2 < 1e-10 and mx < 1e-10, (l2, mx)


@pytest.mark.parametrize("stage", [0, 3])
def test_mixed_split_stage_and_inverse_mass_in_place(stage):
    """Mixed form, split organisation (its M^-1 + stage kernel keeps every cell-component block in registers
    at k = 3): one RK stage on random states of a ragged 5x3x4 box against the oracle (dU to FP32 accuracy,
    U_out - U = B dU at FP64 rounding), and M^-1 in place (in == out) against the oracle's LU solve."""
    g, op = pair((5, 3, 4), 3, precision=1, kernel=0)
    U = inputs.random_state(op.mesh.Nc, op.mesh.n ** 3, 27)
    dU0 = inputs.uniform(U.shape, 28)
    dt = 1e-3
    dUg, Uo = on_gpu(dU0).float().contiguous(), g.empty_state()
    g.rk_stage(stage, dt, 0.0, on_gpu(U), dUg, Uo)
    g.status()
    dU_ref = ork.A[stage] * dU0.float().double() + dt * op.L(U)
    l2, mx = rel_err(dUg, dU_ref)
    assert l2 < 1e-5 and mx < 1e-4, (l2, mx)
    l2, mx = rel_err(Uo.cpu() - U, ork.B[stage] * dUg.double().cpu())
    assert l2 < 1e-10 and mx < 1e-10, (l2, mx)
    R = inputs.uniform(U.shape, 29).float()
    Rg = on_gpu(R).float().contiguous()
    g.inverse_mass(Rg, Rg)
    l2, mx = rel_err(Rg, op.mass_solve(R.double()))
    assert l2 < 1e-5 and mx < 1e-4, (l2, mx)
