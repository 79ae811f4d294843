"""Naive DG operator of Eq. WeakFormulationConservedVariables (oracle; test infrastructure only).

For every element e and every test function V in its space (element-based
form of Sec. 2.2.2), the residual F(U) collects

  - (grad V, F_c(U))                           cell, n_q = nq_conv points
  + (V, F_c* . n)    F_c* = {{F_c}} + Lambda/2 [[U]]           faces, nq_conv
  + (grad V, F_v(U, grad U))                   cell, n_q = nq_visc
  - (V, Q* . n)      Q* = {{F_v}} - tau_IP [[U]]               faces, nq_visc
  - 1/2 (grad V, F_v(U, [[U]]))                faces, nq_visc

with [[U]] . n^- = U^- - U^+ (jump operator of Sec. 2.2.1) and G(U) of the
last term taken at the element's own trace U^-, as in Eq. WeakFormEquation2
where R_h : G(U_h) multiplies the face term of element e.  Integrals are
mapped to the reference cell (Eq. IntegralsReferenceSpace) and replaced by
Gauss sums (Eq. IntegralsNumericalQuadrature) with FULL interpolation
matrices: values phi[p, i] and reference gradients grad[p, i, b] of all
(k+1)^3 basis functions at every point.

The semi-discrete system is M dU/dt = -F(U) + F_rhs(U) = M L(U)
(Eq. SpatiallyDiscretizedProblem).  The mass matrix and the body force use
k+1 points (Sec. 2.2.3); M_e is assembled densely per cell and solved by LU.

Penalty (Eq. TauIP_Element): tau_e = nu (k+1)^2 (A(interior faces)/2 +
A(boundary faces)) / V(e); areas and volume are Gauss sums with nq_conv
points; on interior faces tau = max(tau_e-, tau_e+), on boundary faces tau_e-.
"""
import numpy as np
import torch

from . import physics as ph
from .basis import basis_3d, cell_points, face_points

WHAT_ALL, WHAT_CONV, WHAT_VISC = 0, 1, 2


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64)


class DGOperator:
    def __init__(self, mesh, phys, nq_conv, nq_visc, chunk=1024):
        self.mesh, self.phys = mesh, phys
        self.k, self.n = mesh.k, mesh.n
        self.nq_conv, self.nq_visc, self.nq_mass = int(nq_conv), int(nq_visc), mesh.k + 1
        self.chunk = int(chunk)
        self.xyz = _t(mesh.xyz)  # [Nc, 3, n^3]
        self.nbr = torch.as_tensor(mesh.nbr)
        self._cell = {}
        self._face = {}
        self.tau_cell = self._tau_cells()

    # -- tables ----------------------------------------------------------------
    def cell_tables(self, nq):
        if nq not in self._cell:
            pts, w = cell_points(nq)
            phi, grad = basis_3d(self.mesh.nodes_1d, pts)
            self._cell[nq] = (_t(phi), _t(grad), _t(w))
        return self._cell[nq]

    def face_tables(self, nq, d, s):
        key = (nq, d, s)
        if key not in self._face:
            pts, w = face_points(nq, d, s)
            phi, grad = basis_3d(self.mesh.nodes_1d, pts)
            self._face[key] = (_t(phi), _t(grad), _t(w))
        return self._face[key]

    # -- geometry (Eq. IntegralsReferenceSpace) ----------------------------------
    @staticmethod
    def jacobian(xyz, grad):
        """J[e,p,a,b] = d x_a / d xi_b of the isoparametric map at the table's points."""
        return torch.einsum("ean,pnb->epab", xyz, grad)

    def cell_geometry(self, E, nq):
        _, grad, w = self.cell_tables(nq)
        J = self.jacobian(self.xyz[E], grad)
        return torch.linalg.inv(J), torch.abs(torch.linalg.det(J)) * w

    def face_geometry(self, E, nq, d, s):
        """Inverse Jacobian, outward unit normal n and dA*w at face points of cells E.

        n = J^{-T} n_xi / |J^{-T} n_xi|, dA = |det J| |J^{-T} n_xi| (Eq. IntegralsReferenceSpace).
        """
        _, grad, w = self.face_tables(nq, d, s)
        J = self.jacobian(self.xyz[E], grad)
        Jinv = torch.linalg.inv(J)
        nxi = torch.zeros(3, dtype=torch.float64)
        nxi[d] = 1.0 if s == 1 else -1.0
        v = torch.einsum("epba,b->epa", Jinv, nxi)
        norm = torch.linalg.norm(v, dim=-1)
        dA = torch.abs(torch.linalg.det(J)) * norm
        return Jinv, v / norm[..., None], dA * w

    def _tau_cells(self):
        k, nu = self.k, self.phys.nu
        tau = []
        for E in self._chunks():
            _, JxW = self.cell_geometry(E, self.nq_conv)
            vol = JxW.sum(1)
            a_int = torch.zeros_like(vol)
            a_bnd = torch.zeros_like(vol)
            for d in range(3):
                for s in range(2):
                    _, _, dAw = self.face_geometry(E, self.nq_conv, d, s)
                    area = dAw.sum(1)
                    interior = self.nbr[E, d, s] >= 0
                    a_int = a_int + torch.where(interior, area, torch.zeros_like(area))
                    a_bnd = a_bnd + torch.where(interior, torch.zeros_like(area), area)
            tau.append(nu * (k + 1) ** 2 * (0.5 * a_int + a_bnd) / vol)
        return torch.cat(tau)

    def _chunks(self):
        Nc = self.mesh.Nc
        return [torch.arange(a, min(a + self.chunk, Nc)) for a in range(0, Nc, self.chunk)]

    # -- point evaluation --------------------------------------------------------
    @staticmethod
    def values(phi, Ue):
        return torch.einsum("pn,ecn->epc", phi, Ue)

    @staticmethod
    def gradients(grad, Jinv, Ue):
        """Physical gradients dU_c/dx_a = sum_b Jinv[b,a] dU_c/dxi_b."""
        gxi = torch.einsum("pnb,ecn->epcb", grad, Ue)
        return torch.einsum("epba,epcb->epca", Jinv, gxi)

    @staticmethod
    def test_grad(grad, Jinv, F, wdet):
        """sum_p (grad_xi V_i . J^{-1}) : F  * |det J| w  ->  [e, c, i]."""
        Ft = torch.einsum("epba,epca->epcb", Jinv, F)
        return torch.einsum("pnb,epcb,ep->ecn", grad, Ft, wdet)

    @staticmethod
    def test_val(phi, f, wdet):
        return torch.einsum("pn,epc,ep->ecn", phi, f, wdet)

    # -- residual F(U) -------------------------------------------------------------
    def residual(self, U, what=WHAT_ALL):
        """F(U) [Nc, 5, n^3] of the weak form (cell + face terms, no mass matrix)."""
        out = [self._residual_chunk(U, E, what) for E in self._chunks()]
        return torch.cat(out, 0)

    def _residual_chunk(self, U, E, what):
        g = self.phys.gamma
        Ue = U[E]
        R = torch.zeros_like(Ue)
        if what in (WHAT_ALL, WHAT_CONV):
            phi, grad, _ = self.cell_tables(self.nq_conv)
            Jinv, wdet = self.cell_geometry(E, self.nq_conv)
            Fc = ph.conv_flux(self.values(phi, Ue), g)
            R = R - self.test_grad(grad, Jinv, Fc, wdet)
        if what in (WHAT_ALL, WHAT_VISC):
            phi, grad, _ = self.cell_tables(self.nq_visc)
            Jinv, wdet = self.cell_geometry(E, self.nq_visc)
            Uq = self.values(phi, Ue)
            Fv = ph.visc_flux(Uq, self.gradients(grad, Jinv, Ue), self.phys)
            R = R + self.test_grad(grad, Jinv, Fv, wdet)
        for d in range(3):
            for s in range(2):
                R = R + self._face_chunk(U, E, d, s, what)
        return R

    def _exterior(self, U, E, d, s, nq, Um):
        """Exterior trace: neighbour cell's values/gradients at the shared points, or the wall state."""
        if getattr(self.mesh, "frames", None) is not None:
            return self._exterior_located(U, E, d, s, nq)
        nb = self.nbr[E, d, s]
        interior = nb >= 0
        nb_safe = torch.where(interior, nb, E)
        phi_p, grad_p, _ = self.face_tables(nq, d, 1 - s)
        Up = self.values(phi_p, U[nb_safe])
        J_p = self.jacobian(self.xyz[nb_safe], grad_p)
        Jinv_p = torch.linalg.inv(J_p)
        Gp = self.gradients(grad_p, Jinv_p, U[nb_safe])
        if not bool(interior.all()):
            ghost = ph.wall_ghost_state(Um, self.phys)
            mask = interior[:, None, None]
            Up = torch.where(mask, Up, ghost)
        return Up, Gp, interior, nb_safe

    def _exterior_located(self, U, E, d, s, nq):
        """Rotated-frame meshes: the neighbour's polynomial and its physical gradient at the physical positions
        of this cell's face points, located in the neighbour's own reference frame (periodic boxes, no walls).
        A face point is located through its box coordinates.  On deformed meshes this finds the same physical
        point because both cells interpolate the same deformation at the same face nodes, so their degree-k
        geometries have the same trace on the shared face."""
        m = self.mesh
        En = E.numpy()
        nb = self.nbr[E, d, s]
        pts, _ = face_points(nq, d, s)
        eta = m.to_box(En, pts) - m.offset[En, d, s][:, None, :]  # box coordinates in the neighbour's box
        zeta = m.from_box(nb.numpy(), eta)  # [len(E), P, 3] in the neighbour's frame
        phi, grad = basis_3d(m.nodes_1d, zeta.reshape(-1, 3))
        P, n3 = pts.shape[0], m.n ** 3
        phi = _t(phi).reshape(len(E), P, n3)
        grad = _t(grad).reshape(len(E), P, n3, 3)
        Un = U[nb]
        Up = torch.einsum("epn,ecn->epc", phi, Un)
        Jinv = torch.linalg.inv(torch.einsum("ean,epnb->epab", self.xyz[nb], grad))
        gxi = torch.einsum("epnb,ecn->epcb", grad, Un)
        Gp = torch.einsum("epba,epcb->epca", Jinv, gxi)
        return Up, Gp, torch.ones(len(E), dtype=torch.bool), nb

    def _face_chunk(self, U, E, d, s, what):
        g, phys = self.phys.gamma, self.phys
        Ue = U[E]
        R = torch.zeros_like(Ue)
        if what in (WHAT_ALL, WHAT_CONV):
            nq = self.nq_conv
            phi, _, _ = self.face_tables(nq, d, s)
            _, nrm, dAw = self.face_geometry(E, nq, d, s)
            Um = self.values(phi, Ue)
            Up, _, _, _ = self._exterior(U, E, d, s, nq, Um)
            lam = torch.maximum(torch.linalg.norm(Um[..., 1:4] / Um[..., 0:1], dim=-1) + ph.sound_speed(Um, g),
                                torch.linalg.norm(Up[..., 1:4] / Up[..., 0:1], dim=-1) + ph.sound_speed(Up, g))
            Fn = 0.5 * torch.einsum("epca,epa->epc", ph.conv_flux(Um, g) + ph.conv_flux(Up, g), nrm)
            flux = Fn + 0.5 * lam[..., None] * (Um - Up)
            R = R + self.test_val(phi, flux, dAw)
        if what in (WHAT_ALL, WHAT_VISC):
            nq = self.nq_visc
            phi, grad, _ = self.face_tables(nq, d, s)
            Jinv, nrm, dAw = self.face_geometry(E, nq, d, s)
            Um = self.values(phi, Ue)
            Gm = self.gradients(grad, Jinv, Ue)
            Up, Gp, interior, nb_safe = self._exterior(U, E, d, s, nq, Um)
            Gp = torch.where(interior[:, None, None, None], Gp, Gm)  # wall: grad U+ = grad U-
            tau = torch.where(interior, torch.maximum(self.tau_cell[E], self.tau_cell[nb_safe]), self.tau_cell[E])
            jump = Um - Up
            Fv_avg = 0.5 * (ph.visc_flux(Um, Gm, phys) + ph.visc_flux(Up, Gp, phys))
            Qn = torch.einsum("epca,epa->epc", Fv_avg, nrm) - tau[:, None, None] * jump
            R = R - self.test_val(phi, Qn, dAw)
            Fj = ph.visc_flux(Um, jump[..., :, None] * nrm[..., None, :], phys)
            R = R - 0.5 * self.test_grad(grad, Jinv, Fj, dAw)
        return R

    # -- mass matrix, body force, L(U) -------------------------------------------------
    def mass_matrices(self, E):
        phi, _, _ = self.cell_tables(self.nq_mass)
        _, wdet = self.cell_geometry(E, self.nq_mass)
        return torch.einsum("pi,pj,ep->eij", phi, phi, wdet)

    def mass_solve(self, R):
        """M^{-1} R per cell by a dense LU solve of M_e = B^T diag(|J| w) B (k+1 points)."""
        out = []
        for E in self._chunks():
            M = self.mass_matrices(E)
            out.append(torch.linalg.solve(M, R[E].transpose(1, 2)).transpose(1, 2))
        return torch.cat(out, 0)

    def mass_apply(self, U):
        out = []
        for E in self._chunks():
            out.append(torch.einsum("eij,ecj->eci", self.mass_matrices(E), U[E]))
        return torch.cat(out, 0)

    def body_force(self, U, source=None, t=0.0):
        """(V, F_rhs) with F_rhs = (0, f, f.u) at k+1 points (Sec. 2.2.3).

        ``source(x, t)`` (optional) adds a manufactured source S(x, t) [..., 5]
        integrated at nq_conv points.
        """
        return torch.cat([self.body_force_cells(U, E, source, t) for E in self._chunks()], 0)

    def body_force_cells(self, U, E, source=None, t=0.0):
        f = torch.tensor(self.phys.body_force, dtype=torch.float64)
        Ue = U[E]
        phi, _, _ = self.cell_tables(self.nq_mass)
        _, wdet = self.cell_geometry(E, self.nq_mass)
        Uq = self.values(phi, Ue)
        u = Uq[..., 1:4] / Uq[..., 0:1]
        zero = torch.zeros_like(Uq[..., 0:1])
        Frhs = torch.cat([zero, f.expand(Uq.shape[:-1] + (3,)), (u * f).sum(-1, keepdim=True)], dim=-1)
        r = self.test_val(phi, Frhs, wdet)
        if source is not None:
            phi_s, _, _ = self.cell_tables(self.nq_conv)
            _, wdet_s = self.cell_geometry(E, self.nq_conv)
            xq = torch.einsum("pn,ean->epa", phi_s, self.xyz[E])
            r = r + self.test_val(phi_s, source(xq, t), wdet_s)
        return r

    def residual_cells(self, U, E, what=WHAT_ALL):
        """F(U) restricted to the cells E (element-based form: each cell's rows need only U)."""
        return self._residual_chunk(U, torch.as_tensor(E), what)

    def L_cells(self, U, E):
        """L(U) restricted to the cells E (M is block diagonal)."""
        E = torch.as_tensor(E)
        rhs = -self.residual_cells(U, E)
        if self.has_body_force():
            rhs = rhs + self.body_force_cells(U, E)
        M = self.mass_matrices(E)
        return torch.linalg.solve(M, rhs.transpose(1, 2)).transpose(1, 2)

    def has_body_force(self):
        return any(float(b) != 0.0 for b in self.phys.body_force)

    def L(self, U, what=WHAT_ALL, source=None, t=0.0):
        """L(U) = M^{-1}(-F(U) + F_rhs(U)) (Eq. SpatiallyDiscretizedProblem)."""
        rhs = -self.residual(U, what)
        if self.has_body_force() or source is not None:
            rhs = rhs + self.body_force(U, source, t)
        return self.mass_solve(rhs)

    # -- helpers -------------------------------------------------------------------------
    def integrate(self, U, nq=None):
        """Sum over cells of int U dOmega with a Gauss rule of nq points (default k+1)."""
        nq = self.nq_mass if nq is None else nq
        phi, _, _ = self.cell_tables(nq)
        tot = torch.zeros(U.shape[1], dtype=torch.float64)
        for E in self._chunks():
            _, wdet = self.cell_geometry(E, nq)
            tot = tot + torch.einsum("pn,ecn,ep->c", phi, U[E], wdet)
        return tot
