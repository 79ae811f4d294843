"""Taylor--Green diagnostics and conservation totals (oracle; test infrastructure only).

Sec. 4.2.3 evaluates, as for incompressible flow,
  e_k = 1/V int 1/2 u.u,   eps = nu/V int grad u : grad u,   eps_num = -de_k/dt - eps,
with u = m / rho and nu = mu / rho_0.  -de_k/dt is taken from dU/dt = L(U):
de_k/dt = 1/V int u . (dm/dt - u drho/dt) / rho.  Integrals use the
convective Gauss rule (nq_conv points); the conservation totals
int rho, int m, int rho E use k+1 points, so that they equal 1^T M U.
"""
import torch

from . import physics as ph

NDIAG = 9  # e_k, eps, -de_k/dt, mass, mom_x, mom_y, mom_z, energy, nonfinite


def diagnostics(op, U, LU=None):
    phys = op.phys
    phi, grad, _ = op.cell_tables(op.nq_conv)
    vol = torch.zeros((), dtype=torch.float64)
    ek = torch.zeros((), dtype=torch.float64)
    eps = torch.zeros((), dtype=torch.float64)
    dek = torch.zeros((), dtype=torch.float64)
    for E in op._chunks():
        Jinv, wdet = op.cell_geometry(E, op.nq_conv)
        Uq = op.values(phi, U[E])
        Gq = op.gradients(grad, Jinv, U[E])
        u = Uq[..., 1:4] / Uq[..., 0:1]
        gu = ph.velocity_gradient(Uq, Gq)
        vol = vol + wdet.sum()
        ek = ek + (0.5 * (u * u).sum(-1) * wdet).sum()
        eps = eps + ((gu * gu).sum((-1, -2)) * wdet).sum()
        if LU is not None:
            Lq = op.values(phi, LU[E])
            dudt = (Lq[..., 1:4] - u * Lq[..., 0:1]) / Uq[..., 0:1]
            dek = dek + ((u * dudt).sum(-1) * wdet).sum()
    tot = op.integrate(U)
    out = torch.zeros(NDIAG, dtype=torch.float64)
    out[0] = ek / vol
    out[1] = phys.nu * eps / vol
    out[2] = -dek / vol if LU is not None else 0.0
    out[3:8] = tot
    out[8] = float((~torch.isfinite(U)).sum())
    return out
