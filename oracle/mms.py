"""Manufactured solutions for convergence pins (oracle; test infrastructure only).

A smooth periodic field U_ex(x) is chosen in primitive variables and the
source S = dU/dt + div F_c(U) - div F_v(U, grad U) of
Eq. CompressibleNavierStokesCompact is evaluated exactly by forward-mode
automatic differentiation (torch.func.jacfwd, nested for the second
derivatives inside div F_v): no hand algebra.  The semi-discrete problem
M dU/dt = -F(U) + (V, S) then has U_ex as its smooth steady solution, and the
DG error after a short integration converges with the mesh size.

Euler entropy wave: rho = 1 + 0.2 sin(x+y+z-3t), u = (1,1,1), p = 1 solves
the inviscid equations exactly with no source.
"""
import torch
from torch.func import jacfwd, vmap

from . import physics as ph


def steady_primitive(x):
    """rho = 1 + 0.1 sin(x+y+z), u = 0.1 (sin y, sin z, sin x), p = 1 + 0.1 cos(x - y)."""
    rho = 1.0 + 0.1 * torch.sin(x[0] + x[1] + x[2])
    u = 0.1 * torch.stack([torch.sin(x[1]), torch.sin(x[2]), torch.sin(x[0])])
    p = 1.0 + 0.1 * torch.cos(x[0] - x[1])
    return rho, u, p


def conserved(prim_fun, gamma):
    def U(x):
        rho, u, p = prim_fun(x)
        return torch.cat([rho[None], rho * u, (p / (gamma - 1.0) + 0.5 * rho * (u * u).sum())[None]])
    return U


def steady_source(phys):
    """Return S(xq [..., 3], t) -> [..., 5] for the steady manufactured field."""
    Ufun = conserved(steady_primitive, phys.gamma)

    def flux(x):
        U = Ufun(x)
        G = jacfwd(Ufun)(x)
        return ph.conv_flux(U, phys.gamma) - ph.visc_flux(U, G, phys)

    def S_point(x):
        dF = jacfwd(flux)(x)  # [5, 3, 3]: d F[c, j] / d x_l
        return dF[:, 0, 0] + dF[:, 1, 1] + dF[:, 2, 2]

    Sv = vmap(S_point)

    def source(xq, t):
        shp = xq.shape
        return Sv(xq.reshape(-1, 3)).reshape(shp[:-1] + (5,))

    return source


def steady_exact(xyz, gamma):
    """U_ex at node coordinates xyz [Nc, 3, n^3] -> [Nc, 5, n^3]."""
    Ufun = vmap(conserved(steady_primitive, gamma))
    pts = xyz.permute(0, 2, 1).reshape(-1, 3)
    return Ufun(pts).reshape(xyz.shape[0], xyz.shape[2], 5).permute(0, 2, 1).contiguous()


def entropy_wave_exact(xyz, t, gamma):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rho = 1.0 + 0.2 * torch.sin(x + y + z - 3.0 * t)
    one = torch.ones_like(rho)
    rhoE = one / (gamma - 1.0) + 0.5 * rho * 3.0
    return torch.stack([rho, rho, rho, rho, rhoE], dim=1)
