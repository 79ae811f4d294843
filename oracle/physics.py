"""Compressible Navier--Stokes physics (oracle; test infrastructure only).

Sec. 2.1: conserved variables U = (rho, rho u, rho E); ideal gas p = rho R T;
calorically perfect gas E = c_v T + |u|^2/2, c_v = R/(gamma-1); Newtonian
stress with zero bulk viscosity; Fourier heat flux q = -lambda grad T.
Eq. CompressibleNavierStokesFluxes: F_c, F_v, F_rhs.  F_v is linear in its
gradient argument, F_v(U, grad U) = G(U) : grad U, so visc_flux(U, G) accepts
any 5x3 array in place of grad U (used with the jump [[U]] on faces).

Point values carry the component on the last axis (U[..., 5]) and gradients
carry (component, direction) on the last two axes (G[..., 5, 3]),
G[..., c, j] = dU_c / dx_j.
"""
from dataclasses import dataclass

import torch


@dataclass
class Physics:
    gamma: float
    R: float
    mu: float
    lam: float
    rho0: float
    T_wall: float = 0.0
    body_force: tuple = (0.0, 0.0, 0.0)

    @property
    def c_v(self):
        return self.R / (self.gamma - 1.0)

    @property
    def c_p(self):
        return self.gamma * self.R / (self.gamma - 1.0)

    @property
    def nu(self):
        """Kinematic viscosity nu = mu / rho_0 scaling the penalty (Eq. TauIP_Element)."""
        return self.mu / self.rho0

    @staticmethod
    def from_numbers(Re, Pr, Ma, gamma=1.4, R=287.0, rho0=1.0, U0=1.0, L=1.0, u_mach=None,
                     body_force=(0.0, 0.0, 0.0)):
        """Sec. 4.2.1: Re = rho0 U0 L / mu, Pr = mu c_p / lambda, M = U/c0, T0 = c0^2/(gamma R)."""
        mu = rho0 * U0 * L / Re
        c_p = gamma * R / (gamma - 1.0)
        lam = mu * c_p / Pr
        c0 = (U0 if u_mach is None else u_mach) / Ma
        T0 = c0 * c0 / (gamma * R)
        return Physics(gamma=gamma, R=R, mu=mu, lam=lam, rho0=rho0, T_wall=T0,
                       body_force=tuple(float(b) for b in body_force))


def pressure(U, gamma):
    rho = U[..., 0]
    m = U[..., 1:4]
    return (gamma - 1.0) * (U[..., 4] - 0.5 * (m * m).sum(-1) / rho)


def sound_speed(U, gamma):
    """c = sqrt(|gamma p / rho|) (text after the LLF flux, Sec. 2.2.2)."""
    return torch.sqrt(torch.abs(gamma * pressure(U, gamma) / U[..., 0]))


def conv_flux(U, gamma):
    """F_c(U) of Eq. CompressibleNavierStokesFluxes: rows rho u, rho u (x) u + p I, (rho E + p) u."""
    rho = U[..., 0]
    m = U[..., 1:4]
    u = m / rho[..., None]
    p = pressure(U, gamma)[..., None]
    eye = torch.eye(3, dtype=U.dtype)
    rows = [m]
    for i in range(3):
        rows.append(m[..., i:i + 1] * u + p * eye[i])
    rows.append((U[..., 4:5] + p) * u)
    return torch.stack(rows, dim=-2)


def velocity_gradient(U, G):
    """grad u from conserved gradients: (grad m - u (x) grad rho) / rho."""
    rho = U[..., 0]
    u = U[..., 1:4] / rho[..., None]
    return (G[..., 1:4, :] - u[..., :, None] * G[..., 0:1, :]) / rho[..., None, None]


def temperature_gradient(U, G, phys):
    """grad T with T = (E - |u|^2/2)/c_v, E = rho E / rho: grad T = (grad E - (grad u)^T u) / c_v."""
    rho = U[..., 0]
    u = U[..., 1:4] / rho[..., None]
    E = U[..., 4] / rho
    gradE = (G[..., 4, :] - E[..., None] * G[..., 0, :]) / rho[..., None]
    gu = velocity_gradient(U, G)
    return (gradE - (gu * u[..., :, None]).sum(-2)) / phys.c_v


def visc_flux(U, G, phys):
    """F_v(U, G) of Eq. CompressibleNavierStokesFluxes with G in place of grad U.

    tau = mu (grad u + grad u^T - 2/3 div u I); rows 0, tau, (tau . u)^T + lambda grad T.
    """
    rho = U[..., 0]
    u = U[..., 1:4] / rho[..., None]
    gu = velocity_gradient(U, G)
    div = gu[..., 0, 0] + gu[..., 1, 1] + gu[..., 2, 2]
    eye = torch.eye(3, dtype=U.dtype)
    tau = phys.mu * (gu + gu.transpose(-1, -2) - (2.0 / 3.0) * div[..., None, None] * eye)
    gT = temperature_gradient(U, G, phys)
    energy = (tau * u[..., :, None]).sum(-2) + phys.lam * gT
    zero = torch.zeros_like(energy)
    return torch.cat([zero[..., None, :], tau, energy[..., None, :]], dim=-2)


def wall_ghost_state(U, phys):
    """Exterior state on an isothermal no-slip wall (reading; the paper omits the imposition).

    Sec. 4.3.1 prescribes homogeneous Neumann data for rho, T = T_wall and no
    slip.  Mirror reading: rho+ = rho-, u+ = -u-, T+ = 2 T_wall - T-, so that
    the face averages are u = 0 and T = T_wall; rho E+ follows from rho+, u+, T+.
    """
    rho = U[..., 0]
    u = U[..., 1:4] / rho[..., None]
    ke = 0.5 * (u * u).sum(-1)
    T = (U[..., 4] / rho - ke) / phys.c_v
    Tp = 2.0 * phys.T_wall - T
    return torch.cat([rho[..., None], -U[..., 1:4], (rho * (phys.c_v * Tp + ke))[..., None]], dim=-1)
