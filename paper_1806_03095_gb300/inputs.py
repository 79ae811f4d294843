"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the DG method's arithmetic: it only draws seeded
random numbers and evaluates the closed-form initial fields of the two
workloads at node coordinates supplied by the caller (each side supplies its
own coordinates).  Everything is float64 on the CPU (torch.Generator with
manual seeds), then moved to the requested device.

Taylor--Green vortex (Sec. 4.2.1): u = U0 (sin x cos y cos z, -cos x sin y cos z, 0),
p = p0 + rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2), uniform T0 = c0^2/(gamma R),
c0 = U0/M, p0 = rho0 R T0, rho = p/(R T0), rho E = rho (c_v T0 + |u|^2/2).

Channel (Sec. 4.3.1, laminar start): rho = 1, T = T0 = c^2/(gamma R) with
c = u_max / M, u1 = u_max (1 - y^2) plus a seeded uniform perturbation of
amplitude 5 % of u_max on every velocity component.
"""
import math

import torch


def _gen(seed):
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def uniform(shape, seed, lo=-1.0, hi=1.0):
    """Seeded uniform float64 samples in [lo, hi) on the CPU."""
    r = torch.rand(tuple(shape), generator=_gen(seed), dtype=torch.float64)
    return lo + (hi - lo) * r


def random_state(n_cells, n_nodes, seed, rho0=1.0, mom=0.1, rhoE0=178.57142857142858, amp=0.1):
    """Random conserved state [n_cells, 5, n_nodes] with positive density and pressure.

    rho in rho0 (1 +- amp), momentum components in +-mom, rho E in rhoE0 (1 +- amp).
    Nodal values are independent draws, so the state is discontinuous across
    faces and exercises every jump term.
    """
    r = uniform((n_cells, 5, n_nodes), seed)
    U = torch.empty_like(r)
    U[:, 0] = rho0 * (1.0 + amp * r[:, 0])
    U[:, 1:4] = mom * r[:, 1:4]
    U[:, 4] = rhoE0 * (1.0 + amp * r[:, 4])
    return U


def random_direction(shape, seed):
    """Seeded standard-normal array normalised to unit 2-norm (adjoint test directions)."""
    v = torch.randn(tuple(shape), generator=_gen(seed), dtype=torch.float64)
    return v / torch.linalg.norm(v)


def tgv_state(xyz, gamma=1.4, R=287.0, Ma=0.1, rho0=1.0, U0=1.0, L=1.0):
    """Taylor--Green initial state at node coordinates xyz [Nc, 3, n^3] -> U [Nc, 5, n^3]."""
    x, y, z = xyz[:, 0] / L, xyz[:, 1] / L, xyz[:, 2] / L
    u1 = U0 * torch.sin(x) * torch.cos(y) * torch.cos(z)
    u2 = -U0 * torch.cos(x) * torch.sin(y) * torch.cos(z)
    u3 = torch.zeros_like(u1)
    c0 = U0 / Ma
    T0 = c0 * c0 / (gamma * R)
    p0 = rho0 * R * T0
    p = p0 + rho0 * U0 * U0 / 16.0 * (torch.cos(2 * x) + torch.cos(2 * y)) * (torch.cos(2 * z) + 2.0)
    rho = p / (R * T0)
    cv = R / (gamma - 1.0)
    rhoE = rho * (cv * T0 + 0.5 * (u1 * u1 + u2 * u2 + u3 * u3))
    return torch.stack([rho, rho * u1, rho * u2, rho * u3, rhoE], dim=1)


def channel_state(xyz, seed, u_max=18.3, Ma=0.1, gamma=1.4, R=287.0, rho0=1.0, amp=0.05):
    """Laminar parabolic channel profile plus seeded 5 % uniform velocity perturbation."""
    y = xyz[:, 1]
    pert = uniform((xyz.shape[0], 3, xyz.shape[2]), seed).to(xyz.device)
    u1 = u_max * (1.0 - y * y) + amp * u_max * pert[:, 0]
    u2 = amp * u_max * pert[:, 1]
    u3 = amp * u_max * pert[:, 2]
    c = u_max / Ma
    T0 = c * c / (gamma * R)
    rho = torch.full_like(u1, rho0)
    cv = R / (gamma - 1.0)
    rhoE = rho * (cv * T0 + 0.5 * (u1 * u1 + u2 * u2 + u3 * u3))
    return torch.stack([rho, rho * u1, rho * u2, rho * u3, rhoE], dim=1)


TWO_PI = 2.0 * math.pi
