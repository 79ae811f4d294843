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
amplitude 5 % of u_max on every velocity component, drawn from the counter-based
generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), which libdgcns
implements from the same definition (dg_cns_set_initial_channel), so both sides
produce the same numbers.
"""
import math

import numpy as np
import torch

_PHILOX_M = (0xD2511F53, 0xCD9E8D57)  # round multipliers
_PHILOX_W = (0x9E3779B9, 0xBB67AE85)  # key increments (Weyl sequence)


def philox4x32(ctr, key):
    """Philox4x32-10: counters ctr (4 arrays of uint32 words), key (k0, k1) -> 4 arrays of output words.

    Each of the 10 rounds multiplies words 0 and 2 by the round multipliers (64-bit products split into
    high and low halves), mixes the high halves with words 1 and 3 and the key, and permutes; the key is
    bumped by the Weyl increments between rounds.
    """
    mask = np.uint64(0xFFFFFFFF)
    c = [np.asarray(x, dtype=np.uint64) & mask for x in ctr]
    k0, k1 = np.uint64(key[0]) & mask, np.uint64(key[1]) & mask
    m0, m1 = np.uint64(_PHILOX_M[0]), np.uint64(_PHILOX_M[1])
    for r in range(10):
        p0, p1 = m0 * c[0], m1 * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & mask, p1 & mask, ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & mask,
             p0 & mask]
        k0, k1 = (k0 + np.uint64(_PHILOX_W[0])) & mask, (k1 + np.uint64(_PHILOX_W[1])) & mask
    return c


def philox_uniform(n, seed):
    """n float64 uniforms in [0, 1): element i comes from block i // 2 (counter (i // 2, 0, 0, 0), key (seed mod
    2^32, seed div 2^32)), words (0, 1) for even i and (2, 3) for odd i, as (a >> 5) 2^26 + (b >> 6) times 2^-53."""
    nb = (int(n) + 1) // 2
    j = np.arange(nb, dtype=np.uint64)
    w = philox4x32([j & np.uint64(0xFFFFFFFF), j >> np.uint64(32), np.zeros(nb, np.uint64), np.zeros(nb, np.uint64)],
                   (int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF))
    a = np.stack([w[0], w[2]], 1).reshape(-1)[:n]
    b = np.stack([w[1], w[3]], 1).reshape(-1)[:n]
    k = ((a >> np.uint64(5)) << np.uint64(26)) | (b >> np.uint64(6))
    return torch.from_numpy(k.astype(np.float64) * 2.0 ** -53)


def cell_frames(n_cells, seed):
    """Reference frames of a rotated-frame box mesh: frame e = min(floor(48 u_e), 47) with u_e the e-th Philox
    uniform of the seed (frame g: the (g // 8)-th permutation of the axes in lexicographic order, reflection
    bits g % 8)."""
    u = philox_uniform(n_cells, seed).numpy()
    return np.minimum(np.floor(48.0 * u), 47).astype(np.int64)


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


def parity_state(ncells, n_nodes, seed, rho0=1.0, mom=0.1, rhoE0=178.57142857142858, amp=0.02, contrast=0.4):
    """Random conserved state [cells, 5, n_nodes] on a box of ncells = (nx, ny, nz) cells (x fastest) whose
    energy level alternates between face neighbours: rho E in rhoE0 (1 + contrast)(1 +- amp) on cells with
    i + j + k even and rhoE0 (1 - contrast)(1 +- amp) on odd ones; rho in rho0 (1 +- amp), momentum in +-mom.

    Nodal values are independent draws, so every face carries jumps; with an even cell count along each
    periodic axis the two cells of every face differ in parity, so the sound speeds of the two traces are
    separated by a wide margin at every face point.
    """
    nx, ny, nz = (int(v) for v in ncells)
    r = uniform((nx * ny * nz, 5, n_nodes), seed)
    e = torch.arange(nx * ny * nz)
    odd = ((e % nx) + (e // nx) % ny + e // (nx * ny)) % 2
    level = torch.where(odd == 0, 1.0 + contrast, 1.0 - contrast).to(torch.float64)
    U = torch.empty_like(r)
    U[:, 0] = rho0 * (1.0 + amp * r[:, 0])
    U[:, 1:4] = mom * r[:, 1:4]
    U[:, 4] = rhoE0 * level[:, None] * (1.0 + amp * r[:, 4])
    return U


def smooth_direction(xyz, seed, kmax=1):
    """Seeded smooth velocity direction [Nc, 3, n^3] at node coordinates xyz [Nc, 3, n^3] of a 2 pi periodic
    box: each component is sum_kappa (a cos(kappa . x) + b sin(kappa . x)) over the integer wave vectors
    0 < |kappa|_inf <= kmax with standard-normal a, b, scaled to unit root-mean-square over all nodal
    entries (a step h along it moves every nodal velocity by about h)."""
    g = _gen(seed)
    r = torch.arange(-kmax, kmax + 1, dtype=torch.float64)
    kap = torch.cartesian_prod(r, r, r)
    kap = kap[kap.abs().sum(1) > 0]
    phase = torch.einsum("kd,edn->ekn", kap, xyz.double().cpu())
    out = []
    for _ in range(3):
        a = torch.randn(kap.shape[0], generator=g, dtype=torch.float64)
        b = torch.randn(kap.shape[0], generator=g, dtype=torch.float64)
        out.append(torch.einsum("k,ekn->en", a, torch.cos(phase)) + torch.einsum("k,ekn->en", b, torch.sin(phase)))
    v = torch.stack(out, 1)
    return v / torch.sqrt((v * v).mean())


def fd_direction(u0, xyz, seed):
    """Seeded direction for central differences of a functional of the velocity field u0 [Nc, 3, n^3]: the
    field itself (scaled to unit root-mean-square) plus smooth_direction(xyz, seed), the sum scaled to unit
    root-mean-square.  Its directional derivative stays well above the rounding noise of the differences,
    which a purely random direction (nearly orthogonal to the gradient) does not guarantee."""
    u = u0.double().cpu()
    v = u / torch.sqrt((u * u).mean()) + smooth_direction(xyz, seed)
    return v / torch.sqrt((v * v).mean())


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
    """Laminar parabolic channel profile plus a seeded 5 % uniform velocity perturbation in [-1, 1) (Philox,
    element index (cell * 3 + component) * n^3 + node)."""
    y = xyz[:, 1]
    n = xyz.shape[0] * 3 * xyz.shape[2]
    pert = (-1.0 + 2.0 * philox_uniform(n, seed)).reshape(xyz.shape[0], 3, xyz.shape[2]).to(xyz.device)
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
