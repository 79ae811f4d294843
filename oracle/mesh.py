"""Structured hexahedral box meshes (oracle; test infrastructure only).

Sec. 4.2.1: uniform Cartesian grids (Taylor--Green vortex).  Sec. 4.3.1:
channel grid refined towards the walls by x2 -> delta*tanh(C(2 x2 - 1))/tanh(C)
with an isoparametric mapping of degree k.  A smooth periodic sinusoidal
deformation serves as the "deformed element" mesh of Sec. 4.1 in tests.

Cell index e = cx + nx*(cy + ny*cz); per-cell node index i0 + n*i1 + n^2*i2.
Coordinates of the degree-k geometry are the mapping evaluated at the LGL
nodes of every cell (isoparametric).

RotatedBoxMesh gives every cell of a periodic box its own reference frame, one
of the 48 symmetries of the cube, so that neighbouring cells meet with every
relative orientation a hexahedral mesh generator can produce (the general
unstructured meshes of Sec. 2 and Sec. 3.1, where the two sides of a face see
its points in different orders).
"""
import itertools

import numpy as np

from .basis import lgl_nodes_01

MAP_AFFINE, MAP_CHANNEL, MAP_SINE, MAP_ROTATED = 0, 1, 2, 3


def sine_deformation(x, lo, hi, A):
    """Periodic displacement of box points x [..., 3] with amplitude A (fraction of the box length): a
    different product of phase-shifted sines per component (phase 0.5*a*(b+1) on axis b of component a), so
    J is not the identity plus a rank-one term."""
    L = hi - lo
    X = (x - lo) / L
    disp = []
    for a in range(3):
        s = 1.0
        for b in range(3):
            s = s * np.sin(2 * np.pi * X[..., b] + 0.5 * a * (b + 1))
        disp.append(A * L[a] * s)
    return x + np.stack(disp, axis=-1)


class BoxMesh:
    def __init__(self, ncells, lo, hi, periodic, k, mapping=MAP_AFFINE, map_param=0.0):
        self.ncells = tuple(int(v) for v in ncells)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.periodic = tuple(bool(p) for p in periodic)
        self.k = int(k)
        self.n = self.k + 1
        self.mapping = int(mapping)
        self.map_param = float(map_param)
        self.nodes_1d = lgl_nodes_01(self.k)
        self.Nc = int(np.prod(self.ncells))
        self.h = (self.hi - self.lo) / np.asarray(self.ncells, dtype=np.float64)
        self.xyz = self._node_coords()
        self.nbr = self._neighbors()

    # -- cell indexing ---------------------------------------------------------
    def cell_coords(self):
        nx, ny, nz = self.ncells
        e = np.arange(self.Nc)
        return np.stack([e % nx, (e // nx) % ny, e // (nx * ny)], axis=1)

    def _neighbors(self):
        """nbr[e, d, s]: neighbour across face xi_d = s of cell e, or -1 on a boundary."""
        cc = self.cell_coords()
        nbr = np.full((self.Nc, 3, 2), -1, dtype=np.int64)
        for d in range(3):
            for s in range(2):
                c2 = cc.copy()
                c2[:, d] += 1 if s == 1 else -1
                inside = (c2[:, d] >= 0) & (c2[:, d] < self.ncells[d])
                if self.periodic[d]:
                    c2[:, d] %= self.ncells[d]
                    inside[:] = True
                idx = c2[:, 0] + self.ncells[0] * (c2[:, 1] + self.ncells[1] * c2[:, 2])
                nbr[:, d, s] = np.where(inside, idx, -1)
        return nbr

    # -- geometry --------------------------------------------------------------
    def map_points(self, x):
        """Apply the mesh mapping to affine box coordinates x [..., 3]."""
        x = np.array(x, dtype=np.float64, copy=True)
        L = self.hi - self.lo
        if self.mapping == MAP_CHANNEL:
            # Sec. 4.3.1: f(x2) = delta tanh(C(2 eta - 1))/tanh(C) on the wall-normal axis.
            C = self.map_param
            eta = (x[..., 1] - self.lo[1]) / L[1]
            delta, centre = 0.5 * L[1], 0.5 * (self.lo[1] + self.hi[1])
            x[..., 1] = centre + delta * np.tanh(C * (2.0 * eta - 1.0)) / np.tanh(C)
        elif self.mapping == MAP_SINE:
            x = sine_deformation(x, self.lo, self.hi, self.map_param)
        elif self.mapping != MAP_AFFINE:
            raise ValueError("unknown mapping")
        return x

    def _node_coords(self):
        n = self.n
        xi = self.nodes_1d
        i2, i1, i0 = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ref = np.stack([xi[i0.ravel()], xi[i1.ravel()], xi[i2.ravel()]], axis=1)  # [n^3, 3]
        cc = self.cell_coords().astype(np.float64)
        aff = self.lo + (cc[:, None, :] + ref[None, :, :]) * self.h  # [Nc, n^3, 3]
        phys = self.map_points(aff)
        return np.ascontiguousarray(phys.transpose(0, 2, 1))  # [Nc, 3, n^3]

    def h_min(self):
        """Minimum distance between the 8 vertices of any cell (Sec. 2.4)."""
        n = self.n
        corners = [i0 + n * i1 + n * n * i2 for i2 in (0, n - 1) for i1 in (0, n - 1) for i0 in (0, n - 1)]
        v = self.xyz[:, :, corners].transpose(0, 2, 1)  # [Nc, 8, 3]
        dist = np.linalg.norm(v[:, :, None, :] - v[:, None, :, :], axis=-1)
        dist[:, np.arange(8), np.arange(8)] = np.inf
        return float(dist.min())

    def volume(self):
        return float(np.prod(self.hi - self.lo))


# The permutations of the three axes in lexicographic order; frame g uses the (g // 8)-th.
FRAME_PERMS = np.array(list(itertools.permutations(range(3))), dtype=np.int64)


class RotatedBoxMesh(BoxMesh):
    """Periodic Cartesian box whose cells each have their own reference frame.

    frames[e] in [0, 48): permutation P = FRAME_PERMS[g // 8] and reflection bits g % 8.  A local reference
    point xi in [0,1]^3 of cell e sits at box coordinate eta_a = xi_{P[a]} along box axis a, or 1 - xi_{P[a]}
    when bit a is set; x = lo + (c + eta) h, then moved by the sine deformation of amplitude `deform` (curved
    cells).  Neighbours are found by geometry: the neighbour across a local face is the cell whose box centre
    is the mirror image of this cell's box centre in the face's box centre.
    """

    def __init__(self, ncells, lo, hi, k, frames, deform=0.0):
        frames = np.asarray(frames, dtype=np.int64).reshape(-1)
        if frames.shape[0] != int(np.prod(ncells)) or frames.min() < 0 or frames.max() > 47:
            raise ValueError("one frame in [0, 48) per cell")
        self.frames = frames
        self.perm = FRAME_PERMS[frames // 8]  # [Nc, 3]: box axis a <- local axis perm[e, a]
        self.flip = ((frames[:, None] % 8) >> np.arange(3)[None, :]) & 1 == 1  # [Nc, 3]
        self.deform = float(deform)
        super().__init__(ncells, lo, hi, (True, True, True), k)
        self.mapping = MAP_ROTATED

    def map_points(self, x):
        return sine_deformation(np.asarray(x, dtype=np.float64), self.lo, self.hi, self.deform)

    def to_box(self, E, xi):
        """Box coordinates eta [len(E), P, 3] (in the cell's own box, [0,1]^3) of local points xi of cells E;
        xi is [P, 3] (the same points in every cell) or [len(E), P, 3]."""
        E = np.asarray(E)
        xi = np.broadcast_to(np.asarray(xi, dtype=np.float64), (len(E),) + np.shape(xi)[-2:])
        idx = np.broadcast_to(self.perm[E][:, None, :], xi.shape)
        sel = np.take_along_axis(xi, idx, axis=2)  # sel[e, p, a] = xi[e, p, P[e, a]]
        return np.where(self.flip[E][:, None, :], 1.0 - sel, sel)

    def from_box(self, E, eta):
        """The inverse of to_box: local points xi [len(E), P, 3] of box coordinates eta [len(E), P, 3]."""
        E = np.asarray(E)
        val = np.where(self.flip[E][:, None, :], 1.0 - eta, eta)  # val[e, p, a] = xi[e, p, P[e, a]]
        xi = np.empty_like(val)
        np.put_along_axis(xi, np.broadcast_to(self.perm[E][:, None, :], val.shape), val, axis=2)
        return xi

    def _node_coords(self):
        n = self.n
        xi = self.nodes_1d
        i2, i1, i0 = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ref = np.stack([xi[i0.ravel()], xi[i1.ravel()], xi[i2.ravel()]], axis=1)  # [n^3, 3]
        eta = self.to_box(np.arange(self.Nc), ref)
        cc = self.cell_coords().astype(np.float64)
        phys = self.map_points(self.lo + (cc[:, None, :] + eta) * self.h)
        return np.ascontiguousarray(phys.transpose(0, 2, 1))

    def _neighbors(self):
        """nbr[e, d, s] across local face xi_d = s, and offset[e, d, s] = the neighbour's integer box
        position minus this cell's before the periodic wrap."""
        cc = self.cell_coords()
        E = np.arange(self.Nc)
        nbr = np.empty((self.Nc, 3, 2), dtype=np.int64)
        self.offset = np.empty((self.Nc, 3, 2, 3), dtype=np.int64)
        nc = np.asarray(self.ncells)
        for d in range(3):
            for s in range(2):
                centre = np.full((1, 3), 0.5)
                centre[0, d] = float(s)
                eta = self.to_box(E, centre)[:, 0, :]
                # mirror of the cell centre (box position c + 1/2) in the face centre (c + eta)
                off = np.floor(2.0 * eta - 0.5).astype(np.int64)
                self.offset[:, d, s] = off
                c2 = (cc + off) % nc
                nbr[:, d, s] = c2[:, 0] + nc[0] * (c2[:, 1] + nc[1] * c2[:, 2])
        return nbr
