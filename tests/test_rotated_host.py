"""Host logic of rotated-frame meshes (CPU, no device): the frames and the face table that dg_cns_create
builds, through the host-only dg_cns_face_table, against the input module's generator and the oracle's
geometry (RotatedBoxMesh: neighbours by geometry, node coordinates from the frames)."""
import ctypes
import itertools

import numpy as np
import pytest

from oracle.mesh import RotatedBoxMesh
from paper_1806_03095_gb300 import _lib, inputs

LO, HI = (-1.0, 0.0, 0.5), (2.0, 1.5, 2.5)


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def rotated_mesh(ncells, seed):
    m = _lib.Mesh()
    for d in range(3):
        m.n[d], m.lo[d], m.hi[d], m.periodic[d] = ncells[d], LO[d], HI[d], 1
    m.mapping, m.map_param = 3, float(seed)
    return m


def face_table(lib, ncells, seed):
    Nc = int(np.prod(ncells))
    table, frames = (ctypes.c_int * (12 * Nc))(), (ctypes.c_int * Nc)()
    assert lib.dg_cns_face_table(ctypes.byref(rotated_mesh(ncells, seed)), table, frames) == 0
    return np.array(table).reshape(Nc, 6, 2), np.array(frames)


def decode(code, i, N):
    """The neighbour's own node index of node i = (i0, i1, i2) of the neighbour seen in the cell's frame."""
    j = []
    for b in range(3):
        v = i[(code >> (2 * b)) & 3]
        j.append(N - 1 - v if (code >> (6 + b)) & 1 else v)
    return j[0] + N * (j[1] + N * j[2])


def orientation_gap(table, mesh, decoder=decode):
    """Largest distance, relative to the box, between node q of each neighbour seen in the cell's frame (the
    cell's reference point xi_q moved by one cell across the face) and the neighbour's own node that the code
    names, over every cell, local face and node."""
    N, Nc = mesh.n, mesh.Nc
    L = mesh.hi - mesh.lo
    cc = mesh.cell_coords()
    worst = 0.0
    for e in range(Nc):
        for f in range(6):
            d, s = divmod(f, 2)
            n, code = table[e, f]
            for i in itertools.product(range(N), repeat=3):
                i = (i[2], i[1], i[0])
                xi = mesh.nodes_1d[list(i)].copy()
                xi[d] += 1.0 if s else -1.0
                x = mesh.lo + (cc[e] + mesh.to_box(np.array([e]), xi[None])[0, 0]) * mesh.h
                xn = mesh.xyz[n, :, decoder(code, i, N)]
                g = (x - xn) / L
                worst = max(worst, float(np.abs(g - np.round(g)).max()))
    return worst


@pytest.mark.parametrize("ncells,seed", [((3, 2, 4), 1806), ((4, 3, 3), (1 << 40) + 3), ((1, 3, 2), 7)])
def test_face_table_matches_the_oracle_geometry(lib, ncells, seed):
    table, frames = face_table(lib, ncells, seed)
    # the library's Philox4x32-10 frames are the input module's
    assert np.array_equal(frames, inputs.cell_frames(len(frames), seed))
    mesh = RotatedBoxMesh(ncells, LO, HI, 3, frames)
    # neighbours: the oracle finds them by geometry
    assert np.array_equal(table[:, :, 0], mesh.nbr.reshape(-1, 6))
    # orientation codes: every node lands on the physical node the code names
    assert orientation_gap(table, mesh) < 1e-12


def test_face_table_negative_control(lib):
    """Planted mistake in the decoding: reflection bits ignored."""
    table, frames = face_table(lib, (3, 2, 4), 1806)
    mesh = RotatedBoxMesh((3, 2, 4), LO, HI, 3, frames)

    def no_reflection(code, i, N):
        return decode(code & 63, i, N)

    assert orientation_gap(table, mesh, no_reflection) > 1e-3


def test_face_table_refuses_other_meshes(lib):
    Nc = 24
    table = (ctypes.c_int * (12 * Nc))()
    m = rotated_mesh((3, 2, 4), 1806)
    m.periodic[1] = 0
    assert lib.dg_cns_face_table(ctypes.byref(m), table, None) == -1
    assert lib.dg_cns_last_error(None) == b"rotated-frame meshes must be periodic on every axis"
    m = rotated_mesh((3, 2, 4), 1806)
    m.mapping = 0
    assert lib.dg_cns_face_table(ctypes.byref(m), table, None) == -1
    m = rotated_mesh((3, 2, 4), 2.5)
    assert lib.dg_cns_face_table(ctypes.byref(m), table, None) == -1
    assert lib.dg_cns_face_table(ctypes.byref(rotated_mesh((3, 2, 4), 1806)), None, None) == -1
