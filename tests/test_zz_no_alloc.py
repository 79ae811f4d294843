"""dg_cns_diagnostics_noalloc: the diagnostics variant for callers that may not allocate memory
while they run (their device memory is owned by a pool, or allocation is not permitted at that
point).  Its partial sums live in a static device array; the test calls it through the C ABI
twice in a row and checks both results against dg_cns_diagnostics, and checks that a mesh too
large for the static scratch is refused before anything runs.

tests/conftest.py sorts this file after every other test (full-size cases included), so a run that stops
at its first failure has already run everything else when it reaches this file."""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_1806_03095_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

PI = math.pi


def _ctx(n, k, precision):
    from paper_1806_03095_gb300.api import DGCNS
    return DGCNS((n, n, n), (-PI,) * 3, (PI,) * 3, (1, 1, 1), k, (3 * k) // 2 + 1, k + 1, precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_diagnostics_match_two_calls_in_a_row(precision):
    g = _ctx(6, 3, precision)
    U = inputs.tgv_state(g.node_coords()) + 1e-3 * inputs.uniform(g.shape, 21).cuda()
    LU = g.apply(U.contiguous())
    ref = g.diagnostics(U, LU)
    lib = _lib.load()
    out = torch.full((_lib.NDIAG,), float("nan"), dtype=torch.float64, device=U.device)
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.dg_cns_diagnostics_noalloc(g.ctx, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(LU.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()))
        assert rc == 0, lib.dg_cns_last_error(g.ctx)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the GPU sums the partial rows in another order than the host: the integrals of momentum (about 0
        # on this periodic box) agree to rounding in absolute terms
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), (got, ref)
    # without L(U): -de_k/dt is reported as 0, the rest unchanged
    out2 = g.dg_cns_diagnostics_noalloc(U)
    torch.cuda.synchronize()
    ref2 = g.diagnostics(U)
    assert np.allclose(out2.cpu().numpy(), ref2, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_mesh_beyond_scratch():
    rows = _lib.NOALLOC_SCRATCH_BYTES // 80
    g = _ctx(60, 5, 0)  # 216000 cells, one cell per partial row at k = 5 (nq_conv^3 = 512)
    assert g.n_cells > rows
    lib = _lib.load()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.dg_cns_diagnostics_noalloc(g.ctx, ctypes.c_void_p(dummy.data_ptr()), None,
                                        ctypes.c_void_p(dummy.data_ptr()))
    assert rc == -1
    assert b"too large" in lib.dg_cns_last_error(g.ctx)
