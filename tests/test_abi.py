"""CPU checks of the C ABI: the library loads and exports every symbol the header
declares; argument validation runs on the host (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1806_03095_gb300 import _lib
from paper_1806_03095_gb300.build import LIB, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "dgcns.h")).read()
    return sorted(set(re.findall(r"\b(dg_cns_\w+)\s*\(", text)))


def test_header_and_binding_agree():
    assert header_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_header_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_structs_match_header_layout(tmp_path):
    """Sizes and field offsets of the ctypes structs equal those the C compiler gives the header's."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"dgcns_mesh": (_lib.Mesh, [f[0] for f in _lib.Mesh._fields_]),
              "dgcns_params": (_lib.Params, [f[0] for f in _lib.Params._fields_])}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dgcns.h"', "int main(void) {"]
    for cname, (_, names) in fields.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for n in names:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, n))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = []
    for cname, (st, names) in fields.items():
        want.append(ctypes.sizeof(st))
        want.extend(getattr(st, n).offset for n in names)
    assert got == want


def test_create_validates_on_host(lib):
    m, p, ctx = _lib.Mesh(), _lib.Params(), ctypes.c_void_p()
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -2
    assert b"k must be" in lib.dg_cns_last_error(None)
    p.k, p.nq_conv, p.nq_visc = 3, 3, 4
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -1
    p.nq_conv = 5
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -1  # empty mesh
    assert ctx.value is None
    assert lib.dg_cns_create(None, None, None, ctypes.byref(ctx)) == -1


@pytest.mark.parametrize("n", [(1025, 1024, 1024), (1 << 21, 1 << 21, 1 << 22), (2 ** 31 - 1,) * 3])
def test_create_rejects_too_many_cells_on_host(lib, n):
    """More than 2^30 cells is refused before any device work, also where the product of the three
    counts would overflow 64 bits (2^21 * 2^21 * 2^22 = 2^64)."""
    m, p = _mesh_params(3, 5, 4)
    m.n[0], m.n[1], m.n[2] = n
    ctx = ctypes.c_void_p()
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -1
    assert ctx.value is None
    assert b"too many cells" in lib.dg_cns_last_error(None)


def _no_device():
    import torch
    return not torch.cuda.is_available()


@pytest.mark.skipif(not _no_device(), reason="the failure path of a machine without a GPU")
def test_create_without_a_device_reports_the_cuda_error(lib):
    """A valid configuration on a machine without a GPU: the first CUDA call (the device lookup) fails, the call
    returns DGCNS_ERR_CUDA (not OOM) with the CUDA error in the message, and no context."""
    m, p = _mesh_params(3, 5, 4)
    ctx = ctypes.c_void_p()
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -3
    assert ctx.value is None
    assert lib.dg_cns_last_error(None).startswith(b"CUDA error (cudaGetDevice): ")
    # a later failure of a different kind replaces the message
    m.n[0] = 0
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -1
    assert lib.dg_cns_last_error(None) == b"bad mesh extents"


def _mesh_params(k, qc, qv, precision=0, kernel=2, mapping=0, geometry=0):
    m, p = _lib.Mesh(), _lib.Params()
    for d in range(3):
        m.n[d], m.lo[d], m.hi[d], m.periodic[d] = 2, 0.0, 1.0, 1
    m.mapping, m.map_param = mapping, {1: 1.8, 3: 1806.0}.get(mapping, 0.05)
    if mapping == 1:
        m.periodic[1], m.lo[1] = 0, -1.0
    p.k, p.nq_conv, p.nq_visc = k, qc, qv
    p.gamma, p.Pr, p.Re, p.Ma, p.R, p.rho0, p.U0, p.L = 1.4, 0.71, 1600.0, 0.1, 287.0, 1.0, 1.0, 1.0
    p.precision, p.kernel, p.geometry = precision, kernel, geometry
    return m, p


@pytest.mark.parametrize("case,code", [
    (dict(k=1, qc=2, qv=2, precision=1), -2),            # mixed form not compiled at k = 1
    (dict(k=1, qc=2, qv=2, mapping=1), -2),              # non-affine geometry not compiled at k = 1
    (dict(k=2, qc=4, qv=3, mapping=2, geometry=1), -2),  # geometry on the fly only at k = 3
    (dict(k=3, qc=6, qv=4), -2),                         # no instantiation for this quadrature pair
    (dict(k=7, qc=11, qv=8, precision=1), -2),           # k = 7 only in FP64
    (dict(k=6, qc=13, qv=13), -2),                       # the 2k+1 rule at k = 2..5 and 7 only
    (dict(k=3, qc=5, qv=4, kernel=3), -1),               # unknown kernel organisation
    (dict(k=3, qc=5, qv=4, geometry=2), -1),             # unknown geometry mode
    (dict(k=3, qc=5, qv=4, precision=2), -1),            # unknown precision
    (dict(k=2, qc=4, qv=3, mapping=3, geometry=1, kernel=1), -2),  # geometry on the fly only at k = 3
])
def test_create_rejects_uncompiled_or_invalid_features_on_host(lib, case, code):
    """The feature table of the instantiations answers before any device work."""
    m, p = _mesh_params(**case)
    ctx = ctypes.c_void_p()
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == code
    assert ctx.value is None
    assert lib.dg_cns_last_error(None)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.dg_cns_destroy(None) == -1
    assert lib.dg_cns_apply(None, None, None, 0) == -1
    assert lib.dg_cns_rk_stage(None, 0, 1.0, 0.0, None, None, None) == -1
    c = ctypes.c_int64()
    assert lib.dg_cns_launch_count(None, ctypes.byref(c)) == -1
    assert lib.dg_cns_timing(None, 1) == -1
    assert lib.dg_cns_status(None) == -1
    assert lib.dg_cns_set_initial_tgv(None, None) == -1
    assert lib.dg_cns_set_initial_channel(None, None, 1) == -1
    assert lib.dg_cns_kernel_times(None, None, None, 0) == -1


def test_plain_c_client_links_and_checks_the_host_contract(lib, tmp_path):
    """tests/c_abi_client.c: a C99 program that includes only the header and links only the library."""
    import shutil
    import subprocess

    import torch
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(LIB)
    exe = tmp_path / "client"
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi_client.c"), "-L", libdir, "-ldgcns",
                           "-Wl,-rpath," + libdir, "-o", str(exe)])
    p = subprocess.run([str(exe)] + (["gpu"] if torch.cuda.is_available() else []), stdout=subprocess.PIPE,
                       stderr=subprocess.PIPE, text=True, timeout=120)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.splitlines()[-1] == "failures 0"


def test_kernel_kinds_match_header():
    text = open(os.path.join(ROOT, "include", "dgcns.h")).read()
    kinds = dict((name.lower(), int(v)) for name, v in re.findall(r"#define DGCNS_KT_(\w+) (\d+)", text))
    assert kinds.pop("count") == len(_lib.KERNEL_KINDS)
    assert sorted(kinds, key=kinds.get) == list(_lib.KERNEL_KINDS)


def test_library_is_in_tree():
    assert os.path.dirname(LIB) == os.path.join(ROOT, "paper_1806_03095_gb300")


@pytest.mark.parametrize("change,message", [
    (lambda m: m.periodic.__setitem__(2, 0), b"rotated-frame meshes must be periodic on every axis"),
    (lambda m: setattr(m, "map_param", -1.0), b"the frame seed (map_param) must be a non-negative integer below 2^64"),
    (lambda m: setattr(m, "map_param", 2.5), b"the frame seed (map_param) must be a non-negative integer below 2^64"),
    (lambda m: setattr(m, "map_param", 2.0 ** 64), b"the frame seed (map_param) must be a non-negative integer below 2^64"),
    (lambda m: setattr(m, "deform", float("nan")), b"deform must be finite, and 0 unless the mapping is DGCNS_MAP_ROTATED"),
    (lambda m: (setattr(m, "mapping", 2), setattr(m, "deform", 0.05)),
     b"deform must be finite, and 0 unless the mapping is DGCNS_MAP_ROTATED"),
])
def test_create_validates_rotated_frame_meshes_on_host(lib, change, message):
    m, p = _mesh_params(3, 5, 4, kernel=1, mapping=3, geometry=1)
    change(m)
    ctx = ctypes.c_void_p()
    assert lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), None, ctypes.byref(ctx)) == -1
    assert ctx.value is None
    assert lib.dg_cns_last_error(None) == message
