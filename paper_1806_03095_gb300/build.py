"""Build libdgcns.so in-tree with nvcc for sm_103a (GB300).

One translation unit per (k+1, nq_conv, nq_visc) instantiation and part (FP64
operator, FP32 operator, diagnostics + geometry, adjoint) plus the host file,
compiled in parallel, then linked into paper_1806_03095_gb300/libdgcns.so.
Usage: python -m paper_1806_03095_gb300.build [--jobs N] [--force]
"""
import argparse
import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdgcns.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", INCLUDE]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdgcns")
    return exe


def configs():
    """(N, QC, QV) triples of DGCNS_CONFIGS in dg_launchers.h."""
    text = open(os.path.join(CSRC, "dg_launchers.h")).read()
    block = text[text.index("#define DGCNS_CONFIGS(X)"):]
    block = block[:block.index("\n\n")]
    return [tuple(int(v) for v in m) for m in re.findall(r"X\((\d+),\s*(\d+),\s*(\d+)\)", block)]


def parts():
    text = open(os.path.join(CSRC, "dg_launchers.h")).read()
    return int(re.search(r"#define DGCNS_PARTS (\d+)", text).group(1))


def _sources_digest(extra=()):
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                h.update(name.encode())
                h.update(open(os.path.join(d, name), "rb").read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed: %s\n%s" % (" ".join(cmd), p.stdout))
    return p.stdout


def build(jobs=None, force=False, verbose=False, extra=()):
    """Compile libdgcns.so if the sources changed; returns the library path."""
    digest = _sources_digest(extra)
    stamp = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    jobs = jobs or max(1, min(16, os.cpu_count() or 1))
    cmds = []
    objs = []
    for (N, QC, QV) in configs():
        for part in range(parts()):
            obj = os.path.join(BUILD, "inst_%d_%d_%d_%d.o" % (N, QC, QV, part))
            cmds.append([exe, *ARCH, *FLAGS, *extra, "-DINST_N=%d" % N, "-DINST_QC=%d" % QC, "-DINST_QV=%d" % QV,
                         "-DINST_PART=%d" % part, "-c", os.path.join(CSRC, "dg_inst.cu"), "-o", obj])
            objs.append(obj)
    host_obj = os.path.join(BUILD, "dgcns.o")
    cmds.append([exe, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, "dgcns.cu"), "-o", host_obj])
    objs.append(host_obj)

    # longest translation units first (the operator and adjoint parts of the largest point sets), so that
    # the wall time is not set by a long one started last
    def cost(cmd):
        d = dict(a[2:].split("=") for a in cmd if a.startswith("-DINST_"))
        if not d:
            return 1e6
        q = int(d["INST_QC"]) ** 3 + int(d["INST_QV"]) ** 3
        return q * {"0": 4, "1": 2, "3": 3, "4": 2, "6": 2}.get(d["INST_PART"], 1)

    cmds.sort(key=cost, reverse=True)
    with cf.ThreadPoolExecutor(jobs) as ex:
        outs = list(ex.map(_run, cmds))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp"
    _run([exe, *ARCH, "-shared", "--cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true", help="print register/shared-memory usage")
    a = ap.parse_args(argv)
    extra = ("-Xptxas", "-v") if a.ptxas_info else ()
    print(build(a.jobs, a.force or a.ptxas_info, a.verbose or a.ptxas_info, extra))


if __name__ == "__main__":
    sys.exit(main())
