"""ctypes declaration of the libdgcns C ABI (include/dgcns.h).

Argument marshalling only.  Loading fails loudly when the in-tree library is
missing: there is no CPU fallback.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdgcns.so")

DGCNS_OK = 0
ERR_NAMES = {-1: "INVALID_ARG", -2: "UNSUPPORTED", -3: "CUDA", -4: "OOM", -5: "NONFINITE", -6: "TIMEOUT"}

FP64, MIXED = 0, 1
KERNEL_SPLIT, KERNEL_FUSED, KERNEL_FACES = 0, 1, 2
MAP_AFFINE, MAP_CHANNEL, MAP_SINE, MAP_ROTATED = 0, 1, 2, 3
GEO_STORED, GEO_ON_THE_FLY = 0, 1
OP_L, OP_F, OP_FC, OP_FV = 0, 1, 2, 3
NDIAG = 9
MAX_STAGES = 32  # DGCNS_MAX_STAGES of dg_cns_lsrk_steps
NOALLOC_SCRATCH_BYTES = 16 << 20  # static device scratch of dg_cns_diagnostics_noalloc

# Every symbol include/dgcns.h declares.
EXPORTS = ("dg_cns_create", "dg_cns_destroy", "dg_cns_set_stream", "dg_cns_sizes", "dg_cns_node_coords",
           "dg_cns_set_initial_tgv", "dg_cns_set_initial_channel",
           "dg_cns_apply", "dg_cns_inverse_mass", "dg_cns_rk_stage", "dg_cns_rk_steps", "dg_cns_lsrk_stage",
           "dg_cns_lsrk_steps", "dg_cns_diagnostics",
           "dg_cns_diagnostics_noalloc", "dg_cns_adjoint_apply", "dg_cns_rk_stage_adjoint",
           "dg_cns_kinetic_energy_gradient", "dg_cns_launch_count", "dg_cns_status", "dg_cns_timing", "dg_cns_kernel_times",
           "dg_cns_face_table", "dg_cns_last_error")

# Kernel kinds of dg_cns_kernel_times (DGCNS_KT_*).
KERNEL_KINDS = ("cell", "face", "mass", "fused", "faces", "cell_stage", "dev", "adj_prep", "adj_faces", "adj",
                "other")


class Mesh(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("mapping", ctypes.c_int), ("map_param", ctypes.c_double),
                ("deform", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nq_conv", ctypes.c_int), ("nq_visc", ctypes.c_int),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("Ma", ctypes.c_double), ("R", ctypes.c_double), ("rho0", ctypes.c_double),
                ("U0", ctypes.c_double), ("L", ctypes.c_double), ("u_mach", ctypes.c_double),
                ("body_force", ctypes.c_double * 3), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("geometry", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


_lib = None


def load(path=LIB_PATH):
    """Load libdgcns.so and declare its signatures (cached)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdgcns.so not found at %s: build it with `python -m paper_1806_03095_gb300.build` "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    vp, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    ci, cd = ctypes.c_int, ctypes.c_double
    sig = {
        "dg_cns_create": ([ctypes.POINTER(Mesh), ctypes.POINTER(Params), vp, ctypes.POINTER(vp)], ci),
        "dg_cns_destroy": ([vp], ci),
        "dg_cns_set_stream": ([vp, vp], ci),
        "dg_cns_sizes": ([vp, i64p, i64p, i64p], ci),
        "dg_cns_node_coords": ([vp, vp], ci),
        "dg_cns_set_initial_tgv": ([vp, vp], ci),
        "dg_cns_set_initial_channel": ([vp, vp, ctypes.c_uint64], ci),
        "dg_cns_apply": ([vp, vp, vp, ci], ci),
        "dg_cns_inverse_mass": ([vp, vp, vp], ci),
        "dg_cns_rk_stage": ([vp, ci, cd, cd, vp, vp, vp], ci),
        "dg_cns_rk_steps": ([vp, ci, cd, cd, vp, vp, vp], ci),
        "dg_cns_lsrk_stage": ([vp, cd, cd, cd, vp, vp, vp], ci),
        "dg_cns_lsrk_steps": ([vp, ci, dp, dp, ci, cd, vp, vp, vp], ci),
        "dg_cns_diagnostics": ([vp, vp, vp, dp], ci),
        "dg_cns_diagnostics_noalloc": ([vp, vp, vp, vp], ci),
        "dg_cns_adjoint_apply": ([vp, vp, vp, vp], ci),
        "dg_cns_rk_stage_adjoint": ([vp, ci, cd, vp, vp, vp], ci),
        "dg_cns_kinetic_energy_gradient": ([vp, vp, vp], ci),
        "dg_cns_launch_count": ([vp, i64p], ci),
        "dg_cns_status": ([vp], ci),
        "dg_cns_timing": ([vp, ci], ci),
        "dg_cns_kernel_times": ([vp, dp, i64p, ci], ci),
        "dg_cns_face_table": ([ctypes.POINTER(Mesh), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ci),
        "dg_cns_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class DGCNSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libdgcns error %d (%s): %s" % (code, ERR_NAMES.get(code, "?"), msg))
        self.code = code
