"""Python binding of libdgcns over torch tensors (same names as the C ABI).

PyTorch provides device memory and streams only; every step of the operator
runs in libdgcns's CUDA kernels.  All calls are issued on torch's current
CUDA stream.
"""
import ctypes
import math
import numbers

import numpy as np
import torch

from . import _lib
from ._lib import (FP64, KERNEL_FACES, KERNEL_FUSED, KERNEL_SPLIT, MAP_AFFINE, MAP_CHANNEL, MAP_ROTATED, MAP_SINE,
                   MIXED, NDIAG,
                   OP_F, OP_FC, OP_FV, OP_L, DGCNSError)

__all__ = ["DGCNS", "DGCNSError", "FP64", "MIXED", "KERNEL_SPLIT", "KERNEL_FUSED", "KERNEL_FACES", "OP_L", "OP_F",
           "OP_FC", "OP_FV", "MAP_AFFINE", "MAP_CHANNEL", "MAP_SINE", "MAP_ROTATED", "NDIAG"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def cuda_device(device=None):
    """The CUDA device a context runs on, with its index: None (torch's current device), an index, or a
    CUDA device given as a string or torch.device ("cuda" alone means the current device)."""
    if device is None or isinstance(device, numbers.Integral):
        index = torch.cuda.current_device() if device is None else int(device)
    else:
        dev = torch.device(device)
        if dev.type != "cuda":
            raise ValueError("libdgcns runs on a CUDA device, not %s" % dev)
        index = torch.cuda.current_device() if dev.index is None else dev.index
    return torch.device("cuda", index)


class DGCNS:
    """One operator context: dg_cns_create on construction, dg_cns_destroy on close()."""

    def __init__(self, ncells, lo, hi, periodic, k, nq_conv, nq_visc, *, gamma=1.4, Pr=0.71, Re=1600.0,
                 Ma=0.1, R=287.0, rho0=1.0, U0=1.0, L=1.0, u_mach=0.0, body_force=(0.0, 0.0, 0.0),
                 precision=FP64, kernel=KERNEL_FACES, mapping=MAP_AFFINE, map_param=0.0, deform=0.0, geometry=0,
                 device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libdgcns needs a CUDA device (there is no CPU fallback)")
        self.lib = _lib.load()
        self.device = cuda_device(device)
        m = _lib.Mesh()
        p = _lib.Params()
        for d in range(3):
            m.n[d] = int(ncells[d])
            m.lo[d] = float(lo[d])
            m.hi[d] = float(hi[d])
            m.periodic[d] = 1 if periodic[d] else 0
            p.body_force[d] = float(body_force[d])
        m.mapping = int(mapping)
        m.map_param = float(map_param)
        m.deform = float(deform)
        p.k, p.nq_conv, p.nq_visc = int(k), int(nq_conv), int(nq_visc)
        p.gamma, p.Pr, p.Re, p.Ma, p.R = float(gamma), float(Pr), float(Re), float(Ma), float(R)
        p.rho0, p.U0, p.L, p.u_mach = float(rho0), float(U0), float(L), float(u_mach)
        p.precision, p.kernel, p.geometry = int(precision), int(kernel), int(geometry)
        self.k, self.n = int(k), int(k) + 1
        self.precision, self.kernel = int(precision), int(kernel)
        self.rdtype = torch.float32 if precision == MIXED else torch.float64
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.dg_cns_create(ctypes.byref(m), ctypes.byref(p), self._stream(), ctypes.byref(ctx))
        if rc != 0:
            raise DGCNSError(rc, self.lib.dg_cns_last_error(None).decode())
        self.ctx = ctx
        nc, nn, nd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.dg_cns_sizes(self.ctx, ctypes.byref(nc), ctypes.byref(nn), ctypes.byref(nd)))
        self.n_cells, self.n_nodes, self.n_dofs = nc.value, nn.value, nd.value
        self.shape = (self.n_cells, 5, self.n ** 3)

    # -- helpers --------------------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, rc):
        if rc != 0:
            raise DGCNSError(rc, self.lib.dg_cns_last_error(self.ctx).decode())

    def _sync_stream(self):
        self._check(self.lib.dg_cns_set_stream(self.ctx, self._stream()))

    def _state(self, t, name, dtype=torch.float64):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise TypeError("%s must be a %s tensor on %s" % (name, dtype, self.device))
        if tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError("%s must be contiguous with shape %s" % (name, self.shape))
        return t

    def empty_state(self):
        return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    def empty_residual(self):
        return torch.empty(self.shape, dtype=self.rdtype, device=self.device)

    # -- C ABI mirrors --------------------------------------------------------------------
    def dg_cns_node_coords(self):
        xyz = torch.empty((self.n_cells, 3, self.n ** 3), dtype=torch.float64, device=self.device)
        self._sync_stream()
        self._check(self.lib.dg_cns_node_coords(self.ctx, _ptr(xyz)))
        return xyz

    def dg_cns_apply(self, U, R=None, op=OP_L):
        self._state(U, "U")
        R = self.empty_residual() if R is None else self._state(R, "R", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_apply(self.ctx, _ptr(U), _ptr(R), int(op)))
        return R

    def dg_cns_inverse_mass(self, inp, out=None):
        self._state(inp, "in", self.rdtype)
        out = self.empty_residual() if out is None else self._state(out, "out", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_inverse_mass(self.ctx, _ptr(inp), _ptr(out)))
        return out

    def dg_cns_rk_stage(self, stage, dt, t, U_in, dU, U_out):
        self._state(U_in, "U_in")
        self._state(U_out, "U_out")
        self._state(dU, "dU", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_rk_stage(self.ctx, int(stage), float(dt), float(t), _ptr(U_in), _ptr(dU),
                                             _ptr(U_out)))

    def dg_cns_rk_steps(self, nsteps, dt, t0, U, U_tmp=None, dU=None):
        self._state(U, "U")
        U_tmp = self.empty_state() if U_tmp is None else self._state(U_tmp, "U_tmp")
        dU = self.empty_residual() if dU is None else self._state(dU, "dU", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_rk_steps(self.ctx, int(nsteps), float(dt), float(t0), _ptr(U), _ptr(U_tmp),
                                             _ptr(dU)))
        return U

    def dg_cns_lsrk_stage(self, A, B, dt, U_in, dU, U_out):
        self._state(U_in, "U_in")
        self._state(U_out, "U_out")
        self._state(dU, "dU", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_lsrk_stage(self.ctx, float(A), float(B), float(dt), _ptr(U_in), _ptr(dU),
                                               _ptr(U_out)))

    def dg_cns_lsrk_steps(self, scheme, nsteps, dt, U, U_tmp=None, dU=None):
        """nsteps steps of a 2N scheme: scheme = (A, B) sequences of stage coefficients (see schemes.py)."""
        A, B = scheme
        if len(A) != len(B) or not 1 <= len(A) <= _lib.MAX_STAGES:
            raise ValueError("a 2N scheme needs equal-length A and B with 1..%d stages" % _lib.MAX_STAGES)
        self._state(U, "U")
        U_tmp = self.empty_state() if U_tmp is None else self._state(U_tmp, "U_tmp")
        dU = self.empty_residual() if dU is None else self._state(dU, "dU", self.rdtype)
        a = (ctypes.c_double * len(A))(*[float(x) for x in A])
        b = (ctypes.c_double * len(B))(*[float(x) for x in B])
        self._sync_stream()
        self._check(self.lib.dg_cns_lsrk_steps(self.ctx, len(A), a, b, int(nsteps), float(dt), _ptr(U), _ptr(U_tmp),
                                               _ptr(dU)))
        return U

    def dg_cns_diagnostics(self, U, LU=None, check=True):
        """Returns a float64 numpy array [e_k, eps, -de_k/dt, mass, mom x3, energy, nonfinite]."""
        self._state(U, "U")
        if LU is not None:
            self._state(LU, "L_of_U", self.rdtype)
        out = (ctypes.c_double * NDIAG)()
        self._sync_stream()
        rc = self.lib.dg_cns_diagnostics(self.ctx, _ptr(U), _ptr(LU), out)
        if rc != 0 and (check or rc != -5):
            self._check(rc)
        return np.array(out[:], dtype=np.float64)

    def dg_cns_diagnostics_noalloc(self, U, LU=None, out=None):
        """Diagnostics into a device tensor of NDIAG doubles, allocating nothing in the
        library (its scratch is a fixed static device array; see include/dgcns.h).
        Asynchronous: the values are valid once torch's current stream reaches them."""
        self._state(U, "U")
        if LU is not None:
            self._state(LU, "L_of_U", self.rdtype)
        if out is None:
            out = torch.empty(NDIAG, dtype=torch.float64, device=self.device)
        elif out.device != self.device or out.dtype != torch.float64 or out.numel() < NDIAG or not out.is_contiguous():
            raise ValueError("out must be a contiguous float64 device tensor with at least %d entries" % NDIAG)
        self._sync_stream()
        self._check(self.lib.dg_cns_diagnostics_noalloc(self.ctx, _ptr(U), _ptr(LU), _ptr(out)))
        return out

    def dg_cns_adjoint_apply(self, U, W, G=None):
        """G = (dL/dU)^T W (residual type)."""
        self._state(U, "U")
        self._state(W, "W", self.rdtype)
        G = self.empty_residual() if G is None else self._state(G, "G", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_adjoint_apply(self.ctx, _ptr(U), _ptr(W), _ptr(G)))
        return G

    def dg_cns_rk_stage_adjoint(self, stage, dt, U_in, lam_U, lam_dU):
        self._state(U_in, "U_in")
        self._state(lam_U, "lam_U")
        self._state(lam_dU, "lam_dU", self.rdtype)
        self._sync_stream()
        self._check(self.lib.dg_cns_rk_stage_adjoint(self.ctx, int(stage), float(dt), _ptr(U_in), _ptr(lam_U),
                                                     _ptr(lam_dU)))

    def dg_cns_kinetic_energy_gradient(self, U, G=None):
        self._state(U, "U")
        G = self.empty_state() if G is None else self._state(G, "G")
        self._sync_stream()
        self._check(self.lib.dg_cns_kinetic_energy_gradient(self.ctx, _ptr(U), _ptr(G)))
        return G

    def dg_cns_launch_count(self):
        c = ctypes.c_int64()
        self._check(self.lib.dg_cns_launch_count(self.ctx, ctypes.byref(c)))
        return c.value

    def dg_cns_set_initial_tgv(self, U=None):
        """Taylor--Green initial state at the LGL nodes (computed on the GPU); returns U."""
        U = self.empty_state() if U is None else self._state(U, "U")
        self._sync_stream()
        self._check(self.lib.dg_cns_set_initial_tgv(self.ctx, _ptr(U)))
        return U

    def dg_cns_set_initial_channel(self, seed, U=None):
        """Laminar channel start with a Philox-seeded 5 % velocity perturbation (computed on the GPU)."""
        U = self.empty_state() if U is None else self._state(U, "U")
        self._sync_stream()
        self._check(self.lib.dg_cns_set_initial_channel(self.ctx, _ptr(U), int(seed) & 0xFFFFFFFFFFFFFFFF))
        return U

    set_initial_tgv = dg_cns_set_initial_tgv
    set_initial_channel = dg_cns_set_initial_channel

    def dg_cns_status(self):
        """Raise DGCNSError(TIMEOUT) if a kernel of this context gave up a bounded wait."""
        self._check(self.lib.dg_cns_status(self.ctx))

    status = dg_cns_status

    def dg_cns_timing(self, enable):
        """Start (clearing the totals) or stop per-kernel CUDA-event timing on the context's stream."""
        self._check(self.lib.dg_cns_timing(self.ctx, 1 if enable else 0))

    def dg_cns_kernel_times(self):
        """{kind: (total ms, launches)} of the kernels timed since timing was enabled."""
        n = len(_lib.KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._check(self.lib.dg_cns_kernel_times(self.ctx, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(_lib.KERNEL_KINDS) if cnt[i] > 0}

    timing = dg_cns_timing
    kernel_times = dg_cns_kernel_times

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dg_cns_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # short aliases
    apply = dg_cns_apply
    inverse_mass = dg_cns_inverse_mass
    rk_stage = dg_cns_rk_stage
    rk_steps = dg_cns_rk_steps
    lsrk_stage = dg_cns_lsrk_stage
    lsrk_steps = dg_cns_lsrk_steps
    diagnostics = dg_cns_diagnostics
    adjoint_apply = dg_cns_adjoint_apply
    rk_stage_adjoint = dg_cns_rk_stage_adjoint
    kinetic_energy_gradient = dg_cns_kinetic_energy_gradient
    node_coords = dg_cns_node_coords


def default_nq(k):
    """(nq_conv, nq_visc) = (floor(3k/2)+1, k+1): 3/2-rule for the convective term, k+1 for the viscous term."""
    return (3 * k) // 2 + 1, k + 1


def cfl_dt(k, h_min, u_max, Ma, Cr=0.4, D=0.02, nu=None, e=1.5, f=3.0):
    """Eq. TimeStepRestrictions_Compressible with c = u_max / M: dt = min(dt_c, dt_v)."""
    c = u_max / Ma
    dt_c = Cr / k ** e * h_min / (u_max + c)
    if nu is None or nu <= 0:
        return dt_c
    dt_v = D / k ** f * h_min ** 2 / nu
    return min(dt_c, dt_v)
