"""Algorithmic work of the libdgcns kernels, for roofline reporting.

Counts mirror the kernels' structure: every 1D sweep line with DIN inputs and
DOUT outputs costs 2*DIN*DOUT flops (one FMA = 2 flops), pointwise work uses
per-point operation counts of the flux routines (a division or square root
counts as one flop).  Bytes are the algorithmic HBM traffic of one launch
(each array read or written once).
"""

# per-point operation counts of the pointwise routines (adds, muls, FMAs as 2, div/sqrt as 1)
PT_CELL_CONV = 62      # 1/rho, pressure, 3 directional fluxes, contravariant scaling
PT_CELL_VISC = 150     # velocity/temperature gradients, stress, energy flux, scaling
PT_FACE_CONV = 110     # both traces: 1/rho, pressure, wave speed; LLF combination
PT_FACE_VISC = 420     # F_v on both sides, F_v(U-, [[U]] (x) n), penalty, scaling
PT_FACE_VISC_PAIR = 520  # face-centric: + F_v(U+, [[U]] (x) n) for the other cell
PT_MASS = 1


def _sweep(lines, din, dout):
    return lines * 2 * din * dout


def cell_flops(N, QC, QV):
    """Cell integrals of one cell (5 components)."""
    f = 0
    # convective: interpolate (3), pointwise, 3 collocation tests, 3 transposed interpolations
    f += 5 * (_sweep(N * N, N, QC) + _sweep(N * QC, N, QC) + _sweep(QC * QC, N, QC))
    f += 3 * 5 * _sweep(QC * QC, QC, QC)
    f += 5 * (_sweep(QC * QC, QC, N) + _sweep(QC * N, QC, N) + _sweep(N * N, QC, N))
    f += PT_CELL_CONV * QC ** 3
    # viscous: interpolate (3), 3 collocation gradients, pointwise, 3 tests, 3 transposed
    f += 5 * (_sweep(N * N, N, QV) + _sweep(N * QV, N, QV) + _sweep(QV * QV, N, QV))
    f += 2 * 3 * 5 * _sweep(QV * QV, QV, QV)
    f += 5 * (_sweep(QV * QV, QV, N) + _sweep(QV * N, QV, N) + _sweep(N * N, QV, N))
    f += PT_CELL_VISC * QV ** 3
    return f


def face_flops(N, QC, QV):
    """One face evaluated for one side (element-centric: each cell does its 6 faces)."""
    f = 0
    interp_c = _sweep(N, N, QC) + _sweep(QC, N, QC)
    f += 5 * 2 * interp_c                                # both traces
    f += 5 * (_sweep(QC, QC, N) + _sweep(N, QC, N))      # test
    f += PT_FACE_CONV * QC * QC
    interp_v = _sweep(N, N, QV) + _sweep(QV, N, QV)
    f += 5 * 2 * N * N * 2 * N                           # normal derivatives, both sides
    f += 5 * 4 * interp_v                                # values and normal derivatives, both sides
    f += 5 * 4 * _sweep(QV, QV, QV)                      # tangential collocation derivatives
    f += 5 * 2 * _sweep(QV, QV, QV)                      # tangential gradient tests
    f += 5 * 2 * (_sweep(QV, QV, N) + _sweep(N, QV, N))  # value and normal-gradient tests
    f += 5 * N * N * N * 2                               # scatter along the normal lines
    f += PT_FACE_VISC * QV * QV
    return f


def face_pair_flops(N, QC, QV):
    """One interior face evaluated once for both cells (face-centric kernel): shared traces and fluxes, the
    convective share of the other cell is a negation, the viscous tests are done per side."""
    f = 0
    f += 5 * 2 * (_sweep(N, N, QC) + _sweep(QC, N, QC))      # both traces
    f += 5 * (_sweep(QC, QC, N) + _sweep(N, QC, N))          # one test
    f += PT_FACE_CONV * QC * QC
    interp_v = _sweep(N, N, QV) + _sweep(QV, N, QV)
    f += 5 * 2 * N * N * 2 * N                               # normal derivatives, both sides
    f += 5 * 4 * interp_v                                    # values and normal derivatives, both sides
    f += 5 * 4 * _sweep(QV, QV, QV)                          # tangential collocation derivatives, both sides
    f += 2 * 5 * 2 * _sweep(QV, QV, QV)                      # tangential gradient tests, both sides
    f += 2 * 5 * 2 * (_sweep(QV, QV, N) + _sweep(N, QV, N))  # value and normal-gradient tests, both sides
    f += PT_FACE_VISC_PAIR * QV * QV
    return f


def gather_flops(N):
    """Adding the 6 face shares of a cell (value layer + normal-gradient coefficients along the normal lines)."""
    return 5 * N ** 3 * 6 * 3


def cell_stage_flops_per_cell(N, QC, QV):
    """Face-centric cell kernel: cell integrals + face shares + inverse mass + update."""
    return cell_flops(N, QC, QV) + gather_flops(N) + mass_flops(N) + 4 * 5 * N ** 3


def kernel_flops(kind, N, QC, QV, Nc):
    """Algorithmic flops of one launch of a kernel kind (names of dg_cns_kernel_times) on a periodic mesh of
    Nc cells (3 Nc faces)."""
    per = {"fused": stage_flops_per_cell(N, QC, QV) * Nc,
           "faces": face_pair_flops(N, QC, QV) * 3 * Nc,
           "cell_stage": cell_stage_flops_per_cell(N, QC, QV) * Nc,
           "cell": cell_flops(N, QC, QV) * Nc,
           "face": 6 * face_flops(N, QC, QV) * Nc,
           "mass": (mass_flops(N) + 4 * 5 * N ** 3) * Nc}
    return per.get(kind)


def kernel_bytes(kind, N, Nc, rbytes):
    """Algorithmic HBM bytes of one launch (stages 1..4: dU read), as the kernels run inside dg_cns_rk_steps.

    FP64 (rbytes 8): the operator kernels read U (8 B per value).  Mixed form (rbytes 4): they read the FP32
    deviation state (4 B per value), and the stage kernels of the fused and face-centric organisations also
    read U for the FP64 update and write the next deviation state.  Every stage kernel reads U, reads and
    writes dU and writes U_out; the split M^-1 + stage kernel also reads the residual.  Face shares: 60 n^2
    values per cell."""
    nodes = Nc * N ** 3
    v = nodes * 5
    shares = 60 * N * N * Nc * rbytes
    s = 8 if rbytes == 8 else 4
    dev = 0 if rbytes == 8 else 4 + 4
    upd = v * (8 + rbytes + rbytes + 8)
    per = {"fused": upd + v * dev,
           "faces": v * s + shares,
           "cell_stage": upd + v * dev + shares,
           "cell": v * (s + rbytes),
           "face": v * (s + 2 * rbytes),
           "mass": upd + v * rbytes}
    return per.get(kind)


def mass_flops(N):
    return 5 * 6 * _sweep(N * N, N, N) + 5 * N ** 3 * PT_MASS


def stage_flops_per_cell(N, QC, QV):
    """Fused RK stage: cell integrals + 6 faces + inverse mass + update (4 flops/value)."""
    return cell_flops(N, QC, QV) + 6 * face_flops(N, QC, QV) + mass_flops(N) + 4 * 5 * N ** 3


def stage_bytes_per_node(precision_bytes, first_stage=False):
    """Fused stage: read U (8 B/value), read dU (not at A_1 = 0), write dU, write U_out; 5 values per node."""
    r = precision_bytes
    return 5 * (8 + (0 if first_stage else r) + r + 8)


def split_extra_bytes_per_node(precision_bytes):
    """Split kernels: the residual is written by the cell kernel, read+written by the face kernel, read by the
    mass/stage kernel, and U is read three times."""
    r = precision_bytes
    return 5 * (r + 2 * r + r + 2 * 8)
