/*
 * dgcns.h -- C ABI of libdgcns, a single-GPU (GB300, sm_103a) matrix-free
 * high-order discontinuous Galerkin operator for the compressible
 * Navier--Stokes equations (Fehn, Wall & Kronbichler, arXiv:1806.03095).
 *
 * Operation implemented (paper Sec. 2): the semi-discrete system
 *   M dU/dt = -F_c(U) - F_v(U) + F_rhs(U) = M L(U)      (Eq. SpatiallyDiscretizedProblem)
 * where the residual F = F_c + F_v is the weak form of
 * Eq. WeakFormulationConservedVariables: cell integrals -(grad V, F_c) +
 * (grad V, F_v); face integrals with the local Lax--Friedrichs flux
 * (V, ({{F_c}} + Lambda/2 [[U]]) . n) and the symmetric interior penalty
 * terms -(V, ({{F_v}} - tau_IP [[U]]) . n) - 1/2 (grad V, F_v(U, [[U]])),
 * tau_IP of Eq. TauIP_Element.  Integrals use Gauss--Legendre rules
 * (Eq. IntegralsNumericalQuadrature): nq_conv points per direction for the
 * convective terms, nq_visc for the viscous terms, k+1 for the mass matrix
 * and the body force (Sec. 2.2.3).  Basis: tensor-product Lagrange
 * polynomials of degree k on Legendre--Gauss--Lobatto nodes of [0,1]^3.
 *
 * Time stepping (Sec. 2.4): low-storage explicit Runge--Kutta, here the
 * five-stage fourth-order 2N scheme of Carpenter & Kennedy (1994):
 *   dU <- A_i dU + dt L(U_in, t + C_i dt);   U_out <- U_in + B_i dU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Layout of a state-like array: [n_cells][5][n^3], n = k+1, components
 *   (rho, rho u_x, rho u_y, rho u_z, rho E), node index i0 + n i1 + n^2 i2
 *   (x fastest); cell index cx + nx (cy + ny cz).
 * - All array arguments are DEVICE pointers owned by the caller, contiguous,
 *   16-byte aligned, unless stated otherwise.  U is always double.  "Residual"
 *   arrays (R, dU, W, G) are double in DGCNS_FP64 mode and float in
 *   DGCNS_MIXED mode (FP32 cell/face arithmetic and residual storage, FP64
 *   state accumulation and reductions).
 * - Calls are asynchronous on the context's stream unless stated otherwise.
 * - Every call returns DGCNS_OK (0) or a negative DGCNS_ERR_* code and never
 *   aborts or traps; dg_cns_last_error() gives a message.
 * - The context owns its geometry, 1D tables and scratch buffers.
 */
#ifndef DGCNS_H
#define DGCNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGCNS_OK 0
#define DGCNS_ERR_INVALID_ARG (-1)
#define DGCNS_ERR_UNSUPPORTED (-2)
#define DGCNS_ERR_CUDA (-3)
#define DGCNS_ERR_OOM (-4)
#define DGCNS_ERR_NONFINITE (-5)
#define DGCNS_ERR_TIMEOUT (-6)

#define DGCNS_FP64 0
#define DGCNS_MIXED 1

#define DGCNS_KERNEL_SPLIT 0 /* cell kernel, face kernel, inverse-mass/stage kernel */
#define DGCNS_KERNEL_FUSED 1 /* one kernel per stage: cells, 6 faces, M^-1, update */
/* Face-centric: a face kernel evaluates every face once and stores both cells' shares (a
   context-owned buffer of 60 (k+1)^2 values per cell), then one kernel per stage adds cells and
   face shares, applies M^-1 and the update. */
#define DGCNS_KERNEL_FACES 2

#define DGCNS_MAP_AFFINE 0   /* uniform Cartesian box (Sec. 4.2.1)                     */
#define DGCNS_MAP_CHANNEL 1  /* y -> tanh(C(2 eta - 1))/tanh(C), C = map_param (Sec. 4.3.1) */
#define DGCNS_MAP_SINE 2     /* smooth periodic deformation of amplitude map_param    */
/* Periodic affine box whose cells carry their own reference frames, as the cells of an unstructured
 * hexahedral mesh do (Sec. 4.1.1: meshes that are not Cartesian-aligned).  Cell e's frame is one of the
 * 48 symmetries of the cube, g = floor(48 u_e) with u_e the uniform of element e of Philox4x32-10 with
 * key = (uint64) map_param (as dg_cns_set_initial_channel draws them): permutation
 * P[g / 8] of {(0,1,2), (0,2,1), (1,0,2), (1,2,0), (2,0,1), (2,1,0)} and reflection bits g % 8.  A local
 * reference point xi of the cell lies at the box reference point eta with
 * eta_a = xi_{P[a]} (bit a of g clear) or 1 - xi_{P[a]} (set), so neighbouring cells see each other's
 * face nodes permuted and reflected.  With deform != 0 the node coordinates are then moved by
 * DGCNS_MAP_SINE's deformation of amplitude deform (curved cells with arbitrary relative orientations:
 * the deformed unstructured mesh of Sec. 4.1.1).  Requires all axes periodic; stored geometry or geometry
 * on the fly.  The element-centric kernels reorient each neighbour into the cell's frame as they read it
 * (state, node coordinates, stored face Jacobians); the face-centric face kernel evaluates each face in the
 * frame of the cell that owns it (the cell for which it is a local upper face) and writes the other cell's
 * share into that cell's own face slot and node order.  The adjoint calls return UNSUPPORTED. */
#define DGCNS_MAP_ROTATED 3

#define DGCNS_OP_L 0  /* L(U) = M^-1 (-F(U) + F_rhs(U))        */
#define DGCNS_OP_F 1  /* F(U) = F_c(U) + F_v(U)  (no mass matrix) */
#define DGCNS_OP_FC 2 /* F_c(U) only                           */
#define DGCNS_OP_FV 3 /* F_v(U) only                           */

#define DGCNS_NDIAG 9 /* e_k, eps, -de_k/dt, int rho, int rho u (3), int rho E, nonfinite count */

typedef struct dgcns_ctx dgcns_ctx;

/* Structured hexahedral box of n[0] x n[1] x n[2] cells on [lo, hi]
 * (Sec. 4.2.1 uniform grid, Sec. 4.3.1 stretched channel grid); a
 * non-periodic axis has no-slip isothermal walls on both ends. */
typedef struct {
  int n[3];
  double lo[3], hi[3];
  int periodic[3];
  int mapping;      /* DGCNS_MAP_* ; the geometry is isoparametric of degree k */
  double map_param; /* channel stretch C, sine amplitude (fraction of the box length), or frame seed */
  double deform;    /* DGCNS_MAP_ROTATED: amplitude of DGCNS_MAP_SINE's deformation applied to the box
                       on top of the frames (0: affine cells); must be 0 for the other mappings */
} dgcns_mesh;

/* Discretisation and physics.  mu = rho0 U0 L / Re, lambda = mu c_p / Pr,
 * c_p = gamma R/(gamma-1), c0 = u_mach / Ma (u_mach = U0 when 0),
 * T0 = c0^2/(gamma R) (wall temperature), nu = mu / rho0 (Sec. 4.2.1, 4.3.1). */
typedef struct {
  int k;         /* polynomial degree: 1..8, 11 and 15 in the shipped instantiations */
  int nq_conv;   /* Gauss points per direction for the convective terms   */
  int nq_visc;   /* Gauss points per direction for the viscous terms      */
  double gamma, Pr, Re, Ma, R, rho0, U0, L, u_mach;
  double body_force[3];
  int precision; /* DGCNS_FP64 or DGCNS_MIXED */
  int kernel;    /* DGCNS_KERNEL_SPLIT, DGCNS_KERNEL_FUSED or DGCNS_KERNEL_FACES */
  int geometry;  /* non-affine meshes: DGCNS_GEO_STORED (Jacobians stored per quadrature point, computed
                    once in FP64) or DGCNS_GEO_ON_THE_FLY (the operator kernels recompute them from the
                    node coordinates; diagnostics and the adjoint use the stored FP64 geometry) */
  int reserved[3];
} dgcns_params;

#define DGCNS_GEO_STORED 0
#define DGCNS_GEO_ON_THE_FLY 1

/* Create a context on the current CUDA device.  Every later call with the
 * context runs on that device whatever device is current when it is made: it
 * makes the context's device current for the call and restores the caller's
 * current device before it returns.  `stream` is a cudaStream_t of that
 * device (NULL = legacy default stream).  Builds the host plan (1D tables in FP64,
 * penalty per cell, geometry) and allocates the context's device buffers.  Where one
 * cell's working set exceeds a CTA's shared memory (FP64 from k = 8, and the 2k+1 rule
 * from k = 5), it also allocates a workspace of four cell slices per SM (about 0.2 GB
 * at k = 8 and 1.1 GB at k = 15 on 152 SMs); the operator kernels then run in chunks
 * of that many cells.  Rotated-frame meshes add a face table of 12 ints per cell.
 * Errors: INVALID_ARG (sizes: every n[d] >= 1 and at most 2^30 cells in all;
 * physics), UNSUPPORTED (no instantiation for (k, nq_conv, nq_visc)), OOM,
 * CUDA.  *out is NULL on error. */
int dg_cns_create(const dgcns_mesh* mesh, const dgcns_params* params, void* stream, dgcns_ctx** out);

/* Free every buffer of the context (synchronises its stream first). */
int dg_cns_destroy(dgcns_ctx* ctx);

/* Replace the stream used by later calls.  (Library utility, no counterpart in the paper.) */
int dg_cns_set_stream(dgcns_ctx* ctx, void* stream);

/* Host outputs: number of cells, nodes (n_cells (k+1)^3) and DoFs (5 nodes; the DoF count of
 * Sec. 3, five conserved fields per node). */
int dg_cns_sizes(const dgcns_ctx* ctx, int64_t* n_cells, int64_t* n_nodes, int64_t* n_dofs);

/* Node coordinates of the degree-k geometry, written to xyz [n_cells][3][n^3]
 * (device, double).  Used to set initial conditions. */
int dg_cns_node_coords(dgcns_ctx* ctx, double* xyz);

/* Taylor-Green initial state (Sec. 4.2.1) at the LGL nodes, written to U (device, FP64,
 * [n_cells][5][n^3]): u = U0 (sin x cos y cos z, -cos x sin y cos z, 0) with x = X / L, p = p0 +
 * rho0 U0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2), uniform T0 = (U0 / Ma)^2 / (gamma R), rho = p / (R T0),
 * rho E = rho (c_v T0 + |u|^2 / 2), with the context's gamma, R, Ma, rho0, U0, L.  Allocates and frees
 * a temporary device buffer for the node coordinates; synchronizes the context's stream. */
int dg_cns_set_initial_tgv(dgcns_ctx* ctx, double* U);

/* Laminar channel start (Sec. 4.3.1) at the LGL nodes: rho = rho0, u1 = u_max (1 - y^2) + 0.05 u_max p1,
 * u2 = 0.05 u_max p2, u3 = 0.05 u_max p3, rho E = rho0 (c_v T0 + |u|^2 / 2), T0 = (u_max / Ma)^2 / (gamma R),
 * u_max = the context's u_mach (must be > 0).  The perturbations p in [-1, 1) come from the counter-based
 * generator Philox4x32-10 (Salmon et al., SC'11) with key = seed: element i = (cell 3 + component) n^3 +
 * node uses block i / 2 (counter (i / 2, 0, 0, 0)), output words (0, 1) for even i and (2, 3) for odd i,
 * u = ((a >> 5) 2^26 + (b >> 6)) 2^-53, p = 2u - 1.  Same allocation and synchronization as above. */
int dg_cns_set_initial_channel(dgcns_ctx* ctx, double* U, uint64_t seed);

/* Evaluate one operator of Eq. SpatiallyDiscretizedProblem on U (device,
 * double [n_cells][5][n^3]) into R (device, residual type).  op is
 * DGCNS_OP_L, _F, _FC or _FV.  R must not overlap U (INVALID_ARG). */
int dg_cns_apply(dgcns_ctx* ctx, const double* U, void* R, int op);

/* out = M^-1 in (tensor-product inverse of the block-diagonal mass matrix,
 * Sec. 2.3: M_e^-1 = S^-1 diag(1/(|J| w)) S^-T per cell with the square
 * (k+1) x (k+1) LGL-to-Gauss matrix S).  Residual type; in == out allowed. */
int dg_cns_inverse_mass(dgcns_ctx* ctx, const void* in, void* out);

/* One stage (0..4) of the 2N RK(5,4) scheme:
 *   dU <- A_stage dU + dt L(U_in, t + C_stage dt);  U_out <- U_in + B_stage dU.
 * U_in, U_out: double; dU: residual type (read only when A_stage != 0).
 * Split and face-centric kernels allow U_out == U_in; the fused kernel needs
 * U_out != U_in (neighbours read U_in), else INVALID_ARG.  Otherwise no two of
 * U_in, U_out and dU may overlap, views at an offset included (INVALID_ARG). */
int dg_cns_rk_stage(dgcns_ctx* ctx, int stage, double dt, double t, const double* U_in, void* dU, double* U_out);

/* nsteps full RK(5,4) steps from time t0 with constant dt.  On return U holds
 * the new state; U_tmp (double, state sized) and dU (residual type) are
 * caller-provided work arrays; no two of the three may overlap (else
 * INVALID_ARG). */
int dg_cns_rk_steps(dgcns_ctx* ctx, int nsteps, double dt, double t0, double* U, double* U_tmp, void* dU);

/* One stage of any 2N-storage explicit Runge--Kutta scheme, with the stage's
 * coefficients given by the caller (Sec. 2.4: the paper integrates with a
 * low-storage scheme of this form, the 7-stage third-order scheme of Toulorge
 * and Desmet, whose coefficients it does not print):
 *   dU <- A dU + dt L(U_in);  U_out <- U_in + B dU.
 * Array rules and errors as dg_cns_rk_stage; A and B must be finite
 * (INVALID_ARG).  dU is read only when A != 0. */
int dg_cns_lsrk_stage(dgcns_ctx* ctx, double A, double B, double dt, const double* U_in, void* dU, double* U_out);

/* nsteps steps of the 2N scheme with `stages` stages (1..DGCNS_MAX_STAGES)
 * and coefficients A[stages], B[stages] (HOST arrays, read during the call);
 * arrays and errors as dg_cns_rk_steps.  dg_cns_rk_steps is this call with the
 * RK(5,4) coefficients. */
#define DGCNS_MAX_STAGES 32
int dg_cns_lsrk_steps(dgcns_ctx* ctx, int stages, const double* A, const double* B, int nsteps, double dt, double* U,
                      double* U_tmp, void* dU);

/* Adjoint (vector-Jacobian product) of the operator of dg_cns_apply(DGCNS_OP_L):
 *   G = (dL/dU)^T W = -(dF/dU)^T M^-1 W     (M symmetric)
 * evaluated by transposed sum factorization and transposed pointwise flux
 * Jacobians (LLF, F_c, F_v, the SIPG terms and the wall state).  Faces follow
 * the context's kernel organisation: face-centric (DGCNS_KERNEL_FACES, the
 * default: every face once, both cells' shares through the face buffer) or
 * element-centric (split and fused contexts: each cell transposes its own and
 * its neighbours' face terms).  Not in the paper (it is forward-only): the transpose of
 * Eq. WeakFormulationConservedVariables as discretised here.  U: double state;
 * W, G: residual type; G must not overlap U (INVALID_ARG); G may be W.
 * UNSUPPORTED with a body force. */
int dg_cns_adjoint_apply(dgcns_ctx* ctx, const double* U, const void* W, void* G);

/* Adjoint of one stage of dg_cns_rk_stage (reverse of dU <- A dU + dt L(U_in),
 * U_out <- U_in + B dU).  On entry lam_U (double) and lam_dU (residual type)
 * are the adjoints of (U_out, dU after the stage); on return those of (U_in,
 * dU before the stage):  W = lam_dU + B lam_U;  lam_U += dt (dL/dU)^T W;
 * lam_dU = A W.  U_in is the stage's input state (recomputed from a
 * checkpoint by the caller).  Uses the context's residual scratch.  No two of
 * U_in, lam_U and lam_dU may overlap (INVALID_ARG). */
int dg_cns_rk_stage_adjoint(dgcns_ctx* ctx, int stage, double dt, const double* U_in, double* lam_U, void* lam_dU);

/* G = d e_k / dU (double, state layout) for e_k of dg_cns_diagnostics: the
 * seed of the discrete adjoint of the final kinetic energy.  G must not
 * overlap U (INVALID_ARG). */
int dg_cns_kinetic_energy_gradient(dgcns_ctx* ctx, const double* U, double* G);

/* Taylor--Green diagnostics of Sec. 4.2.3 in FP64 (Gauss rule nq_conv):
 * out[0] e_k = 1/V int |u|^2/2, out[1] eps = nu/V int grad u : grad u,
 * out[2] -de_k/dt from L_of_U (0 when L_of_U is NULL), out[3..7] int rho,
 * int rho u, int rho E (k+1 points, = 1^T M U), out[8] number of non-finite
 * entries of U.  out is a HOST array of DGCNS_NDIAG doubles; the call
 * synchronises the stream.  Returns DGCNS_ERR_NONFINITE when out[8] > 0
 * (out is still filled). */
int dg_cns_diagnostics(dgcns_ctx* ctx, const double* U, const void* L_of_U, double* out);

/* Diagnostics without any memory allocation, for callers that may not
 * allocate while they run: code that owns all device memory through its own
 * pool, loops with a fixed memory budget, or steps recorded while allocation
 * is not permitted.  (No counterpart in the paper: an interface addition.)
 * Computes the same DGCNS_NDIAG values as dg_cns_diagnostics, but writes them
 * to out_dev, a DEVICE array of DGCNS_NDIAG doubles, asynchronously on the
 * context's stream: no host copy, no synchronisation, no cudaMalloc/cudaFree.
 * Scratch: one static device array of DGCNS_NOALLOC_SCRATCH_BYTES (16 MiB)
 * that every GPU loading this library holds until the process exits.  It
 * holds DGCNS_NOALLOC_SCRATCH_BYTES / 80 = 209715 partial-sum rows, one per
 * batch of 2 cells (1 cell when nq_conv^3 > 300); a mesh needing more rows is
 * rejected with DGCNS_ERR_INVALID_ARG before anything is launched.  Every row
 * a call reads it first writes, so nothing needs clearing between calls.  All
 * calls (all contexts on the device) share that array: calls that may overlap
 * on the GPU (different streams, no ordering) race and give wrong results.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  A non-finite state is reported in out_dev[8]
 * only (the call cannot see it without synchronising). */
#define DGCNS_NOALLOC_SCRATCH_BYTES (16u << 20)
int dg_cns_diagnostics_noalloc(dgcns_ctx* ctx, const double* U, const void* L_of_U, double* out_dev);

/* Number of CUDA kernels this context has launched so far (host counter; library utility, no
 * counterpart in the paper). */
int dg_cns_launch_count(const dgcns_ctx* ctx, int64_t* count);

/* Synchronizes the context's stream and reports whether any kernel of this context gave up a
   bounded wait (its pipelined copies did not land within the poll limit) since the last call:
   DGCNS_ERR_TIMEOUT then (the affected results are invalid), else DGCNS_OK.  The flag is cleared.
   (Library utility, no counterpart in the paper.) */
int dg_cns_status(dgcns_ctx* ctx);

/* Kernel kinds of the per-kernel timing. */
#define DGCNS_KT_CELL 0        /* cell integrals alone (split organisation; residual of the face-centric one) */
#define DGCNS_KT_FACE 1        /* element-centric face integrals alone (split organisation) */
#define DGCNS_KT_MASS 2        /* inverse mass / stage update alone (split organisation, adjoint M^-1 W) */
#define DGCNS_KT_FUSED 3       /* fused cells + 6 faces (+ M^-1 + stage update) */
#define DGCNS_KT_FACES 4       /* face-centric face kernel (every face once) */
#define DGCNS_KT_CELL_STAGE 5  /* cells + face shares + M^-1 + stage update (face-centric organisation) */
#define DGCNS_KT_DEV 6         /* FP32 deviation pre-pass of the mixed form */
#define DGCNS_KT_ADJ_PREP 7    /* adjoint stage preparation (W = lam_dU + B lam_U, lam_dU = A W) */
#define DGCNS_KT_ADJ_FACES 8   /* face-centric adjoint face kernel */
#define DGCNS_KT_ADJ 9         /* adjoint cell (+ element-centric face) kernel */
#define DGCNS_KT_OTHER 10      /* diagnostics, kinetic-energy gradient */
#define DGCNS_KT_COUNT 11

/* Per-kernel timing with CUDA events recorded on the context's stream around every kernel the
   context launches.  enable != 0 clears the totals and starts timing; enable == 0 stops it (the
   totals are kept).  Off by default.  (Library utility, no counterpart in the paper.) */
int dg_cns_timing(dgcns_ctx* ctx, int enable);

/* Synchronizes the context's stream, then writes for kinds 0..n-1 (n <= DGCNS_KT_COUNT) the total
   device time ms[i] (milliseconds) and the number of timed launches counts[i] since timing was
   enabled.  Either pointer may be NULL. */
int dg_cns_kernel_times(dgcns_ctx* ctx, double* ms, int64_t* counts, int n);

/* Host only (no device, no context): the reference frames and the face table that dg_cns_create
 * builds for a DGCNS_MAP_ROTATED mesh.  frames[e] (n cells ints): the frame g of cell e.
 * table[(e 6 + 2 d + s) 2] (12 n cells ints): the neighbour across local face (d, s) of cell e;
 * table[(e 6 + 2 d + s) 2 + 1]: its orientation code.  Seen in e's frame and moved across that face,
 * the neighbour's node (i0, i1, i2) is its own node (j0, j1, j2) with j_b = i_a, or N-1-i_a when bit
 * 6 + b of the code is set, where a is held in bits 2b..2b+1.  Either output may be NULL (not both);
 * both are caller-owned.  Errors: INVALID_ARG (not a rotated-frame mesh, a non-periodic axis, bad
 * extents, seed or cell count; message through dg_cns_last_error(NULL)).  (Library utility.) */
int dg_cns_face_table(const dgcns_mesh* mesh, int* table, int* frames);

/* Message of the last error on this context (static string if ctx is NULL; the message of a failed
 * dg_cns_create when ctx is NULL).  (Library utility, no counterpart in the paper.) */
const char* dg_cns_last_error(const dgcns_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGCNS_H */
