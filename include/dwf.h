/*
 * dwf.h -- C ABI of the GB300 (sm_103a) alpha-Mobius domain-wall solver.
 *
 * The library applies the red-black preconditioned alpha domain-wall operator
 *
 *     D_bb = 1_bb - I_bb^-1 D_br I_rr^-1 D_rb            (Sec. 3, Eq. redblack)
 *
 * of H. Neff, "A better conditioned Domain Wall Operator" (arXiv:1501.04950),
 * built on the operator D_alpha(m) of Sec. 2 (Eq. mobius1, Eq. coeff) with the
 * Wilson matrix D_w(M5) of Eq. wilson, and solves D_alpha(m) P z = D_1(1) P b for
 * the 4D propagator z_1 = y_1 (Eq. tosolve1, App. B Eq. tosolve) by conjugate
 * gradient on the normal equations of D_bb (Sec. 3).  The same machinery applies
 * the 4D overlap operator of App. A (dwf_apply_overlap), runs the older red-black
 * forms of Sec. 3 (dwf_options.schur_form) and gives the fermion force of
 * S = phi^+ (D_bb^+ D_bb)^-1 phi (dwf_force).
 *
 * Conventions shared by every entry point
 *   - Status: every call returns an int, DWF_OK (0) on success.  On error the
 *     outputs are unspecified, the handle stays usable and dwf_last_error()
 *     describes the failure.  DWF_ERR_NOT_CONVERGED still fills stats and the
 *     outputs with the last iterate.
 *   - Ownership: the caller owns every buffer passed in; no pointer is kept
 *     after a call returns.  The handle owns its gauge copies, matrices and
 *     workspace (device memory allocated by the library).
 *   - Streams: every call is ordered on the given stream (a cudaStream_t; NULL
 *     is the legacy default stream).  Apply calls do not synchronise.  The
 *     solver calls (dwf_cgne_solve, dwf_apply_overlap, dwf_solve_normal,
 *     dwf_force without X) synchronise internally (convergence polling).
 *   - Gamma basis: chiral, gamma_k = [[0,-i sigma_k],[i sigma_k,0]],
 *     gamma_4 = [[0,1],[1,0]], gamma5 = diag(1,1,-1,-1); mu = 0..3 <-> x,y,z,t.
 *   - Canonical layouts (complex128 stored as interleaved double pairs, C order):
 *       gauge      U[t][z][y][x][mu][3][3]
 *       4D spinor  psi[t][z][y][x][spin 4][colour 3]
 *       5D full    psi[s][t][z][y][x][4][3]
 *       5D half    psi[s][h][4][3], h = (x + Lx*(y + Ly*(z + Lz*t))) / 2 over the
 *                  sites of one checkerboard parity (x + y + z + t) mod 2.
 *     The "black" half-lattice of D_bb is the even parity unless
 *     dwf_options.rb_parity = 1.
 *   - Internal half-fields (inputs/outputs of the apply calls) are opaque,
 *     16-byte aligned device buffers of dwf_field_bytes() bytes per right-hand
 *     side in one of the precisions below; convert with dwf_pack_half /
 *     dwf_unpack_half.  nrhs fields are stored back to back.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_ctx* dwf_handle;
/* Same type as cudaStream_t; keeps the CUDA headers out of C callers. */
typedef struct CUstream_st* dwf_stream;

enum {
  DWF_OK = 0,
  DWF_ERR_INVALID_ARG = 1,
  DWF_ERR_CUDA = 2,
  DWF_ERR_OOM = 3,
  DWF_ERR_NOT_CONVERGED = 4,
  DWF_ERR_BREAKDOWN = 5,
  DWF_ERR_TIMEOUT = 6,
  DWF_ERR_STATE = 7
};

/* Storage precision of internal half-fields.  FP16/BF16 fields carry one FP32
 * scale per 5D site; arithmetic is FP64 for DWF_FP64 and FP32 otherwise. */
enum { DWF_FP64 = 0, DWF_FP32 = 1, DWF_FP16 = 2, DWF_BF16 = 3 };

/* Solver variants of dwf_cgne_solve. */
enum {
  DWF_SOLVER_RELIABLE = 0, /* inner precision CG with FP64 reliable updates (default;
                              FP16/BF16 fields add FP32 ones in between, see
                              reliable_delta); with BF16 inner fields the recurrence
                              restarts at every update (as DWF_SOLVER_DEFECT), and with
                              any precision it restarts after an FP64 update that gained
                              < 10%; five such updates in a row end the solve
                              (DWF_ERR_NOT_CONVERGED) */
  DWF_SOLVER_DEFECT = 1,   /* FP64 defect correction around restarted inner CG      */
  DWF_SOLVER_FP64 = 2      /* plain FP64 CG on the normal equations                 */
};

/* Red-black operator the CG runs on (Sec. 3).  All three have the same solution
 * psi_b; they differ in conditioning, hence in iteration count.
 *   DWF_SCHUR_PRECOND:   D_bb = 1 - I^-1 D_br I^-1 D_rb (Eq. redblack, default);
 *   DWF_SCHUR_PLAIN:     I_bb - D_br I^-1 D_rb = I D_bb (Eq. redblack1), on
 *                        I r'_b;
 *   DWF_SCHUR_ROWSCALED: S I D_bb on S I r'_b, S = diag over the 5th dimension of
 *                        1/(b_s + c_s) where b_s + c_s > 1, else 1 (the left row
 *                        scaling discussed with Eq. redblack1).
 * rel_tol and dwf_stats.true_resid then refer to that operator's own residual
 * |L (r'_b - D_bb x)| / |L r'_b| (L = 1, I or S I); the forms other than
 * DWF_SCHUR_PRECOND use the unfused CG steps and dense site-local kernels. */
enum { DWF_SCHUR_PRECOND = 0, DWF_SCHUR_PLAIN = 1, DWF_SCHUR_ROWSCALED = 2 };

typedef struct {
  int precision_inner;   /* DWF_FP32 (default), DWF_FP16, DWF_BF16 or DWF_FP64     */
  int rb_parity;         /* 0: black = even sites (default), 1: black = odd sites  */
  int bc_t;              /* +1 periodic (default), -1 antiperiodic in t             */
  double rel_tol;        /* target |r'_b - D_bb x| / |r'_b| (default 1e-10)          */
  int maxiter;           /* total inner iterations per right-hand side (default 100000) */
  double reliable_delta; /* reliable update when |r| < delta * max|r|; <= 0 (default):
                            0.5 for FP16/BF16 inner fields, 0.01 otherwise.  With FP16/BF16
                            inner fields (operator DWF_SCHUR_PRECOND) a replacement recomputes
                            the residual in FP32 from the last FP64 one, r = r_64 - D x_32
                            (x_32: the solution accumulated since), until |r| has dropped
                            1e3-fold below |r_64| or reaches rel_tol; then in FP64      */
  int solver;            /* DWF_SOLVER_* (default DWF_SOLVER_RELIABLE)               */
  int check_every;       /* iterations between convergence polls; <= 0 (default): 4 for
                            FP16/BF16 inner fields, 16 otherwise                       */
  int profile;           /* 1: time the inner applies with CUDA events (stats.apply_ms) */
  int graph;             /* 1 (default): replay the CG iterations between polls as a CUDA graph */
  int rhs_block;         /* right-hand sides solved together: 0 (default) = autotuned        */
  int schur_form;        /* DWF_SCHUR_* operator of dwf_cgne_solve (default PRECOND)       */
} dwf_options;

typedef struct {
  int iterations;        /* CG iterations (inner, all restarts)                       */
  int restarts;          /* FP64 reliable updates / defect-correction cycles          */
  double true_resid;     /* FP64 |r'_b - D_bb x| / |r'_b| of the returned solution     */
  double true_resid_5d;  /* FP64 |rhs - D_alpha psi| / |rhs| of the full 5D solution    */
  double seconds;        /* wall time from the start of the batch's CG to this source's
                            convergence (its latency inside the batch)                  */
  int applies;           /* inner-precision D_bb applies                               */
  int applies_dag;       /* inner-precision D_bb^+ applies                             */
  int applies_fp64;      /* FP64 D_bb applies (true residuals)                          */
  int kernel_launches;   /* CUDA kernels the solve launched                             */
  double apply_ms;       /* device time of the batch's timed inner D_bb applies (opt.profile
                            = 1: the applies of the first iteration after each poll)     */
  double apply_dag_ms;   /* same for the D_bb^+ applies                                  */
  int applies_fp32;      /* FP32 D_bb applies: residual replacements of FP16/BF16 solves
                            between two FP64 ones                                       */
  int applies_timed;     /* D_bb (and D_bb^+) applies covered by apply_ms (apply_dag_ms) */
} dwf_stats;

/* Fill *opt with the defaults listed above. */
int dwf_default_options(dwf_options* opt);

/* Create a handle for one operator D_alpha(m) (Sec. 2, Eq. mobius1 / Eq. coeff).
 * lattice = {Lx, Ly, Lz, Lt}, each even and >= 2; 2 <= Ls <= 32; b, c: Ls host
 * doubles (the per-slice Mobius coefficients b_i, c_i); opt may be NULL.
 * Builds the Ls x Ls matrices B, C, I = (4 + M5) B + C, I^-1 and K = B I^-1 per
 * chirality in FP64 on the host and uploads them; uses the current CUDA device. */
int dwf_create(dwf_handle* out, const int lattice[4], int Ls, double M5, double m,
               double alpha, const double* b, const double* c, const dwf_options* opt);
int dwf_destroy(dwf_handle h);
/* Message of the last failed call on h (or, if h is NULL, of the last failed
 * dwf_create or dwf_cgne_solve_multi on the calling thread). */
const char* dwf_last_error(dwf_handle h);

/* Bytes of one internal half-field of precision prec (per right-hand side). */
int dwf_field_bytes(dwf_handle h, int prec, size_t* bytes);

/* Load the gauge field U (canonical layout above; is_device = 0: host memory,
 * 1: device memory).  Converted on the device to the internal per-parity
 * layouts in FP64, FP32 and FP16. */
int dwf_load_gauge(dwf_handle h, const double* U, int is_device, dwf_stream s);

/* Canonical device half-field(s) [nrhs][Ls][Vh][4][3] complex128 <-> internal. */
int dwf_pack_half(dwf_handle h, void* dst_internal, const double* src_canonical, int prec,
                  int nrhs, dwf_stream s);
int dwf_unpack_half(dwf_handle h, double* dst_canonical, const void* src_internal, int prec,
                    int nrhs, dwf_stream s);

/* out = D_bb in (Sec. 3, Eq. redblack) on nrhs internal black half-fields of
 * precision prec.  Two kernels: u = K H_rb (B in) on red sites, then
 * out = in - 1/4 I^-1 H_br u on black sites (D_rb = -1/2 H_rb B, K = B I^-1).
 * in and out must not overlap. */
int dwf_apply_Dbb(dwf_handle h, void* out, const void* in, int prec, int nrhs, dwf_stream s);

/* Same as dwf_apply_Dbb, for callers that cannot allocate device memory (a
 * pool allocator owns the device, or cudaMalloc's implicit synchronisation is
 * not acceptable in their loop).  The paper has no counterpart: this is a
 * library service.  The red intermediate field lives in a static device array
 * of DWF_NOALLOC_SCRATCH_BYTES compiled into the library (every GPU that loads
 * the library holds it until exit) instead of handle workspace; no call
 * allocates or frees anything.  Requires nrhs * dwf_field_bytes(prec) <=
 * DWF_NOALLOC_SCRATCH_BYTES, else DWF_ERR_INVALID_ARG.  dwf_create looks up the
 * array's device address with the handle's device current (create handles
 * outside any stream capture); calls must be made with that device current,
 * else DWF_ERR_INVALID_ARG.  All calls share the array and each call
 * overwrites it completely, so calls that overlap on the GPU (other streams,
 * other handles) race. */
#define DWF_NOALLOC_SCRATCH_BYTES (32u << 20)
int dwf_apply_Dbb_noalloc(dwf_handle h, void* out, const void* in, int prec, int nrhs,
                          dwf_stream s);

/* out = D_bb^dagger in = gamma5 [1 - 1/4 B^T H_br K^T H_rb I^-T] gamma5 in: the
 * adjoint of Eq. redblack (H is gamma5-hermitian; B, C, I are real and commute
 * with gamma5).  in and out must not overlap. */
int dwf_apply_Dbb_dag(dwf_handle h, void* out, const void* in, int prec, int nrhs, dwf_stream s);

/* out = D_alpha'(m') in on canonical FULL 5D device fields [Ls][t][z][y][x][4][3]
 * (FP64), with alpha' and m' given here (the b_i, c_i, M5 of the handle): the
 * operator of Sec. 2, Eq. mobius1, used for right-hand sides and checks. */
int dwf_apply_dalpha(dwf_handle h, double* out_full, const double* in_full, double alpha,
                     double m, dwf_stream s);

/* Batched solves: the nrhs sources are solved in blocks of rhs_block right-hand
 * sides that share every kernel launch (each with its own alpha, scalars and
 * convergence; converged ones are masked off).  With rhs_block = 0 a built-in
 * autotuner times the batched D_bb apply for block sizes that fit in free
 * device memory, for the two CTA tiles of the hop kernels and for the two
 * neighbour staging variants, and keeps the fastest per right-hand side
 * (cached per lattice, Ls, precision and nrhs in the handle, and in the file
 * named by DWF_AUTOTUNE_CACHE if set).  The CG
 * iterations between two convergence polls (check_every, rounded up to even)
 * are captured once as a CUDA graph and replayed.  All solver work runs on a
 * stream owned by the handle; the call first waits for the caller's stream. */

/* Solve D_alpha(m) P z = D_1(1) P b for nrhs sources b = (b_1, 0, ..., 0)
 * (Sec. 2 Eq. tosolve1, App. B Eq. tosolve) and return the 4D propagators
 * z_1 = P_- psi_1 + P_+ psi_Ls.
 *   src4d   nrhs canonical 4D sources b_1 (host or device memory)
 *   prop4d  nrhs canonical 4D outputs z_1 (same memory kind as src4d)
 *   sol5d   optional nrhs canonical FULL 5D solutions psi = P z (device) or NULL
 *   alphas  nrhs host doubles (alpha per source) or NULL for the handle's alpha
 *   stats   nrhs entries or NULL
 * The right-hand side is rhs = D_1(1) P b; red-black: r'_b = I^-1(rhs_b - D_br I^-1 rhs_r),
 * CG on D_bb^+ D_bb x = D_bb^+ r'_b to FP64 true residual opt.rel_tol, then
 * psi_r = I^-1 (rhs_r - D_rb psi_b).  Returns DWF_ERR_NOT_CONVERGED if any
 * source misses the tolerance within maxiter iterations, or if five
 * consecutive FP64 residual replacements fail to lower its true residual by
 * 10% (each such replacement restarts its recurrence; five in a row mean the
 * tolerance is below what the arithmetic can reach), DWF_ERR_BREAKDOWN if a CG
 * scalar is not finite or |D p|^2 <= 0. */
int dwf_cgne_solve(dwf_handle h, const double* src4d, double* prop4d, double* sol5d, int nrhs,
                   const double* alphas, dwf_stats* stats, dwf_stream s);

/* One lattice's propagator solve inside dwf_cgne_solve_multi: the arguments
 * of dwf_cgne_solve for that handle, plus its own status (output). */
typedef struct {
  dwf_handle handle;    /* a distinct handle per job (its lattice, Ls, gauge, options) */
  const double* src4d;  /* as in dwf_cgne_solve */
  double* prop4d;
  double* sol5d;
  int nrhs;
  const double* alphas;
  dwf_stats* stats;
  int status;           /* output: DWF_OK or the job's error code */
} dwf_solve_job;

/* Propagator solves of several lattices at once (Sec. 2 Eq. tosolve1, App. B
 * Eq. tosolve, solved as in dwf_cgne_solve): every job runs the solve of
 * dwf_cgne_solve on its own handle, one host thread per job, each on its
 * handle's stream, so the kernels of small lattices, which alone fill only part
 * of the GPU, overlap.  The paper has no counterpart: it is a batching of
 * independent solves of Sec. 3's operator.
 *   jobs   njobs entries; every handle distinct and created on the current device
 *   s      the caller's stream: the jobs start once it has finished
 * Returns DWF_OK when every job succeeded, else the status of the first failed
 * job (jobs[i].status holds each job's own; dwf_last_error(jobs[i].handle) its
 * message, dwf_last_error(NULL) the first failure's on this thread).  Two jobs
 * with one handle are rejected (DWF_ERR_INVALID_ARG) before any work starts.
 * Returns after every job has finished. */
int dwf_cgne_solve_multi(dwf_solve_job* jobs, int njobs, dwf_stream s);

/* The 4D overlap operator D_OV(m) = 1/2 [(1 + m) + (1 - m) gamma5 eps] of App. A
 * applied to nrhs 4D fields b, through the 5D system with the two masses of
 * Eq. tosolve exchanged (App. B): solve D_alpha(1) P z = D_1(m) P b, b = (b_1, 0,
 * ..., 0), and return out4d = z_1 = D_OV(1)^-1 D_OV(m) b_1 = D_OV(m) b_1.  eps is the
 * sign-function approximation defined by the handle's b_i, c_i (Eq. polar); the
 * solve is the mass-1 (Pauli-Villars) system, whatever the handle's m.  Arguments,
 * layouts, ownership, stream and errors as dwf_cgne_solve (sol5d: optional full
 * 5D solution psi = P z; stats refer to the mass-1 solve).  The paper has no
 * separate entry for this: it is the construction of App. A / B run forward. */
int dwf_apply_overlap(dwf_handle h, const double* src4d, double* out4d, double* sol5d, int nrhs,
                      const double* alphas, dwf_stats* stats, dwf_stream s);

/* CG on the normal equations of D_bb for a black half-field right-hand side:
 * x = (D_bb^+ D_bb)^-1 phi (canonical device half-fields, FP64), with the
 * handle's solver options (inner precision and FP64 reliable updates of the
 * normal residual phi - D_bb^+ D_bb x).  The solve inside dwf_force. */
int dwf_solve_normal(dwf_handle h, double* x_half, const double* phi_half, dwf_stats* stats,
                     dwf_stream s);

/* Pseudofermion action S = phi^+ (D_bb^+ D_bb)^-1 phi = Re phi^+ X of the
 * red-black operator of Sec. 3 (Eq. redblack): X = (D_bb^+ D_bb)^-1 phi by the CG
 * of dwf_solve_normal (the handle's solver options), then S by an FP64 device
 * reduction over the black half-lattice.
 *   S        host double output
 *   phi_half canonical black half-field (device, complex128)
 *   X_half   X (canonical, device) or NULL if not needed
 *   stats    solver statistics or NULL
 * Synchronises (convergence polling).  Errors as dwf_solve_normal; with
 * DWF_ERR_NOT_CONVERGED, S and X refer to the last iterate. */
int dwf_action(dwf_handle h, double* S, const double* phi_half, double* X_half, dwf_stats* stats,
               dwf_stream s);

/* Fermion force of S = phi^+ (D_bb^+ D_bb)^-1 phi.
 *   dSdU     canonical [t][z][y][x][mu][3][3] complex128 device output:
 *            projected = 0: G_ij = dS/dRe U_ij + i dS/dIm U_ij (raw link gradient);
 *            projected = 1: F = TA(U G^+), TA(M) = (M - M^+)/2 - tr(M - M^+)/6.
 *   phi_half canonical black half-field (device)
 *   X_half   X = (D_bb^+ D_bb)^-1 phi (device) or NULL to solve for it here.
 * dS = -2 Re[Y^+ dD_bb X], Y = D_bb X; only D_br and D_rb depend on U. */
int dwf_force(dwf_handle h, double* dSdU, const double* phi_half, const double* X_half,
              int projected, dwf_stream s);

#ifdef __cplusplus
}
#endif
#endif /* DWF_H */
