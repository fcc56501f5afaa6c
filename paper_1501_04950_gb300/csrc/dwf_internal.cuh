// dwf_internal.cuh -- layouts, geometry and kernel launchers shared by the
// translation units of libdwf (GB300, sm_103a).
//
// Internal half-field layout (5th dimension innermost): 5D index n = h * Ls + s,
// h the half-lattice site index of the canonical layout; N5 = Vh * Ls.  The
// slices are stored in pairs (pair m = n >> 1, lane n & 1; dwf_fields.cuh), each
// spinor component of a pair as (re lane 0, re lane 1, im lane 0, im lane 1):
//     FP64  double[12][N5/2][4]
//     FP32  float [12][N5/2][4]
//     FP16/BF16  uint4[6][N5/2] (two components per chunk) + float scale[N5]
//   Spins 0, 1 are the P_+ chirality (gamma5 = +1), spins 2, 3 are P_-.
//
// Gauge layout per parity p (sites of parity p, half index h):
//   FP64  double2 [Vh][4 mu][9]          (row-major 3x3)
//   FP32  float4  [Vh][4 mu][5]          (18 floats + 2 pad, row-major)
//   FP16  uint4   [Vh][4 mu][3]          (9 (re,im) half pairs + 3 pad words)
// The parity-1 copy follows the parity-0 copy in one allocation.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

namespace dwf {

constexpr int kMaxLs = 32;

struct Geom {
  int L[4];      // Lx, Ly, Lz, Lt
  int Lxh;       // Lx / 2
  int Vh;        // sites per parity
  int Ls;
  int N5;        // Vh * Ls
  int bc_t;      // +1 periodic, -1 antiperiodic in t
};

enum Prec { P64 = 0, P32 = 1, P16 = 2, PB16 = 3 };

// Reduction target of a fused |.|^2.  Block b of right-hand side r writes
// partial[r * partial_stride + b]; the last block of r to finish (ticket from
// counter[r]) adds the partials in block order and stores result[r * result_stride].
struct Reduce {
  double* partial;
  unsigned int* counter;
  double* result;
  int partial_stride;
  int result_stride;
};

// ---- the generic hopping pass -------------------------------------------------
//   acc(x,s)  = sum_mu [ (1-g_mu) U_mu(x) v'(x+mu,s) + (1+g_mu) U_mu(x-mu)^+ v'(x-mu,s) ]
//   v'        = B v (cyclic bidiagonal per chirality), gamma5 v, or v
//   out(x,s)  = c_hop * G * post(acc) + c_loc * loc(w)
//   post, loc: dense (s, s') contraction per chirality, or identity / none;
//   G = gamma5 if g5out.  Optional fused |out|^2 per right-hand side.
enum PreOp { PRE_NONE = 0, PRE_B = 1, PRE_G5 = 2 };
enum LocOp { LOC_NONE = 0, LOC_ID = 1, LOC_DENSE = 2 };

struct HopLaunch {
  int prec;                 // Prec of out, v, w
  int p;                    // output parity
  void* out;
  const void* v;            // parity 1-p input
  const void* w;            // parity p input of the local term
  size_t stride;            // bytes between right-hand sides (all three fields)
  int nrhs;
  const void* gauge;        // gauge field of the precision (both parities)
  size_t gauge_parity_bytes;
  int pre;
  const void* pre_diag;     // [2][Ls] compute type
  const void* pre_off;      // [2][Ls]
  const void* post;         // [2][Ls][Ls] compute type, row-major, or nullptr
  int loc;
  const void* locm;         // [2][Ls][Ls] for LOC_DENSE
  double c_hop, c_loc;
  int g5out;
  const Reduce* red;        // nullptr: no norm
  int block_sites;          // 4D sites per CTA (0: default)
  // Tuned path (Ls in {8, 12, 16}): 5th-dimension operators as chain programs
  // (hop2::PR_*) over the recurrence coefficient block, and the neighbour table.
  int post_prog;
  int loc_prog;
  const void* chain;        // hop2 chain coefficient block in the compute type
  const int* nbr;           // [2 parities][Vh][8] neighbour half indices, bit 31 = sign
  int* err;                 // device flag set when a bounded wait gives up
  int use_tma;              // 1: stage neighbours through shared memory with tensor copies
  long long wait_budget;    // clock cycles a bounded wait may take (0: default, ~1 s)
  int* skip_hop;            // test hook: the next staged launch issues no copies for hop
                            // *skip_hop (>= 0), then sets it to -1; nullptr: none
  size_t cstride;           // elements between right-hand sides of every coefficient
                            // array (pre_diag, pre_off, post, locm, chain); 0: shared
  const int* active;        // per right-hand side: 0 skips it (nullptr: all active)
};
// Tries the tuned kernel first, then the generic one.
cudaError_t launch_hop(const Geom& g, const HopLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f64(const Geom& g, const HopLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f32(const Geom& g, const HopLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f16(const Geom& g, const HopLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_bf16(const Geom& g, const HopLaunch& a, cudaStream_t s);
int hop_grid_blocks(const Geom& g, int prec, int block_sites);

// ---- site-local dense contraction: out = c * M (gamma5^g5in in) ---------------
struct LocalLaunch {
  int prec;
  void* out;
  const void* in;
  size_t stride;
  int nrhs;
  const void* m;            // [2][Ls][Ls] compute type
  double c;
  int g5in;
  const Reduce* red;
  int prog;                 // hop2::PR_* equivalent of m (tuned path)
  const void* chain;
  size_t cstride;           // elements between right-hand sides of m / chain (0: shared)
  const int* active;
};
cudaError_t launch_local(const Geom& g, const LocalLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f64_local(const Geom& g, const LocalLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f32_local(const Geom& g, const LocalLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f16_local(const Geom& g, const LocalLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_bf16_local(const Geom& g, const LocalLaunch& a, cudaStream_t s);
// Fused CG residual update of the tuned path (Ls in {8, 12, 16}):
// r -= a w (a = num/den, stored to a_out), |r|^2 -> red, rhat = I^-T gamma5 r.
struct RUpdateLaunch {
  int prec;
  void* r;
  void* rhat;
  const void* w;
  size_t stride;
  int nrhs;
  const void* chain;
  size_t cstride;
  const double* num;
  const double* den;
  double* a_out;
  int sstride;
  const Reduce* red;
  const int* active;
};
cudaError_t launch_rupdate(const Geom& g, const RUpdateLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f64_rupdate(const Geom& g, const RUpdateLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f32_rupdate(const Geom& g, const RUpdateLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_f16_rupdate(const Geom& g, const RUpdateLaunch& a, cudaStream_t s);
cudaError_t launch_hop2_bf16_rupdate(const Geom& g, const RUpdateLaunch& a, cudaStream_t s);
// x += a_prev p; p = z + beta p (a_prev = *a_ptr, beta = num / den); x in xprec.
cudaError_t launch_px_update(const Geom& g, int prec, int xprec, void* x, void* p, const void* z,
                             const double* a_ptr, const double* num, const double* den,
                             int sstride, int nrhs, size_t stride_x, size_t stride,
                             cudaStream_t s, const int* active);
// pnew = z + beta p (beta = num / den), bp = B pnew (B of Eq. mobius1 with D_w -> 1,
// per right-hand side coefficients bdiag/boff [2][Ls] in prec's compute type with
// stride cstride); with do_x also the deferred x += a_prev p.  p and pnew are
// different buffers; 16-bit storage applies B to the stored (rounded) p_new.
// Ls even; prec FP32 (x FP32 or FP64), FP64, or FP16/BF16 with x in FP32.
cudaError_t launch_pxb_update(const Geom& g, int prec, int xprec, void* x, const void* p, void* pnew,
                              void* bp,
                              const void* z, const double* a_ptr, const double* num,
                              const double* den, int sstride, int nrhs, size_t stride_x,
                              size_t stride, const void* bdiag, const void* boff, size_t cstride,
                              cudaStream_t s, const int* active, int do_x);
// x += a p, a = *a_ptr (flush of the deferred solution update).
cudaError_t launch_x_update(const Geom& g, int prec, int xprec, void* x, const void* p,
                            const double* a_ptr, int sstride, int nrhs, size_t stride_x,
                            size_t stride, cudaStream_t s, const int* active);

// Set to 1 to force the generic kernels (tests compare both paths).
extern int g_disable_tuned;

// ---- conversions ---------------------------------------------------------------
size_t field_bytes(const Geom& g, int prec);
size_t gauge_bytes(const Geom& g, int prec);  // both parities
cudaError_t launch_pack_half(const Geom& g, int prec, void* dst, const double* src, int nrhs,
                             cudaStream_t s);
cudaError_t launch_unpack_half(const Geom& g, int prec, double* dst, const void* src, int nrhs,
                               cudaStream_t s);
// Canonical full 5D field <-> two internal FP64 half-fields (parity 0, parity 1).
cudaError_t launch_split_full(const Geom& g, void* par0, void* par1, const double* full,
                              cudaStream_t s);
cudaError_t launch_merge_full(const Geom& g, double* full, const void* par0, const void* par1,
                              cudaStream_t s);
cudaError_t launch_gauge_convert(const Geom& g, const double* U, void* g64, void* g32,
                                 void* g16, cudaStream_t s);
// (P b) for b = (b_1, 0, ..., 0) on both parities, FP64 internal (App. A Eq. eqP):
// (Pb)_1 = P_- b_1, (Pb)_Ls = P_+ b_1.
cudaError_t launch_source_pb(const Geom& g, void* par0, void* par1, const double* src4d,
                             cudaStream_t s);
// z_1 = P_- psi_1 + P_+ psi_Ls (P^-1 of Eq. eqP) -> canonical 4D field.
cudaError_t launch_extract_z1(const Geom& g, double* prop4d, const void* par0, const void* par1,
                              cudaStream_t s);

// ---- BLAS-1 (thread per 5D site; n_rhs right-hand sides back to back) ---------
// x += a p; r -= a w; |r|^2 -> red.  a = num[r*sstride] / den[r*sstride].
// x may be stored in a wider precision xprec (FP32 under FP16/BF16 r, p, w).
cudaError_t launch_xr_update(const Geom& g, int prec, int xprec, void* x, void* r, const void* p,
                             const void* w, const double* num, const double* den, int sstride,
                             int nrhs, size_t stride_x, size_t stride, const Reduce* red,
                             cudaStream_t s, const int* active = nullptr);
// p = z + beta p, beta = num / den.
cudaError_t launch_p_update(const Geom& g, int prec, void* p, const void* z, const double* num,
                            const double* den, int sstride, int nrhs, size_t stride,
                            cudaStream_t s, const int* active = nullptr);
// dst (prec_d) = src (prec_s), optional |dst|^2 (of the converted values).
cudaError_t launch_convert(const Geom& g, int prec_d, void* dst, int prec_s, const void* src,
                           int nrhs, size_t stride_d, size_t stride_s, const Reduce* red,
                           cudaStream_t s, const int* active = nullptr);
// x64 += src (prec_s); then src = 0 if zero_src.
cudaError_t launch_accumulate64(const Geom& g, void* x64, int prec_s, void* src, int zero_src,
                                int nrhs, size_t stride_d, size_t stride_s, cudaStream_t s,
                                const int* active = nullptr);
// out = a - b (FP64), |out|^2 -> red.
cudaError_t launch_sub64_norm(const Geom& g, void* out, const void* a, const void* b, int nrhs,
                              size_t stride, const Reduce* red, cudaStream_t s,
                              const int* active = nullptr);
// dst (prec_d: FP32, FP16 or BF16) = a (FP64) - b (FP32), |dst|^2 of the stored values -> red.
cudaError_t launch_sub_to(const Geom& g, int prec_d, void* dst, const void* a64, const void* b32,
                          int nrhs, size_t stride_d, size_t stride_a, size_t stride_b,
                          const Reduce* red, cudaStream_t s, const int* active = nullptr);
// |x|^2 -> red.
cudaError_t launch_norm(const Geom& g, int prec, const void* x, int nrhs, size_t stride,
                        const Reduce* red, cudaStream_t s);
// Re <a, b> of FP64 half-fields -> red.
cudaError_t launch_dot_re64(const Geom& g, const void* a, const void* b, int nrhs, size_t stride,
                            const Reduce* red, cudaStream_t s);
// Number of blocks the BLAS-1 launches use (partial buffers must hold this many).
int blas_grid_blocks(const Geom& g);

// ---- force (dwf_force.cu) -------------------------------------------------------
// dS/dU of S = phi^+ (D_bb^+ D_bb)^-1 phi from the auxiliary FP64 fields
// eta1 = I^-T Y (black), xi1 = I^-1 D_rb X (red), eta2 = I^-T D_br^+ eta1 (red),
// xi2 = X (black); out: canonical [V][4][3][3] complex128, raw G or TA(U G^+).
cudaError_t launch_force(const Geom& g, double* out, const void* eta1, const void* xi1,
                         const void* eta2, const void* xi2, const double* bd, const double* bo,
                         const void* g64, size_t gpar, int black, int projected, cudaStream_t s);

}  // namespace dwf

typedef struct dwf_ctx* dwf_handle_internal;
namespace dwf {
// D_bb apply using the static scratch array whose address the handle looked up
// at creation (dwf_noalloc.cu); rejects a current device other than the handle's.
int apply_dbb_noalloc(dwf_handle_internal h, void* out, const void* in, int prec, int nrhs,
                      size_t scratch_bytes, cudaStream_t s);
cudaError_t noalloc_scratch_address(void** out);
int set_error(dwf_handle_internal h, int code, const char* msg);
}  // namespace dwf
