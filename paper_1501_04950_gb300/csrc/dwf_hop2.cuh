// dwf_hop2.cuh -- the tuned hopping pass for Ls in {8, 12, 16} (sm_103a).
//
// Work split: one thread per (4D site, pair of 5th-dimension slices s0 = 2t,
// s1 = 2t + 1); Ls / 2 threads per site, block = (Ls/2, S) with S sites.
//   * the half-fields store each spinor component of a slice pair as
//     (re s0, re s1, im s0, im s1) (dwf_fields.cuh), so one vector load gives a
//     thread both slices of a component in lane order, and the projection,
//     SU(3) multiply and reconstruction of the two slices run as paired FP32
//     instructions (FFMA2 / FADD2 / FMUL2 of sm_100+, one link entry feeding
//     both lanes); FP64 runs the same code on scalar lanes;
//   * one link load and one neighbour-table entry serve both slices; the
//     boundary sign of a hop (and the per-site scale of 16-bit storage) rides
//     on the FMAs of the reconstruction;
//   * the B pre-multiplication of D_bb pass A (cyclic bidiagonal per chirality,
//     Eq. mobius1 with D_w -> 1) is applied to the neighbour spinor before the
//     projection: (B v)+(s) = d+ v+(s) + o+ v+(s-1), (B v)-(s) = d- v-(s) + o- v-(s+1),
//     so v+ of the pair below and v- of the pair above are loaded in addition;
//   * the 5th-dimension post operators (I^-1, K = B I^-1, K^T, B^T) run as
//     O(Ls) recurrences on register-resident chains after a transpose through
//     shared memory: every cyclic bidiagonal matrix of the construction, put in
//     "lower" form by reversing the slice order where needed, is either
//     multiplied (y_k = a_k v_k + b_k v_{k-1}) or solved with one forward sweep
//     for the unknown first element and one back-substitution sweep.
#pragma once

#include <atomic>
#include <cstdlib>

#include <cudaTypedefs.h>

#include "dwf_fields.cuh"

namespace dwf {
namespace hop2 {

// Chain coefficient block: [op][chirality][kChainStride(Ls)] in the compute type,
// op = 0 B (mult), 1 B^T (mult), 2 I (mult), 3 I (solve), 4 I^T (solve).
// mult:  a_k = diagonal, b_k = off-diagonal (lower form, sweep order)
// solve: a_k = 1/D_k, b_k = O_k/D_k, c_k = beta_k, then G, O_0.
enum { OP_B = 0, OP_BT = 1, OP_I = 2, OP_ISOLVE = 3, OP_ITSOLVE = 4, NOPS = 5 };
__host__ __device__ constexpr int chain_stride(int Ls) { return ((3 * Ls + 2) + 3) / 4 * 4; }
__host__ __device__ constexpr int chain_block(int Ls) { return NOPS * 2 * chain_stride(Ls); }
// op is transposed -> reversed sweep order for chirality 0, else for chirality 1
__host__ __device__ constexpr bool op_transposed(int op) { return op == OP_BT || op == OP_ITSOLVE; }

// Programs (sequence of ops) used as post / local operators.
enum { PR_NONE = 0, PR_K = 1, PR_IINV = 2, PR_KT = 3, PR_BT = 4, PR_I = 5, PR_ITINV = 6 };
__host__ __device__ constexpr int prog_len(int p) { return p == PR_K || p == PR_KT ? 2 : (p ? 1 : 0); }
__host__ __device__ constexpr int prog_op(int p, int i) {
  return p == PR_K ? (i == 0 ? OP_ISOLVE : OP_B)
       : p == PR_IINV ? OP_ISOLVE
       : p == PR_KT ? (i == 0 ? OP_BT : OP_ITSOLVE)
       : p == PR_BT ? OP_BT
       : p == PR_I ? OP_I
       : p == PR_ITINV ? OP_ITSOLVE : -1;
}
__host__ __device__ constexpr bool op_is_solve(int op) { return op == OP_ISOLVE || op == OP_ITSOLVE; }

// Shared-memory layout of one 4D site for the 5th-dimension programs: the slice
// pair of thread t at t * kPairStride, component c at 4c as (re s0, re s1, im s0,
// im s1); 52 = 20 mod 32 spreads the eight 16-byte stores of a quarter warp
// over all 32 banks.  Sites start 8 words apart modulo 32 banks.
constexpr int kPairStride = 52;
__host__ __device__ constexpr int site_stride(int Ls) {
  return (Ls / 2) * kPairStride + ((8 - ((Ls / 2) * kPairStride) % 32) + 32) % 32;
}
// element of slice s, real component r = 2c + (0 re | 1 im)
__host__ __device__ constexpr int elem(int s, int r) {
  return (s >> 1) * kPairStride + 4 * (r >> 1) + 2 * (r & 1) + (s & 1);
}

// ---------------------------------------------------------------------------
// Lane-pair arithmetic: lane x = slice s0, lane y = slice s1.
// ---------------------------------------------------------------------------
template <typename T>
struct Pr;
template <>
struct Pr<float> {
  using V = float2;
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
  static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ V dup(float v) { return make_float2(v, v); }
  static __device__ __forceinline__ V mk(float x, float y) { return make_float2(x, y); }
};
template <>
struct Pr<double> {
  using V = double2;
  static __device__ __forceinline__ V fma(V a, V b, V c) {
    return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
  }
  static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V neg(V a) { return make_double2(-a.x, -a.y); }
  static __device__ __forceinline__ V dup(double v) { return make_double2(v, v); }
  static __device__ __forceinline__ V mk(double x, double y) { return make_double2(x, y); }
};

// 6 complex lane pairs: one chirality (2 spins x 3 colours), index spin * 3 + colour
template <typename V>
struct HalfP {
  V re[6], im[6];
};
// 12 complex lane pairs: a full spinor for the two slices
template <typename V>
struct SpinP {
  V re[12], im[12];
};

// ---------------------------------------------------------------------------
// Pair access to the half-field layouts of dwf_fields.cuh (pair m, NP pairs).
// load6: components c0 .. c0 + 5 (c0 = 0: P_+ spins, 6: P_- spins), unscaled.
// ---------------------------------------------------------------------------
template <class SP>
struct PairIO;

template <>
struct PairIO<Store32> {
  using V = float2;
  static __device__ __forceinline__ void load6(const void* base, size_t m, size_t NP, int c0, V* re,
                                               V* im) {
    const float4* p = reinterpret_cast<const float4*>(base) + (size_t)c0 * NP + m;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 v = __ldg(p + (size_t)k * NP);
      re[k] = make_float2(v.x, v.y);
      im[k] = make_float2(v.z, v.w);
    }
  }
  static __device__ __forceinline__ V scale(const void*, size_t, size_t) { return make_float2(1.f, 1.f); }
  static __device__ __forceinline__ void quantize(SpinP<V>&) {}
  static __device__ __forceinline__ void store(void* base, size_t m, size_t NP, const SpinP<V>& a) {
    float4* p = reinterpret_cast<float4*>(base) + m;
#pragma unroll
    for (int c = 0; c < 12; c++)
      p[(size_t)c * NP] = make_float4(a.re[c].x, a.re[c].y, a.im[c].x, a.im[c].y);
  }
};

template <>
struct PairIO<Store64> {
  using V = double2;
  static __device__ __forceinline__ void load6(const void* base, size_t m, size_t NP, int c0, V* re,
                                               V* im) {
    const double2* p = reinterpret_cast<const double2*>(base) + ((size_t)c0 * NP + m) * 2;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      re[k] = __ldg(p + (size_t)k * NP * 2);
      im[k] = __ldg(p + (size_t)k * NP * 2 + 1);
    }
  }
  static __device__ __forceinline__ V scale(const void*, size_t, size_t) { return make_double2(1.0, 1.0); }
  static __device__ __forceinline__ void quantize(SpinP<V>&) {}
  static __device__ __forceinline__ void store(void* base, size_t m, size_t NP, const SpinP<V>& a) {
    double2* p = reinterpret_cast<double2*>(base) + m * 2;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      p[(size_t)c * NP * 2] = a.re[c];
      p[(size_t)c * NP * 2 + 1] = a.im[c];
    }
  }
};

template <bool BF>
struct PairIO<Store16<BF>> {
  using V = float2;
  using S = Store16<BF>;
  static __device__ __forceinline__ void load6(const void* base, size_t m, size_t NP, int c0, V* re,
                                               V* im) {
    const uint4* p = reinterpret_cast<const uint4*>(base) + (size_t)(c0 >> 1) * NP + m;
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const uint4 v = __ldg(p + (size_t)j * NP);
      re[2 * j] = S::to_f2(v.x);
      im[2 * j] = S::to_f2(v.y);
      re[2 * j + 1] = S::to_f2(v.z);
      im[2 * j + 1] = S::to_f2(v.w);
    }
  }
  static __device__ __forceinline__ V scale(const void* base, size_t m, size_t NP) {
    return __ldg(reinterpret_cast<const float2*>(reinterpret_cast<const uint4*>(base) + 6 * NP) + m);
  }
  static __device__ __forceinline__ float2 scales_of(const SpinP<V>& a) {
    float mx = 0.f, my = 0.f;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      mx = fmaxf(mx, fmaxf(fabsf(a.re[c].x), fabsf(a.im[c].x)));
      my = fmaxf(my, fmaxf(fabsf(a.re[c].y), fabsf(a.im[c].y)));
    }
    return make_float2(S::scale_of(mx), S::scale_of(my));
  }
  // a <- what store() followed by a load gives back, in registers (a kernel must
  // not re-read through the non-coherent path what it wrote itself)
  static __device__ __forceinline__ void quantize(SpinP<V>& a) {
    const float2 sc = scales_of(a);
    const float2 inv = make_float2(1.f / sc.x, 1.f / sc.y);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      a.re[c] = __fmul2_rn(S::to_f2(S::from_f2(__fmul2_rn(a.re[c], inv))), sc);
      a.im[c] = __fmul2_rn(S::to_f2(S::from_f2(__fmul2_rn(a.im[c], inv))), sc);
    }
  }
  static __device__ __forceinline__ void store(void* base, size_t m, size_t NP, const SpinP<V>& a) {
    float mx = 0.f, my = 0.f;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      mx = fmaxf(mx, fmaxf(fabsf(a.re[c].x), fabsf(a.im[c].x)));
      my = fmaxf(my, fmaxf(fabsf(a.re[c].y), fabsf(a.im[c].y)));
    }
    const float sx = S::scale_of(mx), sy = S::scale_of(my);
    const float2 inv = make_float2(1.f / sx, 1.f / sy);
    uint4* p = reinterpret_cast<uint4*>(base) + m;
#pragma unroll
    for (int j = 0; j < 6; j++)
      p[(size_t)j * NP] = make_uint4(S::from_f2(__fmul2_rn(a.re[2 * j], inv)),
                                     S::from_f2(__fmul2_rn(a.im[2 * j], inv)),
                                     S::from_f2(__fmul2_rn(a.re[2 * j + 1], inv)),
                                     S::from_f2(__fmul2_rn(a.im[2 * j + 1], inv)));
    reinterpret_cast<float2*>(reinterpret_cast<uint4*>(base) + 6 * NP)[m] = make_float2(sx, sy);
  }
};

// full spinor pair (scaled for 16-bit storage)
template <class SP>
__device__ __forceinline__ void load_spin(const void* base, size_t m, size_t NP,
                                          SpinP<typename Pr<typename SP::T>::V>& a) {
  using IO = PairIO<SP>;
  IO::load6(base, m, NP, 0, a.re, a.im);
  IO::load6(base, m, NP, 6, a.re + 6, a.im + 6);
  if constexpr (SP::kScaled) {
    const float2 sc = IO::scale(base, m, NP);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      a.re[c] = __fmul2_rn(a.re[c], sc);
      a.im[c] = __fmul2_rn(a.im[c], sc);
    }
  }
}

// ---------------------------------------------------------------------------
// Spin structure in the chiral basis: (1 - dir gamma_mu) psi = (h, -dir A^+ h),
// h = psi_+ - dir A psi_-, A_x = -i sigma_1, A_y = -i sigma_2, A_z = -i sigma_3,
// A_t = 1.  Row k of h is P_k + cf (i) M_pk; row k of the lower half is
// rs (i) chi_pk, with pk the partner row and (i) present for x and z.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int partner(int mu, int k) { return mu <= 1 ? 1 - k : k; }
__host__ __device__ constexpr bool imag_mu(int mu) { return mu == 0 || mu == 2; }
__host__ __device__ constexpr int proj_sign(int mu, int dir, int k) {
  return mu == 0 ? dir : (mu == 3 ? -dir : (k == 0 ? dir : -dir));
}
__host__ __device__ constexpr int recon_sign(int mu, int dir, int k) {
  return mu == 0 || mu == 3 ? -dir : (k == 0 ? -dir : dir);
}

template <typename T>
struct Args {
  void* out;
  const void* v;
  const void* w;
  size_t stride;
  const void* gauge_p;
  const void* gauge_q;
  const int4* nbr;      // [Vh][2] int4 of output parity: x+ x- y+ y- | z+ z- t+ t- (bit 31: sign)
  const T* bdiag;       // [2][Ls] B diagonal (PRE_B)
  const T* boff;        // [2][Ls] B off-diagonal (PRE_B)
  const T* chain;       // chain coefficient block (programs)
  T c_hop, c_loc;
  Reduce red;
  size_t cstride;       // elements between right-hand sides of bdiag, boff, chain
  const int* active;    // per right-hand side: 0 skips it (nullptr: all active)
  int* err;             // set to 1 when a bounded wait gives up (staged variant)
};

// h = P_+ - dir A P_- (in place into P), chi_k = U' h_k, acc_upper(k) += f chi_k,
// acc_lower(pk) += f rs (i) chi_k; U' = U (dir > 0) or U^+ (dir < 0).
template <class SP, int MU, int DIR>
__device__ __forceinline__ void project_mul_acc(HalfP<typename Pr<typename SP::T>::V>& P,
                                                const HalfP<typename Pr<typename SP::T>::V>& M,
                                                const Link<typename SP::T>& U,
                                                typename Pr<typename SP::T>::V f,
                                                SpinP<typename Pr<typename SP::T>::V>& acc) {
  using T = typename SP::T;
  using A = Pr<T>;
  using V = typename A::V;
  // projection h = P_+ - dir A P_- (in place into P)
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int pk = partner(MU, k);
    const int cs = proj_sign(MU, DIR, k);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const V pr = P.re[3 * k + a], pi = P.im[3 * k + a];
      const V mr = M.re[3 * pk + a], mi = M.im[3 * pk + a];
      if (imag_mu(MU)) {  // P + cs i M
        P.re[3 * k + a] = cs > 0 ? A::sub(pr, mi) : A::add(pr, mi);
        P.im[3 * k + a] = cs > 0 ? A::add(pi, mr) : A::sub(pi, mr);
      } else {            // P + cs M
        P.re[3 * k + a] = cs > 0 ? A::add(pr, mr) : A::sub(pr, mr);
        P.im[3 * k + a] = cs > 0 ? A::add(pi, mi) : A::sub(pi, mi);
      }
    }
  }
  const V fn = A::neg(f);
  // chi_k = U' h_k; acc_upper(k) += f chi_k; acc_lower(pk) += f rs (i) chi_k
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int q = partner(MU, k);  // lower row fed by chi_k
    const int rs = recon_sign(MU, DIR, q);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      V cr, ci;
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const cplx<T> u = DIR > 0 ? U.u[3 * a + b] : U.u[3 * b + a];
        const V ur = A::dup(u.re);
        const V ui = A::dup(DIR > 0 ? u.im : -u.im);
        const V hr = P.re[3 * k + b], hi = P.im[3 * k + b];
        if (b == 0) {
          cr = A::mul(ur, hr);
          ci = A::mul(ur, hi);
        } else {
          cr = A::fma(ur, hr, cr);
          ci = A::fma(ur, hi, ci);
        }
        cr = A::fma(A::neg(ui), hi, cr);
        ci = A::fma(ui, hr, ci);
      }
      acc.re[3 * k + a] = A::fma(f, cr, acc.re[3 * k + a]);
      acc.im[3 * k + a] = A::fma(f, ci, acc.im[3 * k + a]);
      const int l = 6 + 3 * q + a;
      if (imag_mu(MU)) {  // += rs i chi: re -= rs chi_im, im += rs chi_re
        acc.re[l] = A::fma(rs > 0 ? fn : f, ci, acc.re[l]);
        acc.im[l] = A::fma(rs > 0 ? f : fn, cr, acc.im[l]);
      } else {            // += rs chi
        acc.re[l] = A::fma(rs > 0 ? f : fn, cr, acc.re[l]);
        acc.im[l] = A::fma(rs > 0 ? f : fn, ci, acc.im[l]);
      }
    }
  }
}

// acc += f (1 - dir gamma_mu) U' v'(x +- mu) for the two slices of a thread,
// U' = U_mu(x) (dir > 0) or U_mu(x - mu)^+ (dir < 0).
template <class SP, int LS, int PRE, int MU, int DIR>
__device__ __forceinline__ void hop_dir(int nb, int h, int t, size_t NP,
                                        const typename SP::T (&bd)[2][2],
                                        const typename SP::T (&bo)[2][2], const void* v,
                                        const void* gp, const void* gq,
                                        SpinP<typename Pr<typename SP::T>::V>& acc) {
  using T = typename SP::T;
  using A = Pr<T>;
  using V = typename A::V;
  using IO = PairIO<SP>;
  using GP = typename GaugeOf<SP>::type;
  constexpr int HALF = LS / 2;
  const int hn = nb & 0x7fffffff;
  const size_t m = (size_t)hn * HALF + t;
  HalfP<V> P, M;
  IO::load6(v, m, NP, 0, P.re, P.im);
  IO::load6(v, m, NP, 6, M.re, M.im);
  V f = A::dup(nb < 0 ? (T)-1 : (T)1);  // boundary sign of the hop
  if constexpr (PRE == PRE_B) {
    // (B v)+ needs v+(s0 - 1) = lane y of the pair below (cyclic in s),
    // (B v)- needs v-(s1 + 1) = lane x of the pair above.
    const size_t base = (size_t)hn * HALF;
    const size_t mp = base + (t == 0 ? HALF - 1 : t - 1), mn = base + (t + 1 == HALF ? 0 : t + 1);
    HalfP<V> Pb, Ma;
    IO::load6(v, mp, NP, 0, Pb.re, Pb.im);
    IO::load6(v, mn, NP, 6, Ma.re, Ma.im);
    T a1 = bd[0][0], a2 = bo[0][0], a3 = bd[0][1], a4 = bo[0][1];
    T b1 = bd[1][0], b2 = bo[1][0], b3 = bd[1][1], b4 = bo[1][1];
    if constexpr (SP::kScaled) {
      const V sc = IO::scale(v, m, NP), sb = IO::scale(v, mp, NP), sa = IO::scale(v, mn, NP);
      a1 *= sc.x; a2 *= sb.y; a3 *= sc.y; a4 *= sc.x;
      b1 *= sc.x; b2 *= sc.y; b3 *= sc.y; b4 *= sa.x;
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
      P.re[k] = A::mk(::fma(a2, Pb.re[k].y, a1 * P.re[k].x), ::fma(a4, P.re[k].x, a3 * P.re[k].y));
      P.im[k] = A::mk(::fma(a2, Pb.im[k].y, a1 * P.im[k].x), ::fma(a4, P.im[k].x, a3 * P.im[k].y));
      M.re[k] = A::mk(::fma(b2, M.re[k].y, b1 * M.re[k].x), ::fma(b4, Ma.re[k].x, b3 * M.re[k].y));
      M.im[k] = A::mk(::fma(b2, M.im[k].y, b1 * M.im[k].x), ::fma(b4, Ma.im[k].x, b3 * M.im[k].y));
    }
  } else if constexpr (SP::kScaled) {
    f = A::mul(f, IO::scale(v, m, NP));  // per-slice scale of the neighbour site
  }
  Link<T> U;
  if (DIR > 0) GP::load(gp, h, MU, U);
  else GP::load(gq, hn, MU, U);
  project_mul_acc<SP, MU, DIR>(P, M, U, f, acc);
}

// Lower-form cyclic bidiagonal multiply: y_k = a_k v_k + b_k v_{k-1 mod L}.
template <typename T, int LS, int CPT>
__device__ __forceinline__ void chain_mult(T (&V)[CPT][LS], const T* c) {
  T last[CPT];
#pragma unroll
  for (int q = 0; q < CPT; q++) last[q] = V[q][LS - 1];
#pragma unroll
  for (int k = LS - 1; k >= 1; k--) {
    const T a = c[k], b = c[LS + k];
#pragma unroll
    for (int q = 0; q < CPT; q++) V[q][k] = fma(b, V[q][k - 1], a * V[q][k]);
  }
  const T a0 = c[0], b0 = c[LS];
#pragma unroll
  for (int q = 0; q < CPT; q++) V[q][0] = fma(b0, last[q], a0 * V[q][0]);
}

// Lower-form cyclic bidiagonal solve D_k y_k + O_k y_{k-1 mod L} = v_k:
// y_k = alpha_k + beta_k t with t = y_0 from the row-0 equation.
template <typename T, int LS, int CPT>
__device__ __forceinline__ void chain_solve(T (&V)[CPT][LS], const T* c) {
  T h0[CPT], prev[CPT];
#pragma unroll
  for (int q = 0; q < CPT; q++) {
    h0[q] = V[q][0];
    prev[q] = (T)0;
  }
#pragma unroll
  for (int k = 1; k < LS; k++) {
    const T a = c[k], b = c[LS + k];
#pragma unroll
    for (int q = 0; q < CPT; q++) {
      prev[q] = fma(-b, prev[q], a * V[q][k]);
      V[q][k] = prev[q];
    }
  }
  const T G = c[3 * LS], o0 = c[3 * LS + 1];
#pragma unroll
  for (int q = 0; q < CPT; q++) {
    const T t = fma(-o0, prev[q], h0[q]) * G;
    V[q][0] = t;
    prev[q] = t;
  }
#pragma unroll
  for (int k = 1; k < LS; k++) {
    const T bc = c[2 * LS + k];
#pragma unroll
    for (int q = 0; q < CPT; q++) V[q][k] = fma(bc, prev[q], V[q][k]);
  }
}

// Run program PROG on the (Ls x 24) block of one 4D site in shared memory.
// Thread t of the site owns real components cbase .. cbase + CPT - 1 (one chirality).
template <typename T, int LS, int PROG>
__device__ __forceinline__ void run_prog(T* site, const T* coef, int t) {
  constexpr int CPT = 48 / LS;
  const int cbase = t * CPT;
  const int ch = cbase / 12;
  const bool rev = (ch == 1) != op_transposed(prog_op(PROG, 0));
  T V[CPT][LS];
#pragma unroll
  for (int k = 0; k < LS; k++) {
    const int s = rev ? LS - 1 - k : k;
#pragma unroll
    for (int q = 0; q < CPT; q++) V[q][k] = site[elem(s, cbase + q)];
  }
#pragma unroll
  for (int i = 0; i < prog_len(PROG); i++) {
    const int op = prog_op(PROG, i);
    const T* c = coef + (op * 2 + ch) * chain_stride(LS);
    if (op_is_solve(op)) chain_solve<T, LS, CPT>(V, c);
    else chain_mult<T, LS, CPT>(V, c);
  }
#pragma unroll
  for (int k = 0; k < LS; k++) {
    const int s = rev ? LS - 1 - k : k;
#pragma unroll
    for (int q = 0; q < CPT; q++) site[elem(s, cbase + q)] = V[q][k];
  }
}

// thread t's slice pair <-> shared memory
__device__ __forceinline__ void put(float* p, const SpinP<float2>& a) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int c = 0; c < 12; c++) q[c] = make_float4(a.re[c].x, a.re[c].y, a.im[c].x, a.im[c].y);
}
__device__ __forceinline__ void get(const float* p, SpinP<float2>& a) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    const float4 v = q[c];
    a.re[c] = make_float2(v.x, v.y);
    a.im[c] = make_float2(v.z, v.w);
  }
}
__device__ __forceinline__ void put(double* p, const SpinP<double2>& a) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    q[2 * c] = a.re[c];
    q[2 * c + 1] = a.im[c];
  }
}
__device__ __forceinline__ void get(const double* p, SpinP<double2>& a) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int c = 0; c < 12; c++) {
    a.re[c] = q[2 * c];
    a.im[c] = q[2 * c + 1];
  }
}

template <typename V>
__device__ __forceinline__ double sqr(const SpinP<V>& a) {
  V r = a.re[0];
  r.x *= r.x;
  r.y *= r.y;
  using A = Pr<decltype(r.x)>;
  r = A::fma(a.im[0], a.im[0], r);
#pragma unroll
  for (int c = 1; c < 12; c++) {
    r = A::fma(a.re[c], a.re[c], r);
    r = A::fma(a.im[c], a.im[c], r);
  }
  return (double)r.x + (double)r.y;
}

template <typename V>
__device__ __forceinline__ void zero(SpinP<V>& a) {
#pragma unroll
  for (int c = 0; c < 12; c++) {
    a.re[c].x = 0;
    a.re[c].y = 0;
    a.im[c].x = 0;
    a.im[c].y = 0;
  }
}

template <typename T>
constexpr int min_blocks() { return sizeof(T) == 8 ? 2 : 4; }

// Common tail of the hopping kernels: 5th-dimension post program, scaling,
// optional gamma5, local term, store and fused norm.  Every thread of the CTA
// calls it (it contains __syncthreads); threads with part = false (no site of
// their own) only take part in the barriers and the norm.
template <class SP, int LS, int POST, int LOC, bool G5, bool NORM>
__device__ __forceinline__ void epilogue_g(const Args<typename SP::T>& a, const typename SP::T* coef,
                                           typename SP::T* site, size_t NP, int h, int t, bool active,
                                           bool part, int rhs,
                                           SpinP<typename Pr<typename SP::T>::V>& acc) {
  using T = typename SP::T;
  using A = Pr<T>;
  using V = typename A::V;
  if (POST != PR_NONE) {
    if (part) put(site + t * kPairStride, acc);
    __syncthreads();
    if (part) run_prog<T, LS, POST>(site, coef, t);
    __syncthreads();
    if (part) get(site + t * kPairStride, acc);
  }
  const V ch = A::dup(a.c_hop);
  const size_t off = rhs * a.stride;
  const size_t m = (size_t)h * (LS / 2) + t;
  if (LOC == LOC_ID && active) {
    SpinP<V> w;
    load_spin<SP>(reinterpret_cast<const char*>(a.w) + off, m, NP, w);
    const V cl = A::dup(a.c_loc);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      const V f = (G5 && c >= 6) ? A::neg(ch) : ch;
      acc.re[c] = A::fma(f, acc.re[c], A::mul(cl, w.re[c]));
      acc.im[c] = A::fma(f, acc.im[c], A::mul(cl, w.im[c]));
    }
  } else {
#pragma unroll
    for (int c = 0; c < 12; c++) {
      const V f = (G5 && c >= 6) ? A::neg(ch) : ch;
      acc.re[c] = A::mul(f, acc.re[c]);
      acc.im[c] = A::mul(f, acc.im[c]);
    }
  }
  if (active) PairIO<SP>::store(reinterpret_cast<char*>(a.out) + off, m, NP, acc);
  if (NORM) {
    double v = 0.0;
    if (active) {
      if constexpr (SP::kScaled) {
        // 16-bit storage rounds: the norm follows the stored values
        SpinP<V> q = acc;
        PairIO<SP>::quantize(q);
        v = sqr(q);
      } else {
        v = sqr(acc);
      }
    }
    block_sum_to(v, a.red, rhs, gridDim.x, blockIdx.x);
  }
}

// out = c_hop G post(H v') + c_loc loc(w), two 5th-dimension slices per thread.
template <class SP, int LS, int PRE, int POST, int LOC, bool G5, bool NORM, int MINB, int NT = 128>
__global__ void __launch_bounds__(NT, MINB) hop_kernel(const Geom g, const Args<typename SP::T> a) {
  using T = typename SP::T;
  using V = typename Pr<T>::V;
  constexpr int SST = site_stride(LS);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* coef = reinterpret_cast<T*>(smem_raw);
  T* sbuf = coef + chain_block(LS);
  const int t = threadIdx.x, j = threadIdx.y;
  const int nth = blockDim.x * blockDim.y, tid = j * blockDim.x + t;
  const int h = blockIdx.x * blockDim.y + j;
  const bool active = h < g.Vh;
  const int rhs = blockIdx.z;
  if (a.active && !a.active[rhs]) return;
  const size_t co = (size_t)rhs * a.cstride;
  const size_t NP = (size_t)g.N5 >> 1;
  const int s0 = 2 * t;
  if (POST != PR_NONE) {
    for (int i = tid; i < chain_block(LS); i += nth) coef[i] = a.chain[co + i];
  }
  const char* vb = reinterpret_cast<const char*>(a.v) + rhs * a.stride;
  SpinP<V> acc;
  zero(acc);
  if (active) {
    const int4 nb0 = __ldg(a.nbr + 2 * h), nb1 = __ldg(a.nbr + 2 * h + 1);
    T bd[2][2] = {{0, 0}, {0, 0}}, bo[2][2] = {{0, 0}, {0, 0}};
    if (PRE == PRE_B) {
#pragma unroll
      for (int c = 0; c < 2; c++)
#pragma unroll
        for (int k = 0; k < 2; k++) {
          bd[c][k] = __ldg(a.bdiag + co + c * LS + s0 + k);
          bo[c][k] = __ldg(a.boff + co + c * LS + s0 + k);
        }
    }
    const int nb[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};
    hop_dir<SP, LS, PRE, 0, +1>(nb[0], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 0, -1>(nb[1], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 1, +1>(nb[2], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 1, -1>(nb[3], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 2, +1>(nb[4], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 2, -1>(nb[5], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 3, +1>(nb[6], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_dir<SP, LS, PRE, 3, -1>(nb[7], h, t, NP, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
  }
  epilogue_g<SP, LS, POST, LOC, G5, NORM>(a, coef, sbuf + j * SST, NP, h, t, active, true, rhs, acc);
}

// out = c * PROG(gamma5^g5in in), site-local, two slices per thread.
template <class SP, int LS, int PROG>
__global__ void __launch_bounds__(128) local_kernel(const Geom g, void* out, const void* in,
                                                    size_t stride, const typename SP::T* chain,
                                                    typename SP::T c, int g5in, Reduce red,
                                                    int do_norm, size_t cstride,
                                                    const int* rhs_on) {
  using T = typename SP::T;
  using A = Pr<T>;
  using V = typename A::V;
  constexpr int SST = site_stride(LS);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* coef = reinterpret_cast<T*>(smem_raw);
  T* sbuf = coef + chain_block(LS);
  const int t = threadIdx.x, j = threadIdx.y;
  const int nth = blockDim.x * blockDim.y, tid = j * blockDim.x + t;
  const int h = blockIdx.x * blockDim.y + j;
  const bool active = h < g.Vh;
  const int rhs = blockIdx.z;
  if (rhs_on && !rhs_on[rhs]) return;
  const size_t NP = (size_t)g.N5 >> 1;
  for (int i = tid; i < chain_block(LS); i += nth) coef[i] = chain[(size_t)rhs * cstride + i];
  const size_t off = rhs * stride;
  const size_t m = (size_t)h * (LS / 2) + t;
  SpinP<V> x;
  zero(x);
  if (active) load_spin<SP>(reinterpret_cast<const char*>(in) + off, m, NP, x);
  const V cp = A::dup(c), cm = A::dup(g5in ? -c : c);
#pragma unroll
  for (int k = 0; k < 12; k++) {
    x.re[k] = A::mul(k >= 6 ? cm : cp, x.re[k]);
    x.im[k] = A::mul(k >= 6 ? cm : cp, x.im[k]);
  }
  T* site = sbuf + j * SST;
  put(site + t * kPairStride, x);
  __syncthreads();
  run_prog<T, LS, PROG>(site, coef, t);
  __syncthreads();
  get(site + t * kPairStride, x);
  if (active) PairIO<SP>::store(reinterpret_cast<char*>(out) + off, m, NP, x);
  if (do_norm) {
    double v = 0.0;
    if (active) {
      if constexpr (SP::kScaled) {
        SpinP<V> q = x;
        PairIO<SP>::quantize(q);
        v = sqr(q);
      } else {
        v = sqr(x);
      }
    }
    block_sum_to(v, red, rhs, gridDim.x, blockIdx.x);
  }
}

}  // namespace hop2
}  // namespace dwf

#include "dwf_hop_tma.cuh"

namespace dwf {
namespace hop2 {

// 4D sites per CTA: the default tile (128 threads) and the small one (64 threads);
// HopLaunch.block_sites selects the small tile when it equals small_block_sites.
inline int block_sites(int Ls) { return 128 / (Ls / 2); }
inline int small_block_sites(int Ls) { return 64 / (Ls / 2); }

inline size_t smem_bytes(int Ls, int S, size_t ts) {
  return ts * ((size_t)chain_block(Ls) + (size_t)S * site_stride(Ls));
}

// Raises a kernel's dynamic shared-memory limit once per process; safe when
// several host threads launch through different handles at the same time.
template <class K>
cudaError_t smem_limit_once(K k, size_t smem, std::atomic<bool>& done) {
  if (done.load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.store(true, std::memory_order_release);
  return e;
}

// Tensor map of a half-field (nrhs fields back to back) as 32-bit words:
// dim 0 the slice pairs of one row (component or 16-byte chunk row), dim 1 the
// rows, dim 2 the right-hand sides; the box is one site (Ls/2 pairs) x all rows.
template <class SP, int LS>
cudaError_t encode_field_map(CUtensorMap* map, const Geom& g, const void* base, size_t stride,
                             int nrhs) {
  using ST = Stage<SP, LS>;
  static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> enc_fn{nullptr};
  PFN_cuTensorMapEncodeTiled_v12000 enc = enc_fn.load(std::memory_order_acquire);
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    enc_fn.store(enc, std::memory_order_release);
  }
  const size_t NP = (size_t)g.N5 / 2;
  const cuuint64_t dims[3] = {(cuuint64_t)NP * ST::kWpp, (cuuint64_t)ST::kRows, (cuuint64_t)nrhs};
  const cuuint64_t row = (cuuint64_t)NP * ST::kWpp * 4;
  const cuuint64_t strides[2] = {row, (cuuint64_t)(stride ? stride : row * ST::kRows)};
  const cuuint32_t box[3] = {(cuuint32_t)(LS / 2 * ST::kWpp), (cuuint32_t)ST::kRows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void*>(base), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class SP, int LS>
constexpr int tma_stages() { return 2; }

template <class SP, int LS, int PRE, int POST, int LOC, bool G5, bool NORM>
cudaError_t run_tma(const Geom& g, const HopLaunch& L, const Args<typename SP::T>& a, cudaStream_t st) {
  constexpr int NST = tma_stages<SP, LS>();
  constexpr int S = kTmaConsumers / (LS / 2);
  if (((reinterpret_cast<uintptr_t>(L.v) | L.stride) & 15) != 0) return cudaErrorNotSupported;
  CUtensorMap map;
  cudaError_t e = encode_field_map<SP, LS>(&map, g, L.v, L.stride, L.nrhs);
  if (e != cudaSuccess) return e;
  const size_t smem = tma_smem_bytes<SP, LS, NST>();
  auto k = hop_tma_kernel<SP, LS, PRE, POST, LOC, G5, NORM, NST, 1>;
  static std::atomic<bool> attr{false};
  e = smem_limit_once(k, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  int skip = -1;
  if (L.skip_hop && *L.skip_hop >= 0) {
    skip = *L.skip_hop;
    *L.skip_hop = -1;
  }
  k<<<grid, kTmaThreads, smem, st>>>(g, a, map, L.wait_budget > 0 ? L.wait_budget : (1LL << 31),
                                     skip);
  return cudaGetLastError();
}

template <class SP, int LS, int PRE, int POST, int LOC, bool G5, bool NORM>
cudaError_t run(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  Args<T> a;
  a.out = L.out;
  a.v = L.v;
  a.w = L.w;
  a.stride = L.stride;
  const char* gb = reinterpret_cast<const char*>(L.gauge);
  a.gauge_p = gb + (size_t)L.p * L.gauge_parity_bytes;
  a.gauge_q = gb + (size_t)(1 - L.p) * L.gauge_parity_bytes;
  a.nbr = reinterpret_cast<const int4*>(L.nbr) + (size_t)L.p * g.Vh * 2;
  a.bdiag = reinterpret_cast<const T*>(L.pre_diag);
  a.boff = reinterpret_cast<const T*>(L.pre_off);
  a.chain = reinterpret_cast<const T*>(L.chain);
  a.c_hop = (T)L.c_hop;
  a.c_loc = (T)L.c_loc;
  a.red = L.red ? *L.red : Reduce{};
  a.cstride = L.cstride;
  a.active = L.active;
  a.err = L.err;
  if (L.use_tma) return run_tma<SP, LS, PRE, POST, LOC, G5, NORM>(g, L, a, st);
  const bool small = L.block_sites == small_block_sites(LS);
  const int S = small ? small_block_sites(LS) : block_sites(LS);
  dim3 block(LS / 2, S, 1);
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  const size_t smem = smem_bytes(LS, S, sizeof(T));
  constexpr int MB = min_blocks<T>();
  // dynamic shared memory limits, set once per kernel
  if (small) {
    auto k = hop_kernel<SP, LS, PRE, POST, LOC, G5, NORM, 2 * MB, 64>;
    static std::atomic<bool> attr_small{false};
    cudaError_t e = smem_limit_once(k, smem, attr_small);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(g, a);
  } else {
    auto k = hop_kernel<SP, LS, PRE, POST, LOC, G5, NORM, MB>;
    static std::atomic<bool> attr{false};
    cudaError_t e = smem_limit_once(k, smem, attr);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(g, a);
  }
  return cudaGetLastError();
}

// The hot combinations of the CG; anything else returns cudaErrorNotSupported
// and the caller falls back to the generic kernel.
template <class SP, int LS>
cudaError_t dispatch_ls(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  const bool norm = L.red != nullptr;
  if (L.loc == LOC_DENSE) return cudaErrorNotSupported;
  if (L.pre == PRE_B && L.post_prog == PR_K && L.loc == LOC_NONE && !L.g5out && !norm)
    return run<SP, LS, PRE_B, PR_K, LOC_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_K && L.loc == LOC_NONE && !L.g5out && !norm)
    return run<SP, LS, PRE_NONE, PR_K, LOC_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_IINV && L.loc == LOC_ID && !L.g5out)
    return norm ? run<SP, LS, PRE_NONE, PR_IINV, LOC_ID, false, true>(g, L, st)
                : run<SP, LS, PRE_NONE, PR_IINV, LOC_ID, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_KT && L.loc == LOC_NONE && !L.g5out && !norm)
    return run<SP, LS, PRE_NONE, PR_KT, LOC_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_BT && L.loc == LOC_ID && L.g5out)
    return norm ? run<SP, LS, PRE_NONE, PR_BT, LOC_ID, true, true>(g, L, st)
                : run<SP, LS, PRE_NONE, PR_BT, LOC_ID, true, false>(g, L, st);
  return cudaErrorNotSupported;
}

template <class SP, int LS, int PROG>
cudaError_t run_local(const Geom& g, const LocalLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  const int S = block_sites(LS);
  const size_t smem = smem_bytes(LS, S, sizeof(T));
  auto k = local_kernel<SP, LS, PROG>;
  static std::atomic<bool> attr{false};
  cudaError_t e = smem_limit_once(k, smem, attr);
  if (e != cudaSuccess) return e;
  Reduce red{};
  if (L.red) red = *L.red;
  dim3 block(LS / 2, S, 1);
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  k<<<grid, block, smem, st>>>(g, L.out, L.in, L.stride, reinterpret_cast<const T*>(L.chain),
                               (T)L.c, L.g5in, red, L.red != nullptr, L.cstride, L.active);
  return cudaGetLastError();
}

template <class SP>
cudaError_t dispatch(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  if (L.chain == nullptr || L.nbr == nullptr) return cudaErrorNotSupported;
  switch (g.Ls) {
    case 8: return dispatch_ls<SP, 8>(g, L, st);
    case 12: return dispatch_ls<SP, 12>(g, L, st);
    case 16: return dispatch_ls<SP, 16>(g, L, st);
  }
  return cudaErrorNotSupported;
}

template <class SP>
cudaError_t dispatch_local(const Geom& g, const LocalLaunch& L, cudaStream_t st) {
  if (L.chain == nullptr || L.prog != PR_ITINV) return cudaErrorNotSupported;
  switch (g.Ls) {
    case 8: return run_local<SP, 8, PR_ITINV>(g, L, st);
    case 12: return run_local<SP, 12, PR_ITINV>(g, L, st);
    case 16: return run_local<SP, 16, PR_ITINV>(g, L, st);
  }
  return cudaErrorNotSupported;
}


// Fused CG residual update: r -= a w with a = num / den, |r|^2, and
// r^ = I^-T gamma5 r (the input of the next D_bb^+ pass A), two slices per
// thread; a is also stored to a_out (read by the next p/x update).
template <class SP, int LS>
__global__ void __launch_bounds__(128) rupdate_kernel(const Geom g, void* r, void* rhat,
                                                      const void* w, size_t stride,
                                                      const typename SP::T* chain, size_t cstride,
                                                      const double* num, const double* den,
                                                      double* a_out, int sstride, Reduce red,
                                                      const int* rhs_on) {
  using T = typename SP::T;
  using A = Pr<T>;
  using V = typename A::V;
  constexpr int SST = site_stride(LS);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* coef = reinterpret_cast<T*>(smem_raw);
  T* sbuf = coef + chain_block(LS);
  const int t = threadIdx.x, j = threadIdx.y;
  const int nth = blockDim.x * blockDim.y, tid = j * blockDim.x + t;
  const int h = blockIdx.x * blockDim.y + j;
  const bool active = h < g.Vh;
  const int rhs = blockIdx.z;
  if (rhs_on && !rhs_on[rhs]) return;
  const size_t NP = (size_t)g.N5 >> 1;
  const double ad = num[(size_t)rhs * sstride] / den[(size_t)rhs * sstride];
  if (blockIdx.x == 0 && tid == 0) a_out[(size_t)rhs * sstride] = ad;
  const V na = A::dup(-(T)ad);
  for (int i = tid; i < chain_block(LS); i += nth) coef[i] = chain[(size_t)rhs * cstride + i];
  const size_t off = rhs * stride;
  const size_t m = (size_t)h * (LS / 2) + t;
  SpinP<V> x;
  zero(x);
  double nrm = 0.0;
  if (active) {
    SpinP<V> wv;
    load_spin<SP>(reinterpret_cast<const char*>(r) + off, m, NP, x);
    load_spin<SP>(reinterpret_cast<const char*>(w) + off, m, NP, wv);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      x.re[k] = A::fma(na, wv.re[k], x.re[k]);
      x.im[k] = A::fma(na, wv.im[k], x.im[k]);
    }
    PairIO<SP>::store(reinterpret_cast<char*>(r) + off, m, NP, x);
    // 16-bit storage rounds: r^ and |r|^2 follow the stored residual
    PairIO<SP>::quantize(x);
    nrm = sqr(x);
  }
#pragma unroll
  for (int k = 6; k < 12; k++) {
    x.re[k] = A::neg(x.re[k]);
    x.im[k] = A::neg(x.im[k]);
  }
  T* site = sbuf + j * SST;
  put(site + t * kPairStride, x);
  __syncthreads();
  run_prog<T, LS, PR_ITINV>(site, coef, t);
  __syncthreads();
  get(site + t * kPairStride, x);
  if (active) PairIO<SP>::store(reinterpret_cast<char*>(rhat) + off, m, NP, x);
  block_sum_to(nrm, red, rhs, gridDim.x, blockIdx.x);
}

template <class SP, int LS>
cudaError_t run_rupdate(const Geom& g, const RUpdateLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  const int S = block_sites(LS);
  const size_t smem = smem_bytes(LS, S, sizeof(T));
  auto k = rupdate_kernel<SP, LS>;
  static std::atomic<bool> attr{false};
  cudaError_t e = smem_limit_once(k, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 block(LS / 2, S, 1);
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  k<<<grid, block, smem, st>>>(g, L.r, L.rhat, L.w, L.stride, reinterpret_cast<const T*>(L.chain),
                               L.cstride, L.num, L.den, L.a_out, L.sstride, *L.red, L.active);
  return cudaGetLastError();
}

template <class SP>
cudaError_t dispatch_rupdate(const Geom& g, const RUpdateLaunch& L, cudaStream_t st) {
  switch (g.Ls) {
    case 8: return run_rupdate<SP, 8>(g, L, st);
    case 12: return run_rupdate<SP, 12>(g, L, st);
    case 16: return run_rupdate<SP, 16>(g, L, st);
  }
  return cudaErrorNotSupported;
}
}  // namespace hop2
}  // namespace dwf

#define DWF_HOP2_INSTANTIATE(NAME, SP)                                                    \
  namespace dwf {                                                                        \
  cudaError_t NAME(const Geom& g, const HopLaunch& L, cudaStream_t st) {                 \
    return hop2::dispatch<SP>(g, L, st);                                                 \
  }                                                                                      \
  cudaError_t NAME##_local(const Geom& g, const LocalLaunch& L, cudaStream_t st) {       \
    return hop2::dispatch_local<SP>(g, L, st);                                           \
  }                                                                                      \
  cudaError_t NAME##_rupdate(const Geom& g, const RUpdateLaunch& L, cudaStream_t st) {   \
    return hop2::dispatch_rupdate<SP>(g, L, st);                                         \
  }                                                                                      \
  }
