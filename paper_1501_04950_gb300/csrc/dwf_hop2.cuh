// dwf_hop2.cuh -- the tuned hopping pass for Ls in {8, 12, 16} (sm_103a).
//
// Work split: one thread per (4D site, pair of 5th-dimension slices s0 = 2t,
// s1 = 2t + 1); Ls / 2 threads per site, block = (Ls/2, S) with S sites.
//   * one link load and one neighbour-table entry serve both slices;
//   * the B pre-multiplication of D_bb pass A (cyclic bidiagonal per
//     chirality, Eq. mobius1 with D_w -> 1) is folded into the spin projection:
//     proj(B v)(s) = d+ v+(s) + o+ v+(s-1) - sg A (d- v-(s) + o- v-(s+1)),
//     so only the two extra half spinors v+(s0-1) and v-(s1+1) are loaded;
//   * the 5th-dimension post operators (I^-1, K = B I^-1, K^T, B^T) run as
//     O(Ls) recurrences on register-resident chains after a transpose through
//     shared memory: every cyclic bidiagonal matrix of the construction, put
//     in "lower" form by reversing the slice order where needed, is either
//     multiplied (y_k = a_k v_k + b_k v_{k-1}) or solved with one forward
//     sweep for the unknown first element and one back-substitution sweep.
#pragma once

#include <cstdlib>

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

// Shared-memory layout of one 4D site: the two slices of thread t are stored
// together at t * kPairStride (24 reals each); 52 = 20 mod 32 spreads the eight
// 16-byte stores of a quarter warp over all 32 banks.  Sites start 8 words
// apart modulo 32 banks.
constexpr int kPairStride = 52;
__host__ __device__ constexpr int slot(int s) { return (s >> 1) * kPairStride + (s & 1) * 24; }
__host__ __device__ constexpr int site_stride(int Ls) {
  return (Ls / 2) * kPairStride + ((8 - ((Ls / 2) * kPairStride) % 32) + 32) % 32;
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
  int* err;             // set to 1 when a bounded wait gives up (TMA path)
  size_t cstride;       // elements between right-hand sides of bdiag, boff, chain
  const int* active;    // per right-hand side: 0 skips it (nullptr: all active)
};

// h_k = cp1 P_k + cp2 P'_k - SG phi_k (cm1 M_pi(k) + cm2 M'_pi(k)), with
// (A psi_-)_k = phi_k psi_-pi(k):  x: pi=(1,0), phi=(-i,-i);  y: (1,0), (-1,+1);
// z: (0,1), (-i,+i);  t: (0,1), (+1,+1).
template <typename T, int MU, int SG, bool TWO>
__device__ __forceinline__ void proj(cplx<T> h[2][3], T cp1, const cplx<T>* P, T cp2,
                                     const cplx<T>* Pp, T cm1, const cplx<T>* M, T cm2,
                                     const cplx<T>* Mp) {
  constexpr bool imag = (MU == 0 || MU == 2);
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int pk = (MU <= 1) ? 1 - k : k;
    const int phs = MU == 0 ? -1 : (MU == 3 ? 1 : (k == 0 ? -1 : 1));
    const T f = (T)(-SG * phs);
    const T f1 = f * cm1, f2 = f * cm2;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const cplx<T> p = P[3 * k + a], m = M[3 * pk + a];
      T re = cp1 * p.re, im = cp1 * p.im;
      if (TWO) {
        const cplx<T> pp = Pp[3 * k + a];
        re = fma(cp2, pp.re, re);
        im = fma(cp2, pp.im, im);
      }
      if (imag) {
        re = fma(-f1, m.im, re);
        im = fma(f1, m.re, im);
      } else {
        re = fma(f1, m.re, re);
        im = fma(f1, m.im, im);
      }
      if (TWO) {
        const cplx<T> mp = Mp[3 * pk + a];
        if (imag) {
          re = fma(-f2, mp.im, re);
          im = fma(f2, mp.re, im);
        } else {
          re = fma(f2, mp.re, re);
          im = fma(f2, mp.im, im);
        }
      }
      h[k][a] = cmake(re, im);
    }
  }
}

// chi = U h (DAG = false) or U^+ h for the two slices of a thread at once, for
// 16-bit storage: FP32 lanes (x: slice s0, y: slice s1) through the paired FMA
// of sm_100+ (FFMA2), the same link entry feeding both lanes, in the FMA order of
// cmac / cmac_conj (each lane rounds as the scalar multiply); measured 3-6%
// faster there.  FP32 storage keeps two scalar multiplies (the pairs raise its
// register pressure and measured 3-4% slower), FP64 too.
template <bool DAG>
__device__ __forceinline__ void su3_mul_pair(const Link<float>& U, const cplx<float> ha[2][3],
                                             const cplx<float> hb[2][3], cplx<float> ca[2][3],
                                             cplx<float> cb[2][3]) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const cplx<float> u = DAG ? U.u[3 * b + a] : U.u[3 * a + b];
        const float2 hr = make_float2(ha[k][b].re, hb[k][b].re);
        const float2 hi = make_float2(ha[k][b].im, hb[k][b].im);
        const float2 ur = make_float2(u.re, u.re);
        const float2 ui = DAG ? make_float2(u.im, u.im) : make_float2(-u.im, -u.im);
        const float2 uj = DAG ? make_float2(-u.im, -u.im) : make_float2(u.im, u.im);
        re = __ffma2_rn(ur, hr, re);
        re = __ffma2_rn(ui, hi, re);
        im = __ffma2_rn(ur, hi, im);
        im = __ffma2_rn(uj, hr, im);
      }
      ca[k][a] = cmake(re.x, im.x);
      cb[k][a] = cmake(re.y, im.y);
    }
}

// Boundary sign of a hop without the B pre-multiplication: for 16-bit and FP64
// storage it rides on the accumulating FMAs of the reconstruction (fewer
// instructions, measured faster); for FP32 it scales the projection
// coefficients (the folded form spills registers there and measured slower).
template <class SP>
__host__ __device__ constexpr bool fold_sign() { return SP::kPrec != P32; }

template <class SP, int PRE, int MU, int DIR>
__device__ __forceinline__ void proj_plain(cplx<typename SP::T> h[2][3], typename SP::T sg,
                                           const cplx<typename SP::T>* P,
                                           const cplx<typename SP::T>* M) {
  using T = typename SP::T;
  if constexpr (fold_sign<SP>()) {
    constexpr T cm = PRE == PRE_G5 ? (T)-1 : (T)1;
    proj<T, MU, DIR, false>(h, (T)1, P, (T)0, P, cm, M, (T)0, M);
  } else {
    const T cm = PRE == PRE_G5 ? -sg : sg;
    proj<T, MU, DIR, false>(h, sg, P, (T)0, P, cm, M, (T)0, M);
  }
}

template <class SP, int PRE, int MU, int DIR>
__device__ __forceinline__ void accumulate(Spinor<typename SP::T>& acc,
                                           const cplx<typename SP::T> c0[3],
                                           const cplx<typename SP::T> c1[3], typename SP::T sg) {
  using T = typename SP::T;
  if constexpr (PRE != PRE_B && fold_sign<SP>()) reconstruct_add<T, MU, DIR>(acc, c0, c1, sg);
  else reconstruct_add<T, MU, DIR>(acc, c0, c1);
}

template <class SP, class GP, int PRE, int MU, int DIR>
__device__ __forceinline__ void hop_dir(const Geom& g, int nb, int h, int s0, int sm, int sp2,
                                        const typename SP::T (&bd)[2][2],
                                        const typename SP::T (&bo)[2][2], const void* v,
                                        const void* gp, const void* gq,
                                        Spinor<typename SP::T>& acc0,
                                        Spinor<typename SP::T>& acc1) {
  using T = typename SP::T;
  const int hn = nb & 0x7fffffff;
  const T sg = nb < 0 ? (T)-1 : (T)1;
  // slice s0 = 2t sits at position t, s0 + 1 at Ls/2 + t (even slices first)
  const int base = hn * g.Ls;
  const int half = g.Ls >> 1, t0 = s0 >> 1;
  cplx<T> h0[2][3], h1[2][3];
  if (PRE == PRE_B) {
    cplx<T> P0[6], M0[6], P1[6], M1[6], Pa[6], Mb[6];
    SP::load_half(v, base + t0, g.N5, 0, P0);
    SP::load_half(v, base + t0, g.N5, 1, M0);
    SP::load_half(v, base + half + t0, g.N5, 0, P1);
    SP::load_half(v, base + half + t0, g.N5, 1, M1);
    SP::load_half(v, base + half + (sm >> 1), g.N5, 0, Pa);  // sm odd
    SP::load_half(v, base + (sp2 >> 1), g.N5, 1, Mb);        // sp2 even
    proj<T, MU, DIR, true>(h0, sg * bd[0][0], P0, sg * bo[0][0], Pa, sg * bd[1][0], M0,
                           sg * bo[1][0], M1);
    proj<T, MU, DIR, true>(h1, sg * bd[0][1], P1, sg * bo[0][1], P0, sg * bd[1][1], M1,
                           sg * bo[1][1], Mb);
  } else {
    cplx<T> P0[6], M0[6], P1[6], M1[6];
    SP::load_half(v, base + t0, g.N5, 0, P0);
    SP::load_half(v, base + t0, g.N5, 1, M0);
    SP::load_half(v, base + half + t0, g.N5, 0, P1);
    SP::load_half(v, base + half + t0, g.N5, 1, M1);
    proj_plain<SP, PRE, MU, DIR>(h0, sg, P0, M0);
    proj_plain<SP, PRE, MU, DIR>(h1, sg, P1, M1);
  }
  Link<T> U;
  if (DIR > 0) GP::load(gp, h, MU, U);
  else GP::load(gq, hn, MU, U);
  if constexpr (SP::kScaled) {
    cplx<T> ca[2][3], cb[2][3];
    su3_mul_pair<(DIR < 0)>(U, h0, h1, ca, cb);
    accumulate<SP, PRE, MU, DIR>(acc0, ca[0], ca[1], sg);
    accumulate<SP, PRE, MU, DIR>(acc1, cb[0], cb[1], sg);
  } else {
    cplx<T> c0[3], c1[3];
    su3_mul<T, (DIR < 0)>(U, h0[0], h0[1], c0, c1);
    accumulate<SP, PRE, MU, DIR>(acc0, c0, c1, sg);
    su3_mul<T, (DIR < 0)>(U, h1[0], h1[1], c0, c1);
    accumulate<SP, PRE, MU, DIR>(acc1, c0, c1, sg);
  }
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
    for (int q = 0; q < CPT; q++) V[q][k] = site[slot(s) + cbase + q];
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
    for (int q = 0; q < CPT; q++) site[slot(s) + cbase + q] = V[q][k];
  }
}


template <typename T>
__device__ __forceinline__ void put(T* p, const Spinor<T>& a) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    p[2 * k] = a.c[k].re;
    p[2 * k + 1] = a.c[k].im;
  }
}
template <typename T>
__device__ __forceinline__ void get(const T* p, Spinor<T>& a) {
#pragma unroll
  for (int k = 0; k < 12; k++) a.c[k] = cmake(p[2 * k], p[2 * k + 1]);
}
__device__ __forceinline__ void put(float* p, const Spinor<float>& a) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < 6; k++)
    q[k] = make_float4(a.c[2 * k].re, a.c[2 * k].im, a.c[2 * k + 1].re, a.c[2 * k + 1].im);
}
__device__ __forceinline__ void get(const float* p, Spinor<float>& a) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const float4 v = q[k];
    a.c[2 * k] = cmake(v.x, v.y);
    a.c[2 * k + 1] = cmake(v.z, v.w);
  }
}

__device__ __forceinline__ void reduce_finish(double v, const Reduce& red, int rhs, int nblocks,
                                              int bid) {
  __shared__ double wsum[32];
  const int nth = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = (nth + 31) >> 5;
    v = lane < nw ? wsum[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    double* part = red.partial + (size_t)rhs * red.partial_stride;
    unsigned int ticket = 0;
    if (lane == 0) {
      part[bid] = v;
      __threadfence();
      ticket = atomicAdd(red.counter + rhs, 1u);
    }
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    if (ticket == (unsigned)(nblocks - 1)) {
      __threadfence();
      double acc = 0.0;
      for (int b = lane; b < nblocks; b += 32) acc += *((volatile double*)(part + b));
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        red.result[(size_t)rhs * red.result_stride] = acc;
        red.counter[rhs] = 0u;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ double sqr(const Spinor<T>& a) {
  T r = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) r += a.c[k].re * a.c[k].re + a.c[k].im * a.c[k].im;
  return (double)r;
}

template <typename T>
constexpr int min_blocks() { return sizeof(T) == 8 ? 2 : 4; }

// Common tail of the hopping kernels: 5th-dimension post program, scaling,
// optional gamma5, local term, store and fused norm.  Every thread of the CTA
// calls it (it contains __syncthreads).
template <class SP, int LS, int POST, int LOC, int LOCP, bool G5, bool NORM>
__device__ __forceinline__ void epilogue(const Geom& g, const Args<typename SP::T>& a,
                                         const typename SP::T* coef, typename SP::T* site,
                                         int h, int t, bool active, int rhs,
                                         Spinor<typename SP::T>& acc0,
                                         Spinor<typename SP::T>& acc1) {
  using T = typename SP::T;
  const int s0 = 2 * t;
  if (POST != PR_NONE) {
    put(site + slot(s0), acc0);
    put(site + slot(s0) + 24, acc1);
    __syncthreads();
    run_prog<T, LS, POST>(site, coef, t);
    __syncthreads();
    get(site + slot(s0), acc0);
    get(site + slot(s0) + 24, acc1);
  }
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const T f = (G5 && k >= 6) ? -a.c_hop : a.c_hop;
    acc0.c[k] = cmake(f * acc0.c[k].re, f * acc0.c[k].im);
    acc1.c[k] = cmake(f * acc1.c[k].re, f * acc1.c[k].im);
  }
  const size_t off = rhs * a.stride;
  const int n = h * LS + t, n1 = n + LS / 2;
  if (LOC == LOC_ID) {
    if (active) {
      Spinor<T> w0, w1;
      SP::load(reinterpret_cast<const char*>(a.w) + off, n, g.N5, w0);
      SP::load(reinterpret_cast<const char*>(a.w) + off, n1, g.N5, w1);
#pragma unroll
      for (int k = 0; k < 12; k++) {
        acc0.c[k] = cmake(fma(a.c_loc, w0.c[k].re, acc0.c[k].re), fma(a.c_loc, w0.c[k].im, acc0.c[k].im));
        acc1.c[k] = cmake(fma(a.c_loc, w1.c[k].re, acc1.c[k].re), fma(a.c_loc, w1.c[k].im, acc1.c[k].im));
      }
    }
  } else if (LOC == LOC_DENSE) {  // chain program LOCP on w
    Spinor<T> w0, w1;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      w0.c[k] = cmake<T>(0, 0);
      w1.c[k] = cmake<T>(0, 0);
    }
    if (active) {
      SP::load(reinterpret_cast<const char*>(a.w) + off, n, g.N5, w0);
      SP::load(reinterpret_cast<const char*>(a.w) + off, n1, g.N5, w1);
    }
    if (POST == PR_NONE) __syncthreads();  // coefficients staged
    put(site + slot(s0), w0);
    put(site + slot(s0) + 24, w1);
    __syncthreads();
    run_prog<T, LS, LOCP>(site, coef, t);
    __syncthreads();
    get(site + slot(s0), w0);
    get(site + slot(s0) + 24, w1);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      acc0.c[k] = cmake(fma(a.c_loc, w0.c[k].re, acc0.c[k].re), fma(a.c_loc, w0.c[k].im, acc0.c[k].im));
      acc1.c[k] = cmake(fma(a.c_loc, w1.c[k].re, acc1.c[k].re), fma(a.c_loc, w1.c[k].im, acc1.c[k].im));
    }
  }
  if (active) {
    SP::store(reinterpret_cast<char*>(a.out) + off, n, g.N5, acc0);
    SP::store(reinterpret_cast<char*>(a.out) + off, n1, g.N5, acc1);
  }
  if (NORM) {
    const double v = active ? sqr(acc0) + sqr(acc1) : 0.0;
    reduce_finish(v, a.red, rhs, gridDim.x, blockIdx.x);
  }
}

// out = c_hop G post(H v') + c_loc loc(w), two 5th-dimension slices per thread.
template <class SP, int LS, int PRE, int POST, int LOC, int LOCP, bool G5, bool NORM, int MINB>
__global__ void __launch_bounds__(128, MINB)
    hop_kernel(const Geom g, const Args<typename SP::T> a) {
  using T = typename SP::T;
  using GP = typename GaugeOf<SP>::type;
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
  const int s0 = 2 * t;
  constexpr bool kChain = POST != PR_NONE || LOCP != PR_NONE;
  if (kChain) {
    for (int i = tid; i < chain_block(LS); i += nth) coef[i] = a.chain[co + i];
  }
  const char* vb = reinterpret_cast<const char*>(a.v) + rhs * a.stride;
  Spinor<T> acc0, acc1;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    acc0.c[k] = cmake<T>(0, 0);
    acc1.c[k] = cmake<T>(0, 0);
  }
  if (active) {
    const int4 nb0 = __ldg(a.nbr + 2 * h), nb1 = __ldg(a.nbr + 2 * h + 1);
    T bd[2][2] = {{0, 0}, {0, 0}}, bo[2][2] = {{0, 0}, {0, 0}};
    if (PRE == PRE_B) {
#pragma unroll
      for (int ch = 0; ch < 2; ch++)
#pragma unroll
        for (int k = 0; k < 2; k++) {
          bd[ch][k] = __ldg(a.bdiag + co + ch * LS + s0 + k);
          bo[ch][k] = __ldg(a.boff + co + ch * LS + s0 + k);
        }
    }
    const int sm = s0 == 0 ? LS - 1 : s0 - 1;
    const int sp2 = s0 + 2 == LS ? 0 : s0 + 2;
    hop_dir<SP, GP, PRE, 0, +1>(g, nb0.x, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 0, -1>(g, nb0.y, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 1, +1>(g, nb0.z, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 1, -1>(g, nb0.w, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 2, +1>(g, nb1.x, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 2, -1>(g, nb1.y, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 3, +1>(g, nb1.z, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
    hop_dir<SP, GP, PRE, 3, -1>(g, nb1.w, h, s0, sm, sp2, bd, bo, vb, a.gauge_p, a.gauge_q, acc0, acc1);
  }
  epilogue<SP, LS, POST, LOC, LOCP, G5, NORM>(g, a, coef, sbuf + j * SST, h, t, active, rhs, acc0, acc1);
}


// ---------------------------------------------------------------------------
// TMA-staged variant (FP32 and 16-bit storage).  For each of the 8 hopping
// directions the CTA copies, with cp.async.bulk into shared memory, the full
// Ls-slice block of every neighbour site (all 16-byte chunks, the 16-bit
// scales) and the link it needs; two stages alternate so that the copies of
// direction d+2 run while direction d is computed.  Completion is tracked by
// one mbarrier per stage (expect_tx by thread 0, complete_tx by the copies).
// Every wait is bounded: after kWaitLimit polls the kernel sets *err and
// carries on (the host reports DWF_ERR_TIMEOUT), so no wait can hang.
// ---------------------------------------------------------------------------
constexpr unsigned kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  const uint32_t addr = smem_addr(bar);
  for (unsigned i = 0; i < kWaitLimit; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  if (err) atomicOr(err, 1);
  return false;
}

// Byte layout of one neighbour site inside a stage.
template <class SP, int LS>
struct StageSite {
  static constexpr int kChunkBytes = SP::kChunks * LS * 16;
  static constexpr int kScaleBytes = SP::kScaled ? ((LS * 4 + 15) / 16) * 16 : 0;
  static constexpr int kLinkBytes = GaugeOf<SP>::type::kLinkBytes;
  static constexpr int kBytes = kChunkBytes + kScaleBytes + kLinkBytes;
  static constexpr int kCopies = SP::kChunks + (SP::kScaled ? 1 : 0) + 1;
};

// One chirality of slice position pos from a staged site (plain shared loads).
__device__ __forceinline__ void smem_half(const Store32*, const unsigned char* site, int LS, int pos,
                                          int chir, cplx<float>* o) {
  const float4* b = reinterpret_cast<const float4*>(site);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float4 v = b[(3 * chir + k) * LS + pos];
    o[2 * k] = cmake(v.x, v.y);
    o[2 * k + 1] = cmake(v.z, v.w);
  }
}
template <bool BF>
__device__ __forceinline__ void smem_half(const Store16<BF>*, const unsigned char* site, int LS,
                                          int pos, int chir, cplx<float>* o) {
  const uint4* b = reinterpret_cast<const uint4*>(site);
  const float sc = reinterpret_cast<const float*>(site + 3 * LS * 16)[pos];
  const uint4 v1 = b[LS + pos];
  const uint4 v0 = b[(chir ? 2 : 0) * LS + pos];
  uint32_t w[6];
  if (chir == 0) {
    w[0] = v0.x; w[1] = v0.y; w[2] = v0.z; w[3] = v0.w; w[4] = v1.x; w[5] = v1.y;
  } else {
    w[0] = v1.z; w[1] = v1.w; w[2] = v0.x; w[3] = v0.y; w[4] = v0.z; w[5] = v0.w;
  }
#pragma unroll
  for (int q = 0; q < 6; q++)
    o[q] = cmake(sc * Store16<BF>::to_f((uint16_t)(w[q] & 0xffffu)),
                 sc * Store16<BF>::to_f((uint16_t)(w[q] >> 16)));
}
__device__ __forceinline__ void smem_link(const Store32*, const unsigned char* p, Link<float>& U) {
  const float4* b = reinterpret_cast<const float4*>(p);
  float f[20];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    const float4 v = b[k];
    f[4 * k] = v.x;
    f[4 * k + 1] = v.y;
    f[4 * k + 2] = v.z;
    f[4 * k + 3] = v.w;
  }
#pragma unroll
  for (int k = 0; k < 9; k++) U.u[k] = cmake(f[2 * k], f[2 * k + 1]);
}
template <bool BF>
__device__ __forceinline__ void smem_link(const Store16<BF>*, const unsigned char* p, Link<float>& U) {
  const uint4* b = reinterpret_cast<const uint4*>(p);
  uint32_t w[12];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const uint4 v = b[k];
    w[4 * k] = v.x;
    w[4 * k + 1] = v.y;
    w[4 * k + 2] = v.z;
    w[4 * k + 3] = v.w;
  }
#pragma unroll
  for (int k = 0; k < 9; k++)
    U.u[k] = cmake(__half2float(__ushort_as_half((uint16_t)(w[k] & 0xffffu))),
                   __half2float(__ushort_as_half((uint16_t)(w[k] >> 16))));
}

template <class SP, int LS, int PRE, int MU, int DIR>
__device__ __forceinline__ void staged_dir(const unsigned char* site, bool neg, int t,
                                           const typename SP::T (&bd)[2][2],
                                           const typename SP::T (&bo)[2][2],
                                           Spinor<typename SP::T>& acc0,
                                           Spinor<typename SP::T>& acc1) {
  using T = typename SP::T;
  constexpr int half = LS / 2;
  const SP* tag = nullptr;
  const T sg = neg ? (T)-1 : (T)1;
  cplx<T> h0[2][3], h1[2][3];
  if (PRE == PRE_B) {
    const int pa = half + (t == 0 ? half - 1 : t - 1);  // slice 2t-1 (odd)
    const int pb = t + 1 == half ? 0 : t + 1;           // slice 2t+2 (even)
    cplx<T> P0[6], M0[6], P1[6], M1[6], Pa[6], Mb[6];
    smem_half(tag, site, LS, t, 0, P0);
    smem_half(tag, site, LS, t, 1, M0);
    smem_half(tag, site, LS, half + t, 1, M1);
    smem_half(tag, site, LS, pa, 0, Pa);
    proj<T, MU, DIR, true>(h0, sg * bd[0][0], P0, sg * bo[0][0], Pa, sg * bd[1][0], M0,
                           sg * bo[1][0], M1);
    smem_half(tag, site, LS, half + t, 0, P1);
    smem_half(tag, site, LS, pb, 1, Mb);
    proj<T, MU, DIR, true>(h1, sg * bd[0][1], P1, sg * bo[0][1], P0, sg * bd[1][1], M1,
                           sg * bo[1][1], Mb);
  } else {
    cplx<T> P[6], M[6];
    smem_half(tag, site, LS, t, 0, P);
    smem_half(tag, site, LS, t, 1, M);
    proj_plain<SP, PRE, MU, DIR>(h0, sg, P, M);
    smem_half(tag, site, LS, half + t, 0, P);
    smem_half(tag, site, LS, half + t, 1, M);
    proj_plain<SP, PRE, MU, DIR>(h1, sg, P, M);
  }
  Link<T> U;
  smem_link(tag, site + StageSite<SP, LS>::kChunkBytes + StageSite<SP, LS>::kScaleBytes, U);
  if constexpr (SP::kScaled) {
    cplx<T> ca[2][3], cb[2][3];
    su3_mul_pair<(DIR < 0)>(U, h0, h1, ca, cb);
    accumulate<SP, PRE, MU, DIR>(acc0, ca[0], ca[1], sg);
    accumulate<SP, PRE, MU, DIR>(acc1, cb[0], cb[1], sg);
  } else {
    cplx<T> c0[3], c1[3];
    su3_mul<T, (DIR < 0)>(U, h0[0], h0[1], c0, c1);
    accumulate<SP, PRE, MU, DIR>(acc0, c0, c1, sg);
    su3_mul<T, (DIR < 0)>(U, h1[0], h1[1], c0, c1);
    accumulate<SP, PRE, MU, DIR>(acc1, c0, c1, sg);
  }
}

template <class SP, int LS>
__device__ __forceinline__ void issue_stage(const Geom& g, const Args<typename SP::T>& a,
                                            const char* vb, unsigned char* stage, uint64_t* bar,
                                            int d, int h, int j, int t, bool active, int nb_d,
                                            int active_sites, int tid) {
  using SS = StageSite<SP, LS>;
  if (tid == 0) mbar_expect_tx(bar, (unsigned)(active_sites * (SS::kBytes)));
  if (!active) return;
  const int y = nb_d & 0x7fffffff;
  unsigned char* dst = stage + j * SS::kBytes;
  for (int c = t; c < SS::kCopies; c += LS / 2) {
    if (c < SP::kChunks) {
      bulk_copy(dst + c * LS * 16, vb + ((size_t)c * g.N5 + (size_t)y * LS) * 16, LS * 16, bar);
    } else if (SP::kScaled && c == SP::kChunks) {
      bulk_copy(dst + SS::kChunkBytes,
                vb + (size_t)SP::kChunks * g.N5 * 16 + (size_t)y * LS * 4, SS::kScaleBytes, bar);
    } else {
      const int mu = d >> 1;
      const char* gsrc = (d & 1) == 0
                             ? reinterpret_cast<const char*>(a.gauge_p) + ((size_t)h * 4 + mu) * SS::kLinkBytes
                             : reinterpret_cast<const char*>(a.gauge_q) + ((size_t)y * 4 + mu) * SS::kLinkBytes;
      bulk_copy(dst + SS::kChunkBytes + SS::kScaleBytes, gsrc, SS::kLinkBytes, bar);
    }
  }
}

template <int D, class SP, int LS, int PRE>
__device__ __forceinline__ void staged_dispatch(const unsigned char* site, bool neg, int t,
                                                const typename SP::T (&bd)[2][2],
                                                const typename SP::T (&bo)[2][2],
                                                Spinor<typename SP::T>& acc0,
                                                Spinor<typename SP::T>& acc1) {
  staged_dir<SP, LS, PRE, D / 2, (D % 2 == 0) ? 1 : -1>(site, neg, t, bd, bo, acc0, acc1);
}

template <class SP, int LS, int PRE, int POST, int LOC, int LOCP, bool G5, bool NORM>
__global__ void __launch_bounds__(128, 4)
    hop_tma_kernel(const Geom g, const Args<typename SP::T> a) {
  using T = typename SP::T;
  using SS = StageSite<SP, LS>;
  constexpr int SST = site_stride(LS);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int t = threadIdx.x, j = threadIdx.y, S = blockDim.y;
  const int nth = blockDim.x * blockDim.y, tid = j * blockDim.x + t;
  const int h = blockIdx.x * S + j;
  const bool active = h < g.Vh;
  const int rhs = blockIdx.z;
  if (a.active && !a.active[rhs]) return;
  const size_t co = (size_t)rhs * a.cstride;
  const int s0 = 2 * t;
  // [mbar 2][coef][stage 0][stage 1]; the chain buffer aliases the stages
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  T* coef = reinterpret_cast<T*>(smem_raw + 128);
  unsigned char* stages = smem_raw + 128 + ((chain_block(LS) * sizeof(T) + 127) / 128) * 128;
  const int stage_bytes = S * SS::kBytes;
  T* sbuf = reinterpret_cast<T*>(stages);
  const int active_sites = min(S, g.Vh - (int)blockIdx.x * S);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr bool kChain = POST != PR_NONE || LOCP != PR_NONE;
  if (kChain) {
    for (int i = tid; i < chain_block(LS); i += nth) coef[i] = a.chain[co + i];
  }
  int nb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  T bd[2][2] = {{0, 0}, {0, 0}}, bo[2][2] = {{0, 0}, {0, 0}};
  if (active) {
    const int4 nb0 = __ldg(a.nbr + 2 * h), nb1 = __ldg(a.nbr + 2 * h + 1);
    nb[0] = nb0.x; nb[1] = nb0.y; nb[2] = nb0.z; nb[3] = nb0.w;
    nb[4] = nb1.x; nb[5] = nb1.y; nb[6] = nb1.z; nb[7] = nb1.w;
    if (PRE == PRE_B) {
#pragma unroll
      for (int ch = 0; ch < 2; ch++)
#pragma unroll
        for (int k = 0; k < 2; k++) {
          bd[ch][k] = __ldg(a.bdiag + co + ch * LS + s0 + k);
          bo[ch][k] = __ldg(a.boff + co + ch * LS + s0 + k);
        }
    }
  }
  __syncthreads();  // barriers initialised
  const char* vb = reinterpret_cast<const char*>(a.v) + rhs * a.stride;
  issue_stage<SP, LS>(g, a, vb, stages, &bar[0], 0, h, j, t, active, nb[0], active_sites, tid);
  issue_stage<SP, LS>(g, a, vb, stages + stage_bytes, &bar[1], 1, h, j, t, active, nb[1],
                      active_sites, tid);
  Spinor<T> acc0, acc1;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    acc0.c[k] = cmake<T>(0, 0);
    acc1.c[k] = cmake<T>(0, 0);
  }
#pragma unroll
  for (int d = 0; d < 8; d++) {
    const int st = d & 1;
    unsigned char* stg = stages + st * stage_bytes;
    mbar_wait(&bar[st], (unsigned)((d >> 1) & 1), a.err);
    if (active) {
      const unsigned char* site = stg + j * SS::kBytes;
      const bool neg = nb[d] < 0;
      switch (d) {
        case 0: staged_dispatch<0, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        case 1: staged_dispatch<1, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        case 2: staged_dispatch<2, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        case 3: staged_dispatch<3, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        case 4: staged_dispatch<4, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        case 5: staged_dispatch<5, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        case 6: staged_dispatch<6, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
        default: staged_dispatch<7, SP, LS, PRE>(site, neg, t, bd, bo, acc0, acc1); break;
      }
    }
    __syncthreads();  // stage st fully read
    if (d + 2 < 8) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_stage<SP, LS>(g, a, vb, stg, &bar[st], d + 2, h, j, t, active, nb[d + 2],
                          active_sites, tid);
    }
  }
  epilogue<SP, LS, POST, LOC, LOCP, G5, NORM>(g, a, coef, sbuf + j * SST, h, t, active, rhs, acc0,
                                              acc1);
}

template <class SP, int LS>
constexpr size_t tma_smem_bytes(int S) {
  return 128 + ((chain_block(LS) * sizeof(typename SP::T) + 127) / 128) * 128 +
         (size_t)(2 * S * StageSite<SP, LS>::kBytes > S * site_stride(LS) * (int)sizeof(typename SP::T)
                      ? 2 * S * StageSite<SP, LS>::kBytes
                      : S * site_stride(LS) * (int)sizeof(typename SP::T));
}

// out = c * PROG(gamma5^g5in in), site-local, two slices per thread.
template <class SP, int LS, int PROG>
__global__ void __launch_bounds__(128) local_kernel(const Geom g, void* out, const void* in,
                                                    size_t stride, const typename SP::T* chain,
                                                    typename SP::T c, int g5in, Reduce red,
                                                    int do_norm, size_t cstride,
                                                    const int* rhs_on) {
  using T = typename SP::T;
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
  const int s0 = 2 * t;
  for (int i = tid; i < chain_block(LS); i += nth) coef[i] = chain[(size_t)rhs * cstride + i];
  const size_t off = rhs * stride;
  const int n = h * LS + t, n1 = n + LS / 2;
  Spinor<T> x0, x1;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    x0.c[k] = cmake<T>(0, 0);
    x1.c[k] = cmake<T>(0, 0);
  }
  if (active) {
    SP::load(reinterpret_cast<const char*>(in) + off, n, g.N5, x0);
    SP::load(reinterpret_cast<const char*>(in) + off, n1, g.N5, x1);
  }
  const T c5 = g5in ? -c : c;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const T f = k >= 6 ? c5 : c;
    x0.c[k] = cmake(f * x0.c[k].re, f * x0.c[k].im);
    x1.c[k] = cmake(f * x1.c[k].re, f * x1.c[k].im);
  }
  T* site = sbuf + j * SST;
  put(site + slot(s0), x0);
  put(site + slot(s0) + 24, x1);
  __syncthreads();
  run_prog<T, LS, PROG>(site, coef, t);
  __syncthreads();
  get(site + slot(s0), x0);
  get(site + slot(s0) + 24, x1);
  if (active) {
    SP::store(reinterpret_cast<char*>(out) + off, n, g.N5, x0);
    SP::store(reinterpret_cast<char*>(out) + off, n1, g.N5, x1);
  }
  if (do_norm) {
    const double v = active ? sqr(x0) + sqr(x1) : 0.0;
    reduce_finish(v, red, rhs, gridDim.x, blockIdx.x);
  }
}

}  // namespace hop2
}  // namespace dwf

namespace dwf {
namespace hop2 {

inline int block_sites(int Ls) { return 128 / (Ls / 2); }

inline size_t smem_bytes(int Ls, int S, size_t ts) {
  return ts * ((size_t)chain_block(Ls) + (size_t)S * site_stride(Ls));
}

template <class SP, int LS, int PRE, int POST, int LOC, int LOCP, bool G5, bool NORM>
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
  if (L.red) a.red = *L.red;
  a.err = L.err;
  a.cstride = L.cstride;
  a.active = L.active;
  const int S = block_sites(LS);
  dim3 block(LS / 2, S, 1);
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  const bool aligned = ((reinterpret_cast<uintptr_t>(L.v) | L.stride) & 15) == 0;
  if constexpr (SP::kPrec != P64) {
    if (aligned && L.use_tma) {
      const size_t smem = tma_smem_bytes<SP, LS>(S);
      auto k = hop_tma_kernel<SP, LS, PRE, POST, LOC, LOCP, G5, NORM>;
      static bool attr = false;
      if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
      }
      k<<<grid, block, smem, st>>>(g, a);
      return cudaGetLastError();
    }
  }
  const size_t smem = smem_bytes(LS, S, sizeof(T));
  constexpr int MB = min_blocks<T>();
  auto k = hop_kernel<SP, LS, PRE, POST, LOC, LOCP, G5, NORM, MB>;
  static bool attr = false;  // dynamic shared memory limit, set once per kernel
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<grid, block, smem, st>>>(g, a);
  return cudaGetLastError();
}

// The hot combinations of the CG; anything else returns cudaErrorNotSupported
// and the caller falls back to the generic kernel.
template <class SP, int LS>
cudaError_t dispatch_ls(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  const bool norm = L.red != nullptr;
  if (L.loc == LOC_DENSE) return cudaErrorNotSupported;
  if (L.pre == PRE_B && L.post_prog == PR_K && L.loc == LOC_NONE && !L.g5out && !norm)
    return run<SP, LS, PRE_B, PR_K, LOC_NONE, PR_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_IINV && L.loc == LOC_ID && !L.g5out)
    return norm ? run<SP, LS, PRE_NONE, PR_IINV, LOC_ID, PR_NONE, false, true>(g, L, st)
                : run<SP, LS, PRE_NONE, PR_IINV, LOC_ID, PR_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_KT && L.loc == LOC_NONE && !L.g5out && !norm)
    return run<SP, LS, PRE_NONE, PR_KT, LOC_NONE, PR_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && L.post_prog == PR_BT && L.loc == LOC_ID && L.g5out)
    return norm ? run<SP, LS, PRE_NONE, PR_BT, LOC_ID, PR_NONE, true, true>(g, L, st)
                : run<SP, LS, PRE_NONE, PR_BT, LOC_ID, PR_NONE, true, false>(g, L, st);
  return cudaErrorNotSupported;
}

template <class SP, int LS, int PROG>
cudaError_t run_local(const Geom& g, const LocalLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  const int S = block_sites(LS);
  const size_t smem = smem_bytes(LS, S, sizeof(T));
  auto k = local_kernel<SP, LS, PROG>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
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
  const double ad = num[(size_t)rhs * sstride] / den[(size_t)rhs * sstride];
  if (blockIdx.x == 0 && tid == 0) a_out[(size_t)rhs * sstride] = ad;
  const T a = (T)ad;
  for (int i = tid; i < chain_block(LS); i += nth) coef[i] = chain[(size_t)rhs * cstride + i];
  const size_t off = rhs * stride;
  const int n = h * LS + t, n1 = n + LS / 2;
  Spinor<T> x0, x1;
  double nrm = 0.0;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    x0.c[k] = cmake<T>(0, 0);
    x1.c[k] = cmake<T>(0, 0);
  }
  if (active) {
    Spinor<T> w0, w1;
    SP::load(reinterpret_cast<const char*>(r) + off, n, g.N5, x0);
    SP::load(reinterpret_cast<const char*>(r) + off, n1, g.N5, x1);
    SP::load(reinterpret_cast<const char*>(w) + off, n, g.N5, w0);
    SP::load(reinterpret_cast<const char*>(w) + off, n1, g.N5, w1);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      x0.c[k] = cmake(fma(-a, w0.c[k].re, x0.c[k].re), fma(-a, w0.c[k].im, x0.c[k].im));
      x1.c[k] = cmake(fma(-a, w1.c[k].re, x1.c[k].re), fma(-a, w1.c[k].im, x1.c[k].im));
    }
    SP::store(reinterpret_cast<char*>(r) + off, n, g.N5, x0);
    SP::store(reinterpret_cast<char*>(r) + off, n1, g.N5, x1);
    if constexpr (SP::kScaled) {
      // 16-bit storage rounds: r^ and |r|^2 follow the stored residual
      SP::quantize(x0);
      SP::quantize(x1);
    }
    nrm = sqr(x0) + sqr(x1);
  }
#pragma unroll
  for (int k = 6; k < 12; k++) {
    x0.c[k] = cmake(-x0.c[k].re, -x0.c[k].im);
    x1.c[k] = cmake(-x1.c[k].re, -x1.c[k].im);
  }
  T* site = sbuf + j * SST;
  const int s0 = 2 * t;
  put(site + slot(s0), x0);
  put(site + slot(s0) + 24, x1);
  __syncthreads();
  run_prog<T, LS, PR_ITINV>(site, coef, t);
  __syncthreads();
  get(site + slot(s0), x0);
  get(site + slot(s0) + 24, x1);
  if (active) {
    SP::store(reinterpret_cast<char*>(rhat) + off, n, g.N5, x0);
    SP::store(reinterpret_cast<char*>(rhat) + off, n1, g.N5, x1);
  }
  reduce_finish(nrm, red, rhs, gridDim.x, blockIdx.x);
}

template <class SP, int LS>
cudaError_t run_rupdate(const Geom& g, const RUpdateLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  const int S = block_sites(LS);
  const size_t smem = smem_bytes(LS, S, sizeof(T));
  auto k = rupdate_kernel<SP, LS>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
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
