// dwf_blas.cu -- layout conversions, sources, propagator extraction and the
// fused BLAS-1 kernels of the CG on the normal equations (sm_103a).
#include "dwf_fields.cuh"

namespace dwf {

namespace {

constexpr int kBlasThreads = 256;

template <typename T>
__device__ __forceinline__ double sqd(const Spinor<T>& a) {
  T r = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) r += a.c[k].re * a.c[k].re + a.c[k].im * a.c[k].im;
  return (double)r;
}

template <typename TD, typename TS>
__device__ __forceinline__ void cvt(Spinor<TD>& d, const Spinor<TS>& s) {
#pragma unroll
  for (int k = 0; k < 12; k++) d.c[k] = cmake((TD)s.c[k].re, (TD)s.c[k].im);
}

// ---- conversions --------------------------------------------------------------

template <class SP>
__global__ void pack_half_kernel(const Geom g, void* dst, const double* src, size_t stride,
                                 int nrhs) {
  using T = typename SP::T;
  const size_t total = (size_t)g.N5 * nrhs;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / g.N5);
    const int q = (int)(i % g.N5);
    const int s = q / g.Vh, h = q % g.Vh;  // canonical order [s][h]
    const double2* in = reinterpret_cast<const double2*>(src) + ((size_t)r * g.N5 + q) * 12;
    Spinor<T> a;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = in[k];
      a.c[k] = cmake((T)v.x, (T)v.y);
    }
    SP::store(reinterpret_cast<char*>(dst) + r * stride, site5(h, s, g.Ls), g.N5, a);
  }
}

template <class SP>
__global__ void unpack_half_kernel(const Geom g, double* dst, const void* src, size_t stride,
                                   int nrhs) {
  using T = typename SP::T;
  const size_t total = (size_t)g.N5 * nrhs;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / g.N5);
    const int q = (int)(i % g.N5);
    const int s = q / g.Vh, h = q % g.Vh;
    Spinor<T> a;
    SP::load(reinterpret_cast<const char*>(src) + r * stride, site5(h, s, g.Ls), g.N5, a);
    double2* out = reinterpret_cast<double2*>(dst) + ((size_t)r * g.N5 + q) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) out[k] = make_double2((double)a.c[k].re, (double)a.c[k].im);
  }
}

__device__ __forceinline__ void lex_coords(const Geom& g, int i, int& x, int& y, int& z, int& t) {
  x = i % g.L[0];
  int r = i / g.L[0];
  y = r % g.L[1];
  r /= g.L[1];
  z = r % g.L[2];
  t = r / g.L[2];
}

// full canonical [Ls][V][4][3] <-> FP64 internal halves
__global__ void split_full_kernel(const Geom g, void* p0, void* p1, const double* full, int to_full) {
  const size_t V = (size_t)g.Vh * 2;
  const size_t total = V * g.Ls;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / V);
    const int site = (int)(i % V);
    int x, y, z, t;
    lex_coords(g, site, x, y, z, t);
    const int par = (x + y + z + t) & 1;
    const int h = site >> 1;
    void* half = par ? p1 : p0;
    double2* cf = reinterpret_cast<double2*>(const_cast<double*>(full)) + i * 12;
    Spinor<double> a;
    if (!to_full) {
#pragma unroll
      for (int k = 0; k < 12; k++) a.c[k] = cmake(cf[k].x, cf[k].y);
      Store64::store(half, site5(h, s, g.Ls), g.N5, a);
    } else {
      Store64::load(half, site5(h, s, g.Ls), g.N5, a);
#pragma unroll
      for (int k = 0; k < 12; k++) cf[k] = make_double2(a.c[k].re, a.c[k].im);
    }
  }
}

__global__ void gauge_convert_kernel(const Geom g, const double* U, double2* g64, float4* g32,
                                     uint4* g16) {
  const size_t V = (size_t)g.Vh * 2;
  const size_t total = V * 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int site = (int)(i / 4), mu = (int)(i % 4);
    int x, y, z, t;
    lex_coords(g, site, x, y, z, t);
    const int par = (x + y + z + t) & 1;
    const size_t slot = (size_t)par * g.Vh + (site >> 1);
    const double2* u = reinterpret_cast<const double2*>(U) + i * 9;
    double2 v[9];
#pragma unroll
    for (int k = 0; k < 9; k++) v[k] = u[k];
    double2* d64 = g64 + (slot * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) d64[k] = v[k];
    float f[20];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      f[2 * k] = (float)v[k].x;
      f[2 * k + 1] = (float)v[k].y;
    }
    f[18] = 0.f;
    f[19] = 0.f;
    float4* d32 = g32 + (slot * 4 + mu) * 5;
#pragma unroll
    for (int k = 0; k < 5; k++) d32[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    uint32_t w[12];
#pragma unroll
    for (int k = 0; k < 9; k++)
      w[k] = (uint32_t)__half_as_ushort(__float2half_rn((float)v[k].x)) |
             ((uint32_t)__half_as_ushort(__float2half_rn((float)v[k].y)) << 16);
    w[9] = w[10] = w[11] = 0u;
    uint4* d16 = g16 + (slot * 4 + mu) * 3;
#pragma unroll
    for (int k = 0; k < 3; k++) d16[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  }
}

// (Pb)_1 = P_- b_1 (spins 2,3), (Pb)_Ls = P_+ b_1 (spins 0,1); zero elsewhere.
__global__ void source_pb_kernel(const Geom g, void* p0, void* p1, const double* src) {
  const size_t V = (size_t)g.Vh * 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V;
       i += (size_t)gridDim.x * blockDim.x) {
    int x, y, z, t;
    lex_coords(g, (int)i, x, y, z, t);
    const int par = (x + y + z + t) & 1;
    const int h = (int)(i >> 1);
    void* half = par ? p1 : p0;
    const double2* b = reinterpret_cast<const double2*>(src) + i * 12;
    for (int s = 0; s < g.Ls; s++) {
      Spinor<double> a;
#pragma unroll
      for (int k = 0; k < 12; k++) a.c[k] = cmake(0.0, 0.0);
      if (s == 0) {
#pragma unroll
        for (int k = 6; k < 12; k++) a.c[k] = cmake(b[k].x, b[k].y);
      }
      if (s == g.Ls - 1) {
#pragma unroll
        for (int k = 0; k < 6; k++) a.c[k] = cmake(b[k].x, b[k].y);
      }
      Store64::store(half, site5(h, s, g.Ls), g.N5, a);
    }
  }
}

// z_1 = P_- psi_1 + P_+ psi_Ls
__global__ void extract_z1_kernel(const Geom g, double* prop, const void* p0, const void* p1) {
  const size_t V = (size_t)g.Vh * 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V;
       i += (size_t)gridDim.x * blockDim.x) {
    int x, y, z, t;
    lex_coords(g, (int)i, x, y, z, t);
    const int par = (x + y + z + t) & 1;
    const int h = (int)(i >> 1);
    const void* half = par ? p1 : p0;
    Spinor<double> a, b;
    Store64::load(half, site5(h, 0, g.Ls), g.N5, a);
    Store64::load(half, site5(h, g.Ls - 1, g.Ls), g.N5, b);
    double2* o = reinterpret_cast<double2*>(prop) + i * 12;
#pragma unroll
    for (int k = 0; k < 6; k++) o[k] = make_double2(b.c[k].re, b.c[k].im);
#pragma unroll
    for (int k = 6; k < 12; k++) o[k] = make_double2(a.c[k].re, a.c[k].im);
  }
}

// ---- BLAS-1 -------------------------------------------------------------------
// One thread per slice pair m (two 5D sites), vector loads of the pair layout.

template <class SPX, class SP>
__global__ void __launch_bounds__(kBlasThreads) xr_update_kernel(
    const Geom g, void* x, void* r, const void* p, const void* w, const double* num,
    const double* den, int sstride, size_t stride_x, size_t stride, Reduce red, const int* active) {
  using T = typename SP::T;
  using TX = typename SPX::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const size_t off = rhs * stride, offx = rhs * stride_x;
  const double ad = num[rhs * sstride] / den[rhs * sstride];
  const T a = (T)ad;
  const TX ax = (TX)ad;
  const int NP = g.N5 >> 1;
  double acc = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<TX> xv[2];
    Spinor<T> rv[2], pv[2], wv[2];
    SPX::load_pair(reinterpret_cast<const char*>(x) + offx, m, NP, xv[0], xv[1]);
    SP::load_pair(reinterpret_cast<const char*>(r) + off, m, NP, rv[0], rv[1]);
    SP::load_pair(reinterpret_cast<const char*>(p) + off, m, NP, pv[0], pv[1]);
    SP::load_pair(reinterpret_cast<const char*>(w) + off, m, NP, wv[0], wv[1]);
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        xv[l].c[k] = cmake(fma(ax, (TX)pv[l].c[k].re, xv[l].c[k].re), fma(ax, (TX)pv[l].c[k].im, xv[l].c[k].im));
        rv[l].c[k] = cmake(fma(-a, wv[l].c[k].re, rv[l].c[k].re), fma(-a, wv[l].c[k].im, rv[l].c[k].im));
      }
    SPX::store_pair(reinterpret_cast<char*>(x) + offx, m, NP, xv[0], xv[1]);
    SP::store_pair(reinterpret_cast<char*>(r) + off, m, NP, rv[0], rv[1]);
    acc += sqd(rv[0]) + sqd(rv[1]);
  }
  block_sum_to(acc, red, rhs, gridDim.x, blockIdx.x);
}

template <class SP>
__global__ void __launch_bounds__(kBlasThreads) p_update_kernel(
    const Geom g, void* p, const void* z, const double* num, const double* den, int sstride,
    size_t stride, const int* active) {
  using T = typename SP::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const size_t off = rhs * stride;
  const T beta = (T)(num[rhs * sstride] / den[rhs * sstride]);
  const int NP = g.N5 >> 1;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<T> pv[2], zv[2];
    SP::load_pair(reinterpret_cast<const char*>(p) + off, m, NP, pv[0], pv[1]);
    SP::load_pair(reinterpret_cast<const char*>(z) + off, m, NP, zv[0], zv[1]);
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++)
        pv[l].c[k] = cmake(fma(beta, pv[l].c[k].re, zv[l].c[k].re), fma(beta, pv[l].c[k].im, zv[l].c[k].im));
    SP::store_pair(reinterpret_cast<char*>(p) + off, m, NP, pv[0], pv[1]);
  }
}


template <class SPX, class SP>
__global__ void __launch_bounds__(kBlasThreads) px_update_kernel(
    const Geom g, void* x, void* p, const void* z, const double* a_ptr, const double* num,
    const double* den, int sstride, size_t stride_x, size_t stride, const int* active, int do_p) {
  using T = typename SP::T;
  using TX = typename SPX::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const size_t off = rhs * stride, offx = rhs * stride_x;
  const TX a = (TX)a_ptr[(size_t)rhs * sstride];
  const T beta = do_p ? (T)(num[(size_t)rhs * sstride] / den[(size_t)rhs * sstride]) : (T)0;
  const int NP = g.N5 >> 1;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<T> pv[2];
    Spinor<TX> xv[2];
    SP::load_pair(reinterpret_cast<const char*>(p) + off, m, NP, pv[0], pv[1]);
    SPX::load_pair(reinterpret_cast<const char*>(x) + offx, m, NP, xv[0], xv[1]);
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++)
        xv[l].c[k] = cmake(fma(a, (TX)pv[l].c[k].re, xv[l].c[k].re), fma(a, (TX)pv[l].c[k].im, xv[l].c[k].im));
    SPX::store_pair(reinterpret_cast<char*>(x) + offx, m, NP, xv[0], xv[1]);
    if (do_p) {
      Spinor<T> zv[2];
      SP::load_pair(reinterpret_cast<const char*>(z) + off, m, NP, zv[0], zv[1]);
#pragma unroll
      for (int l = 0; l < 2; l++)
#pragma unroll
        for (int k = 0; k < 12; k++)
          pv[l].c[k] = cmake(fma(beta, pv[l].c[k].re, zv[l].c[k].re), fma(beta, pv[l].c[k].im, zv[l].c[k].im));
      SP::store_pair(reinterpret_cast<char*>(p) + off, m, NP, pv[0], pv[1]);
    }
  }
}

// p_new = z + beta p_old (and, with do_x, the deferred x += a_prev p_old) for one
// slice pair m of site h, t = m mod (Ls/2), plus bp = B p_new: B is cyclic
// bidiagonal per chirality (Eq. mobius1 with D_w -> 1),
//   (B v)+(s) = d+(s) v+(s) + o+(s) v+(s-1),  (B v)-(s) = d-(s) v-(s) + o-(s) v-(s+1),
// so v+ of slice 2t-1 (pair below) and v- of slice 2t+2 (pair above) are formed
// from z and p of those pairs as well.  Used by the CG on the tuned path, whose
// D_bb pass A then hops B p directly.  p_old and p_new are different buffers
// (neighbouring pairs of p_old are read while p_new is written).
// FP32 fields: two CTAs per SM (128 registers, 48 bytes spilled) so that one
// CTA's loads overlap the other's stores; the other combinations would spill
// hundreds of bytes at that cap and keep one CTA per SM.
template <class SPX, class SP>
constexpr int pxb_min_blocks() {
  return SP::kPrec == P32 && SPX::kPrec == P32 ? 2 : 1;
}

template <class SPX, class SP>
__global__ void __launch_bounds__(kBlasThreads, (pxb_min_blocks<SPX, SP>())) pxb_update_kernel(
    const Geom g, void* x, const void* p, void* pnew, void* bp, const void* z, const double* a_ptr,
    const double* num, const double* den, int sstride, size_t stride_x, size_t stride,
    const typename SP::T* bdiag, const typename SP::T* boff, size_t cstride, const int* active,
    int do_x) {
  using T = typename SP::T;
  using TX = typename SPX::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const size_t off = rhs * stride, offx = rhs * stride_x;
  const TX a = do_x ? (TX)a_ptr[(size_t)rhs * sstride] : (TX)0;
  const T beta = (T)(num[(size_t)rhs * sstride] / den[(size_t)rhs * sstride]);
  const int NP = g.N5 >> 1, half = g.Ls >> 1;
  const T* bd = bdiag + (size_t)rhs * cstride;
  const T* bo = boff + (size_t)rhs * cstride;
  const char* pb = reinterpret_cast<const char*>(p) + off;
  const char* zb = reinterpret_cast<const char*>(z) + off;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    const int t = m % half, base = m - t;
    const int mp = base + (t == 0 ? half - 1 : t - 1), mn = base + (t + 1 == half ? 0 : t + 1);
    // the slice below the pair (lane 1 of pair mp) enters through its v+ half,
    // the slice above (lane 0 of pair mn) through its v- half; 16-bit storage
    // loads all 12 components of those slices (the scale of their stored p_new)
    const int n_below = 2 * mp + 1, n_above = 2 * mn;
    Spinor<T> pv[2], zv[2], pl, zl, pu, zu;
    SP::load_pair(pb, m, NP, pv[0], pv[1]);
    SP::load_pair(zb, m, NP, zv[0], zv[1]);
    SP::load_chir(pb, n_below, g.N5, 0, pl);
    SP::load_chir(zb, n_below, g.N5, 0, zl);
    SP::load_chir(pb, n_above, g.N5, 1, pu);
    SP::load_chir(zb, n_above, g.N5, 1, zu);
    if (do_x) {
      Spinor<TX> xv[2];
      SPX::load_pair(reinterpret_cast<const char*>(x) + offx, m, NP, xv[0], xv[1]);
#pragma unroll
      for (int l = 0; l < 2; l++)
#pragma unroll
        for (int k = 0; k < 12; k++)
          xv[l].c[k] = cmake(fma(a, (TX)pv[l].c[k].re, xv[l].c[k].re), fma(a, (TX)pv[l].c[k].im, xv[l].c[k].im));
      SPX::store_pair(reinterpret_cast<char*>(x) + offx, m, NP, xv[0], xv[1]);
    }
    // p_new on the pair, v+ of the slice below and v- of the slice above
    Spinor<T> q[2], qb, qa;
#pragma unroll
    for (int k = 0; k < 12; k++) {
#pragma unroll
      for (int l = 0; l < 2; l++)
        q[l].c[k] = cmake(fma(beta, pv[l].c[k].re, zv[l].c[k].re), fma(beta, pv[l].c[k].im, zv[l].c[k].im));
      if (SP::kScaled || k < 6)
        qb.c[k] = cmake(fma(beta, pl.c[k].re, zl.c[k].re), fma(beta, pl.c[k].im, zl.c[k].im));
      if (SP::kScaled || k >= 6)
        qa.c[k] = cmake(fma(beta, pu.c[k].re, zu.c[k].re), fma(beta, pu.c[k].im, zu.c[k].im));
    }
    SP::store_pair(reinterpret_cast<char*>(pnew) + off, m, NP, q[0], q[1]);
    if constexpr (SP::kScaled) {
      // 16-bit storage: B acts on the stored (rounded) p_new, as pass B's local
      // term sees it; the slices below and above round with their own scales
      SP::quantize(q[0]);
      SP::quantize(q[1]);
      SP::quantize(qb);
      SP::quantize(qa);
    }
    cplx<T> below[6], above[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      below[k] = qb.c[k];
      above[k] = qa.c[6 + k];
    }
    const int s0 = 2 * t;
    const T dp0 = bd[s0], dp1 = bd[s0 + 1], op0 = bo[s0], op1 = bo[s0 + 1];
    const T dm0 = bd[g.Ls + s0], dm1 = bd[g.Ls + s0 + 1], om0 = bo[g.Ls + s0], om1 = bo[g.Ls + s0 + 1];
    Spinor<T> b[2];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      b[0].c[k] = cmake(fma(op0, below[k].re, dp0 * q[0].c[k].re), fma(op0, below[k].im, dp0 * q[0].c[k].im));
      b[1].c[k] = cmake(fma(op1, q[0].c[k].re, dp1 * q[1].c[k].re), fma(op1, q[0].c[k].im, dp1 * q[1].c[k].im));
      b[0].c[6 + k] = cmake(fma(om0, q[1].c[6 + k].re, dm0 * q[0].c[6 + k].re),
                            fma(om0, q[1].c[6 + k].im, dm0 * q[0].c[6 + k].im));
      b[1].c[6 + k] = cmake(fma(om1, above[k].re, dm1 * q[1].c[6 + k].re),
                            fma(om1, above[k].im, dm1 * q[1].c[6 + k].im));
    }
    SP::store_pair(reinterpret_cast<char*>(bp) + off, m, NP, b[0], b[1]);
  }
}

// dst <- src converted; the norm (optional) is that of the stored dst values.
template <class SPD, class SPS>
__global__ void __launch_bounds__(kBlasThreads) convert_kernel(
    const Geom g, void* dst, const void* src, size_t sd, size_t ss, Reduce red, int do_norm,
    const int* active) {
  using TD = typename SPD::T;
  using TS = typename SPS::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int NP = g.N5 >> 1;
  double acc = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<TS> a[2];
    SPS::load_pair(reinterpret_cast<const char*>(src) + rhs * ss, m, NP, a[0], a[1]);
    Spinor<TD> b[2];
    cvt(b[0], a[0]);
    cvt(b[1], a[1]);
    SPD::store_pair(reinterpret_cast<char*>(dst) + rhs * sd, m, NP, b[0], b[1]);
    if (do_norm) {
      if constexpr (SPD::kScaled) {
        SPD::quantize(b[0]);
        SPD::quantize(b[1]);
      }
      acc += sqd(b[0]) + sqd(b[1]);
    }
  }
  if (do_norm) block_sum_to(acc, red, rhs, gridDim.x, blockIdx.x);
}

template <class SPS>
__global__ void __launch_bounds__(kBlasThreads) accumulate64_kernel(
    const Geom g, void* x64, void* src, int zero_src, size_t sd, size_t ss, const int* active) {
  using TS = typename SPS::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int NP = g.N5 >> 1;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<TS> a[2];
    SPS::load_pair(reinterpret_cast<const char*>(src) + rhs * ss, m, NP, a[0], a[1]);
    Spinor<double> x[2];
    Store64::load_pair(reinterpret_cast<const char*>(x64) + rhs * sd, m, NP, x[0], x[1]);
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++)
        x[l].c[k] = cmake(x[l].c[k].re + (double)a[l].c[k].re, x[l].c[k].im + (double)a[l].c[k].im);
    Store64::store_pair(reinterpret_cast<char*>(x64) + rhs * sd, m, NP, x[0], x[1]);
    if (zero_src) {
      Spinor<TS> zz;
#pragma unroll
      for (int k = 0; k < 12; k++) zz.c[k] = cmake<TS>(0, 0);
      SPS::store_pair(reinterpret_cast<char*>(src) + rhs * ss, m, NP, zz, zz);
    }
  }
}

__global__ void __launch_bounds__(kBlasThreads) sub64_norm_kernel(
    const Geom g, void* out, const void* a, const void* b, size_t stride, Reduce red,
    const int* active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const size_t off = rhs * stride;
  const int NP = g.N5 >> 1;
  double acc = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<double> x[2], y[2];
    Store64::load_pair(reinterpret_cast<const char*>(a) + off, m, NP, x[0], x[1]);
    Store64::load_pair(reinterpret_cast<const char*>(b) + off, m, NP, y[0], y[1]);
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++) x[l].c[k] = x[l].c[k] - y[l].c[k];
    Store64::store_pair(reinterpret_cast<char*>(out) + off, m, NP, x[0], x[1]);
    acc += sqd(x[0]) + sqd(x[1]);
  }
  block_sum_to(acc, red, rhs, gridDim.x, blockIdx.x);
}

// dst <- a - b with a FP64 and b FP32 (the difference in FP64), stored in the
// precision of SPD; |dst|^2 of the stored values.
template <class SPD>
__global__ void __launch_bounds__(kBlasThreads) sub_to_kernel(
    const Geom g, void* dst, const void* a, const void* b, size_t sd, size_t sa, size_t sb,
    Reduce red, const int* active) {
  using TD = typename SPD::T;
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const int NP = g.N5 >> 1;
  double acc = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<double> x[2];
    Spinor<float> y[2];
    Store64::load_pair(reinterpret_cast<const char*>(a) + rhs * sa, m, NP, x[0], x[1]);
    Store32::load_pair(reinterpret_cast<const char*>(b) + rhs * sb, m, NP, y[0], y[1]);
    Spinor<TD> d[2];
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++)
        d[l].c[k] = cmake<TD>((TD)(x[l].c[k].re - (double)y[l].c[k].re),
                              (TD)(x[l].c[k].im - (double)y[l].c[k].im));
    SPD::store_pair(reinterpret_cast<char*>(dst) + rhs * sd, m, NP, d[0], d[1]);
    if constexpr (SPD::kScaled) {
      SPD::quantize(d[0]);
      SPD::quantize(d[1]);
    }
    acc += sqd(d[0]) + sqd(d[1]);
  }
  block_sum_to(acc, red, rhs, gridDim.x, blockIdx.x);
}

template <class SP>
__global__ void __launch_bounds__(kBlasThreads) norm_kernel(const Geom g, const void* x,
                                                             size_t stride, Reduce red) {
  using T = typename SP::T;
  const int rhs = blockIdx.y;
  const int NP = g.N5 >> 1;
  double acc = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<T> a[2];
    SP::load_pair(reinterpret_cast<const char*>(x) + rhs * stride, m, NP, a[0], a[1]);
    acc += sqd(a[0]) + sqd(a[1]);
  }
  block_sum_to(acc, red, rhs, gridDim.x, blockIdx.x);
}

// Re <a, b> of two FP64 half-fields (one right-hand side per blockIdx.y).
__global__ void __launch_bounds__(kBlasThreads) dot_re64_kernel(const Geom g, const void* a,
                                                                 const void* b, size_t stride,
                                                                 Reduce red) {
  const int rhs = blockIdx.y;
  const int NP = g.N5 >> 1;
  double acc = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < NP; m += gridDim.x * blockDim.x) {
    Spinor<double> x[2], y[2];
    Store64::load_pair(reinterpret_cast<const char*>(a) + rhs * stride, m, NP, x[0], x[1]);
    Store64::load_pair(reinterpret_cast<const char*>(b) + rhs * stride, m, NP, y[0], y[1]);
#pragma unroll
    for (int l = 0; l < 2; l++)
#pragma unroll
      for (int k = 0; k < 12; k++)
        acc = fma(x[l].c[k].re, y[l].c[k].re, fma(x[l].c[k].im, y[l].c[k].im, acc));
  }
  block_sum_to(acc, red, rhs, gridDim.x, blockIdx.x);
}

int elementwise_blocks(size_t n) {
  size_t b = (n + kBlasThreads - 1) / kBlasThreads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int blas_grid_blocks(const Geom& g) { return elementwise_blocks((size_t)g.N5 / 2); }

size_t field_bytes(const Geom& g, int prec) {
  size_t b = 0;
  switch (prec) {
    case P64: b = (size_t)g.N5 * 192; break;
    case P32: b = (size_t)g.N5 * 96; break;
    case P16:
    case PB16: b = (size_t)g.N5 * 52; break;
    default: return 0;
  }
  return (b + 255) / 256 * 256;
}

size_t gauge_bytes(const Geom& g, int prec) {
  const size_t links = (size_t)g.Vh * 2 * 4;
  switch (prec) {
    case P64: return links * 144;
    case P32: return links * 80;
    default: return links * 48;
  }
}

#define DWF_PREC_SWITCH(prec, SP, ...)                 \
  switch (prec) {                                      \
    case P64: { using SP = Store64; __VA_ARGS__; } break;        \
    case P32: { using SP = Store32; __VA_ARGS__; } break;        \
    case P16: { using SP = Store16<false>; __VA_ARGS__; } break; \
    case PB16: { using SP = Store16<true>; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;             \
  }

cudaError_t launch_pack_half(const Geom& g, int prec, void* dst, const double* src, int nrhs,
                             cudaStream_t s) {
  const size_t stride = field_bytes(g, prec);
  const int blocks = elementwise_blocks((size_t)g.N5 * nrhs);
  DWF_PREC_SWITCH(prec, SP, pack_half_kernel<SP><<<blocks, kBlasThreads, 0, s>>>(g, dst, src, stride, nrhs));
  return cudaGetLastError();
}

cudaError_t launch_unpack_half(const Geom& g, int prec, double* dst, const void* src, int nrhs,
                               cudaStream_t s) {
  const size_t stride = field_bytes(g, prec);
  const int blocks = elementwise_blocks((size_t)g.N5 * nrhs);
  DWF_PREC_SWITCH(prec, SP, unpack_half_kernel<SP><<<blocks, kBlasThreads, 0, s>>>(g, dst, src, stride, nrhs));
  return cudaGetLastError();
}

cudaError_t launch_split_full(const Geom& g, void* p0, void* p1, const double* full, cudaStream_t s) {
  split_full_kernel<<<elementwise_blocks((size_t)g.N5 * 2), kBlasThreads, 0, s>>>(g, p0, p1, full, 0);
  return cudaGetLastError();
}

cudaError_t launch_merge_full(const Geom& g, double* full, const void* p0, const void* p1,
                              cudaStream_t s) {
  split_full_kernel<<<elementwise_blocks((size_t)g.N5 * 2), kBlasThreads, 0, s>>>(
      g, const_cast<void*>(p0), const_cast<void*>(p1), full, 1);
  return cudaGetLastError();
}

cudaError_t launch_gauge_convert(const Geom& g, const double* U, void* g64, void* g32, void* g16,
                                 cudaStream_t s) {
  gauge_convert_kernel<<<elementwise_blocks((size_t)g.Vh * 8), kBlasThreads, 0, s>>>(
      g, U, reinterpret_cast<double2*>(g64), reinterpret_cast<float4*>(g32),
      reinterpret_cast<uint4*>(g16));
  return cudaGetLastError();
}

cudaError_t launch_source_pb(const Geom& g, void* p0, void* p1, const double* src, cudaStream_t s) {
  source_pb_kernel<<<elementwise_blocks((size_t)g.Vh * 2), kBlasThreads, 0, s>>>(g, p0, p1, src);
  return cudaGetLastError();
}

cudaError_t launch_extract_z1(const Geom& g, double* prop, const void* p0, const void* p1,
                              cudaStream_t s) {
  extract_z1_kernel<<<elementwise_blocks((size_t)g.Vh * 2), kBlasThreads, 0, s>>>(g, prop, p0, p1);
  return cudaGetLastError();
}

cudaError_t launch_xr_update(const Geom& g, int prec, int xprec, void* x, void* r, const void* p,
                             const void* w, const double* num, const double* den, int sstride,
                             int nrhs, size_t stride_x, size_t stride, const Reduce* red,
                             cudaStream_t s, const int* active) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  if (xprec == prec) {
    DWF_PREC_SWITCH(prec, SP, xr_update_kernel<SP, SP><<<grid, kBlasThreads, 0, s>>>(g, x, r, p, w, num, den, sstride, stride_x, stride, *red, active));
  } else if (xprec == P32) {
    DWF_PREC_SWITCH(prec, SP, xr_update_kernel<Store32, SP><<<grid, kBlasThreads, 0, s>>>(g, x, r, p, w, num, den, sstride, stride_x, stride, *red, active));
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_p_update(const Geom& g, int prec, void* p, const void* z, const double* num,
                            const double* den, int sstride, int nrhs, size_t stride,
                            cudaStream_t s, const int* active) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  DWF_PREC_SWITCH(prec, SP, p_update_kernel<SP><<<grid, kBlasThreads, 0, s>>>(g, p, z, num, den, sstride, stride, active));
  return cudaGetLastError();
}

template <class SPD>
cudaError_t convert_from(const Geom& g, void* dst, int prec_s, const void* src, int nrhs, size_t sd,
                         size_t ss, const Reduce* red, cudaStream_t s, const int* active) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  Reduce r{};
  if (red) r = *red;
  const int dn = red != nullptr;
  DWF_PREC_SWITCH(prec_s, SPS, convert_kernel<SPD, SPS><<<grid, kBlasThreads, 0, s>>>(g, dst, src, sd, ss, r, dn, active));
  return cudaGetLastError();
}

cudaError_t launch_convert(const Geom& g, int prec_d, void* dst, int prec_s, const void* src,
                           int nrhs, size_t sd, size_t ss, const Reduce* red, cudaStream_t s,
                           const int* active) {
  switch (prec_d) {
    case P64: return convert_from<Store64>(g, dst, prec_s, src, nrhs, sd, ss, red, s, active);
    case P32: return convert_from<Store32>(g, dst, prec_s, src, nrhs, sd, ss, red, s, active);
    case P16: return convert_from<Store16<false>>(g, dst, prec_s, src, nrhs, sd, ss, red, s, active);
    case PB16: return convert_from<Store16<true>>(g, dst, prec_s, src, nrhs, sd, ss, red, s, active);
  }
  return cudaErrorInvalidValue;
}


template <class SPX>
cudaError_t px_from(const Geom& g, int prec, void* x, void* p, const void* z, const double* a_ptr,
                    const double* num, const double* den, int sstride, int nrhs, size_t sx,
                    size_t sp, cudaStream_t s, const int* active, int do_p) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  DWF_PREC_SWITCH(prec, SP, px_update_kernel<SPX, SP><<<grid, kBlasThreads, 0, s>>>(g, x, p, z, a_ptr, num, den, sstride, sx, sp, active, do_p));
  return cudaGetLastError();
}

cudaError_t launch_px_update(const Geom& g, int prec, int xprec, void* x, void* p, const void* z,
                             const double* a_ptr, const double* num, const double* den,
                             int sstride, int nrhs, size_t sx, size_t sp, cudaStream_t s,
                             const int* active) {
  if (xprec == P64) return px_from<Store64>(g, prec, x, p, z, a_ptr, num, den, sstride, nrhs, sx, sp, s, active, 1);
  return px_from<Store32>(g, prec, x, p, z, a_ptr, num, den, sstride, nrhs, sx, sp, s, active, 1);
}

cudaError_t launch_x_update(const Geom& g, int prec, int xprec, void* x, const void* p,
                            const double* a_ptr, int sstride, int nrhs, size_t sx, size_t sp,
                            cudaStream_t s, const int* active) {
  void* pp = const_cast<void*>(p);
  if (xprec == P64) return px_from<Store64>(g, prec, x, pp, nullptr, a_ptr, a_ptr, a_ptr, sstride, nrhs, sx, sp, s, active, 0);
  return px_from<Store32>(g, prec, x, pp, nullptr, a_ptr, a_ptr, a_ptr, sstride, nrhs, sx, sp, s, active, 0);
}

cudaError_t launch_pxb_update(const Geom& g, int prec, int xprec, void* x, const void* p,
                              void* pnew, void* bp, const void* z, const double* a_ptr, const double* num,
                              const double* den, int sstride, int nrhs, size_t sx, size_t sp,
                              const void* bdiag, const void* boff, size_t cstride, cudaStream_t s,
                              const int* active, int do_x) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  if (prec == P32 && xprec == P32) {
    pxb_update_kernel<Store32, Store32><<<grid, kBlasThreads, 0, s>>>(
        g, x, p, pnew, bp, z, a_ptr, num, den, sstride, sx, sp, reinterpret_cast<const float*>(bdiag),
        reinterpret_cast<const float*>(boff), cstride, active, do_x);
  } else if (prec == P32 && xprec == P64) {
    pxb_update_kernel<Store64, Store32><<<grid, kBlasThreads, 0, s>>>(
        g, x, p, pnew, bp, z, a_ptr, num, den, sstride, sx, sp, reinterpret_cast<const float*>(bdiag),
        reinterpret_cast<const float*>(boff), cstride, active, do_x);
  } else if (prec == P64 && xprec == P64) {
    pxb_update_kernel<Store64, Store64><<<grid, kBlasThreads, 0, s>>>(
        g, x, p, pnew, bp, z, a_ptr, num, den, sstride, sx, sp, reinterpret_cast<const double*>(bdiag),
        reinterpret_cast<const double*>(boff), cstride, active, do_x);
  } else if (prec == P16 && xprec == P32) {
    pxb_update_kernel<Store32, Store16<false>><<<grid, kBlasThreads, 0, s>>>(
        g, x, p, pnew, bp, z, a_ptr, num, den, sstride, sx, sp, reinterpret_cast<const float*>(bdiag),
        reinterpret_cast<const float*>(boff), cstride, active, do_x);
  } else if (prec == PB16 && xprec == P32) {
    pxb_update_kernel<Store32, Store16<true>><<<grid, kBlasThreads, 0, s>>>(
        g, x, p, pnew, bp, z, a_ptr, num, den, sstride, sx, sp, reinterpret_cast<const float*>(bdiag),
        reinterpret_cast<const float*>(boff), cstride, active, do_x);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_accumulate64(const Geom& g, void* x64, int prec_s, void* src, int zero_src,
                                int nrhs, size_t sd, size_t ss, cudaStream_t s, const int* active) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  DWF_PREC_SWITCH(prec_s, SPS, accumulate64_kernel<SPS><<<grid, kBlasThreads, 0, s>>>(g, x64, src, zero_src, sd, ss, active));
  return cudaGetLastError();
}

cudaError_t launch_sub64_norm(const Geom& g, void* out, const void* a, const void* b, int nrhs,
                              size_t stride, const Reduce* red, cudaStream_t s, const int* active) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  sub64_norm_kernel<<<grid, kBlasThreads, 0, s>>>(g, out, a, b, stride, *red, active);
  return cudaGetLastError();
}

cudaError_t launch_sub_to(const Geom& g, int prec_d, void* dst, const void* a64, const void* b32,
                          int nrhs, size_t sd, size_t sa, size_t sb, const Reduce* red,
                          cudaStream_t s, const int* active) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  switch (prec_d) {
    case P32:
      sub_to_kernel<Store32><<<grid, kBlasThreads, 0, s>>>(g, dst, a64, b32, sd, sa, sb, *red, active);
      break;
    case P16:
      sub_to_kernel<Store16<false>><<<grid, kBlasThreads, 0, s>>>(g, dst, a64, b32, sd, sa, sb, *red,
                                                                  active);
      break;
    case PB16:
      sub_to_kernel<Store16<true>><<<grid, kBlasThreads, 0, s>>>(g, dst, a64, b32, sd, sa, sb, *red,
                                                                 active);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_norm(const Geom& g, int prec, const void* x, int nrhs, size_t stride,
                        const Reduce* red, cudaStream_t s) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  DWF_PREC_SWITCH(prec, SP, norm_kernel<SP><<<grid, kBlasThreads, 0, s>>>(g, x, stride, *red));
  return cudaGetLastError();
}

cudaError_t launch_dot_re64(const Geom& g, const void* a, const void* b, int nrhs, size_t stride,
                            const Reduce* red, cudaStream_t s) {
  dim3 grid(elementwise_blocks((size_t)g.N5 / 2), nrhs);
  dot_re64_kernel<<<grid, kBlasThreads, 0, s>>>(g, a, b, stride, *red);
  return cudaGetLastError();
}

}  // namespace dwf
