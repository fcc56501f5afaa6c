// dwf_fields.cuh -- device-side complex numbers, spinors, storage policies and
// the chiral-basis spin projection used by the hopping kernels.
#pragma once

#include "dwf_internal.cuh"

namespace dwf {

template <typename T>
struct cplx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmake(T r, T i) {
  cplx<T> c;
  c.re = r;
  c.im = i;
  return c;
}
template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return cmake(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return cmake(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return cmake(s * a.re, s * a.im); }
// i * a
template <typename T>
__device__ __forceinline__ cplx<T> times_i(cplx<T> a) { return cmake(-a.im, a.re); }
// acc += u * v
template <typename T>
__device__ __forceinline__ void cmac(cplx<T>& acc, cplx<T> u, cplx<T> v) {
  acc.re = fma(u.re, v.re, acc.re);
  acc.re = fma(-u.im, v.im, acc.re);
  acc.im = fma(u.re, v.im, acc.im);
  acc.im = fma(u.im, v.re, acc.im);
}
// acc += conj(u) * v
template <typename T>
__device__ __forceinline__ void cmac_conj(cplx<T>& acc, cplx<T> u, cplx<T> v) {
  acc.re = fma(u.re, v.re, acc.re);
  acc.re = fma(u.im, v.im, acc.re);
  acc.im = fma(u.re, v.im, acc.im);
  acc.im = fma(-u.im, v.re, acc.im);
}

// 4 spins x 3 colours; index spin * 3 + colour.  Spins 0,1: P_+, spins 2,3: P_-.
template <typename T>
struct Spinor {
  cplx<T> c[12];
};

template <typename T>
struct Link {
  cplx<T> u[9];  // row-major U[a][b] = u[3a+b]
};

// 5D index of slice s of half-site h: n = h * Ls + s.  Slices are stored in
// pairs: pair m = n >> 1 holds the slices 2j, 2j + 1 of one site (Ls even) in
// its two lanes l = n & 1, so that a thread owning a slice pair reads both with
// one vector load and computes on them with paired FP32 instructions.
__host__ __device__ __forceinline__ int site5(int h, int s, int Ls) { return h * Ls + s; }

// ---------------------------------------------------------------------------
// Storage policies.  Half-field layout with NP = N5 / 2 slice pairs; for each
// spinor component c = spin * 3 + colour, pair m stores
// (re lane 0, re lane 1, im lane 0, im lane 1):
//   FP64       double[12][NP][4]                                  192 B / site
//   FP32       float [12][NP][4]                                   96 B / site
//   FP16/BF16  uint4 [6][NP]: chunk j = components 2j, 2j+1 as the
//              words (re c, im c, re c+1, im c+1), each word the 16-bit
//              values of lane 0 (low half) and lane 1 (high half);
//              then float scale[N5] (index n)                      52 B / site
// load/store move one 5D site n (scalar lanes; the generic kernels and the
// conversions); load_pair/store_pair move the two sites of pair m.
// ---------------------------------------------------------------------------
struct Store64 {
  using T = double;
  static constexpr int kPrec = P64;
  static constexpr bool kScaled = false;
  __device__ static const double* at(const void* base, int c, int n, int N5) {
    return reinterpret_cast<const double*>(base) + ((size_t)c * (N5 >> 1) + (n >> 1)) * 4 + (n & 1);
  }
  __device__ static void load(const void* base, int n, int N5, Spinor<double>& o) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double* q = at(base, k, n, N5);
      o.c[k] = cmake(__ldg(q), __ldg(q + 2));
    }
  }
  // spins of one chirality only (chir 0: spins 0,1; chir 1: spins 2,3)
  __device__ static void load_chir(const void* base, int n, int N5, int chir, Spinor<double>& o) {
#pragma unroll
    for (int k = 6 * chir; k < 6 * chir + 6; k++) {
      const double* q = at(base, k, n, N5);
      o.c[k] = cmake(__ldg(q), __ldg(q + 2));
    }
  }
  __device__ static void store(void* base, int n, int N5, const Spinor<double>& o) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double* q = const_cast<double*>(at(base, k, n, N5));
      q[0] = o.c[k].re;
      q[2] = o.c[k].im;
    }
  }
  __device__ static void load_pair(const void* base, int m, int NP, Spinor<double>& a, Spinor<double>& b) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double2 re = __ldg(p + ((size_t)k * NP + m) * 2), im = __ldg(p + ((size_t)k * NP + m) * 2 + 1);
      a.c[k] = cmake(re.x, im.x);
      b.c[k] = cmake(re.y, im.y);
    }
  }
  __device__ static void store_pair(void* base, int m, int NP, const Spinor<double>& a,
                                    const Spinor<double>& b) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      p[((size_t)k * NP + m) * 2] = make_double2(a.c[k].re, b.c[k].re);
      p[((size_t)k * NP + m) * 2 + 1] = make_double2(a.c[k].im, b.c[k].im);
    }
  }
};

struct Store32 {
  using T = float;
  static constexpr int kPrec = P32;
  static constexpr bool kScaled = false;
  __device__ static const float* at(const void* base, int c, int n, int N5) {
    return reinterpret_cast<const float*>(base) + ((size_t)c * (N5 >> 1) + (n >> 1)) * 4 + (n & 1);
  }
  __device__ static void load(const void* base, int n, int N5, Spinor<float>& o) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const float* q = at(base, k, n, N5);
      o.c[k] = cmake(__ldg(q), __ldg(q + 2));
    }
  }
  __device__ static void load_chir(const void* base, int n, int N5, int chir, Spinor<float>& o) {
#pragma unroll
    for (int k = 6 * chir; k < 6 * chir + 6; k++) {
      const float* q = at(base, k, n, N5);
      o.c[k] = cmake(__ldg(q), __ldg(q + 2));
    }
  }
  __device__ static void store(void* base, int n, int N5, const Spinor<float>& o) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      float* q = const_cast<float*>(at(base, k, n, N5));
      q[0] = o.c[k].re;
      q[2] = o.c[k].im;
    }
  }
  __device__ static void load_pair(const void* base, int m, int NP, Spinor<float>& a, Spinor<float>& b) {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const float4 v = __ldg(p + (size_t)k * NP + m);
      a.c[k] = cmake(v.x, v.z);
      b.c[k] = cmake(v.y, v.w);
    }
  }
  __device__ static void store_pair(void* base, int m, int NP, const Spinor<float>& a,
                                    const Spinor<float>& b) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++)
      p[(size_t)k * NP + m] = make_float4(a.c[k].re, b.c[k].re, a.c[k].im, b.c[k].im);
  }
};

// 16-bit storage with one FP32 scale per 5D site: value = stored * scale,
// scale = max |real component| of the site.
template <bool BF>
struct Store16 {
  using T = float;
  static constexpr int kPrec = BF ? PB16 : P16;
  static constexpr bool kScaled = true;
  __device__ static float to_f(uint16_t v) {
    if (BF) return __bfloat162float(__ushort_as_bfloat16(v));
    return __half2float(__ushort_as_half(v));
  }
  __device__ static uint16_t from_f(float f) {
    if (BF) return __bfloat16_as_ushort(__float2bfloat16_rn(f));
    return __half_as_ushort(__float2half_rn(f));
  }
  // both lanes of a 32-bit word -> (lane 0, lane 1) as FP32
  __device__ static float2 to_f2(uint32_t w) {
    if (BF) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
  }
  // (lane 0, lane 1) -> one word, round to nearest
  __device__ static uint32_t from_f2(float2 v) {
    if (BF) {
      const __nv_bfloat162 h = __float22bfloat162_rn(v);
      return *reinterpret_cast<const uint32_t*>(&h);
    }
    const __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static const float* scales(const void* base, int N5) {
    return reinterpret_cast<const float*>(reinterpret_cast<const uint4*>(base) + (size_t)3 * N5);
  }
  // the 16-bit entries of component c of site n: re at [0], im at [2] (units of uint16)
  __device__ static const uint16_t* at(const void* base, int c, int n, int N5) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint4*>(base) +
                                                         (size_t)(c >> 1) * (N5 >> 1) + (n >> 1));
    return reinterpret_cast<const uint16_t*>(w + 2 * (c & 1)) + (n & 1);
  }
  __device__ static void load(const void* base, int n, int N5, Spinor<float>& o) {
    const float sc = __ldg(scales(base, N5) + n);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const uint16_t* q = at(base, k, n, N5);
      o.c[k] = cmake(sc * to_f(__ldg(q)), sc * to_f(__ldg(q + 2)));
    }
  }
  __device__ static void load_chir(const void* base, int n, int N5, int chir, Spinor<float>& o) {
    load(base, n, N5, o);
  }
  // Per-site scale from the largest |component|.  Below the smallest normal float
  // (subnormal or zero, e.g. the far tail of a point-source solve) 1/max would
  // overflow to inf: such a site keeps scale 1, and its components, far below
  // 16-bit resolution, store as zero.  A NaN component still stores as NaN.
  __device__ static float scale_of(float mx) { return mx >= 1.17549435e-38f ? mx : 1.f; }
  __device__ static float maxabs(const Spinor<float>& o) {
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) mx = fmaxf(mx, fmaxf(fabsf(o.c[k].re), fabsf(o.c[k].im)));
    return mx;
  }
  // o <- what store() followed by load() gives back, computed in registers (a
  // kernel must not re-read through __ldg what it wrote itself).
  __device__ static void quantize(Spinor<float>& o) {
    const float sc = scale_of(maxabs(o));
    const float inv = 1.f / sc;
#pragma unroll
    for (int k = 0; k < 12; k++)
      o.c[k] = cmake(sc * to_f(from_f(o.c[k].re * inv)), sc * to_f(from_f(o.c[k].im * inv)));
  }
  // One site: 16-bit stores of its own lane only (the other lane of each word
  // belongs to the neighbouring slice, possibly written by another thread).
  __device__ static void store(void* base, int n, int N5, const Spinor<float>& o) {
    const float sc = scale_of(maxabs(o));
    const float inv = 1.f / sc;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      uint16_t* q = const_cast<uint16_t*>(at(base, k, n, N5));
      q[0] = from_f(o.c[k].re * inv);
      q[2] = from_f(o.c[k].im * inv);
    }
    const_cast<float*>(scales(base, N5))[n] = sc;
  }
  __device__ static void load_pair(const void* base, int m, int NP, Spinor<float>& a, Spinor<float>& b) {
    const uint4* p = reinterpret_cast<const uint4*>(base);
    const float2 sc = __ldg(reinterpret_cast<const float2*>(p + (size_t)6 * NP) + m);
#pragma unroll
    for (int j = 0; j < 6; j++) {
      const uint4 v = __ldg(p + (size_t)j * NP + m);
      const float2 r0 = to_f2(v.x), i0 = to_f2(v.y), r1 = to_f2(v.z), i1 = to_f2(v.w);
      a.c[2 * j] = cmake(sc.x * r0.x, sc.x * i0.x);
      b.c[2 * j] = cmake(sc.y * r0.y, sc.y * i0.y);
      a.c[2 * j + 1] = cmake(sc.x * r1.x, sc.x * i1.x);
      b.c[2 * j + 1] = cmake(sc.y * r1.y, sc.y * i1.y);
    }
  }
  __device__ static void store_pair(void* base, int m, int NP, const Spinor<float>& a,
                                    const Spinor<float>& b) {
    uint4* p = reinterpret_cast<uint4*>(base);
    const float sa = scale_of(maxabs(a)), sb = scale_of(maxabs(b));
    const float ia = 1.f / sa, ib = 1.f / sb;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      const int c0 = 2 * j, c1 = 2 * j + 1;
      p[(size_t)j * NP + m] =
          make_uint4(from_f2(make_float2(a.c[c0].re * ia, b.c[c0].re * ib)),
                     from_f2(make_float2(a.c[c0].im * ia, b.c[c0].im * ib)),
                     from_f2(make_float2(a.c[c1].re * ia, b.c[c1].re * ib)),
                     from_f2(make_float2(a.c[c1].im * ia, b.c[c1].im * ib)));
    }
    reinterpret_cast<float2*>(p + (size_t)6 * NP)[m] = make_float2(sa, sb);
  }
};

// ---------------------------------------------------------------------------
// Deterministic two-level sum of one double per thread into red.result[rhs]:
// warp shuffles, one partial per block (block bid of nblocks), and the last
// block of the right-hand side to finish (ticket from red.counter) adds the
// partials in block order.  Every thread of the block must call it (it
// synchronises the block); works for 1D and 2D blocks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum_to(double v, const Reduce& red, int rhs, int nblocks,
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

// ---------------------------------------------------------------------------
// Gauge policies: link of a half-site h in direction mu.
// ---------------------------------------------------------------------------
struct Gauge64 {
  using T = double;
  static constexpr int kLinkBytes = 144;
  __device__ static void load(const void* base, int h, int mu, Link<double>& U) {
    const double2* b = reinterpret_cast<const double2*>(base) + ((size_t)h * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      double2 v = __ldg(b + k);
      U.u[k] = cmake(v.x, v.y);
    }
  }
};
struct Gauge32 {
  using T = float;
  static constexpr int kLinkBytes = 80;
  __device__ static void load(const void* base, int h, int mu, Link<float>& U) {
    const float4* b = reinterpret_cast<const float4*>(base) + ((size_t)h * 4 + mu) * 5;
    float f[20];
#pragma unroll
    for (int k = 0; k < 5; k++) {
      float4 v = __ldg(b + k);
      f[4 * k] = v.x;
      f[4 * k + 1] = v.y;
      f[4 * k + 2] = v.z;
      f[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < 9; k++) U.u[k] = cmake(f[2 * k], f[2 * k + 1]);
  }
};
struct Gauge16 {
  using T = float;
  static constexpr int kLinkBytes = 48;
  __device__ static void load(const void* base, int h, int mu, Link<float>& U) {
    const uint4* b = reinterpret_cast<const uint4*>(base) + ((size_t)h * 4 + mu) * 3;
    uint32_t w[12];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 v = __ldg(b + k);
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
};

template <typename S> struct GaugeOf;
template <> struct GaugeOf<Store64> { using type = Gauge64; };
template <> struct GaugeOf<Store32> { using type = Gauge32; };
template <> struct GaugeOf<Store16<false>> { using type = Gauge16; };
template <> struct GaugeOf<Store16<true>> { using type = Gauge16; };

// ---------------------------------------------------------------------------
// Lattice geometry: half index h of parity p <-> coordinates, neighbours.
// ---------------------------------------------------------------------------
struct Coords {
  int x, y, z, t;
};

__device__ __forceinline__ Coords site_coords(const Geom& g, int h, int p) {
  Coords c;
  int xh = h % g.Lxh;
  int r = h / g.Lxh;
  c.y = r % g.L[1];
  r /= g.L[1];
  c.z = r % g.L[2];
  c.t = r / g.L[2];
  c.x = 2 * xh + ((c.y + c.z + c.t + p) & 1);
  return c;
}

__device__ __forceinline__ int half_index(const Geom& g, int x, int y, int z, int t) {
  return (x >> 1) + g.Lxh * (y + g.L[1] * (z + g.L[2] * t));
}

// Neighbour x + dir * mu: half index and boundary sign (bc_t across the t edge).
__device__ __forceinline__ int neighbour(const Geom& g, Coords c, int mu, int dir, int& sign) {
  sign = 1;
  int x = c.x, y = c.y, z = c.z, t = c.t;
  if (mu == 0) {
    x += dir;
    x = x < 0 ? x + g.L[0] : (x >= g.L[0] ? x - g.L[0] : x);
  } else if (mu == 1) {
    y += dir;
    y = y < 0 ? y + g.L[1] : (y >= g.L[1] ? y - g.L[1] : y);
  } else if (mu == 2) {
    z += dir;
    z = z < 0 ? z + g.L[2] : (z >= g.L[2] ? z - g.L[2] : z);
  } else {
    t += dir;
    if (t < 0) {
      t += g.L[3];
      sign = g.bc_t;
    } else if (t >= g.L[3]) {
      t -= g.L[3];
      sign = g.bc_t;
    }
  }
  return half_index(g, x, y, z, t);
}

// ---------------------------------------------------------------------------
// Spin projection in the chiral basis.  gamma_mu = [[0, A],[A^+, 0]] with
// A_x = -i sigma_1, A_y = -i sigma_2, A_z = -i sigma_3, A_t = 1.
// (1 - sg gamma_mu) psi = (h, -sg A^+ h),  h = psi_+ - sg A psi_-   (sg = +-1)
// so only the two-spin half spinor h is multiplied by the link.
// ---------------------------------------------------------------------------
template <typename T, int MU, int SG>
__device__ __forceinline__ void project(const Spinor<T>& s, cplx<T> h0[3], cplx<T> h1[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cplx<T> p0 = s.c[a], p1 = s.c[3 + a], p2 = s.c[6 + a], p3 = s.c[9 + a];
    if (MU == 0) {         // A psi_- = (-i p3, -i p2)
      h0[a] = SG > 0 ? p0 + times_i(p3) : p0 - times_i(p3);
      h1[a] = SG > 0 ? p1 + times_i(p2) : p1 - times_i(p2);
    } else if (MU == 1) {  // A psi_- = (-p3, p2)
      h0[a] = SG > 0 ? p0 + p3 : p0 - p3;
      h1[a] = SG > 0 ? p1 - p2 : p1 + p2;
    } else if (MU == 2) {  // A psi_- = (-i p2, i p3)
      h0[a] = SG > 0 ? p0 + times_i(p2) : p0 - times_i(p2);
      h1[a] = SG > 0 ? p1 - times_i(p3) : p1 + times_i(p3);
    } else {               // A psi_- = (p2, p3)
      h0[a] = SG > 0 ? p0 - p2 : p0 + p2;
      h1[a] = SG > 0 ? p1 - p3 : p1 + p3;
    }
  }
}

// acc += (chi, -sg A^+ chi)
template <typename T, int MU, int SG>
__device__ __forceinline__ void reconstruct_add(Spinor<T>& acc, const cplx<T> c0[3], const cplx<T> c1[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    acc.c[a] = acc.c[a] + c0[a];
    acc.c[3 + a] = acc.c[3 + a] + c1[a];
    if (MU == 0) {         // A^+ chi = (i c1, i c0)
      acc.c[6 + a] = SG > 0 ? acc.c[6 + a] - times_i(c1[a]) : acc.c[6 + a] + times_i(c1[a]);
      acc.c[9 + a] = SG > 0 ? acc.c[9 + a] - times_i(c0[a]) : acc.c[9 + a] + times_i(c0[a]);
    } else if (MU == 1) {  // A^+ chi = (c1, -c0)
      acc.c[6 + a] = SG > 0 ? acc.c[6 + a] - c1[a] : acc.c[6 + a] + c1[a];
      acc.c[9 + a] = SG > 0 ? acc.c[9 + a] + c0[a] : acc.c[9 + a] - c0[a];
    } else if (MU == 2) {  // A^+ chi = (i c0, -i c1)
      acc.c[6 + a] = SG > 0 ? acc.c[6 + a] - times_i(c0[a]) : acc.c[6 + a] + times_i(c0[a]);
      acc.c[9 + a] = SG > 0 ? acc.c[9 + a] + times_i(c1[a]) : acc.c[9 + a] - times_i(c1[a]);
    } else {               // A^+ chi = (c0, c1)
      acc.c[6 + a] = SG > 0 ? acc.c[6 + a] - c0[a] : acc.c[6 + a] + c0[a];
      acc.c[9 + a] = SG > 0 ? acc.c[9 + a] - c1[a] : acc.c[9 + a] + c1[a];
    }
  }
}

// acc += f (chi, -sg A^+ chi) with a runtime factor f (the +-1 of a hop across
// an antiperiodic boundary): the factor rides on the accumulating FMAs.
template <typename T>
__device__ __forceinline__ void fmac(cplx<T>& acc, T f, const cplx<T>& c) {
  acc = cmake(fma(f, c.re, acc.re), fma(f, c.im, acc.im));
}
template <typename T>
__device__ __forceinline__ void fmac_i(cplx<T>& acc, T f, const cplx<T>& c) {  // acc += f i c
  acc = cmake(fma(-f, c.im, acc.re), fma(f, c.re, acc.im));
}
template <typename T, int MU, int SG>
__device__ __forceinline__ void reconstruct_add(Spinor<T>& acc, const cplx<T> c0[3], const cplx<T> c1[3],
                                                T f) {
  const T m = SG > 0 ? -f : f;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    fmac(acc.c[a], f, c0[a]);
    fmac(acc.c[3 + a], f, c1[a]);
    if (MU == 0) {         // A^+ chi = (i c1, i c0)
      fmac_i(acc.c[6 + a], m, c1[a]);
      fmac_i(acc.c[9 + a], m, c0[a]);
    } else if (MU == 1) {  // A^+ chi = (c1, -c0)
      fmac(acc.c[6 + a], m, c1[a]);
      fmac(acc.c[9 + a], -m, c0[a]);
    } else if (MU == 2) {  // A^+ chi = (i c0, -i c1)
      fmac_i(acc.c[6 + a], m, c0[a]);
      fmac_i(acc.c[9 + a], -m, c1[a]);
    } else {               // A^+ chi = (c0, c1)
      fmac(acc.c[6 + a], m, c0[a]);
      fmac(acc.c[9 + a], m, c1[a]);
    }
  }
}

// chi = U h (DAG = false) or U^+ h (DAG = true), for both half-spinor rows.
template <typename T, bool DAG>
__device__ __forceinline__ void su3_mul(const Link<T>& U, const cplx<T> h0[3], const cplx<T> h1[3],
                                        cplx<T> c0[3], cplx<T> c1[3]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    c0[a] = cmake<T>(0, 0);
    c1[a] = cmake<T>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; b++) {
      if (DAG) {
        cmac_conj(c0[a], U.u[3 * b + a], h0[b]);
        cmac_conj(c1[a], U.u[3 * b + a], h1[b]);
      } else {
        cmac(c0[a], U.u[3 * a + b], h0[b]);
        cmac(c1[a], U.u[3 * a + b], h1[b]);
      }
    }
  }
}

}  // namespace dwf
