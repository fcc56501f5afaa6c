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

// Position of slice s inside a 4D site's Ls consecutive 5D entries: even
// slices first, then odd ones, so that threads owning the slice pairs
// (2t, 2t+1) read and write contiguous memory for each of the two slices.
__host__ __device__ __forceinline__ int slice_pos(int s, int Ls) {
  return (s & 1) ? ((Ls + 1) >> 1) + (s >> 1) : (s >> 1);
}
__host__ __device__ __forceinline__ int site5(int h, int s, int Ls) { return h * Ls + slice_pos(s, Ls); }

// ---------------------------------------------------------------------------
// Storage policies.  load/store one 5D site (index n) of one half-field.
// ---------------------------------------------------------------------------
struct Store64 {
  using T = double;
  static constexpr int kPrec = P64;
  static constexpr int kChunks = 12;     // 16-byte chunks per 5D site
  static constexpr bool kScaled = false;
  __device__ static void load(const void* base, int n, int N5, Spinor<double>& o) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 v = __ldg(b + (size_t)k * N5 + n);
      o.c[k] = cmake(v.x, v.y);
    }
  }
  // spins of one chirality only (chir 0: spins 0,1; chir 1: spins 2,3)
  __device__ static void load_chir(const void* base, int n, int N5, int chir, Spinor<double>& o) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      double2 v = __ldg(b + (size_t)(k + 6 * chir) * N5 + n);
      o.c[k + 6 * chir] = cmake(v.x, v.y);
    }
  }
  // the 6 complex components of one chirality into o[0..5]
  __device__ static void load_half(const void* base, int n, int N5, int chir, cplx<double>* o) {
    const double2* b = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      double2 v = __ldg(b + (size_t)(k + 6 * chir) * N5 + n);
      o[k] = cmake(v.x, v.y);
    }
  }
  __device__ static void store(void* base, int n, int N5, const Spinor<double>& o) {
    double2* b = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) b[(size_t)k * N5 + n] = make_double2(o.c[k].re, o.c[k].im);
  }
};

struct Store32 {
  using T = float;
  static constexpr int kPrec = P32;
  static constexpr int kChunks = 6;
  static constexpr bool kScaled = false;
  __device__ static void load(const void* base, int n, int N5, Spinor<float>& o) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = __ldg(b + (size_t)k * N5 + n);
      o.c[2 * k] = cmake(v.x, v.y);
      o.c[2 * k + 1] = cmake(v.z, v.w);
    }
  }
  __device__ static void load_chir(const void* base, int n, int N5, int chir, Spinor<float>& o) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = __ldg(b + (size_t)(k + 3 * chir) * N5 + n);
      o.c[2 * k + 6 * chir] = cmake(v.x, v.y);
      o.c[2 * k + 1 + 6 * chir] = cmake(v.z, v.w);
    }
  }
  __device__ static void load_half(const void* base, int n, int N5, int chir, cplx<float>* o) {
    const float4* b = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = __ldg(b + (size_t)(k + 3 * chir) * N5 + n);
      o[2 * k] = cmake(v.x, v.y);
      o[2 * k + 1] = cmake(v.z, v.w);
    }
  }
  __device__ static void store(void* base, int n, int N5, const Spinor<float>& o) {
    float4* b = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++)
      b[(size_t)k * N5 + n] = make_float4(o.c[2 * k].re, o.c[2 * k].im, o.c[2 * k + 1].re,
                                          o.c[2 * k + 1].im);
  }
};

// 16-bit storage: 3 chunks of 8 values (uint4) per site, then one FP32 scale per
// site after the 3 * N5 chunks.  value = stored * scale, scale = max |real|.
template <bool BF>
struct Store16 {
  using T = float;
  static constexpr int kPrec = BF ? PB16 : P16;
  static constexpr int kChunks = 3;
  static constexpr bool kScaled = true;
  __device__ static float to_f(uint16_t v) {
    if (BF) return __bfloat162float(__ushort_as_bfloat16(v));
    return __half2float(__ushort_as_half(v));
  }
  __device__ static uint16_t from_f(float f) {
    if (BF) return __bfloat16_as_ushort(__float2bfloat16_rn(f));
    return __half_as_ushort(__float2half_rn(f));
  }
  __device__ static void load(const void* base, int n, int N5, Spinor<float>& o) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    const float sc = __ldg(reinterpret_cast<const float*>(b + (size_t)3 * N5) + n);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 v = __ldg(b + (size_t)k * N5 + n);
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        o.c[4 * k + q] = cmake(sc * to_f((uint16_t)(w[q] & 0xffffu)), sc * to_f((uint16_t)(w[q] >> 16)));
      }
    }
  }
  __device__ static void load_chir(const void* base, int n, int N5, int chir, Spinor<float>& o) {
    load(base, n, N5, o);
  }
  // chirality 0: complex 0..5 = chunk 0 (0..3) + low half of chunk 1 (4, 5);
  // chirality 1: complex 6..11 = high half of chunk 1 (6, 7) + chunk 2 (8..11).
  __device__ static void load_half(const void* base, int n, int N5, int chir, cplx<float>* o) {
    const uint4* b = reinterpret_cast<const uint4*>(base);
    const float sc = __ldg(reinterpret_cast<const float*>(b + (size_t)3 * N5) + n);
    const uint4 v1 = __ldg(b + (size_t)N5 + n);
    const uint4 v0 = __ldg(b + (size_t)(chir ? 2 : 0) * N5 + n);
    uint32_t w[6];
    if (chir == 0) {
      w[0] = v0.x; w[1] = v0.y; w[2] = v0.z; w[3] = v0.w; w[4] = v1.x; w[5] = v1.y;
    } else {
      w[0] = v1.z; w[1] = v1.w; w[2] = v0.x; w[3] = v0.y; w[4] = v0.z; w[5] = v0.w;
    }
#pragma unroll
    for (int q = 0; q < 6; q++)
      o[q] = cmake(sc * to_f((uint16_t)(w[q] & 0xffffu)), sc * to_f((uint16_t)(w[q] >> 16)));
  }
  // Per-site scale from the largest |component|.  Below the smallest normal float
  // (subnormal or zero, e.g. the far tail of a point-source solve) 1/max would
  // overflow to inf: such a site keeps scale 1, and its components, far below
  // 16-bit resolution, store as zero.  A NaN component still stores as NaN.
  __device__ static float scale_of(float mx) { return mx >= 1.17549435e-38f ? mx : 1.f; }
  // o <- what store() followed by load() gives back, computed in registers (a
  // kernel must not re-read through __ldg what it wrote itself).
  __device__ static void quantize(Spinor<float>& o) {
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) mx = fmaxf(mx, fmaxf(fabsf(o.c[k].re), fabsf(o.c[k].im)));
    const float sc = scale_of(mx);
    const float inv = 1.f / sc;
#pragma unroll
    for (int k = 0; k < 12; k++)
      o.c[k] = cmake(sc * to_f(from_f(o.c[k].re * inv)), sc * to_f(from_f(o.c[k].im * inv)));
  }
  __device__ static void store(void* base, int n, int N5, const Spinor<float>& o) {
    uint4* b = reinterpret_cast<uint4*>(base);
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) mx = fmaxf(mx, fmaxf(fabsf(o.c[k].re), fabsf(o.c[k].im)));
    const float sc = scale_of(mx);
    const float inv = 1.f / sc;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        w[q] = (uint32_t)from_f(o.c[4 * k + q].re * inv) | ((uint32_t)from_f(o.c[4 * k + q].im * inv) << 16);
      }
      b[(size_t)k * N5 + n] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    reinterpret_cast<float*>(b + (size_t)3 * N5)[n] = sc;
  }
};

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
