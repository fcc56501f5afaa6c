// dwf_hop.cu -- the hopping pass and the site-local contraction (sm_103a).
//
// One thread per 5D site (h, s); a CTA owns all Ls slices of block_sites 4D
// sites (blockDim = (Ls, block_sites)), so the 5th-dimension contractions of
// I^-1, K = B I^-1 and B^T (dense real Ls x Ls per chirality, Sec. 3
// Eq. redblack with Eq. mobius1) run from shared memory inside the CTA.  The
// gauge link of a 4D site is read once per CTA-warp and broadcast to its Ls
// threads; neighbour spinors are read with the 5th dimension contiguous.
#include "dwf_fields.cuh"

namespace dwf {

namespace {

constexpr int kSitePad = 4;  // shared-memory padding per 4D site (bank spread)

template <typename T>
__device__ __forceinline__ T sq(const Spinor<T>& a) {
  T r = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) r += a.c[k].re * a.c[k].re + a.c[k].im * a.c[k].im;
  return r;
}

template <typename T>
struct HopArgs {
  void* out;
  const void* v;
  const void* w;
  size_t stride;
  const void* gauge_p;  // links of parity-p sites
  const void* gauge_q;  // links of parity-(1-p) sites
  const T* pre_diag;
  const T* pre_off;
  const T* post;
  const T* locm;
  T c_hop, c_loc;
  int p;
  Reduce red;
  size_t cstride;
  const int* active;
};

template <class SP, class GP, int PRE, int MU, int DIR>
__device__ __forceinline__ void hop_term(const Geom& g, const Coords& c, int h, int s, int sp,
                                         int sn, const typename SP::T* bd,
                                         const typename SP::T* bo, const void* v,
                                         const void* gp, const void* gq,
                                         Spinor<typename SP::T>& acc) {
  using T = typename SP::T;
  int sign;
  const int hn = neighbour(g, c, MU, DIR, sign);
  Spinor<T> in;
  SP::load(v, site5(hn, s, g.Ls), g.N5, in);
  if (PRE == PRE_B) {
    Spinor<T> a, b;
    SP::load_chir(v, site5(hn, sp, g.Ls), g.N5, 0, a);
    SP::load_chir(v, site5(hn, sn, g.Ls), g.N5, 1, b);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      in.c[k] = cmake(fma(bd[0], in.c[k].re, bo[0] * a.c[k].re), fma(bd[0], in.c[k].im, bo[0] * a.c[k].im));
      in.c[k + 6] = cmake(fma(bd[1], in.c[k + 6].re, bo[1] * b.c[k + 6].re),
                          fma(bd[1], in.c[k + 6].im, bo[1] * b.c[k + 6].im));
    }
  } else if (PRE == PRE_G5) {
#pragma unroll
    for (int k = 6; k < 12; k++) in.c[k] = cmake(-in.c[k].re, -in.c[k].im);
  }
  cplx<T> h0[3], h1[3], c0[3], c1[3];
  project<T, MU, DIR>(in, h0, h1);
  if (sign < 0) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      h0[a] = cmake(-h0[a].re, -h0[a].im);
      h1[a] = cmake(-h1[a].re, -h1[a].im);
    }
  }
  Link<T> U;
  if (DIR > 0) {
    GP::load(gp, h, MU, U);
    su3_mul<T, false>(U, h0, h1, c0, c1);
  } else {
    GP::load(gq, hn, MU, U);
    su3_mul<T, true>(U, h0, h1, c0, c1);
  }
  reconstruct_add<T, MU, DIR>(acc, c0, c1);
}

// res += sum_{s'} M_chir[s][s'] buf[j][s'] with smat[chir][s'][s] = M_chir[s][s'].
template <typename T>
__device__ __forceinline__ void contract(const T* smat, const T* sbuf_site, int Ls, int s,
                                         Spinor<T>& res) {
  const int LL = Ls * Ls;
  for (int q = 0; q < Ls; q++) {
    const T m0 = smat[q * Ls + s];
    const T m1 = smat[LL + q * Ls + s];
    const T* e = sbuf_site + q * 24;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      res.c[k].re = fma(m0, e[2 * k], res.c[k].re);
      res.c[k].im = fma(m0, e[2 * k + 1], res.c[k].im);
      res.c[k + 6].re = fma(m1, e[2 * k + 12], res.c[k + 6].re);
      res.c[k + 6].im = fma(m1, e[2 * k + 13], res.c[k + 6].im);
    }
  }
}

template <typename T>
__device__ __forceinline__ void put_site(T* slot, const Spinor<T>& a) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    slot[2 * k] = a.c[k].re;
    slot[2 * k + 1] = a.c[k].im;
  }
}

template <typename T>
__device__ void load_matrix_T(T* dst, const T* src, int Ls, int tid, int nth) {
  // dst[chir][col][row] = src[chir][row][col]
  const int LL = Ls * Ls;
  for (int i = tid; i < 2 * LL; i += nth) {
    const int ch = i / LL, r = i % LL, row = r / Ls, col = r % Ls;
    dst[ch * LL + col * Ls + row] = src[i];
  }
}

template <class SP, int PRE, bool POST, int LOC, bool G5, bool NORM>
__global__ void __launch_bounds__(256) hop_kernel(const Geom g, const HopArgs<typename SP::T> a) {
  using T = typename SP::T;
  using GP = typename GaugeOf<SP>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smat = reinterpret_cast<T*>(smem_raw);
  const int Ls = g.Ls, LL = Ls * Ls;
  T* smat_loc = smat + 2 * LL;
  T* sbuf = smat + 4 * LL;
  const int SST = Ls * 24 + kSitePad;
  const int s = threadIdx.x, j = threadIdx.y;
  const int tid = j * Ls + s, nth = Ls * blockDim.y;
  const int h = blockIdx.x * blockDim.y + j;
  const bool active = h < g.Vh;
  const int rhs = blockIdx.z;
  if (a.active && !a.active[rhs]) return;
  const size_t co = (size_t)rhs * a.cstride;

  if (POST) load_matrix_T(smat, a.post + co, Ls, tid, nth);
  if (LOC == LOC_DENSE) load_matrix_T(smat_loc, a.locm + co, Ls, tid, nth);
  if (POST || LOC == LOC_DENSE) __syncthreads();

  const char* vb = reinterpret_cast<const char*>(a.v) + rhs * a.stride;
  Spinor<T> acc;
#pragma unroll
  for (int k = 0; k < 12; k++) acc.c[k] = cmake<T>(0, 0);

  if (active) {
    const Coords c = site_coords(g, h, a.p);
    T bd[2] = {0, 0}, bo[2] = {0, 0};
    if (PRE == PRE_B) {
      bd[0] = a.pre_diag[co + s];
      bd[1] = a.pre_diag[co + Ls + s];
      bo[0] = a.pre_off[co + s];
      bo[1] = a.pre_off[co + Ls + s];
    }
    const int sp = s == 0 ? Ls - 1 : s - 1;
    const int sn = s == Ls - 1 ? 0 : s + 1;
    hop_term<SP, GP, PRE, 0, +1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 0, -1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 1, +1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 1, -1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 2, +1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 2, -1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 3, +1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
    hop_term<SP, GP, PRE, 3, -1>(g, c, h, s, sp, sn, bd, bo, vb, a.gauge_p, a.gauge_q, acc);
  }

  Spinor<T> res;
  if (POST) {
    put_site(sbuf + j * SST + s * 24, acc);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 12; k++) res.c[k] = cmake<T>(0, 0);
    contract(smat, sbuf + j * SST, Ls, s, res);
  } else {
    res = acc;
  }
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const T f = (G5 && k >= 6) ? -a.c_hop : a.c_hop;
    res.c[k] = cmake(f * res.c[k].re, f * res.c[k].im);
  }
  const size_t off = rhs * a.stride;
  if (LOC == LOC_ID) {
    if (active) {
      Spinor<T> w;
      SP::load(reinterpret_cast<const char*>(a.w) + off, site5(h, s, Ls), g.N5, w);
#pragma unroll
      for (int k = 0; k < 12; k++)
        res.c[k] = cmake(fma(a.c_loc, w.c[k].re, res.c[k].re), fma(a.c_loc, w.c[k].im, res.c[k].im));
    }
  } else if (LOC == LOC_DENSE) {
    Spinor<T> w;
#pragma unroll
    for (int k = 0; k < 12; k++) w.c[k] = cmake<T>(0, 0);
    if (active) SP::load(reinterpret_cast<const char*>(a.w) + off, site5(h, s, Ls), g.N5, w);
    if (POST) __syncthreads();  // everyone is done reading sbuf
    put_site(sbuf + j * SST + s * 24, w);
    __syncthreads();
    Spinor<T> lw;
#pragma unroll
    for (int k = 0; k < 12; k++) lw.c[k] = cmake<T>(0, 0);
    contract(smat_loc, sbuf + j * SST, Ls, s, lw);
#pragma unroll
    for (int k = 0; k < 12; k++)
      res.c[k] = cmake(fma(a.c_loc, lw.c[k].re, res.c[k].re), fma(a.c_loc, lw.c[k].im, res.c[k].im));
  }
  if (active) SP::store(reinterpret_cast<char*>(a.out) + off, site5(h, s, Ls), g.N5, res);
  if (NORM) {
    double v = active ? (double)sq(res) : 0.0;
    block_sum_to(v, a.red, rhs, gridDim.x, blockIdx.x);
  }
}

template <class SP>
__global__ void __launch_bounds__(256) local_kernel(const Geom g, void* out, const void* in,
                                                    size_t stride, const typename SP::T* m,
                                                    typename SP::T c, int g5in, Reduce red,
                                                    int do_norm, size_t cstride,
                                                    const int* rhs_on) {
  using T = typename SP::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smat = reinterpret_cast<T*>(smem_raw);
  const int Ls = g.Ls, LL = Ls * Ls;
  T* sbuf = smat + 2 * LL;
  const int SST = Ls * 24 + kSitePad;
  const int s = threadIdx.x, j = threadIdx.y;
  const int tid = j * Ls + s, nth = Ls * blockDim.y;
  const int h = blockIdx.x * blockDim.y + j;
  const bool active = h < g.Vh;
  const int rhs = blockIdx.z;
  if (rhs_on && !rhs_on[rhs]) return;
  const size_t off = rhs * stride;
  load_matrix_T(smat, m + (size_t)rhs * cstride, Ls, tid, nth);
  Spinor<T> x;
#pragma unroll
  for (int k = 0; k < 12; k++) x.c[k] = cmake<T>(0, 0);
  if (active) SP::load(reinterpret_cast<const char*>(in) + off, site5(h, s, Ls), g.N5, x);
  if (g5in) {
#pragma unroll
    for (int k = 6; k < 12; k++) x.c[k] = cmake(-x.c[k].re, -x.c[k].im);
  }
  put_site(sbuf + j * SST + s * 24, x);
  __syncthreads();
  Spinor<T> res;
#pragma unroll
  for (int k = 0; k < 12; k++) res.c[k] = cmake<T>(0, 0);
  contract(smat, sbuf + j * SST, Ls, s, res);
#pragma unroll
  for (int k = 0; k < 12; k++) res.c[k] = cmake(c * res.c[k].re, c * res.c[k].im);
  if (active) SP::store(reinterpret_cast<char*>(out) + off, site5(h, s, Ls), g.N5, res);
  if (do_norm) {
    double v = active ? (double)sq(res) : 0.0;
    block_sum_to(v, red, rhs, gridDim.x, blockIdx.x);
  }
}

int default_block_sites(int prec, int Ls) {
  const int target = prec == P64 ? 128 : 256;
  int S = target / Ls;
  if (S < 1) S = 1;
  return S;
}

size_t hop_smem(int prec, int Ls, int S) {
  const size_t ts = prec == P64 ? 8 : 4;
  return ts * (4 * (size_t)Ls * Ls + (size_t)S * (Ls * 24 + kSitePad));
}

template <class SP, int PRE, bool POST, int LOC, bool G5, bool NORM>
cudaError_t run_hop(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  HopArgs<T> a;
  a.out = L.out;
  a.v = L.v;
  a.w = L.w;
  a.stride = L.stride;
  const char* gb = reinterpret_cast<const char*>(L.gauge);
  a.gauge_p = gb + (size_t)L.p * L.gauge_parity_bytes;
  a.gauge_q = gb + (size_t)(1 - L.p) * L.gauge_parity_bytes;
  a.pre_diag = reinterpret_cast<const T*>(L.pre_diag);
  a.pre_off = reinterpret_cast<const T*>(L.pre_off);
  a.post = reinterpret_cast<const T*>(L.post);
  a.locm = reinterpret_cast<const T*>(L.locm);
  a.c_hop = (T)L.c_hop;
  a.c_loc = (T)L.c_loc;
  a.p = L.p;
  a.cstride = L.cstride;
  a.active = L.active;
  if (L.red) a.red = *L.red;
  const int S = L.block_sites > 0 ? L.block_sites : default_block_sites(L.prec, g.Ls);
  const size_t smem = hop_smem(L.prec, g.Ls, S);
  auto k = hop_kernel<SP, PRE, POST, LOC, G5, NORM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 block(g.Ls, S, 1);
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  k<<<grid, block, smem, st>>>(g, a);
  return cudaGetLastError();
}

template <class SP>
cudaError_t dispatch_hop(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  const bool post = L.post != nullptr;
  const bool norm = L.red != nullptr;
  // The combinations the library uses (see dwf_api.cu):
  //  D_bb pass A        PRE_B,    post K,     no local
  //  D_bb pass B        PRE_NONE, post I^-1,  LOC_ID, (norm)
  //  D_bb^+ pass A      PRE_NONE, post K^T,   no local
  //  D_bb^+ pass B      PRE_NONE, post B^T,   LOC_ID, gamma5 out, (norm)
  //  D_alpha parity     PRE_B,    no post,    LOC_DENSE (I)
  //  Schur rhs/recon    PRE_NONE / PRE_B, post I^-1, LOC_DENSE (I^-1)
  //  force eta2         PRE_G5,   post K^T,   gamma5 out
  if (L.pre == PRE_B && post && L.loc == LOC_NONE && !L.g5out && !norm)
    return run_hop<SP, PRE_B, true, LOC_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && post && L.loc == LOC_ID && !L.g5out)
    return norm ? run_hop<SP, PRE_NONE, true, LOC_ID, false, true>(g, L, st)
                : run_hop<SP, PRE_NONE, true, LOC_ID, false, false>(g, L, st);
  if (L.pre == PRE_NONE && post && L.loc == LOC_NONE && !L.g5out && !norm)
    return run_hop<SP, PRE_NONE, true, LOC_NONE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && post && L.loc == LOC_ID && L.g5out)
    return norm ? run_hop<SP, PRE_NONE, true, LOC_ID, true, true>(g, L, st)
                : run_hop<SP, PRE_NONE, true, LOC_ID, true, false>(g, L, st);
  if (L.pre == PRE_B && !post && L.loc == LOC_DENSE && !L.g5out && !norm)
    return run_hop<SP, PRE_B, false, LOC_DENSE, false, false>(g, L, st);
  if (L.pre == PRE_NONE && post && L.loc == LOC_DENSE && !L.g5out && !norm)
    return run_hop<SP, PRE_NONE, true, LOC_DENSE, false, false>(g, L, st);
  if (L.pre == PRE_B && post && L.loc == LOC_DENSE && !L.g5out && !norm)
    return run_hop<SP, PRE_B, true, LOC_DENSE, false, false>(g, L, st);
  if (L.pre == PRE_B && post && L.loc == LOC_NONE && !L.g5out && !norm)
    return run_hop<SP, PRE_B, true, LOC_NONE, false, false>(g, L, st);
  if (L.pre == PRE_G5 && post && L.loc == LOC_NONE && L.g5out && !norm)
    return run_hop<SP, PRE_G5, true, LOC_NONE, true, false>(g, L, st);
  return cudaErrorInvalidValue;
}

template <class SP>
cudaError_t run_local(const Geom& g, const LocalLaunch& L, cudaStream_t st) {
  using T = typename SP::T;
  const int S = default_block_sites(L.prec, g.Ls);
  const size_t ts = sizeof(T);
  const size_t smem = ts * (2 * (size_t)g.Ls * g.Ls + (size_t)S * (g.Ls * 24 + kSitePad));
  auto k = local_kernel<SP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  Reduce red{};
  if (L.red) red = *L.red;
  dim3 block(g.Ls, S, 1);
  dim3 grid((g.Vh + S - 1) / S, 1, L.nrhs);
  k<<<grid, block, smem, st>>>(g, L.out, L.in, L.stride, reinterpret_cast<const T*>(L.m), (T)L.c,
                               L.g5in, red, L.red != nullptr, L.cstride, L.active);
  return cudaGetLastError();
}

}  // namespace

int hop_grid_blocks(const Geom& g, int prec, int block_sites) {
  const int S = block_sites > 0 ? block_sites : default_block_sites(prec, g.Ls);
  return (g.Vh + S - 1) / S;
}

int g_disable_tuned = 0;

cudaError_t launch_hop(const Geom& g, const HopLaunch& L, cudaStream_t st) {
  if (!g_disable_tuned) {
    cudaError_t e = cudaErrorNotSupported;
    switch (L.prec) {
      case P64: e = launch_hop2_f64(g, L, st); break;
      case P32: e = launch_hop2_f32(g, L, st); break;
      case P16: e = launch_hop2_f16(g, L, st); break;
      case PB16: e = launch_hop2_bf16(g, L, st); break;
    }
    if (e != cudaErrorNotSupported) return e;
  }
  // block_sites is the tuned kernels' tile: the generic kernel takes its own default
  HopLaunch G = L;
  G.block_sites = 0;
  switch (G.prec) {
    case P64: return dispatch_hop<Store64>(g, G, st);
    case P32: return dispatch_hop<Store32>(g, G, st);
    case P16: return dispatch_hop<Store16<false>>(g, G, st);
    case PB16: return dispatch_hop<Store16<true>>(g, G, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rupdate(const Geom& g, const RUpdateLaunch& L, cudaStream_t st) {
  if (g_disable_tuned) return cudaErrorNotSupported;
  switch (L.prec) {
    case P64: return launch_hop2_f64_rupdate(g, L, st);
    case P32: return launch_hop2_f32_rupdate(g, L, st);
    case P16: return launch_hop2_f16_rupdate(g, L, st);
    case PB16: return launch_hop2_bf16_rupdate(g, L, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_local(const Geom& g, const LocalLaunch& L, cudaStream_t st) {
  if (!g_disable_tuned) {
    cudaError_t e = cudaErrorNotSupported;
    switch (L.prec) {
      case P64: e = launch_hop2_f64_local(g, L, st); break;
      case P32: e = launch_hop2_f32_local(g, L, st); break;
      case P16: e = launch_hop2_f16_local(g, L, st); break;
      case PB16: e = launch_hop2_bf16_local(g, L, st); break;
    }
    if (e != cudaErrorNotSupported) return e;
  }
  switch (L.prec) {
    case P64: return run_local<Store64>(g, L, st);
    case P32: return run_local<Store32>(g, L, st);
    case P16: return run_local<Store16<false>>(g, L, st);
    case PB16: return run_local<Store16<true>>(g, L, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dwf
