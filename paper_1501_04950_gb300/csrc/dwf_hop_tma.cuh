// dwf_hop_tma.cuh -- the tuned hopping pass with neighbour staging by the Tensor
// Memory Accelerator (sm_103a): a producer warp copies, for each of the 8 hops,
// the slice-pair block of every neighbour site of the CTA (one 2D tensor copy per
// site: the spinor component rows x the site's Ls/2 slice pairs) and its link
// (1D bulk copy) into a ring of NST shared-memory stages; four consumer warps
// compute the hop of stage d while the copies of the following hops are in
// flight.  The data lands in shared memory, not registers, so several hops per
// CTA are in flight at once; pass A's B pre-multiplication reads the neighbour
// slice pairs of the other threads from the same staged block.
//
// Synchronisation: per stage a "full" mbarrier (one producer arrival with the
// expected byte count; the copies complete the transaction) and an "empty"
// mbarrier (every consumer thread arrives after reading).  Every wait is
// bounded by a clock budget: when it runs out the thread sets *err (the host
// reports DWF_ERR_TIMEOUT), skips the stage and carries on, so no wait can hang.
#pragma once

#include <cuda.h>

namespace dwf {
namespace hop2 {

constexpr int kTmaConsumers = 128;
constexpr int kTmaThreads = kTmaConsumers + 32;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Bounded wait for the completion of phase `parity`; false when the clock
// budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long budget) {
  const uint32_t addr = smem_u32(bar);
  long long t0 = 0;
  for (int i = 0;; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    const long long now = clock64();
    if (i == 0) t0 = now;
    else if (now - t0 > budget) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Staged site block: the tensor box ([kRows][Ls/2] 16-byte units of kWpp/4 ...),
// then (16-bit) the slice-pair scales, then the link; each part 16-byte aligned,
// the block padded to 128 bytes (tensor copies land on 128-byte boundaries).
template <class SP, int LS>
struct Stage {
  static constexpr int HALF = LS / 2;
  static constexpr int kRows = SP::kPrec == P64 ? 12 : (SP::kScaled ? 6 : 12);
  static constexpr int kWpp = SP::kPrec == P64 ? 8 : 4;  // 32-bit words per pair and row
  static constexpr int kBoxBytes = kRows * HALF * kWpp * 4;
  static constexpr int kScaleOff = kBoxBytes;
  static constexpr int kScaleBytes = SP::kScaled ? (HALF * 8 + 15) / 16 * 16 : 0;
  static constexpr int kLinkOff = kScaleOff + kScaleBytes;
  static constexpr int kLinkBytes = GaugeOf<SP>::type::kLinkBytes;
  static constexpr int kBytes = (kLinkOff + kLinkBytes + 127) / 128 * 128;
  static constexpr int kTx = kBoxBytes + kScaleBytes + kLinkBytes;  // bytes per site and hop
};

// Staged-block readers (pair t, components c0 .. c0 + 5, unscaled).
template <class SP, int LS>
struct StageIO;
template <int LS>
struct StageIO<Store32, LS> {
  using V = float2;
  static __device__ __forceinline__ void load6(const unsigned char* sb, int t, int c0, V* re, V* im) {
    const float4* b = reinterpret_cast<const float4*>(sb) + c0 * (LS / 2) + t;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 v = b[k * (LS / 2)];
      re[k] = make_float2(v.x, v.y);
      im[k] = make_float2(v.z, v.w);
    }
  }
  static __device__ __forceinline__ V scale(const unsigned char*, int) { return make_float2(1.f, 1.f); }
  static __device__ __forceinline__ void link(const unsigned char* p, Link<float>& U) {
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
};
template <int LS>
struct StageIO<Store64, LS> {
  using V = double2;
  static __device__ __forceinline__ void load6(const unsigned char* sb, int t, int c0, V* re, V* im) {
    const double2* b = reinterpret_cast<const double2*>(sb) + (c0 * (LS / 2) + t) * 2;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      re[k] = b[k * LS];
      im[k] = b[k * LS + 1];
    }
  }
  static __device__ __forceinline__ V scale(const unsigned char*, int) { return make_double2(1.0, 1.0); }
  static __device__ __forceinline__ void link(const unsigned char* p, Link<double>& U) {
    const double2* b = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const double2 v = b[k];
      U.u[k] = cmake(v.x, v.y);
    }
  }
};
template <bool BF, int LS>
struct StageIO<Store16<BF>, LS> {
  using V = float2;
  using S = Store16<BF>;
  static __device__ __forceinline__ void load6(const unsigned char* sb, int t, int c0, V* re, V* im) {
    const uint4* b = reinterpret_cast<const uint4*>(sb) + (c0 >> 1) * (LS / 2) + t;
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const uint4 v = b[j * (LS / 2)];
      re[2 * j] = S::to_f2(v.x);
      im[2 * j] = S::to_f2(v.y);
      re[2 * j + 1] = S::to_f2(v.z);
      im[2 * j + 1] = S::to_f2(v.w);
    }
  }
  static __device__ __forceinline__ V scale(const unsigned char* sb, int t) {
    return reinterpret_cast<const float2*>(sb + Stage<S, LS>::kScaleOff)[t];
  }
  static __device__ __forceinline__ void link(const unsigned char* p, Link<float>& U) {
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
    for (int k = 0; k < 9; k++) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
      U.u[k] = cmake(f.x, f.y);
    }
  }
};

// One hop from a staged neighbour block sb (pair t of the site); the link of the
// hop is the staged one.
template <class SP, int LS, int PRE, int MU, int DIR>
__device__ __forceinline__ void hop_staged(const unsigned char* sb, bool neg, int t,
                                           const typename SP::T (&bd)[2][2],
                                           const typename SP::T (&bo)[2][2],
                                           SpinP<typename Pr<typename SP::T>::V>& acc) {
  using T = typename SP::T;
  using A = Pr<T>;
  using V = typename A::V;
  using IO = StageIO<SP, LS>;
  constexpr int HALF = LS / 2;
  HalfP<V> P, M;
  IO::load6(sb, t, 0, P.re, P.im);
  IO::load6(sb, t, 6, M.re, M.im);
  V f = A::dup(neg ? (T)-1 : (T)1);
  if constexpr (PRE == PRE_B) {
    const int tp = t == 0 ? HALF - 1 : t - 1, tn = t + 1 == HALF ? 0 : t + 1;
    HalfP<V> Pb, Ma;
    IO::load6(sb, tp, 0, Pb.re, Pb.im);
    IO::load6(sb, tn, 6, Ma.re, Ma.im);
    T a1 = bd[0][0], a2 = bo[0][0], a3 = bd[0][1], a4 = bo[0][1];
    T b1 = bd[1][0], b2 = bo[1][0], b3 = bd[1][1], b4 = bo[1][1];
    if constexpr (SP::kScaled) {
      const V sc = IO::scale(sb, t), sb_ = IO::scale(sb, tp), sa = IO::scale(sb, tn);
      a1 *= sc.x; a2 *= sb_.y; a3 *= sc.y; a4 *= sc.x;
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
    f = A::mul(f, IO::scale(sb, t));
  }
  Link<T> U;
  IO::link(sb + Stage<SP, LS>::kLinkOff, U);
  project_mul_acc<SP, MU, DIR>(P, M, U, f, acc);
}

template <class SP, int LS, int PRE, int POST, int LOC, bool G5, bool NORM, int NST, int MINB>
__global__ void __launch_bounds__(kTmaThreads, MINB)
    hop_tma_kernel(const Geom g, const Args<typename SP::T> a, const __grid_constant__ CUtensorMap tmap,
                   long long budget, int skip_hop) {
  using T = typename SP::T;
  using V = typename Pr<T>::V;
  using ST = Stage<SP, LS>;
  constexpr int HALF = LS / 2;
  constexpr int S = kTmaConsumers / HALF;
  constexpr int SST = site_stride(LS);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + NST;
  T* coef = reinterpret_cast<T*>(smem_raw + 128);
  unsigned char* stages = smem_raw + 128 + (chain_block(LS) * (int)sizeof(T) + 127) / 128 * 128;
  const int tid = threadIdx.x;
  const bool producer = tid >= kTmaConsumers;
  const int t = tid % HALF, j = tid / HALF;
  const bool cons = !producer && j < S;
  const int h = blockIdx.x * S + j;
  const bool active = cons && h < g.Vh;
  const int rhs = blockIdx.z;
  if (a.active && !a.active[rhs]) return;
  const size_t co = (size_t)rhs * a.cstride;
  const size_t NP = (size_t)g.N5 >> 1;
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NST; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kTmaConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (POST != PR_NONE) {
    for (int i = tid; i < chain_block(LS); i += kTmaThreads) coef[i] = a.chain[co + i];
  }
  __syncthreads();
  SpinP<V> acc;
  zero(acc);
  bool timed_out = false;
  if (producer) {
    const int lane = tid - kTmaConsumers;
    const int hs = blockIdx.x * S + lane;
    const bool ok = lane < S && hs < g.Vh;
    const int nsites = min(S, g.Vh - (int)blockIdx.x * S);
    int nb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ok) {
      const int4 n0 = __ldg(a.nbr + 2 * hs), n1 = __ldg(a.nbr + 2 * hs + 1);
      nb[0] = n0.x; nb[1] = n0.y; nb[2] = n0.z; nb[3] = n0.w;
      nb[4] = n1.x; nb[5] = n1.y; nb[6] = n1.z; nb[7] = n1.w;
    }
    const char* vb = reinterpret_cast<const char*>(a.v) + rhs * a.stride;
    int armed[NST];
#pragma unroll
    for (int i = 0; i < NST; i++) armed[i] = 0;
#pragma unroll
    for (int d = 0; d < 8; d++) {
      const int st = d % NST;
      if (d >= NST) {
        if (!mbar_wait(&empty[st], (unsigned)((d / NST - 1) & 1), budget)) timed_out = true;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      // the test hook skip_hop leaves this stage unarmed: its consumers' bounded
      // waits run out (no arrival, no copy in flight)
      if (d == skip_hop) continue;
      if (lane == 0) mbar_expect_tx(&full[st], (unsigned)(nsites * ST::kTx));
      armed[st]++;
      __syncwarp();
      if (ok) {
        unsigned char* dst = stages + (size_t)st * S * ST::kBytes + (size_t)lane * ST::kBytes;
        const int hn = nb[d] & 0x7fffffff;
        tma_load_3d(dst, &tmap, hn * HALF * ST::kWpp, 0, rhs, &full[st]);
        if constexpr (SP::kScaled)
          bulk_load(dst + ST::kScaleOff, vb + (size_t)6 * NP * 16 + (size_t)hn * HALF * 8,
                    ST::kScaleBytes, &full[st]);
        const int mu = d >> 1;
        const char* lk = (d & 1) == 0
                             ? reinterpret_cast<const char*>(a.gauge_p) + ((size_t)hs * 4 + mu) * ST::kLinkBytes
                             : reinterpret_cast<const char*>(a.gauge_q) + ((size_t)hn * 4 + mu) * ST::kLinkBytes;
        bulk_load(dst + ST::kLinkOff, lk, ST::kLinkBytes, &full[st]);
      }
    }
    // every armed phase has landed before the stages are reused or the CTA exits
    // (phases complete in order, so waiting for the last one of a stage suffices)
#pragma unroll
    for (int i = 0; i < NST; i++)
      if (armed[i] > 0 && !mbar_wait(&full[i], (unsigned)((armed[i] - 1) & 1), budget)) timed_out = true;
  } else {
    T bd[2][2] = {{0, 0}, {0, 0}}, bo[2][2] = {{0, 0}, {0, 0}};
    int4 n0 = make_int4(0, 0, 0, 0), n1 = n0;
    if (active) {
      n0 = __ldg(a.nbr + 2 * h);
      n1 = __ldg(a.nbr + 2 * h + 1);
      if (PRE == PRE_B) {
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
          for (int k = 0; k < 2; k++) {
            bd[c][k] = __ldg(a.bdiag + co + c * LS + 2 * t + k);
            bo[c][k] = __ldg(a.boff + co + c * LS + 2 * t + k);
          }
      }
    }
    const int nbv[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#define DWF_TMA_STEP(D, MU, DIR)                                                               \
  {                                                                                           \
    const int st = D % NST;                                                                   \
    const bool ready = mbar_wait(&full[st], (unsigned)((D / NST) & 1), budget);               \
    if (!ready) timed_out = true;                                                             \
    if (ready && active)                                                                      \
      hop_staged<SP, LS, PRE, MU, DIR>(stages + (size_t)st * S * ST::kBytes + (size_t)j * ST::kBytes, \
                                       nbv[D] < 0, t, bd, bo, acc);                           \
    mbar_arrive(&empty[st]);                                                                  \
  }
    DWF_TMA_STEP(0, 0, +1)
    DWF_TMA_STEP(1, 0, -1)
    DWF_TMA_STEP(2, 1, +1)
    DWF_TMA_STEP(3, 1, -1)
    DWF_TMA_STEP(4, 2, +1)
    DWF_TMA_STEP(5, 2, -1)
    DWF_TMA_STEP(6, 3, +1)
    DWF_TMA_STEP(7, 3, -1)
#undef DWF_TMA_STEP
  }
  if (timed_out && a.err) atomicOr(a.err, 1);
  // the stages are consumed (every full phase waited for): reuse them for the
  // 5th-dimension transpose of the epilogue
  __syncthreads();
  T* site = reinterpret_cast<T*>(stages) + (size_t)(cons ? j : 0) * SST;
  epilogue_g<SP, LS, POST, LOC, G5, NORM>(a, coef, site, NP, h, t, active, cons, rhs, acc);
}

template <class SP, int LS, int NST>
constexpr size_t tma_smem_bytes() {
  using T = typename SP::T;
  constexpr int S = kTmaConsumers / (LS / 2);
  constexpr size_t ring = (size_t)NST * S * Stage<SP, LS>::kBytes;
  constexpr size_t tr = (size_t)S * site_stride(LS) * sizeof(T);
  return 128 + ((size_t)chain_block(LS) * sizeof(T) + 127) / 128 * 128 + (ring > tr ? ring : tr);
}

}  // namespace hop2
}  // namespace dwf
