// dwf_api.cu -- the C ABI of libdwf: handle, 5th-dimension matrices, gauge
// loading, the D_bb / D_bb^dagger applies, the propagator solve and the force.
//
// Operator factorisation (Sec. 2 Eq. mobius1 with Eq. coeff and Eq. wilson):
// D_alpha = D_w B + C with B, C real Ls x Ls matrices acting on the 5th index of
// each chirality (B: D_w -> 1, C: D_w -> 0 in the block list).  With
// D_w = (4 + M5) - H/2 (H the Wilson hopping term) the site-local part is
// I = (4 + M5) B + C and the hopping part is -1/2 H B, so the red-black operator
// of Sec. 3 Eq. redblack becomes
//     D_bb = 1 - 1/4 I^-1 H_br K H_rb B,          K = B I^-1,
//     D_bb^+ = gamma5 [1 - 1/4 B^T H_br K^T H_rb I^-T] gamma5.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <limits>
#include <sstream>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dwf.h"
#include "dwf_internal.cuh"
#include "dwf_hop2.cuh"

using namespace dwf;

namespace {

thread_local std::string g_create_error;

// Real Ls x Ls matrices of one (alpha, m) for both chiralities, FP64 host copy
// and device copies in FP64 and FP32.  Device layout (in elements):
//   K[2][Ls][Ls] KT IinvM IinvT Ifull BT  then Bdiag[2][Ls] Boff[2][Ls]
struct MatSet {
  double alpha = 1.0, m = 0.0;
  int Ls = 0;
  std::vector<double> host;
  void* dev[2] = {nullptr, nullptr};  // [0] double, [1] float
  // IT = I^T, SI = S I and SIT = (S I)^T for the operator forms of Eq. redblack1
  enum { K = 0, KT = 1, IINV = 2, IINVT = 3, IFULL = 4, BT = 5, IT = 6, SI = 7, SIT = 8, NMAT = 9 };
  size_t mat_off(int which) const { return (size_t)which * 2 * Ls * Ls; }
  size_t bdiag_off() const { return (size_t)NMAT * 2 * Ls * Ls; }
  size_t boff_off() const { return bdiag_off() + 2 * (size_t)Ls; }
  size_t chain_off() const { return boff_off() + 2 * (size_t)Ls; }
  size_t count() const { return chain_off() + (size_t)hop2::chain_block(Ls); }
  const void* ptr(int prec, size_t off) const {
    const int f = prec == P64 ? 0 : 1;
    const size_t es = f == 0 ? 8 : 4;
    return reinterpret_cast<const char*>(dev[f]) + off * es;
  }
};

bool invert(std::vector<double> a, int n, std::vector<double>& inv) {
  // Gauss-Jordan elimination with partial pivoting.
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; col++) {
    int piv = col;
    for (int r = col + 1; r < n; r++)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    if (a[(size_t)piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int k = 0; k < n; k++) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double d = 1.0 / a[(size_t)col * n + col];
    for (int k = 0; k < n; k++) {
      a[(size_t)col * n + k] *= d;
      inv[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; r++) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; k++) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  return true;
}

// B_+-, C_+- of Eq. mobius1: row s of the P_+ (chir 0) and P_- (chir 1) blocks.
// fb = b (B) or 1 (C); fc = c (B) or -1 (C).
void chiral_blocks(int Ls, double alpha, double m, const double* fb, const double* fc,
                   std::vector<double>& Mp, std::vector<double>& Mm) {
  Mp.assign((size_t)Ls * Ls, 0.0);
  Mm.assign((size_t)Ls * Ls, 0.0);
  auto P = [&](int r, int c) -> double& { return Mp[(size_t)r * Ls + c]; };
  auto M = [&](int r, int c) -> double& { return Mm[(size_t)r * Ls + c]; };
  const int l = Ls - 1;
  // row 1: D_1+(P_- + alpha P_+), alpha D_1- P_- (col 2), -m D_1- P_+ (col Ls)
  P(0, 0) += alpha * fb[0];
  M(0, 0) += fb[0];
  M(0, 1) += alpha * fc[0];
  P(0, l) += -m * fc[0];
  // rows 2 .. Ls-1: alpha D_i- P_+ (col i-1), alpha D_i+ (col i), alpha D_i- P_- (col i+1)
  for (int i = 1; i < l; i++) {
    P(i, i - 1) += alpha * fc[i];
    P(i, i) += alpha * fb[i];
    M(i, i) += alpha * fb[i];
    M(i, i + 1) += alpha * fc[i];
  }
  // row Ls: -m D_Ls- P_- (col 1), alpha D_Ls- P_+ (col Ls-1), D_Ls+(P_+ + alpha P_-)
  M(l, 0) += -m * fc[l];
  P(l, l - 1) += alpha * fc[l];
  P(l, l) += fb[l];
  M(l, l) += alpha * fb[l];
}

std::vector<double> matmul(const std::vector<double>& a, const std::vector<double>& b, int n) {
  std::vector<double> c((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++)
    for (int k = 0; k < n; k++)
      for (int j = 0; j < n; j++) c[(size_t)i * n + j] += a[(size_t)i * n + k] * b[(size_t)k * n + j];
  return c;
}

std::vector<double> transpose(const std::vector<double>& a, int n) {
  std::vector<double> t((size_t)n * n);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) t[(size_t)j * n + i] = a[(size_t)i * n + j];
  return t;
}

// Cyclic bidiagonal matrix (M y)_s = d_s y_s + o_s y_{(s + dir) mod Ls}.
struct CycBidiag {
  std::vector<double> d, o;
  int dir;
};

CycBidiag extract_cb(const std::vector<double>& M, int Ls, int dir) {
  CycBidiag r;
  r.dir = dir;
  r.d.resize(Ls);
  r.o.resize(Ls);
  for (int s = 0; s < Ls; s++) {
    r.d[s] = M[(size_t)s * Ls + s];
    r.o[s] = M[(size_t)s * Ls + (s + dir + Ls) % Ls];
  }
  return r;
}

// (M^T y)_s = d_s y_s + o_{s - dir} y_{s - dir}
CycBidiag transpose_cb(const CycBidiag& m, int Ls) {
  CycBidiag r;
  r.dir = -m.dir;
  r.d = m.d;
  r.o.resize(Ls);
  for (int s = 0; s < Ls; s++) r.o[s] = m.o[(s - m.dir + Ls) % Ls];
  return r;
}

// Coefficients of the tuned kernels' recurrences in "lower" sweep order
// (slice order reversed when dir = +1): multiply y_k = D_k v_k + O_k v_{k-1};
// solve D_k y_k + O_k y_{k-1} = v_k by y_k = alpha_k + beta_k y_0.
void chain_coeffs(const CycBidiag& m, int Ls, bool solve, double* out) {
  const bool rev = m.dir == +1;
  std::vector<double> D(Ls), O(Ls);
  for (int k = 0; k < Ls; k++) {
    const int s = rev ? Ls - 1 - k : k;
    D[k] = m.d[s];
    O[k] = m.o[s];
  }
  if (!solve) {
    for (int k = 0; k < Ls; k++) {
      out[k] = D[k];
      out[Ls + k] = O[k];
    }
    return;
  }
  std::vector<double> beta(Ls);
  beta[0] = 1.0;
  for (int k = 1; k < Ls; k++) beta[k] = -(O[k] / D[k]) * beta[k - 1];
  for (int k = 0; k < Ls; k++) {
    out[k] = 1.0 / D[k];
    out[Ls + k] = O[k] / D[k];
    out[2 * Ls + k] = beta[k];
  }
  out[3 * Ls] = 1.0 / (D[0] + O[0] * beta[Ls - 1]);
  out[3 * Ls + 1] = O[0];
}

}  // namespace

struct dwf_ctx {
  Geom g{};
  int Ls = 0;
  double M5 = 0, m = 0, alpha = 1;
  std::vector<double> b, c;
  dwf_options opt{};
  int device = 0;
  void* noalloc_scratch = nullptr;               // device address of the static scratch array
  std::string err;
  std::map<std::pair<double, double>, MatSet> mats;
  void* gauge[3] = {nullptr, nullptr, nullptr};  // FP64, FP32, FP16
  int* nbr = nullptr;                            // [2][Vh][8] neighbour table
  int* dev_err = nullptr;                        // set by a kernel whose bounded wait gave up
  int use_tma = 0;                               // tensor-copy staged tuned kernels (autotuned)
  int env_tma = 0;                               // DWF_TMA set: staging fixed to tensor copies
  long long wait_budget = 0;                     // DWF_WAIT_BUDGET: clock cycles per bounded wait
  int skip_hop = -1;                             // DWF_TEST_SKIP_HOP: the first staged launch
                                                 // issues no copies for this hop (timeout test)
  bool fused_cg = true;                          // DWF_UNFUSED_CG unset: fused CG BLAS steps
  bool bp_fused = true;                          // DWF_NO_BP_FUSED unset: p update forms B p
  int check = 16;                                // effective iterations between polls
  bool gauge_loaded = false;
  std::vector<void*> allocs;
  // workspace
  std::map<std::string, void*> ws;
  std::map<std::string, size_t> ws_size;
  double* scal = nullptr;          // per-rhs scalars, kScal doubles each
  double* partial = nullptr;       // reduction partials
  unsigned int* counter = nullptr; // reduction counters
  int partial_stride = 0;
  int scal_rhs = 0;
  double* pinned = nullptr;        // host mirror of scal
  long long launches = 0;          // kernels launched through this handle
  // CUDA-event timing of the inner applies (opt.profile): pool and pending pairs
  std::vector<cudaEvent_t> events;
  std::vector<int> pending;        // (start index) of recorded pairs, kind in pending_kind
  std::vector<int> pending_kind;
  size_t next_event = 0;
  double timed_ms[2] = {0, 0};
  int timed_n[2] = {0, 0};         // applies covered by timed_ms
  cudaStream_t cstream = nullptr;  // solver stream (graph capture needs a non-legacy stream)
  int* d_active = nullptr;         // per right-hand-side active mask of a batched solve
  int* pinned_i = nullptr;         // host staging of the mask
  int active_cap = 0;
  struct Tuned {
    int nb, tma, tile;  // right-hand-side block, staging variant, 4D sites per CTA (0: default)
  };
  std::map<std::string, Tuned> tune;  // autotuned launch shapes
  int tile = 0;                      // 4D sites per CTA of the tuned hop kernels (0: default)
  int env_tile = -1;                 // DWF_HOP_TILE set: tile fixed (-1: autotuned)
  double tier_eta = 1e-3;            // 16-bit solves: FP64 replacement once |r| < eta |r_64|
                                     // (DWF_TIER_ETA; <= 0: every replacement in FP64)
};

namespace {

constexpr int kScal = 16;
enum { S_ZZ0 = 0, S_ZZ1 = 1, S_WW = 2, S_RR = 3, S_RRHI = 4, S_BB = 5, S_T0 = 6, S_T1 = 7, S_T2 = 8, S_A = 9 };

int fail(dwf_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

#define KLAUNCH(h, expr)            \
  do {                              \
    (h)->launches++;                \
    CUCHK(h, expr);                 \
  } while (0)

#define CUCHK(h, expr)                                                                       \
  do {                                                                                      \
    cudaError_t _e = (expr);                                                                \
    if (_e != cudaSuccess)                                                                  \
      return fail(h, _e == cudaErrorMemoryAllocation ? DWF_ERR_OOM : DWF_ERR_CUDA,         \
                  std::string(#expr) + ": " + cudaGetErrorString(_e));                      \
  } while (0)

bool valid_prec(int p) { return p >= DWF_FP64 && p <= DWF_BF16; }

int build_matset(dwf_ctx* h, double alpha, double m, MatSet** out) {
  auto key = std::make_pair(alpha, m);
  auto it = h->mats.find(key);
  if (it != h->mats.end()) {
    *out = &it->second;
    return DWF_OK;
  }
  const int Ls = h->Ls;
  MatSet ms;
  ms.alpha = alpha;
  ms.m = m;
  ms.Ls = Ls;
  std::vector<double> ones(Ls, 1.0), mones(Ls, -1.0);
  std::vector<double> Bm[2], Cm[2];
  chiral_blocks(Ls, alpha, m, h->b.data(), h->c.data(), Bm[0], Bm[1]);
  chiral_blocks(Ls, alpha, m, ones.data(), mones.data(), Cm[0], Cm[1]);
  ms.host.assign(ms.count(), 0.0);
  const size_t LL = (size_t)Ls * Ls;
  for (int ch = 0; ch < 2; ch++) {
    std::vector<double> I(LL), Iinv;
    for (size_t k = 0; k < LL; k++) I[k] = (4.0 + h->M5) * Bm[ch][k] + Cm[ch][k];
    if (!invert(I, Ls, Iinv))
      return fail(h, DWF_ERR_INVALID_ARG, "the site-local matrix I = (4+M5)B + C is singular");
    std::vector<double> K = matmul(Bm[ch], Iinv, Ls);
    // S I: row s of I scaled by 1/(b_s + c_s) where that coefficient exceeds one
    std::vector<double> SI = I;
    for (int s = 0; s < Ls; s++) {
      const double a = h->b[s] + h->c[s];
      if (a > 1.0)
        for (int q = 0; q < Ls; q++) SI[(size_t)s * Ls + q] /= a;
    }
    std::vector<double> mats[MatSet::NMAT] = {K, transpose(K, Ls), Iinv, transpose(Iinv, Ls), I,
                                              transpose(Bm[ch], Ls), transpose(I, Ls), SI,
                                              transpose(SI, Ls)};
    for (int w = 0; w < MatSet::NMAT; w++)
      std::copy(mats[w].begin(), mats[w].end(), ms.host.begin() + ms.mat_off(w) + ch * LL);
    // cyclic bidiagonal form of B
    for (int s = 0; s < Ls; s++) {
      const int col = ch == 0 ? (s + Ls - 1) % Ls : (s + 1) % Ls;
      for (int q = 0; q < Ls; q++) {
        if (q == s || q == col) continue;
        if (Bm[ch][(size_t)s * Ls + q] != 0.0)
          return fail(h, DWF_ERR_STATE, "B is not cyclic bidiagonal");
      }
      ms.host[ms.bdiag_off() + ch * Ls + s] = Bm[ch][(size_t)s * Ls + s];
      ms.host[ms.boff_off() + ch * Ls + s] = Ls == 1 ? 0.0 : Bm[ch][(size_t)s * Ls + col];
    }
  }
  // recurrence coefficients of the tuned kernels
  for (int ch = 0; ch < 2; ch++) {
    std::vector<double> I(LL);
    for (size_t k = 0; k < LL; k++) I[k] = (4.0 + h->M5) * Bm[ch][k] + Cm[ch][k];
    const int dir = ch == 0 ? -1 : +1;
    const CycBidiag Bc = extract_cb(Bm[ch], Ls, dir), Ic = extract_cb(I, Ls, dir);
    const int cs = hop2::chain_stride(Ls);
    double* base = ms.host.data() + ms.chain_off();
    chain_coeffs(Bc, Ls, false, base + (hop2::OP_B * 2 + ch) * cs);
    chain_coeffs(transpose_cb(Bc, Ls), Ls, false, base + (hop2::OP_BT * 2 + ch) * cs);
    chain_coeffs(Ic, Ls, false, base + (hop2::OP_I * 2 + ch) * cs);
    chain_coeffs(Ic, Ls, true, base + (hop2::OP_ISOLVE * 2 + ch) * cs);
    chain_coeffs(transpose_cb(Ic, Ls), Ls, true, base + (hop2::OP_ITSOLVE * 2 + ch) * cs);
  }
  std::vector<float> hf(ms.count());
  for (size_t k = 0; k < hf.size(); k++) hf[k] = (float)ms.host[k];
  CUCHK(h, cudaMalloc(&ms.dev[0], ms.count() * 8));
  CUCHK(h, cudaMalloc(&ms.dev[1], ms.count() * 4));
  CUCHK(h, cudaMemcpy(ms.dev[0], ms.host.data(), ms.count() * 8, cudaMemcpyHostToDevice));
  CUCHK(h, cudaMemcpy(ms.dev[1], hf.data(), ms.count() * 4, cudaMemcpyHostToDevice));
  h->allocs.push_back(ms.dev[0]);
  h->allocs.push_back(ms.dev[1]);
  auto res = h->mats.emplace(key, std::move(ms));
  *out = &res.first->second;
  return DWF_OK;
}

int get_ws(dwf_ctx* h, const std::string& name, size_t bytes, void** out) {
  auto it = h->ws.find(name);
  if (it != h->ws.end() && h->ws_size[name] >= bytes) {
    *out = it->second;
    return DWF_OK;
  }
  if (it != h->ws.end()) {
    cudaFree(it->second);
    h->ws.erase(it);
  }
  void* p = nullptr;
  CUCHK(h, cudaMalloc(&p, bytes));
  h->ws[name] = p;
  h->ws_size[name] = bytes;
  *out = p;
  return DWF_OK;
}

int ensure_reduce(dwf_ctx* h, int nrhs) {
  int need_blocks =
      std::max(hop_grid_blocks(h->g, P64, 0), std::max(hop_grid_blocks(h->g, P32, 0),
                                                       blas_grid_blocks(h->g)));
  if (h->Ls == 8 || h->Ls == 12 || h->Ls == 16)  // the small tile of the tuned kernels
    need_blocks = std::max(need_blocks, hop_grid_blocks(h->g, P32, hop2::small_block_sites(h->Ls)));
  if (h->scal && h->scal_rhs >= nrhs && h->partial_stride >= need_blocks) return DWF_OK;
  if (h->scal) {
    cudaFree(h->scal);
    cudaFree(h->partial);
    cudaFree(h->counter);
    cudaFreeHost(h->pinned);
  }
  h->scal_rhs = std::max(nrhs, 1);
  h->partial_stride = need_blocks;
  CUCHK(h, cudaMalloc(&h->scal, sizeof(double) * kScal * h->scal_rhs));
  CUCHK(h, cudaMalloc(&h->partial, sizeof(double) * (size_t)need_blocks * h->scal_rhs * 4));
  CUCHK(h, cudaMalloc(&h->counter, sizeof(unsigned int) * h->scal_rhs * 4));
  CUCHK(h, cudaMemset(h->counter, 0, sizeof(unsigned int) * h->scal_rhs * 4));
  CUCHK(h, cudaMemset(h->scal, 0, sizeof(double) * kScal * h->scal_rhs));
  CUCHK(h, cudaMallocHost(&h->pinned, sizeof(double) * (kScal * h->scal_rhs + 1)));
  return DWF_OK;
}

// Reduction slot k (0..3) into scalar index which.
Reduce make_reduce(dwf_ctx* h, int slot, int which) {
  Reduce r;
  r.partial = h->partial + (size_t)slot * h->partial_stride * h->scal_rhs;
  r.counter = h->counter + (size_t)slot * h->scal_rhs;
  r.result = h->scal + which;
  r.partial_stride = h->partial_stride;
  r.result_stride = kScal;
  return r;
}

const void* gauge_for(dwf_ctx* h, int prec) {
  return prec == P64 ? h->gauge[0] : (prec == P32 ? h->gauge[1] : h->gauge[2]);
}

HopLaunch base_hop(dwf_ctx* h, int prec, int p, int nrhs, size_t stride) {
  HopLaunch L{};
  L.prec = prec;
  L.p = p;
  L.nrhs = nrhs;
  L.stride = stride;
  L.gauge = gauge_for(h, prec);
  L.gauge_parity_bytes = gauge_bytes(h->g, prec) / 2;
  L.c_hop = 1.0;
  L.c_loc = 0.0;
  L.nbr = h->nbr;
  L.err = h->dev_err;
  L.use_tma = h->use_tma;
  L.block_sites = h->tile;
  L.wait_budget = h->wait_budget;
  L.skip_hop = &h->skip_hop;  // one-shot test hook, consumed by the first staged launch
  return L;
}

// Coefficient arrays of one or more right-hand sides: the layout (offsets) of a
// MatSet, base pointers of the FP64 / FP32 copies, the element stride between
// right-hand sides (0: all share one set) and the per-RHS active mask.
struct CoefView {
  const MatSet* layout;
  const void* dev[2];
  size_t cstride;
  const int* active;
  const void* ptr(int prec, size_t off) const {
    const int f = prec == P64 ? 0 : 1;
    return reinterpret_cast<const char*>(dev[f]) + off * (f == 0 ? 8 : 4);
  }
};
CoefView view_of(const MatSet& ms) { return CoefView{&ms, {ms.dev[0], ms.dev[1]}, 0, nullptr}; }

void set_coef(HopLaunch& L, const CoefView& cv) {
  L.cstride = cv.cstride;
  L.active = cv.active;
}

// out = D_bb in.  tmp: red half-field(s) of the same precision.
int apply_dbb(dwf_ctx* h, const CoefView& cv, int prec, void* out, const void* in, void* tmp, int nrhs,
              const Reduce* norm, cudaStream_t s) {
  const MatSet& ms = *cv.layout;
  const int black = h->opt.rb_parity, red = 1 - black;
  const size_t st = field_bytes(h->g, prec);
  HopLaunch A = base_hop(h, prec, red, nrhs, st);
  A.out = tmp;
  A.v = in;
  A.pre = PRE_B;
  A.pre_diag = cv.ptr(prec, ms.bdiag_off());
  A.pre_off = cv.ptr(prec, ms.boff_off());
  A.post = cv.ptr(prec, ms.mat_off(MatSet::K));
  A.post_prog = hop2::PR_K;
  A.chain = cv.ptr(prec, ms.chain_off());
  set_coef(A, cv);
  KLAUNCH(h, launch_hop(h->g, A, s));
  HopLaunch B = base_hop(h, prec, black, nrhs, st);
  B.out = out;
  B.v = tmp;
  B.w = in;
  B.post = cv.ptr(prec, ms.mat_off(MatSet::IINV));
  B.post_prog = hop2::PR_IINV;
  B.chain = cv.ptr(prec, ms.chain_off());
  B.loc = LOC_ID;
  B.c_hop = -0.25;
  B.c_loc = 1.0;
  B.red = norm;
  set_coef(B, cv);
  KLAUNCH(h, launch_hop(h->g, B, s));
  return DWF_OK;
}

// out = D_bb p given bp = B p (the fused CG forms B p with p): pass A hops bp
// without the B pre-multiplication, pass B as in apply_dbb.
int apply_dbb_bp(dwf_ctx* h, const CoefView& cv, int prec, void* out, const void* p, const void* bp,
                 void* tmp, int nrhs, const Reduce* norm, cudaStream_t s) {
  const MatSet& ms = *cv.layout;
  const int black = h->opt.rb_parity, red = 1 - black;
  const size_t st = field_bytes(h->g, prec);
  HopLaunch A = base_hop(h, prec, red, nrhs, st);
  A.out = tmp;
  A.v = bp;
  A.post = cv.ptr(prec, ms.mat_off(MatSet::K));
  A.post_prog = hop2::PR_K;
  A.chain = cv.ptr(prec, ms.chain_off());
  set_coef(A, cv);
  KLAUNCH(h, launch_hop(h->g, A, s));
  HopLaunch B = base_hop(h, prec, black, nrhs, st);
  B.out = out;
  B.v = tmp;
  B.w = p;
  B.post = cv.ptr(prec, ms.mat_off(MatSet::IINV));
  B.post_prog = hop2::PR_IINV;
  B.chain = cv.ptr(prec, ms.chain_off());
  B.loc = LOC_ID;
  B.c_hop = -0.25;
  B.c_loc = 1.0;
  B.red = norm;
  set_coef(B, cv);
  KLAUNCH(h, launch_hop(h->g, B, s));
  return DWF_OK;
}

// hat = I^-T gamma5 in (the local first factor of D_bb^+).
int apply_hat(dwf_ctx* h, const CoefView& cv, int prec, void* hat, const void* in, int nrhs,
              cudaStream_t s) {
  const MatSet& ms = *cv.layout;
  LocalLaunch L{};
  L.prec = prec;
  L.out = hat;
  L.in = in;
  L.stride = field_bytes(h->g, prec);
  L.nrhs = nrhs;
  L.m = cv.ptr(prec, ms.mat_off(MatSet::IINVT));
  L.prog = hop2::PR_ITINV;
  L.chain = cv.ptr(prec, ms.chain_off());
  L.c = 1.0;
  L.g5in = 1;
  L.cstride = cv.cstride;
  L.active = cv.active;
  KLAUNCH(h, launch_local(h->g, L, s));
  return DWF_OK;
}

// out = D_bb^+ in given hat = I^-T gamma5 in.  tmp_red: red field(s).
int apply_dbb_dag_hat(dwf_ctx* h, const CoefView& cv, int prec, void* out, const void* in,
                      const void* hat, void* tmp_red, int nrhs, const Reduce* norm, cudaStream_t s) {
  const MatSet& ms = *cv.layout;
  const int black = h->opt.rb_parity, red = 1 - black;
  const size_t st = field_bytes(h->g, prec);
  HopLaunch A = base_hop(h, prec, red, nrhs, st);
  A.out = tmp_red;
  A.v = hat;
  A.post = cv.ptr(prec, ms.mat_off(MatSet::KT));
  A.post_prog = hop2::PR_KT;
  A.chain = cv.ptr(prec, ms.chain_off());
  set_coef(A, cv);
  KLAUNCH(h, launch_hop(h->g, A, s));
  HopLaunch B = base_hop(h, prec, black, nrhs, st);
  B.out = out;
  B.v = tmp_red;
  B.w = in;
  B.post = cv.ptr(prec, ms.mat_off(MatSet::BT));
  B.post_prog = hop2::PR_BT;
  B.chain = cv.ptr(prec, ms.chain_off());
  B.loc = LOC_ID;
  B.c_hop = -0.25;
  B.c_loc = 1.0;
  B.g5out = 1;
  B.red = norm;
  set_coef(B, cv);
  KLAUNCH(h, launch_hop(h->g, B, s));
  return DWF_OK;
}

// out = D_bb^+ in.  tmp_red: red field(s); tmp_blk: black field(s).
int apply_dbb_dag(dwf_ctx* h, const CoefView& cv, int prec, void* out, const void* in, void* tmp_red,
                  void* tmp_blk, int nrhs, const Reduce* norm, cudaStream_t s) {
  int rc;
  if ((rc = apply_hat(h, cv, prec, tmp_blk, in, nrhs, s))) return rc;
  return apply_dbb_dag_hat(h, cv, prec, out, in, tmp_blk, tmp_red, nrhs, norm, s);
}

// out = L in for the site-local dense matrix L = MatSet matrix `which` of each
// right-hand side (generic local kernel), optional fused |out|^2.
int apply_local_dense(dwf_ctx* h, const CoefView& cv, int prec, int which, void* out,
                      const void* in, int nrhs, const Reduce* norm, cudaStream_t s) {
  LocalLaunch L{};
  L.prec = prec;
  L.out = out;
  L.in = in;
  L.stride = field_bytes(h->g, prec);
  L.nrhs = nrhs;
  L.m = cv.ptr(prec, cv.layout->mat_off(which));
  L.c = 1.0;
  L.red = norm;
  L.prog = hop2::PR_NONE;
  L.cstride = cv.cstride;
  L.active = cv.active;
  KLAUNCH(h, launch_local(h->g, L, s));
  return DWF_OK;
}

// (out0, out1) = D_alpha(ms) (in0, in1), FP64 internal halves by parity.
int apply_dalpha_halves(dwf_ctx* h, const MatSet& ms, void* out[2], const void* in[2], cudaStream_t s) {
  const size_t st = field_bytes(h->g, P64);
  for (int p = 0; p < 2; p++) {
    HopLaunch L = base_hop(h, P64, p, 1, st);
    L.out = out[p];
    L.v = in[1 - p];
    L.w = in[p];
    L.pre = PRE_B;
    L.pre_diag = ms.ptr(P64, ms.bdiag_off());
    L.pre_off = ms.ptr(P64, ms.boff_off());
    L.loc = LOC_DENSE;
    L.locm = ms.ptr(P64, ms.mat_off(MatSet::IFULL));
    L.c_hop = -0.5;
    L.c_loc = 1.0;
    KLAUNCH(h, launch_hop(h->g, L, s));
  }
  return DWF_OK;
}

int sync_read(dwf_ctx* h, int nrhs, cudaStream_t s) {
  CUCHK(h, cudaMemcpyAsync(h->pinned, h->scal, sizeof(double) * kScal * nrhs, cudaMemcpyDeviceToHost, s));
  CUCHK(h, cudaMemcpyAsync(h->pinned + kScal * h->scal_rhs, h->dev_err, sizeof(int),
                           cudaMemcpyDeviceToHost, s));
  CUCHK(h, cudaStreamSynchronize(s));
  int flag;
  std::memcpy(&flag, h->pinned + kScal * h->scal_rhs, sizeof(int));
  if (flag) {
    cudaMemsetAsync(h->dev_err, 0, sizeof(int), s);
    return fail(h, DWF_ERR_TIMEOUT, "a kernel's bounded wait for its shared-memory copies gave up");
  }
  return DWF_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct SolveWork {
  void *b_hi, *x_hi, *r_hi, *t64, *t64r;  // FP64 black (t64r red)
  void *p, *r, *w, *z, *xlo, *tb, *tr;    // inner precision
  void *p2, *bp;                          // second p buffer and B p (fused CG)
};

int alloc_solve_work(dwf_ctx* h, int prec, SolveWork& W, int nb = 1) {
  const size_t f64 = field_bytes(h->g, P64) * nb, fi = field_bytes(h->g, prec) * nb;
  const std::string sfx = "_" + std::to_string(prec);
  int rc;
  if ((rc = get_ws(h, "b_hi", f64, &W.b_hi))) return rc;
  if ((rc = get_ws(h, "x_hi", f64, &W.x_hi))) return rc;
  if ((rc = get_ws(h, "r_hi", f64, &W.r_hi))) return rc;
  if ((rc = get_ws(h, "t64", f64, &W.t64))) return rc;
  if ((rc = get_ws(h, "t64r", f64, &W.t64r))) return rc;
  if ((rc = get_ws(h, "p" + sfx, fi, &W.p))) return rc;
  if ((rc = get_ws(h, "r" + sfx, fi, &W.r))) return rc;
  if ((rc = get_ws(h, "w" + sfx, fi, &W.w))) return rc;
  if ((rc = get_ws(h, "z" + sfx, fi, &W.z))) return rc;
  const int xprec = (prec == P16 || prec == PB16) ? P32 : prec;
  if ((rc = get_ws(h, "xlo" + sfx, field_bytes(h->g, xprec) * nb, &W.xlo))) return rc;
  if ((rc = get_ws(h, "tb" + sfx, fi, &W.tb))) return rc;
  if ((rc = get_ws(h, "tr" + sfx, fi, &W.tr))) return rc;
  W.p2 = W.bp = nullptr;
  {
    if ((rc = get_ws(h, "p2" + sfx, fi, &W.p2))) return rc;
    if ((rc = get_ws(h, "bp" + sfx, fi, &W.bp))) return rc;
  }
  return DWF_OK;
}

// Bytes of solver workspace per right-hand side (used by the autotuner's memory check).
size_t solve_bytes_per_rhs(const Geom& g, int prec) {
  const int xprec = (prec == P16 || prec == PB16) ? P32 : prec;
  const int extra = 2;  // second p buffer, B p
  return 5 * field_bytes(g, P64) + (6 + extra) * field_bytes(g, prec) + field_bytes(g, xprec);
}

// Start/stop events around one apply (kind 0: D_bb, 1: D_bb^+) when profiling.
int timer_mark(dwf_ctx* h, cudaStream_t s, bool start, int kind) {
  if (!h->opt.profile) return DWF_OK;
  if (h->next_event >= h->events.size()) {
    cudaEvent_t e;
    CUCHK(h, cudaEventCreate(&e));
    h->events.push_back(e);
  }
  const int idx = (int)h->next_event++;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CUCHK(h, cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    CUCHK(h, cudaEventRecordWithFlags(h->events[idx], s, cudaEventRecordExternal));
  else
    CUCHK(h, cudaEventRecord(h->events[idx], s));
  if (start) {
    h->pending.push_back(idx);
    h->pending_kind.push_back(kind);
  }
  return DWF_OK;
}

// After a stream synchronisation: add the elapsed time of all recorded pairs.
// keep = true for pairs recorded inside a CUDA graph (re-recorded at every replay).
int timer_harvest(dwf_ctx* h, bool keep = false) {
  if (!h->opt.profile) return DWF_OK;
  for (size_t k = 0; k < h->pending.size(); k++) {
    float ms = 0.f;
    const int i = h->pending[k];
    CUCHK(h, cudaEventElapsedTime(&ms, h->events[i], h->events[i + 1]));
    h->timed_ms[h->pending_kind[k]] += ms;
    h->timed_n[h->pending_kind[k]]++;
  }
  if (!keep) {
    h->pending.clear();
    h->pending_kind.clear();
    h->next_event = 0;
  }
  return DWF_OK;
}

int ensure_active(dwf_ctx* h, int nb) {
  if (h->active_cap >= nb) return DWF_OK;
  if (h->d_active) {
    cudaFree(h->d_active);
    cudaFreeHost(h->pinned_i);
  }
  CUCHK(h, cudaMalloc(&h->d_active, sizeof(int) * nb));
  CUCHK(h, cudaMallocHost(&h->pinned_i, sizeof(double) * (nb + 2)));
  h->active_cap = nb;
  return DWF_OK;
}

// CG on D^+ D x = D^+ b for nb right-hand sides at once (CGNR form: r = b - D x
// is tracked, z = D^+ r), inner precision prec with FP64 reliable updates
// (residual replacement once |r| drops below delta times its maximum since the
// last replacement) or, with restart = true, FP64 defect correction (beta = 0
// after every replacement).  One iteration:
//   z = D^+ r (fused |z|^2), beta = |z|^2 / |z_prev|^2, p = z + beta p,
//   w = D p (fused |w|^2), a = |z|^2 / |w|^2, x += a p, r -= a w (fused |r|^2);
// the first beta is 0 (|z_prev|^2 starts at +inf).  With the tuned kernels
// (Ls in {8, 12, 16}) the BLAS steps are fused differently, same arithmetic:
// the residual update also writes r^ = I^-T gamma5 r (the first factor of the
// next D^+ r) and stores a, and x += a p is deferred into the next p update
// (flushed before every poll).  The check iterations
// between two convergence polls are captured once as a CUDA graph.  Each right-
// hand side has its own scalars, coefficients (cv.cstride) and convergence; the
// device mask skips converged ones.  W.b_hi holds the nb FP64 sources, W.x_hi
// receives the solutions.
int cgnr_batched(dwf_ctx* h, const CoefView& cv_in, int prec, double tol, int maxiter,
                 double delta, bool restart, SolveWork& W, int nb, dwf_stats* st, cudaStream_t s) {
  const int xprec = (prec == P16 || prec == PB16) ? P32 : prec;
  const size_t f64 = field_bytes(h->g, P64), fi = field_bytes(h->g, prec),
               fx = field_bytes(h->g, xprec);
  Reduce red_ww = make_reduce(h, 0, S_WW), red_rr = make_reduce(h, 1, S_RR);
  Reduce red_zz[2] = {make_reduce(h, 2, S_ZZ0), make_reduce(h, 2, S_ZZ1)};
  Reduce red_hi = make_reduce(h, 3, S_RRHI), red_bb = make_reduce(h, 3, S_BB);
  int rc;
  if ((rc = ensure_active(h, nb))) return rc;
  const long long launches0 = h->launches;
  h->timed_ms[0] = h->timed_ms[1] = 0.0;
  h->timed_n[0] = h->timed_n[1] = 0;
  h->pending.clear();
  h->pending_kind.clear();
  h->next_event = 0;
  std::vector<int> act(nb, 1), conv(nb, 0), its(nb, 0), rst(nb, 0), stalled(nb, 0), code(nb, 0);
  std::vector<double> bnorm(nb), rmax(nb), true_res(nb, 1.0), best(nb, 1.0), t_done(nb, -1.0);
  // two-tier replacement (16-bit inner fields): |r_64| of the last FP64 replacement,
  // best FP32-tier residual since, escalation flag, FP32 replacements
  std::vector<double> anchor(nb, 0.0), best32(nb, 0.0);
  std::vector<int> esc(nb, 0), n32(nb, 0);
  const auto t_start = std::chrono::steady_clock::now();
  auto now_s = [&]() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  };
  CoefView cv = cv_in;
  cv.active = h->d_active;
  auto push_mask = [&](const std::vector<int>& mask) -> int {
    for (int r = 0; r < nb; r++) h->pinned_i[r] = mask[r];
    CUCHK(h, cudaMemcpyAsync(h->d_active, h->pinned_i, sizeof(int) * nb, cudaMemcpyHostToDevice, s));
    return DWF_OK;
  };
  auto push_active = [&]() -> int { return push_mask(act); };
  // |z_prev|^2 = +inf for the listed right-hand sides (first beta = 0)
  double* inf_src = reinterpret_cast<double*>(h->pinned_i + ((nb + 1) & ~1));
  auto reset_beta = [&](const std::vector<int>& which) -> int {
    *inf_src = std::numeric_limits<double>::infinity();
    for (int r = 0; r < nb; r++)
      if (which[r])
        CUCHK(h, cudaMemcpyAsync(h->scal + (size_t)r * kScal + S_ZZ0, inf_src, sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    return DWF_OK;
  };
  if ((rc = push_active())) return rc;
  // Operator form (Sec. 3): M = L D_bb with L = 1, I (Eq. redblack1) or S I (row scaled)
  const int form = h->opt.schur_form;
  const int Lw = form == DWF_SCHUR_ROWSCALED ? MatSet::SI : MatSet::IFULL;
  const int LTw = form == DWF_SCHUR_ROWSCALED ? MatSet::SIT : MatSet::IT;
  void *tb2 = nullptr, *t64b = nullptr;
  if (form != DWF_SCHUR_PRECOND) {
    if ((rc = get_ws(h, "tb2_" + std::to_string(prec), fi * nb, &tb2)) ||
        (rc = get_ws(h, "t64b", f64 * nb, &t64b)))
      return rc;
    // right-hand side L r'_b
    if ((rc = apply_local_dense(h, cv, P64, Lw, t64b, W.b_hi, nb, nullptr, s))) return rc;
    CUCHK(h, cudaMemcpyAsync(W.b_hi, t64b, f64 * nb, cudaMemcpyDeviceToDevice, s));
  }
  CUCHK(h, cudaMemsetAsync(W.x_hi, 0, f64 * nb, s));
  CUCHK(h, cudaMemsetAsync(W.xlo, 0, fx * nb, s));
  CUCHK(h, cudaMemsetAsync(W.p, 0, fi * nb, s));
  KLAUNCH(h, launch_convert(h->g, P64, W.r_hi, P64, W.b_hi, nb, f64, f64, &red_bb, s));
  KLAUNCH(h, launch_convert(h->g, prec, W.r, P64, W.b_hi, nb, fi, f64, nullptr, s));
  if ((rc = reset_beta(act))) return rc;
  if ((rc = sync_read(h, nb, s))) return rc;
  for (int r = 0; r < nb; r++) {
    const double bb = h->pinned[(size_t)r * kScal + S_BB];
    bnorm[r] = std::sqrt(bb);
    rmax[r] = bnorm[r];
    anchor[r] = best32[r] = bnorm[r];
    if (!(bb > 0.0)) {
      act[r] = 0;
      if (bb == 0.0) {
        conv[r] = 1;
        true_res[r] = 0.0;
      } else {
        code[r] = DWF_ERR_BREAKDOWN;
      }
    }
  }
  if ((rc = push_active())) return rc;
  const int Ls = h->g.Ls;
  const bool fused = form == DWF_SCHUR_PRECOND && h->fused_cg && !g_disable_tuned &&
                     (Ls == 8 || Ls == 12 || Ls == 16);
  if (fused && (rc = apply_hat(h, cv, prec, W.tb, W.r, nb, s))) return rc;
  // the p update also forms B p (of the stored p) for D_bb pass A; with BF16
  // fields the rounding of B p to 8 significand bits costs more iterations than
  // pass A saves (Zolotarev 24^3x48: 3288 against 2600), so BF16 folds B into pass A
  const bool with_bp = fused && W.bp != nullptr && h->bp_fused && prec != PB16;
  // Two-tier residual replacement for 16-bit inner fields: between FP64
  // replacements r = r_64 - D x_lo in FP32, where r_64 is the FP64 residual of the
  // last FP64 replacement and x_lo (FP32) the solution accumulated since; its
  // error is ~1e-6 |r_64|, small against |r| while |r| > tier_eta |r_64|.
  const bool tiered = (prec == P16 || prec == PB16) && form == DWF_SCHUR_PRECOND && h->tier_eta > 0;
  if (with_bp) CUCHK(h, cudaMemsetAsync(W.p2, 0, fi * nb, s));

  // with opt.profile, the first iteration after each poll times its two applies
  // (a sample: every timed apply adds two event records to the replayed graph)
  auto mark = [&](bool first, bool start, int kind) -> int {
    return first ? timer_mark(h, s, start, kind) : DWF_OK;
  };
  auto enqueue_fused = [&](int cur, bool first) -> int {
    const int nxt = 1 - cur;
    double* zz_new = h->scal + (nxt ? S_ZZ1 : S_ZZ0);
    double* zz_old = h->scal + (cur ? S_ZZ1 : S_ZZ0);
    int r;
    if ((r = mark(first, true, 1))) return r;
    if ((r = apply_dbb_dag_hat(h, cv, prec, W.z, W.r, W.tb, W.tr, nb, &red_zz[nxt], s))) return r;
    if ((r = mark(first, false, 1))) return r;
    void* pcur = W.p;
    if (with_bp) {
      // p_new = z + beta p and B p_new into the other p buffer (even/odd iterations
      // alternate, so after the even number of iterations between polls W.p is current)
      void* pold = cur ? W.p2 : W.p;
      pcur = cur ? W.p : W.p2;
      KLAUNCH(h, launch_pxb_update(h->g, prec, xprec, W.xlo, pold, pcur, W.bp, W.z, h->scal + S_A,
                                   zz_new, zz_old, kScal, nb, fx, fi,
                                   cv.ptr(prec, cv.layout->bdiag_off()),
                                   cv.ptr(prec, cv.layout->boff_off()), cv.cstride, s, h->d_active,
                                   first ? 0 : 1));
    } else if (first) {
      KLAUNCH(h, launch_p_update(h->g, prec, W.p, W.z, zz_new, zz_old, kScal, nb, fi, s, h->d_active));
    } else {
      KLAUNCH(h, launch_px_update(h->g, prec, xprec, W.xlo, W.p, W.z, h->scal + S_A, zz_new, zz_old,
                                  kScal, nb, fx, fi, s, h->d_active));
    }
    if ((r = mark(first, true, 0))) return r;
    if (with_bp) {
      if ((r = apply_dbb_bp(h, cv, prec, W.w, pcur, W.bp, W.tr, nb, &red_ww, s))) return r;
    } else if ((r = apply_dbb(h, cv, prec, W.w, W.p, W.tr, nb, &red_ww, s))) {
      return r;
    }
    if ((r = mark(first, false, 0))) return r;
    RUpdateLaunch U{};
    U.prec = prec;
    U.r = W.r;
    U.rhat = W.tb;
    U.w = W.w;
    U.stride = fi;
    U.nrhs = nb;
    U.chain = cv.ptr(prec, cv.layout->chain_off());
    U.cstride = cv.cstride;
    U.num = zz_new;
    U.den = h->scal + S_WW;
    U.a_out = h->scal + S_A;
    U.sstride = kScal;
    U.red = &red_rr;
    U.active = h->d_active;
    KLAUNCH(h, launch_rupdate(h->g, U, s));
    return DWF_OK;
  };
  auto flush_x = [&]() -> int {
    if (fused)
      KLAUNCH(h, launch_x_update(h->g, prec, xprec, W.xlo, W.p, h->scal + S_A, kScal, nb, fx, fi, s,
                                 h->d_active));
    return DWF_OK;
  };
  auto enqueue_iter = [&](int cur, bool first) -> int {
    if (fused) return enqueue_fused(cur, first);
    const int nxt = 1 - cur;
    int r;
    if ((r = mark(first, true, 1))) return r;
    if (form != DWF_SCHUR_PRECOND) {  // z = D_bb^+ L^T r
      if ((r = apply_local_dense(h, cv, prec, LTw, tb2, W.r, nb, nullptr, s))) return r;
      if ((r = apply_dbb_dag(h, cv, prec, W.z, tb2, W.tr, W.tb, nb, &red_zz[nxt], s))) return r;
    } else if ((r = apply_dbb_dag(h, cv, prec, W.z, W.r, W.tr, W.tb, nb, &red_zz[nxt], s))) {
      return r;
    }
    if ((r = mark(first, false, 1))) return r;
    KLAUNCH(h, launch_p_update(h->g, prec, W.p, W.z, h->scal + (nxt ? S_ZZ1 : S_ZZ0),
                               h->scal + (cur ? S_ZZ1 : S_ZZ0), kScal, nb, fi, s, h->d_active));
    if ((r = mark(first, true, 0))) return r;
    if (form != DWF_SCHUR_PRECOND) {  // w = L D_bb p
      if ((r = apply_dbb(h, cv, prec, tb2, W.p, W.tr, nb, nullptr, s))) return r;
      if ((r = apply_local_dense(h, cv, prec, Lw, W.w, tb2, nb, &red_ww, s))) return r;
    } else if ((r = apply_dbb(h, cv, prec, W.w, W.p, W.tr, nb, &red_ww, s))) {
      return r;
    }
    if ((r = mark(first, false, 0))) return r;
    KLAUNCH(h, launch_xr_update(h->g, prec, xprec, W.xlo, W.r, W.p, W.w,
                                h->scal + (nxt ? S_ZZ1 : S_ZZ0), h->scal + S_WW, kScal, nb, fx, fi,
                                &red_rr, s, h->d_active));
    return DWF_OK;
  };
  int check = std::max(2, h->check);
  if (check & 1) check++;
  const bool use_graph = h->opt.graph != 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long lpc = 0;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  };
  if (use_graph) {
    const long long l0 = h->launches;
    CUCHK(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    int cur = 0;
    for (int k = 0; k <= check; k++) {
      if ((rc = k < check ? enqueue_iter(cur, k == 0) : flush_x())) {
        cudaStreamEndCapture(s, &graph);
        cleanup();
        return rc;
      }
      cur = 1 - cur;
    }
    CUCHK(h, cudaStreamEndCapture(s, &graph));
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      cleanup();
      return fail(h, DWF_ERR_CUDA, "cudaGraphInstantiate failed");
    }
    lpc = h->launches - l0;
    h->launches = l0;
  }
  int it = 0;
  bool any_active = std::any_of(act.begin(), act.end(), [](int a) { return a != 0; });
  while (any_active && it < maxiter) {
    if (use_graph) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess) {
        cleanup();
        return fail(h, DWF_ERR_CUDA, "cudaGraphLaunch failed");
      }
      h->launches += lpc;
    } else {
      int cur = 0;
      for (int k = 0; k < check; k++) {
        if ((rc = enqueue_iter(cur, k == 0))) return rc;
        cur = 1 - cur;
      }
      if ((rc = flush_x())) return rc;
    }
    it += check;
    for (int r = 0; r < nb; r++)
      if (act[r]) its[r] += check;
    if ((rc = sync_read(h, nb, s)) || (rc = timer_harvest(h, use_graph))) {
      cleanup();
      return rc;
    }
    bool update = false, update32 = false, changed = false;
    std::vector<int> upd(nb, 0), upd32(nb, 0);
    for (int r = 0; r < nb; r++) {
      if (!act[r]) continue;
      const double rr = h->pinned[(size_t)r * kScal + S_RR], ww = h->pinned[(size_t)r * kScal + S_WW];
      if (!std::isfinite(rr) || !std::isfinite(ww) || !(ww > 0.0)) {
        act[r] = 0;
        code[r] = DWF_ERR_BREAKDOWN;
        changed = true;
        continue;
      }
      const double rn = std::sqrt(rr);
      if (rn < delta * rmax[r] || rn <= tol * bnorm[r] || it >= maxiter) {
        if (tiered && !esc[r] && rn > h->tier_eta * anchor[r] && rn > tol * bnorm[r] &&
            it < maxiter) {
          upd32[r] = 1;
          update32 = true;
        } else {
          upd[r] = 1;
          update = true;
        }
      }
    }
    if (update32) {
      // FP32-tier replacement: r = r_64 - D x_lo (x_lo keeps accumulating)
      if ((rc = push_mask(upd32)) ||
          (rc = apply_dbb(h, cv, P32, W.t64, W.xlo, W.t64r, nb, nullptr, s))) {
        cleanup();
        return rc;
      }
      KLAUNCH(h, launch_sub_to(h->g, prec, W.r, W.r_hi, W.t64, nb, fi, f64, fx, &red_rr, s,
                               h->d_active));
      if (fused && (rc = apply_hat(h, cv, prec, W.tb, W.r, nb, s))) {
        cleanup();
        return rc;
      }
      if ((rc = sync_read(h, nb, s))) {
        cleanup();
        return rc;
      }
      std::vector<int> restarted(nb, 0);
      for (int r = 0; r < nb; r++) {
        if (!upd32[r]) continue;
        const double rn = std::sqrt(h->pinned[(size_t)r * kScal + S_RR]);
        n32[r]++;
        if (!std::isfinite(rn)) {
          act[r] = 0;
          code[r] = DWF_ERR_BREAKDOWN;
          continue;
        }
        rmax[r] = rn;
        // no 10% gain over the best FP32-tier residual: the next replacement is FP64
        if (rn < 0.9 * best32[r]) best32[r] = rn;
        else esc[r] = 1;
        if (restart) restarted[r] = 1;
      }
      if (std::any_of(restarted.begin(), restarted.end(), [](int v) { return v != 0; }) &&
          (rc = reset_beta(restarted))) {
        cleanup();
        return rc;
      }
      changed = true;
    }
    if (changed && !update && (rc = push_active())) {
      cleanup();
      return rc;
    }
    if (update) {
      // reliable update of the right-hand sides that reached their threshold (the
      // device mask selects them): x_hi += x_lo, r = b - D x_hi (FP64)
      if ((rc = push_mask(upd))) {
        cleanup();
        return rc;
      }
      KLAUNCH(h, launch_accumulate64(h->g, W.x_hi, xprec, W.xlo, 1, nb, f64, fx, s, h->d_active));
      if (form != DWF_SCHUR_PRECOND) {
        if ((rc = apply_dbb(h, cv, P64, t64b, W.x_hi, W.t64r, nb, nullptr, s)) ||
            (rc = apply_local_dense(h, cv, P64, Lw, W.t64, t64b, nb, nullptr, s))) {
          cleanup();
          return rc;
        }
      } else if ((rc = apply_dbb(h, cv, P64, W.t64, W.x_hi, W.t64r, nb, nullptr, s))) {
        cleanup();
        return rc;
      }
      KLAUNCH(h, launch_sub64_norm(h->g, W.r_hi, W.b_hi, W.t64, nb, f64, &red_hi, s, h->d_active));
      KLAUNCH(h, launch_convert(h->g, prec, W.r, P64, W.r_hi, nb, fi, f64, nullptr, s, h->d_active));
      if (fused && (rc = apply_hat(h, cv, prec, W.tb, W.r, nb, s))) {
        cleanup();
        return rc;
      }
      if ((rc = sync_read(h, nb, s))) {
        cleanup();
        return rc;
      }
      std::vector<int> restarted(nb, 0);
      for (int r = 0; r < nb; r++) {
        if (!upd[r]) continue;
        const double rrh = h->pinned[(size_t)r * kScal + S_RRHI];
        true_res[r] = std::sqrt(rrh) / bnorm[r];
        rmax[r] = std::sqrt(rrh);
        anchor[r] = best32[r] = rmax[r];
        esc[r] = 0;
        rst[r]++;
        if (true_res[r] <= tol) {
          conv[r] = 1;
          act[r] = 0;
          t_done[r] = now_s();
          continue;
        }
        // A replacement without a 10% gain of the true residual means the
        // low-precision recurrence has lost conjugacy: restart it (beta = 0).
        // Five such replacements in a row: stagnation, stop.
        if (true_res[r] < 0.9 * best[r]) {
          best[r] = true_res[r];
          stalled[r] = 0;
        } else if (++stalled[r] >= 5) {
          act[r] = 0;
          code[r] = DWF_ERR_NOT_CONVERGED;
          t_done[r] = now_s();
          continue;
        } else {
          restarted[r] = 1;
        }
        if (restart) restarted[r] = 1;
      }
      if (std::any_of(restarted.begin(), restarted.end(), [](int v) { return v != 0; }) &&
          (rc = reset_beta(restarted))) {
        cleanup();
        return rc;
      }
      if ((rc = push_active())) {
        cleanup();
        return rc;
      }
    }
    any_active = std::any_of(act.begin(), act.end(), [](int a) { return a != 0; });
  }
  cleanup();
  int result = DWF_OK;
  for (int r = 0; r < nb; r++) {
    if (!conv[r] && !code[r]) code[r] = DWF_ERR_NOT_CONVERGED;
    if (code[r] == DWF_ERR_BREAKDOWN) result = DWF_ERR_BREAKDOWN;
    else if (code[r] && result == DWF_OK) result = code[r];
    if (st) {
      st[r].iterations = its[r];
      st[r].restarts = rst[r];
      st[r].true_resid = true_res[r];
      st[r].applies = its[r];
      st[r].applies_dag = its[r];
      st[r].applies_fp64 = rst[r];
      st[r].applies_fp32 = n32[r];
      st[r].apply_ms = h->timed_ms[0];
      st[r].apply_dag_ms = h->timed_ms[1];
      st[r].applies_timed = h->timed_n[0];
      st[r].kernel_launches = (int)(h->launches - launches0);
      st[r].seconds = t_done[r] >= 0.0 ? t_done[r] : now_s();
    }
  }
  if (result == DWF_ERR_BREAKDOWN) return fail(h, result, "CG breakdown (|Dp|^2 <= 0 or not finite)");
  if (result)
    return fail(h, result,
                "CG did not reach the tolerance (maxiter reached or the true residual stagnated)");
  return DWF_OK;
}

// CG on A x = phi with A = D_bb^+ D_bb (Hestenes-Stiefel), inner precision prec
// with FP64 reliable updates of the normal residual phi - A x_hi.  phi in
// W.b_hi, solution in W.x_hi (FP64 black fields).  Per iteration: w = D p
// (|w|^2 = p^+ A p), z = D^+ w, x += a p, r -= a z, p = r + beta p.
int cgnormal_solve(dwf_ctx* h, const MatSet& ms, int prec, double tol, int maxiter, double delta,
                   SolveWork& W, void* t64b, dwf_stats* st, cudaStream_t s) {
  const int xprec = (prec == P16 || prec == PB16) ? P32 : prec;
  const size_t f64 = field_bytes(h->g, P64), fi = field_bytes(h->g, prec),
               fx = field_bytes(h->g, xprec);
  Reduce red_ww = make_reduce(h, 0, S_WW);
  Reduce red_rr[2] = {make_reduce(h, 1, S_ZZ0), make_reduce(h, 1, S_ZZ1)};
  Reduce red_hi = make_reduce(h, 3, S_RRHI), red_bb = make_reduce(h, 3, S_BB);
  int rc;
  const long long launches0 = h->launches;
  int n_app = 0, n_dag = 0, n_64 = 0;
  CUCHK(h, cudaMemsetAsync(W.x_hi, 0, f64, s));
  CUCHK(h, cudaMemsetAsync(W.xlo, 0, fx, s));
  KLAUNCH(h, launch_convert(h->g, P64, W.r_hi, P64, W.b_hi, 1, f64, f64, &red_bb, s));
  int cur = 0;
  KLAUNCH(h, launch_convert(h->g, prec, W.r, P64, W.b_hi, 1, fi, f64, &red_rr[cur], s));
  if ((rc = sync_read(h, 1, s))) return rc;
  const double bb = h->pinned[S_BB];
  auto fill = [&](int it, int restarts, double res) {
    if (!st) return;
    st->iterations = it;
    st->restarts = restarts;
    st->true_resid = res;
    st->applies = n_app;
    st->applies_dag = n_dag;
    st->applies_fp64 = n_64;
    st->kernel_launches = (int)(h->launches - launches0);
  };
  if (!(bb > 0.0)) {
    fill(0, 0, 0.0);
    return bb == 0.0 ? DWF_OK : fail(h, DWF_ERR_BREAKDOWN, "source norm is not finite");
  }
  const double bnorm = std::sqrt(bb);
  CUCHK(h, cudaMemcpyAsync(W.p, W.r, fi, cudaMemcpyDeviceToDevice, s));
  double rmax = bnorm, true_res = 1.0, best_res = 1.0;
  int it = 0, restarts = 0, stalled = 0;
  bool converged = false;
  const int check = std::max(1, h->check);
  while (it < maxiter) {
    if ((rc = apply_dbb(h, view_of(ms), prec, W.w, W.p, W.tr, 1, &red_ww, s))) return rc;
    if ((rc = apply_dbb_dag(h, view_of(ms), prec, W.z, W.w, W.tr, W.tb, 1, nullptr, s))) return rc;
    n_app++;
    n_dag++;
    const int nxt = 1 - cur;
    KLAUNCH(h, launch_xr_update(h->g, prec, xprec, W.xlo, W.r, W.p, W.z,
                                h->scal + (cur ? S_ZZ1 : S_ZZ0), h->scal + S_WW, kScal, 1, fx, fi,
                                &red_rr[nxt], s));
    it++;
    if (it % check == 0 || it >= maxiter) {
      if ((rc = sync_read(h, 1, s))) return rc;
      const double rr = h->pinned[nxt ? S_ZZ1 : S_ZZ0], ww = h->pinned[S_WW];
      if (!std::isfinite(rr) || !std::isfinite(ww) || !(ww > 0.0)) {
        fill(it, restarts, true_res);
        return fail(h, DWF_ERR_BREAKDOWN, "CG breakdown (p^+ A p <= 0 or not finite)");
      }
      const double rn = std::sqrt(rr);
      if (rn < delta * rmax || rn <= tol * bnorm || it >= maxiter) {
        KLAUNCH(h, launch_accumulate64(h->g, W.x_hi, xprec, W.xlo, 1, 1, f64, fx, s));
        if ((rc = apply_dbb(h, view_of(ms), P64, W.t64, W.x_hi, W.t64r, 1, nullptr, s))) return rc;
        if ((rc = apply_dbb_dag(h, view_of(ms), P64, t64b, W.t64, W.t64r, W.r_hi, 1, nullptr, s))) return rc;
        n_64 += 2;
        KLAUNCH(h, launch_sub64_norm(h->g, W.r_hi, W.b_hi, t64b, 1, f64, &red_hi, s));
        KLAUNCH(h, launch_convert(h->g, prec, W.r, P64, W.r_hi, 1, fi, f64, &red_rr[nxt], s));
        if ((rc = sync_read(h, 1, s))) return rc;
        true_res = std::sqrt(h->pinned[S_RRHI]) / bnorm;
        rmax = std::sqrt(h->pinned[S_RRHI]);
        restarts++;
        if (true_res <= tol) {
          converged = true;
          break;
        }
        if (true_res < 0.9 * best_res) {
          best_res = true_res;
          stalled = 0;
        } else if (++stalled >= 3) {
          break;
        }
        if (it >= maxiter) break;
      }
    }
    KLAUNCH(h, launch_p_update(h->g, prec, W.p, W.r, h->scal + (nxt ? S_ZZ1 : S_ZZ0),
                               h->scal + (cur ? S_ZZ1 : S_ZZ0), kScal, 1, fi, s));
    cur = nxt;
  }
  fill(it, restarts, true_res);
  if (!converged)
    return fail(h, DWF_ERR_NOT_CONVERGED,
                "CG did not reach the tolerance (maxiter reached or the true residual stagnated)");
  return DWF_OK;
}

// Effective solver settings.  reliable_delta <= 0 and check_every <= 0 select
// precision-dependent defaults, measured on 8^4 x 16 point-source solves:
//   FP32: delta 0.01, poll every 16 iterations (delta 0.1 .. 0.002 give the same
//         iteration counts on 16^3x32 and the Zolotarev 24^3x48 system; 0.01
//         needs the fewest FP64 replacements without costing iterations there);
//   FP16: delta 0.5, every 4 (its 11-bit significand drifts from the true
//         residual within a few iterations);
//   BF16: delta 0.5, every 4, and the reliable-update solver restarts the
//         recurrence at every replacement (defect correction): with an 8-bit
//         significand the unrestarted recurrence loses conjugacy, and at
//         delta 0.1 the inner solve of a Zolotarev m = 0.005 system never
//         reached its threshold.
int solver_params(dwf_ctx* h, int* prec, double* delta, bool* restart) {
  *prec = h->opt.precision_inner;
  const bool b16 = *prec == PB16, half = *prec == P16 || b16;
  *delta = h->opt.reliable_delta > 0.0 ? h->opt.reliable_delta : (half ? 0.5 : 0.01);
  h->check = h->opt.check_every > 0 ? h->opt.check_every : (half ? 4 : 16);
  *restart = b16;
  if (h->opt.solver == DWF_SOLVER_FP64) {
    *prec = P64;
    *delta = 0.0;
    *restart = false;
  } else if (h->opt.solver == DWF_SOLVER_DEFECT) {
    *restart = true;
  }
  return DWF_OK;
}

// Autotuner of the launch shapes of the solver: times the (batched) D_bb apply
// of the inner precision for every right-hand-side block size that fits in free
// device memory (batched solves), every CTA tile of the tuned hop kernels
// (default and small) and both neighbour staging variants (direct loads,
// tensor-copy staging), and keeps the fastest per right-hand side (within 3%,
// the larger block).  Results are cached per (lattice, Ls, precision, nrhs) in
// the handle and, if DWF_AUTOTUNE_CACHE names a file, there as
// "key nb staging tile" lines.  An explicit rhs_block option fixes the block;
// DWF_TMA (set at dwf_create) fixes the staging.
int choose_rhs_block(dwf_ctx* h, int nrhs, int prec, cudaStream_t st, int* nb_out) {
  const int Ls = h->g.Ls;
  const bool tuned = !g_disable_tuned && (Ls == 8 || Ls == 12 || Ls == 16);
  const bool fixed_nb = h->opt.rhs_block > 0 || nrhs == 1;
  const int fnb = nrhs == 1 ? 1 : std::min(std::max(h->opt.rhs_block, 1), nrhs);
  if (!tuned) {  // one generic kernel shape: only the block is tuned (or fixed)
    if (fixed_nb) {
      *nb_out = fnb;
      return DWF_OK;
    }
  }
  std::ostringstream key;
  key << "v2_" << h->g.L[0] << "x" << h->g.L[1] << "x" << h->g.L[2] << "x" << h->g.L[3] << "_Ls" << Ls
      << "_p" << prec << "_n" << nrhs << "_b" << (fixed_nb ? fnb : 0) << "_t" << h->env_tma
      << "_s" << h->env_tile;
  auto it = h->tune.find(key.str());
  const char* cache_file = std::getenv("DWF_AUTOTUNE_CACHE");
  if (it == h->tune.end() && cache_file) {
    std::ifstream in(cache_file);
    std::string k;
    int nb, tma, tile;
    while (in >> k >> nb >> tma >> tile)
      if (k == key.str()) h->tune[k] = dwf_ctx::Tuned{nb, tma, tile};
    it = h->tune.find(key.str());
  }
  if (it != h->tune.end()) {
    *nb_out = std::min(it->second.nb, nrhs);
    h->use_tma = it->second.tma;
    h->tile = it->second.tile;
    return DWF_OK;
  }
  std::vector<int> ok;
  if (fixed_nb) {
    ok.push_back(fnb);
  } else {
    size_t freeb = 0, totalb = 0;
    CUCHK(h, cudaMemGetInfo(&freeb, &totalb));
    const size_t per = solve_bytes_per_rhs(h->g, prec) + 3 * field_bytes(h->g, prec);
    const double budget = 0.8 * (double)freeb;
    const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    for (int c : cand)
      if (c <= nrhs && (double)c * per <= budget) ok.push_back(c);
    if (ok.empty()) ok.push_back(1);
  }
  const int maxnb = ok.back();
  const size_t fi = field_bytes(h->g, prec);
  void *x, *y, *t;
  int rc;
  if ((rc = get_ws(h, "tune_x", fi * maxnb, &x)) || (rc = get_ws(h, "tune_y", fi * maxnb, &y)) ||
      (rc = get_ws(h, "tune_t", fi * maxnb, &t)))
    return rc;
  CUCHK(h, cudaMemsetAsync(x, 0, fi * maxnb, st));
  MatSet* ms;
  if ((rc = build_matset(h, h->alpha, h->m, &ms))) return rc;
  cudaEvent_t e0, e1;
  CUCHK(h, cudaEventCreate(&e0));
  CUCHK(h, cudaEventCreate(&e1));
  std::vector<int> tmas = {h->env_tma};
  std::vector<int> tiles = {h->env_tile >= 0 ? h->env_tile : 0};
  if (tuned) {
    if (!h->env_tma) tmas.push_back(1);
    if (h->env_tile < 0) tiles.push_back(hop2::small_block_sites(Ls));
  }
  double best = 1e300;
  int best_nb = ok.front(), best_tma = tmas.front(), best_tile = 0;
  const bool single = ok.size() == 1 && tmas.size() == 1 && (tiles.size() == 1 || tmas[0]);
  best_tile = tiles.front();
  if (!single)
  for (int nb : ok)
    for (int tma : tmas)
      for (int tile : tiles) {
        if (tma && tile) continue;  // the staged variant has one tile
        h->use_tma = tma;
        h->tile = tile;
        if ((rc = apply_dbb(h, view_of(*ms), prec, y, x, t, nb, nullptr, st))) return rc;
        // best of two timed passes of 3 applies (one slow pass does not decide)
        double per_rhs = 1e300;
        for (int pass = 0; pass < 2; pass++) {
          CUCHK(h, cudaEventRecord(e0, st));
          for (int k = 0; k < 3; k++)
            if ((rc = apply_dbb(h, view_of(*ms), prec, y, x, t, nb, nullptr, st))) return rc;
          CUCHK(h, cudaEventRecord(e1, st));
          CUCHK(h, cudaEventSynchronize(e1));
          float ms_t = 0.f;
          CUCHK(h, cudaEventElapsedTime(&ms_t, e0, e1));
          per_rhs = std::min(per_rhs, ms_t / (3.0 * nb));
        }
        if (per_rhs < 0.97 * best || (per_rhs <= best * 1.03 && nb > best_nb)) {
          if (per_rhs < best) best = per_rhs;
          best_nb = nb;
          best_tma = tma;
          best_tile = tile;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->use_tma = best_tma;
  h->tile = best_tile;
  h->tune[key.str()] = dwf_ctx::Tuned{best_nb, best_tma, best_tile};
  if (cache_file) {
    // handles tuned on several host threads at once append whole lines
    static std::mutex cache_mutex;
    std::lock_guard<std::mutex> lock(cache_mutex);
    std::ofstream out(cache_file, std::ios::app);
    out << key.str() << " " << best_nb << " " << best_tma << " " << best_tile << "\n";
  }
  *nb_out = best_nb;
  return DWF_OK;
}

}  // namespace

extern "C" {

int dwf_default_options(dwf_options* opt) {
  if (!opt) return DWF_ERR_INVALID_ARG;
  opt->precision_inner = DWF_FP32;
  opt->rb_parity = 0;
  opt->bc_t = 1;
  opt->rel_tol = 1e-10;
  opt->maxiter = 100000;
  opt->reliable_delta = 0.0;
  opt->solver = DWF_SOLVER_RELIABLE;
  opt->check_every = 0;
  opt->profile = 0;
  opt->graph = 1;
  opt->rhs_block = 0;
  opt->schur_form = DWF_SCHUR_PRECOND;
  return DWF_OK;
}

int dwf_create(dwf_handle* out, const int lattice[4], int Ls, double M5, double m, double alpha,
               const double* b, const double* c, const dwf_options* opt) {
  if (!out || !lattice || !b || !c) return fail(nullptr, DWF_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  for (int k = 0; k < 4; k++)
    if (lattice[k] < 2 || lattice[k] % 2)
      return fail(nullptr, DWF_ERR_INVALID_ARG, "lattice extents must be even and >= 2");
  if (Ls < 2 || Ls > kMaxLs) return fail(nullptr, DWF_ERR_INVALID_ARG, "Ls must be in [2, 32]");
  const double V = (double)lattice[0] * lattice[1] * lattice[2] * lattice[3];
  if (V / 2 * Ls * 24 > 2147483647.0)
    return fail(nullptr, DWF_ERR_INVALID_ARG, "lattice too large for 32-bit 5D indexing");
  dwf_ctx* h = new dwf_ctx();
  for (int k = 0; k < 4; k++) h->g.L[k] = lattice[k];
  h->g.Lxh = lattice[0] / 2;
  h->g.Vh = (int)(V / 2);
  h->g.Ls = Ls;
  h->g.N5 = h->g.Vh * Ls;
  h->Ls = Ls;
  h->M5 = M5;
  h->m = m;
  h->alpha = alpha;
  h->b.assign(b, b + Ls);
  h->c.assign(c, c + Ls);
  dwf_default_options(&h->opt);
  if (opt) h->opt = *opt;
  if (h->opt.bc_t != 1 && h->opt.bc_t != -1) {
    delete h;
    return fail(nullptr, DWF_ERR_INVALID_ARG, "bc_t must be +1 or -1");
  }
  if (h->opt.schur_form < DWF_SCHUR_PRECOND || h->opt.schur_form > DWF_SCHUR_ROWSCALED) {
    delete h;
    return fail(nullptr, DWF_ERR_INVALID_ARG, "schur_form must be 0, 1 or 2");
  }
  if (!valid_prec(h->opt.precision_inner) || (h->opt.rb_parity != 0 && h->opt.rb_parity != 1)) {
    delete h;
    return fail(nullptr, DWF_ERR_INVALID_ARG, "bad precision_inner or rb_parity");
  }
  h->g.bc_t = h->opt.bc_t;
  // DWF_GENERIC_KERNELS=1 selects the generic (any Ls, dense 5th-dimension)
  // kernels instead of the tuned ones; used to cross-check the two paths.
  g_disable_tuned = std::getenv("DWF_GENERIC_KERNELS") != nullptr;
  // DWF_TMA=1 stages the neighbour blocks of the tuned kernels through shared
  // memory with tensor copies (measured slower than direct loads on the
  // 16^3x32 workload; kept as an alternative staging strategy).
  h->use_tma = std::getenv("DWF_TMA") != nullptr;
  h->env_tma = h->use_tma;
  // DWF_HOP_TILE=small|default fixes the CTA tile of the tuned hop kernels
  if (const char* e = std::getenv("DWF_HOP_TILE")) {
    const bool tuned_ls = Ls == 8 || Ls == 12 || Ls == 16;
    h->env_tile = (std::string(e) == "small" && tuned_ls) ? hop2::small_block_sites(Ls) : 0;
    h->tile = h->env_tile;
  }
  h->bp_fused = std::getenv("DWF_NO_BP_FUSED") == nullptr;
  if (const char* e = std::getenv("DWF_TIER_ETA")) h->tier_eta = std::atof(e);
  if (const char* e = std::getenv("DWF_WAIT_BUDGET")) h->wait_budget = std::atoll(e);
  if (const char* e = std::getenv("DWF_TEST_SKIP_HOP")) h->skip_hop = std::atoi(e);
  h->fused_cg = std::getenv("DWF_UNFUSED_CG") == nullptr;
  cudaGetDevice(&h->device);
  // address of the static scratch of dwf_apply_Dbb_noalloc on this device
  if (noalloc_scratch_address(&h->noalloc_scratch) != cudaSuccess) {
    cudaGetLastError();
    h->noalloc_scratch = nullptr;
  }
  if (cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(nullptr, DWF_ERR_CUDA, "stream creation failed");
  }
  MatSet* ms;
  int rc = build_matset(h, alpha, m, &ms);
  if (!rc) rc = build_matset(h, 1.0, 1.0, &ms);
  if (rc) {
    g_create_error = h->err;
    dwf_destroy(h);
    return rc;
  }
  {
    // neighbour table: for each parity p and half index h the half indices of
    // x+mu and x-mu (mu = x, y, z, t), bit 31 set where the hop crosses the t
    // boundary with antiperiodic fermions
    const int Lx = lattice[0], Ly = lattice[1], Lz = lattice[2], Lt = lattice[3];
    const int Vh = h->g.Vh, Lxh = Lx / 2;
    std::vector<int> tab((size_t)2 * Vh * 8);
    for (int p = 0; p < 2; p++)
      for (int hh = 0; hh < Vh; hh++) {
        const int xh = hh % Lxh;
        int r = hh / Lxh;
        const int y = r % Ly;
        r /= Ly;
        const int z = r % Lz, t = r / Lz;
        const int x = 2 * xh + ((y + z + t + p) & 1);
        int* e = &tab[((size_t)p * Vh + hh) * 8];
        const int c[4] = {x, y, z, t}, L4[4] = {Lx, Ly, Lz, Lt};
        for (int mu = 0; mu < 4; mu++)
          for (int d = 0; d < 2; d++) {
            int cc[4] = {c[0], c[1], c[2], c[3]};
            const int step = d == 0 ? 1 : -1;
            cc[mu] += step;
            bool cross = false;
            if (cc[mu] < 0) { cc[mu] += L4[mu]; cross = true; }
            if (cc[mu] >= L4[mu]) { cc[mu] -= L4[mu]; cross = true; }
            int idx = (cc[0] >> 1) + Lxh * (cc[1] + Ly * (cc[2] + Lz * cc[3]));
            if (mu == 3 && cross && h->opt.bc_t < 0) idx |= (int)0x80000000u;
            e[mu * 2 + d] = idx;
          }
      }
    if (cudaMalloc(&h->dev_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->dev_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->nbr, tab.size() * sizeof(int)) != cudaSuccess ||
        cudaMemcpy(h->nbr, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      dwf_destroy(h);
      return fail(nullptr, DWF_ERR_OOM, "neighbour table allocation failed");
    }
  }
  for (int p = 0; p < 3; p++) {
    const int prec = p == 0 ? P64 : (p == 1 ? P32 : P16);
    if (cudaMalloc(&h->gauge[p], gauge_bytes(h->g, prec)) != cudaSuccess) {
      cudaGetLastError();
      dwf_destroy(h);
      return fail(nullptr, DWF_ERR_OOM, "gauge allocation failed");
    }
  }
  *out = h;
  return DWF_OK;
}

int dwf_destroy(dwf_handle h) {
  if (!h) return DWF_OK;
  for (void* p : h->allocs) cudaFree(p);
  for (auto& kv : h->ws) cudaFree(kv.second);
  for (int p = 0; p < 3; p++) cudaFree(h->gauge[p]);
  if (h->nbr) cudaFree(h->nbr);
  if (h->dev_err) cudaFree(h->dev_err);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  if (h->d_active) {
    cudaFree(h->d_active);
    cudaFreeHost(h->pinned_i);
  }
  if (h->scal) {
    cudaFree(h->scal);
    cudaFree(h->partial);
    cudaFree(h->counter);
    cudaFreeHost(h->pinned);
  }
  delete h;
  return DWF_OK;
}

const char* dwf_last_error(dwf_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int dwf_field_bytes(dwf_handle h, int prec, size_t* bytes) {
  if (!h || !bytes || !valid_prec(prec)) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  *bytes = field_bytes(h->g, prec);
  return DWF_OK;
}

int dwf_load_gauge(dwf_handle h, const double* U, int is_device, dwf_stream s) {
  if (!h || !U) return fail(h, DWF_ERR_INVALID_ARG, "null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  const size_t bytes = (size_t)h->g.Vh * 2 * 4 * 9 * 16;
  const double* src = U;
  if (!is_device) {
    void* tmp;
    int rc = get_ws(h, "gauge_in", bytes, &tmp);
    if (rc) return rc;
    CUCHK(h, cudaMemcpyAsync(tmp, U, bytes, cudaMemcpyHostToDevice, st));
    src = reinterpret_cast<const double*>(tmp);
  }
  KLAUNCH(h, launch_gauge_convert(h->g, src, h->gauge[0], h->gauge[1], h->gauge[2], st));
  h->gauge_loaded = true;
  return DWF_OK;
}

int dwf_pack_half(dwf_handle h, void* dst, const double* src, int prec, int nrhs, dwf_stream s) {
  if (!h || !dst || !src || !valid_prec(prec) || nrhs < 1)
    return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  KLAUNCH(h, launch_pack_half(h->g, prec, dst, src, nrhs, reinterpret_cast<cudaStream_t>(s)));
  return DWF_OK;
}

int dwf_unpack_half(dwf_handle h, double* dst, const void* src, int prec, int nrhs, dwf_stream s) {
  if (!h || !dst || !src || !valid_prec(prec) || nrhs < 1)
    return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  KLAUNCH(h, launch_unpack_half(h->g, prec, dst, src, nrhs, reinterpret_cast<cudaStream_t>(s)));
  return DWF_OK;
}

int dwf_apply_Dbb(dwf_handle h, void* out, const void* in, int prec, int nrhs, dwf_stream s) {
  if (!h || !out || !in || !valid_prec(prec) || nrhs < 1 || out == in)
    return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  MatSet* ms;
  int rc = build_matset(h, h->alpha, h->m, &ms);
  if (rc) return rc;
  void* tmp;
  if ((rc = get_ws(h, "apply_red_" + std::to_string(prec), field_bytes(h->g, prec) * nrhs, &tmp))) return rc;
  return apply_dbb(h, view_of(*ms), prec, out, in, tmp, nrhs, nullptr, reinterpret_cast<cudaStream_t>(s));
}

int dwf_apply_Dbb_dag(dwf_handle h, void* out, const void* in, int prec, int nrhs, dwf_stream s) {
  if (!h || !out || !in || !valid_prec(prec) || nrhs < 1 || out == in)
    return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  MatSet* ms;
  int rc = build_matset(h, h->alpha, h->m, &ms);
  if (rc) return rc;
  void *tr, *tb;
  const size_t fb = field_bytes(h->g, prec) * nrhs;
  if ((rc = get_ws(h, "apply_red_" + std::to_string(prec), fb, &tr))) return rc;
  if ((rc = get_ws(h, "apply_blk_" + std::to_string(prec), fb, &tb))) return rc;
  return apply_dbb_dag(h, view_of(*ms), prec, out, in, tr, tb, nrhs, nullptr, reinterpret_cast<cudaStream_t>(s));
}

int dwf_apply_dalpha(dwf_handle h, double* out_full, const double* in_full, double alpha, double m,
                     dwf_stream s) {
  if (!h || !out_full || !in_full) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  MatSet* ms;
  int rc = build_matset(h, alpha, m, &ms);
  if (rc) return rc;
  const size_t f64 = field_bytes(h->g, P64);
  void *i0, *i1, *o0, *o1;
  if ((rc = get_ws(h, "da_i0", f64, &i0)) || (rc = get_ws(h, "da_i1", f64, &i1)) ||
      (rc = get_ws(h, "da_o0", f64, &o0)) || (rc = get_ws(h, "da_o1", f64, &o1)))
    return rc;
  KLAUNCH(h, launch_split_full(h->g, i0, i1, in_full, st));
  void* outs[2] = {o0, o1};
  const void* ins[2] = {i0, i1};
  if ((rc = apply_dalpha_halves(h, *ms, outs, ins, st))) return rc;
  KLAUNCH(h, launch_merge_full(h->g, out_full, o0, o1, st));
  return DWF_OK;
}

int dwf_solve_normal(dwf_handle h, double* x_half, const double* phi_half, dwf_stats* stats,
                     dwf_stream s) {
  if (!h || !x_half || !phi_half) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  int rc;
  if ((rc = ensure_reduce(h, 1))) return rc;
  int prec;
  double delta;
  bool restart;
  solver_params(h, &prec, &delta, &restart);
  SolveWork W;
  if ((rc = alloc_solve_work(h, prec, W))) return rc;
  void* t64b;
  if ((rc = get_ws(h, "t64b", field_bytes(h->g, P64), &t64b))) return rc;
  MatSet* ms;
  if ((rc = build_matset(h, h->alpha, h->m, &ms))) return rc;
  auto t0 = std::chrono::steady_clock::now();
  KLAUNCH(h, launch_pack_half(h->g, P64, W.b_hi, phi_half, 1, st));
  dwf_stats sk{};
  rc = cgnormal_solve(h, *ms, prec, h->opt.rel_tol, h->opt.maxiter, delta, W, t64b, &sk, st);
  if (rc && rc != DWF_ERR_NOT_CONVERGED) return rc;
  KLAUNCH(h, launch_unpack_half(h->g, P64, x_half, W.x_hi, 1, st));
  CUCHK(h, cudaStreamSynchronize(st));
  sk.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = sk;
  return rc;
}

int dwf_action(dwf_handle h, double* S, const double* phi_half, double* X_half, dwf_stats* stats,
               dwf_stream s) {
  if (!h || !S || !phi_half) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  int rc;
  if ((rc = ensure_reduce(h, 1))) return rc;
  int prec;
  double delta;
  bool restart;
  solver_params(h, &prec, &delta, &restart);
  SolveWork W;
  if ((rc = alloc_solve_work(h, prec, W))) return rc;
  void* t64b;
  if ((rc = get_ws(h, "t64b", field_bytes(h->g, P64), &t64b))) return rc;
  MatSet* ms;
  if ((rc = build_matset(h, h->alpha, h->m, &ms))) return rc;
  auto t0 = std::chrono::steady_clock::now();
  KLAUNCH(h, launch_pack_half(h->g, P64, W.b_hi, phi_half, 1, st));
  dwf_stats sk{};
  rc = cgnormal_solve(h, *ms, prec, h->opt.rel_tol, h->opt.maxiter, delta, W, t64b, &sk, st);
  if (rc && rc != DWF_ERR_NOT_CONVERGED) return rc;
  // S = Re phi^+ X, FP64 device reduction over the black half-lattice
  Reduce red = make_reduce(h, 0, S_T0);
  KLAUNCH(h, launch_dot_re64(h->g, W.b_hi, W.x_hi, 1, field_bytes(h->g, P64), &red, st));
  if (X_half) KLAUNCH(h, launch_unpack_half(h->g, P64, X_half, W.x_hi, 1, st));
  int rc2;
  if ((rc2 = sync_read(h, 1, st))) return rc2;
  *S = h->pinned[S_T0];
  sk.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = sk;
  return rc;
}

// Red-black solves of D_alpha(solve_m) P z = D_1(rhs_m) P b for nrhs sources,
// z_1 -> prop4d: the propagator (solve_m = m, rhs_m = 1) or D_OV(m) b
// (solve_m = 1, rhs_m = m).
static int solve_5d(dwf_ctx* h, const double* src4d, double* prop4d, double* sol5d, int nrhs,
                    const double* alphas, dwf_stats* stats, dwf_stream s, double solve_m,
                    double rhs_m);

int dwf_cgne_solve(dwf_handle h, const double* src4d, double* prop4d, double* sol5d, int nrhs,
                   const double* alphas, dwf_stats* stats, dwf_stream s) {
  if (!h) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  return solve_5d(h, src4d, prop4d, sol5d, nrhs, alphas, stats, s, h->m, 1.0);
}

int dwf_apply_overlap(dwf_handle h, const double* src4d, double* out4d, double* sol5d, int nrhs,
                      const double* alphas, dwf_stats* stats, dwf_stream s) {
  if (!h) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  return solve_5d(h, src4d, out4d, sol5d, nrhs, alphas, stats, s, 1.0, h->m);
}

int dwf_cgne_solve_multi(dwf_solve_job* jobs, int njobs, dwf_stream s) {
  // failures before any job starts: reported on the job's handle and on this thread
  auto reject = [](dwf_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    g_create_error = msg;
    return code;
  };
  if (!jobs || njobs < 1) return reject(nullptr, DWF_ERR_INVALID_ARG, "bad argument");
  for (int i = 0; i < njobs; i++) {
    if (!jobs[i].handle) return reject(nullptr, DWF_ERR_INVALID_ARG, "job without a handle");
    for (int j = 0; j < i; j++)
      if (jobs[j].handle == jobs[i].handle)
        return reject(jobs[i].handle, DWF_ERR_INVALID_ARG,
                      "two jobs of one dwf_cgne_solve_multi call share a handle");
  }
  for (int i = 0; i < njobs; i++) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != jobs[i].handle->device)
      return reject(jobs[i].handle, DWF_ERR_INVALID_ARG, "handle created on another device");
  }
  // the jobs start after the caller's stream; each then runs on its handle's stream
  {
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return reject(jobs[0].handle, DWF_ERR_CUDA, cudaGetErrorString(e));
  }
  int dev = 0;
  cudaGetDevice(&dev);
  auto run = [&](int i) {
    dwf_solve_job& J = jobs[i];
    if (cudaSetDevice(dev) != cudaSuccess) {
      J.status = fail(J.handle, DWF_ERR_CUDA, "cudaSetDevice failed on a worker thread");
      return;
    }
    J.status = solve_5d(J.handle, J.src4d, J.prop4d, J.sol5d, J.nrhs, J.alphas, J.stats,
                        reinterpret_cast<dwf_stream>(J.handle->cstream), J.handle->m, 1.0);
  };
  // one thread per job beyond the first; a job whose thread cannot be started
  // runs on the calling thread (no exception crosses the C ABI)
  std::vector<std::thread> pool;
  std::vector<int> inline_jobs;
  for (int i = 1; i < njobs; i++) {
    try {
      pool.emplace_back(run, i);
    } catch (...) {
      inline_jobs.push_back(i);
    }
  }
  run(0);
  for (int i : inline_jobs) run(i);
  for (auto& t : pool) t.join();
  int rc = DWF_OK;
  for (int i = 0; i < njobs && rc == DWF_OK; i++) rc = jobs[i].status;
  if (rc != DWF_OK)
    for (int i = 0; i < njobs; i++)
      if (jobs[i].status != DWF_OK) {
        g_create_error = "job " + std::to_string(i) + ": " + jobs[i].handle->err;
        break;
      }
  return rc;
}

static int solve_5d(dwf_ctx* h, const double* src4d, double* prop4d, double* sol5d, int nrhs,
                    const double* alphas, dwf_stats* stats, dwf_stream s, double solve_m,
                    double rhs_m) {
  if (!h || !src4d || !prop4d || nrhs < 1) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  // all solver work runs on the handle's stream, after the caller's stream
  CUCHK(h, cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s)));
  cudaStream_t st = h->cstream;
  const Geom& g = h->g;
  const size_t src_bytes = (size_t)g.Vh * 2 * 12 * 16;
  const bool host = !is_device_ptr(src4d);
  int rc;
  int prec;
  double delta;
  bool restart;
  solver_params(h, &prec, &delta, &restart);
  std::vector<MatSet*> ms(nrhs);
  for (int k = 0; k < nrhs; k++)
    if ((rc = build_matset(h, alphas ? alphas[k] : h->alpha, solve_m, &ms[k]))) return rc;
  MatSet* rhs_set;
  if ((rc = build_matset(h, 1.0, rhs_m, &rhs_set))) return rc;
  int nb = 1;
  if ((rc = choose_rhs_block(h, nrhs, prec, st, &nb))) return rc;
  if ((rc = ensure_reduce(h, nb))) return rc;
  SolveWork W;
  if ((rc = alloc_solve_work(h, prec, W, nb))) return rc;
  const size_t f64 = field_bytes(g, P64), cnt = ms[0]->count();
  void *pb[2], *rhs[2], *psi_r, *src_d = nullptr, *prop_d = nullptr, *tmp5[2], *bc64, *bc32;
  if ((rc = get_ws(h, "pb0", f64, &pb[0])) || (rc = get_ws(h, "pb1", f64, &pb[1])) ||
      (rc = get_ws(h, "rhs0", f64, &rhs[0])) || (rc = get_ws(h, "rhs1", f64, &rhs[1])) ||
      (rc = get_ws(h, "psi_r", f64, &psi_r)) || (rc = get_ws(h, "t5a", f64, &tmp5[0])) ||
      (rc = get_ws(h, "t5b", f64, &tmp5[1])) || (rc = get_ws(h, "bcoef64", cnt * 8 * nb, &bc64)) ||
      (rc = get_ws(h, "bcoef32", cnt * 4 * nb, &bc32)))
    return rc;
  if (host) {
    if ((rc = get_ws(h, "src_d", src_bytes, &src_d)) || (rc = get_ws(h, "prop_d", src_bytes, &prop_d)))
      return rc;
  }
  const int black = h->opt.rb_parity, red = 1 - black;
  // rhs = D_1(1) P b for source k (full 5D, FP64) into rhs[0], rhs[1]
  auto make_rhs = [&](int k) -> int {
    const double* src_k = src4d + (size_t)k * src_bytes / 8;
    if (host) {
      CUCHK(h, cudaMemcpyAsync(src_d, src_k, src_bytes, cudaMemcpyHostToDevice, st));
      src_k = reinterpret_cast<const double*>(src_d);
    }
    KLAUNCH(h, launch_source_pb(g, pb[0], pb[1], src_k, st));
    const void* pbc[2] = {pb[0], pb[1]};
    return apply_dalpha_halves(h, *rhs_set, rhs, pbc, st);
  };
  int result = DWF_OK;
  for (int blk = 0; blk < nrhs; blk += nb) {
    const int n = std::min(nb, nrhs - blk);
    auto t0 = std::chrono::steady_clock::now();
    const long long l0 = h->launches;
    for (int r = 0; r < n; r++) {
      const MatSet& m = *ms[blk + r];
      CUCHK(h, cudaMemcpyAsync(reinterpret_cast<char*>(bc64) + r * cnt * 8, m.dev[0], cnt * 8,
                               cudaMemcpyDeviceToDevice, st));
      CUCHK(h, cudaMemcpyAsync(reinterpret_cast<char*>(bc32) + r * cnt * 4, m.dev[1], cnt * 4,
                               cudaMemcpyDeviceToDevice, st));
      if ((rc = make_rhs(blk + r))) return rc;
      // r'_b = I^-1 rhs_b + 1/2 I^-1 H_br (K rhs_r)
      LocalLaunch Lk{};
      Lk.prec = P64;
      Lk.out = W.t64r;
      Lk.in = rhs[red];
      Lk.stride = f64;
      Lk.nrhs = 1;
      Lk.m = m.ptr(P64, m.mat_off(MatSet::K));
      Lk.c = 1.0;
      KLAUNCH(h, launch_local(g, Lk, st));
      HopLaunch Hs = base_hop(h, P64, black, 1, f64);
      Hs.out = reinterpret_cast<char*>(W.b_hi) + r * f64;
      Hs.v = W.t64r;
      Hs.w = rhs[black];
      Hs.post = m.ptr(P64, m.mat_off(MatSet::IINV));
      Hs.loc = LOC_DENSE;
      Hs.locm = m.ptr(P64, m.mat_off(MatSet::IINV));
      Hs.c_hop = 0.5;
      Hs.c_loc = 1.0;
      KLAUNCH(h, launch_hop(g, Hs, st));
    }
    std::vector<dwf_stats> sk(n);
    CoefView cv{ms[blk], {bc64, bc32}, cnt, nullptr};
    rc = cgnr_batched(h, cv, prec, h->opt.rel_tol, h->opt.maxiter, delta, restart, W, n, sk.data(), st);
    if (rc && rc != DWF_ERR_NOT_CONVERGED && rc != DWF_ERR_BREAKDOWN) return rc;
    if (rc) result = rc;
    for (int r = 0; r < n; r++) {
      const int k = blk + r;
      const MatSet& m = *ms[k];
      void* xb = reinterpret_cast<char*>(W.x_hi) + r * f64;
      if ((rc = make_rhs(k))) return rc;
      // psi_r = I^-1 rhs_r + 1/2 I^-1 H_rb (B psi_b)
      HopLaunch Hr = base_hop(h, P64, red, 1, f64);
      Hr.out = psi_r;
      Hr.v = xb;
      Hr.w = rhs[red];
      Hr.pre = PRE_B;
      Hr.pre_diag = m.ptr(P64, m.bdiag_off());
      Hr.pre_off = m.ptr(P64, m.boff_off());
      Hr.post = m.ptr(P64, m.mat_off(MatSet::IINV));
      Hr.loc = LOC_DENSE;
      Hr.locm = m.ptr(P64, m.mat_off(MatSet::IINV));
      Hr.c_hop = 0.5;
      Hr.c_loc = 1.0;
      KLAUNCH(h, launch_hop(g, Hr, st));
      void* psi[2];
      psi[black] = xb;
      psi[red] = psi_r;
      double* prop_k = prop4d + (size_t)k * src_bytes / 8;
      KLAUNCH(h, launch_extract_z1(g, host ? reinterpret_cast<double*>(prop_d) : prop_k, psi[0],
                                   psi[1], st));
      if (host) CUCHK(h, cudaMemcpyAsync(prop_k, prop_d, src_bytes, cudaMemcpyDeviceToHost, st));
      if (sol5d) KLAUNCH(h, launch_merge_full(g, sol5d + (size_t)k * g.N5 * 2 * 24, psi[0], psi[1], st));
      // full 5D residual |rhs - D_alpha psi| / |rhs|
      const void* psic[2] = {psi[0], psi[1]};
      if ((rc = apply_dalpha_halves(h, m, tmp5, psic, st))) return rc;
      Reduce r0 = make_reduce(h, 0, S_T0), r1 = make_reduce(h, 1, S_T1);
      Reduce n0 = make_reduce(h, 2, S_T2), n1 = make_reduce(h, 3, S_ZZ0);
      KLAUNCH(h, launch_sub64_norm(g, tmp5[0], rhs[0], tmp5[0], 1, f64, &r0, st));
      KLAUNCH(h, launch_sub64_norm(g, tmp5[1], rhs[1], tmp5[1], 1, f64, &r1, st));
      KLAUNCH(h, launch_norm(g, P64, rhs[0], 1, f64, &n0, st));
      KLAUNCH(h, launch_norm(g, P64, rhs[1], 1, f64, &n1, st));
      if ((rc = sync_read(h, 1, st))) return rc;
      sk[r].true_resid_5d =
          std::sqrt((h->pinned[S_T0] + h->pinned[S_T1]) / (h->pinned[S_T2] + h->pinned[S_ZZ0]));
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    (void)secs;
    for (int r = 0; r < n; r++) {
      sk[r].kernel_launches = (int)(h->launches - l0);
      if (stats) stats[blk + r] = sk[r];
    }
  }
  CUCHK(h, cudaStreamSynchronize(st));
  if (result == DWF_ERR_NOT_CONVERGED)
    return fail(h, result, "CG did not reach the tolerance for at least one source");
  if (result == DWF_ERR_BREAKDOWN) return fail(h, result, "CG breakdown for at least one source");
  return DWF_OK;
}

int dwf_force(dwf_handle h, double* dSdU, const double* phi_half, const double* X_half,
              int projected, dwf_stream s) {
  if (!h || !dSdU || !phi_half) return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  const Geom& g = h->g;
  int rc;
  MatSet* ms;
  if ((rc = build_matset(h, h->alpha, h->m, &ms))) return rc;
  const size_t f64 = field_bytes(g, P64);
  const int black = h->opt.rb_parity, red = 1 - black;
  void *X, *Y, *eta1, *xi1, *eta2;
  if ((rc = get_ws(h, "f_Y", f64, &Y)) || (rc = get_ws(h, "f_eta1", f64, &eta1)) ||
      (rc = get_ws(h, "f_xi1", f64, &xi1)) || (rc = get_ws(h, "f_eta2", f64, &eta2)) ||
      (rc = get_ws(h, "f_red", f64, &X)))
    return rc;
  void* tred = X;  // red scratch of the FP64 applies
  if (X_half) {
    if ((rc = get_ws(h, "x_hi", f64, &X))) return rc;
    KLAUNCH(h, launch_pack_half(g, P64, X, X_half, 1, st));
  } else {
    // recompute X = (D^+ D)^-1 phi (no solver history is kept)
    if ((rc = ensure_reduce(h, 1))) return rc;
    int prec;
    double delta;
    bool restart;
    solver_params(h, &prec, &delta, &restart);
    SolveWork W;
    if ((rc = alloc_solve_work(h, prec, W))) return rc;
    void* t64b;
    if ((rc = get_ws(h, "t64b", f64, &t64b))) return rc;
    KLAUNCH(h, launch_pack_half(g, P64, W.b_hi, phi_half, 1, st));
    rc = cgnormal_solve(h, *ms, prec, h->opt.rel_tol, h->opt.maxiter, delta, W, t64b, nullptr, st);
    if (rc) return rc;
    X = W.x_hi;
    tred = W.t64r;
  }
  // Y = D_bb X
  if ((rc = apply_dbb(h, view_of(*ms), P64, Y, X, tred, 1, nullptr, st))) return rc;
  // eta1 = I^-T Y
  LocalLaunch Le{};
  Le.prec = P64;
  Le.out = eta1;
  Le.in = Y;
  Le.stride = f64;
  Le.nrhs = 1;
  Le.m = ms->ptr(P64, ms->mat_off(MatSet::IINVT));
  Le.prog = hop2::PR_ITINV;
  Le.chain = ms->ptr(P64, ms->chain_off());
  Le.c = 1.0;
  KLAUNCH(h, launch_local(g, Le, st));
  // xi1 = I^-1 D_rb X = -1/2 I^-1 H_rb (B X)
  HopLaunch Hx = base_hop(h, P64, red, 1, f64);
  Hx.out = xi1;
  Hx.v = X;
  Hx.pre = PRE_B;
  Hx.pre_diag = ms->ptr(P64, ms->bdiag_off());
  Hx.pre_off = ms->ptr(P64, ms->boff_off());
  Hx.post = ms->ptr(P64, ms->mat_off(MatSet::IINV));
  Hx.c_hop = -0.5;
  KLAUNCH(h, launch_hop(g, Hx, st));
  // eta2 = I^-T D_br^+ eta1 = -1/2 K^T gamma5 H_rb (gamma5 eta1)
  HopLaunch He = base_hop(h, P64, red, 1, f64);
  He.out = eta2;
  He.v = eta1;
  He.pre = PRE_G5;
  He.post = ms->ptr(P64, ms->mat_off(MatSet::KT));
  He.g5out = 1;
  He.c_hop = -0.5;
  KLAUNCH(h, launch_hop(g, He, st));
  KLAUNCH(h, launch_force(g, dSdU, eta1, xi1, eta2, X,
                          reinterpret_cast<const double*>(ms->ptr(P64, ms->bdiag_off())),
                          reinterpret_cast<const double*>(ms->ptr(P64, ms->boff_off())), h->gauge[0],
                          gauge_bytes(g, P64) / 2, black, projected, st));
  return DWF_OK;
}

}  // extern "C"

namespace dwf {

int set_error(dwf_handle h, int code, const char* msg) { return fail(h, code, msg); }

// D_bb apply with the static scratch array as the red intermediate field (at
// least nrhs * field_bytes(prec) bytes); allocates nothing (the handle's
// matrices for its own alpha and m exist since dwf_create).
int apply_dbb_noalloc(dwf_handle h, void* out, const void* in, int prec, int nrhs,
                      size_t scratch_bytes, cudaStream_t s) {
  if (!h || !out || !in || !valid_prec(prec) || nrhs < 1 || out == in)
    return fail(h, DWF_ERR_INVALID_ARG, "bad argument");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
    return fail(h, DWF_ERR_INVALID_ARG,
                "dwf_apply_Dbb_noalloc: the current device is not the handle's device");
  if (!h->noalloc_scratch)
    return fail(h, DWF_ERR_CUDA, "the static scratch array has no device address on this device");
  void* scratch = h->noalloc_scratch;
  if (!h->gauge_loaded) return fail(h, DWF_ERR_STATE, "gauge field not loaded");
  const size_t need = field_bytes(h->g, prec) * (size_t)nrhs;
  if (need > scratch_bytes)
    return fail(h, DWF_ERR_INVALID_ARG,
                "dwf_apply_Dbb_noalloc: the red intermediate field needs " + std::to_string(need) +
                    " bytes, more than the " + std::to_string(scratch_bytes) +
                    "-byte static scratch buffer; use dwf_apply_Dbb");
  auto it = h->mats.find(std::make_pair(h->alpha, h->m));
  if (it == h->mats.end()) return fail(h, DWF_ERR_STATE, "operator matrices missing");
  return apply_dbb(h, view_of(it->second), prec, out, in, scratch, nrhs, nullptr, s);
}

}  // namespace dwf
