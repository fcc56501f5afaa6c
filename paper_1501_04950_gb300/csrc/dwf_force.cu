// dwf_force.cu -- fermion force of S = phi^+ (D_bb^+ D_bb)^-1 phi (sm_103a).
//
// With X = (D^+ D)^-1 phi and Y = D_bb X, the variation of S under a change of
// the links is dS = -2 Re[Y^+ dD_bb X].  Only the hopping blocks of Eq. redblack
// depend on U (D_rb = -1/2 H_rb B, D_br = -1/2 H_br B), which gives
//   dS = 2 Re[eta1^+ dD_br xi1] + 2 Re[eta2^+ dD_rb xi2],
//   eta1 = I^-T Y (black),  xi1 = I^-1 D_rb X (red),
//   eta2 = I^-T D_br^+ eta1 = -1/2 K^T gamma5 H_rb gamma5 eta1 (red),  xi2 = X (black).
// Each term is -1/2 sum_s over the hops of Eq. wilson that contain U_mu(x):
//   forward  x <- x+mu:  eta(x)^+ (1 - gamma_mu) dU w(x+mu)
//   backward x+mu <- x:  eta(x+mu)^+ (1 + gamma_mu) dU^+ w(x),      w = B xi.
// With the convention G_ij = dS/dRe U_ij + i dS/dIm U_ij a term Re[a^+ dU b]
// contributes a b^+, and sum_spin a_spin (P b)_spin^+ for P = 1 -+ gamma_mu
// reduces to the two rows of the projected half spinors: sum_k h(a)_k h(b)_k^+.
#include <algorithm>

#include "dwf_fields.cuh"

namespace dwf {

namespace {

// Half spinor of (1 - sg gamma_mu) psi (two rows of 3 colours), runtime mu.
__device__ __forceinline__ void project_rt(const Spinor<double>& s, int mu, int sg,
                                           cplx<double> h[2][3]) {
  cplx<double> h0[3], h1[3];
  switch (mu * 2 + (sg > 0 ? 0 : 1)) {
    case 0: project<double, 0, +1>(s, h0, h1); break;
    case 1: project<double, 0, -1>(s, h0, h1); break;
    case 2: project<double, 1, +1>(s, h0, h1); break;
    case 3: project<double, 1, -1>(s, h0, h1); break;
    case 4: project<double, 2, +1>(s, h0, h1); break;
    case 5: project<double, 2, -1>(s, h0, h1); break;
    case 6: project<double, 3, +1>(s, h0, h1); break;
    default: project<double, 3, -1>(s, h0, h1); break;
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    h[0][a] = h0[a];
    h[1][a] = h1[a];
  }
}

// w = B xi at (site hs, slice s): B_+ row s = d+ e_s + o+ e_{s-1}, B_- row s = d- e_s + o- e_{s+1}.
__device__ __forceinline__ void load_bxi(const Geom& g, const void* xi, int hs, int s,
                                         const double* bd, const double* bo, Spinor<double>& w) {
  const int Ls = g.Ls;
  const int sp = s == 0 ? Ls - 1 : s - 1, sn = s == Ls - 1 ? 0 : s + 1;
  Spinor<double> a, b;
  Store64::load(xi, site5(hs, s, Ls), g.N5, w);
  Store64::load_chir(xi, site5(hs, sp, Ls), g.N5, 0, a);
  Store64::load_chir(xi, site5(hs, sn, Ls), g.N5, 1, b);
  const double dp = bd[s], dm = bd[Ls + s], op = bo[s], om = bo[Ls + s];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    w.c[k] = cmake(dp * w.c[k].re + op * a.c[k].re, dp * w.c[k].im + op * a.c[k].im);
    w.c[k + 6] = cmake(dm * w.c[k + 6].re + om * b.c[k + 6].re, dm * w.c[k + 6].im + om * b.c[k + 6].im);
  }
}

// acc_ij += sum_k a_k,i conj(b_k,j)
__device__ __forceinline__ void outer_add(cplx<double> acc[9], const cplx<double> a[2][3],
                                          const cplx<double> b[2][3], int sign) {
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const cplx<double> x = a[k][i], y = b[k][j];
        acc[3 * i + j].re += sign * (x.re * y.re + x.im * y.im);
        acc[3 * i + j].im += sign * (x.im * y.re - x.re * y.im);
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

struct ForceArgs {
  const void* eta1;  // black
  const void* xi1;   // red
  const void* eta2;  // red
  const void* xi2;   // black
  const double* bd;  // B diagonal [2][Ls]
  const double* bo;  // B off-diagonal [2][Ls]
  const void* g64;   // internal FP64 gauge (both parities)
  size_t gpar;       // bytes per parity
  double* out;       // canonical [V][4][3][3] complex
  int black;
  int projected;
};

// One thread per link (x, mu): G = -(term1(eta_a(x), B xi_a(x+mu)) + term2(B xi_b(x), eta_b(x+mu))),
// (a, b) = (1, 2) on black x and (2, 1) on red x.
__global__ void force_kernel(const Geom g, const ForceArgs a) {
  const size_t V = (size_t)g.Vh * 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < V * 4;
       i += (size_t)gridDim.x * blockDim.x) {
    const int site = (int)(i / 4), mu = (int)(i % 4);
    int x, y, z, t;
    lex_coords(g, site, x, y, z, t);
    const int q = (x + y + z + t) & 1;
    const int h = site >> 1;
    int c[4] = {x, y, z, t};
    double sign = 1.0;
    c[mu] += 1;
    if (c[mu] == g.L[mu]) {
      c[mu] = 0;
      if (mu == 3) sign = g.bc_t;
    }
    const int hn = (c[0] >> 1) + g.Lxh * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
    const bool is_black = q == a.black;
    const void* eta_a = is_black ? a.eta1 : a.eta2;
    const void* xi_a = is_black ? a.xi1 : a.xi2;
    const void* eta_b = is_black ? a.eta2 : a.eta1;
    const void* xi_b = is_black ? a.xi2 : a.xi1;
    cplx<double> G[9];
#pragma unroll
    for (int k = 0; k < 9; k++) G[k] = cmake(0.0, 0.0);
    for (int s = 0; s < g.Ls; s++) {
      Spinor<double> e, w;
      cplx<double> he[2][3], hw[2][3];
      // term 1: eta_a(x)^+ (1 - gamma_mu) dU w_a(x+mu)
      Store64::load(eta_a, site5(h, s, g.Ls), g.N5, e);
      load_bxi(g, xi_a, hn, s, a.bd, a.bo, w);
      project_rt(e, mu, +1, he);
      project_rt(w, mu, +1, hw);
      outer_add(G, he, hw, 1);
      // term 2: eta_b(x+mu)^+ (1 + gamma_mu) dU^+ w_b(x)  ->  w_b(x) (proj eta_b)^+
      Store64::load(eta_b, site5(hn, s, g.Ls), g.N5, e);
      load_bxi(g, xi_b, h, s, a.bd, a.bo, w);
      project_rt(e, mu, -1, he);
      project_rt(w, mu, -1, hw);
      outer_add(G, hw, he, 1);
    }
    // 2 * (-1/2) and the antiperiodic sign of a hop across the t boundary
#pragma unroll
    for (int k = 0; k < 9; k++) G[k] = cmake(-sign * G[k].re, -sign * G[k].im);
    double2* o = reinterpret_cast<double2*>(a.out) + i * 9;
    if (!a.projected) {
#pragma unroll
      for (int k = 0; k < 9; k++) o[k] = make_double2(G[k].re, G[k].im);
    } else {
      // F = TA(U G^+), TA(M) = (M - M^+)/2 - tr(M - M^+)/6
      const double2* u = reinterpret_cast<const double2*>(reinterpret_cast<const char*>(a.g64) +
                                                          (size_t)q * a.gpar) +
                         ((size_t)h * 4 + mu) * 9;
      cplx<double> M[9];
#pragma unroll
      for (int r = 0; r < 3; r++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {
          cplx<double> acc = cmake(0.0, 0.0);
#pragma unroll
          for (int k = 0; k < 3; k++) {
            const double2 uu = u[3 * r + k];
            const cplx<double> gg = G[3 * cc + k];  // (G^+)_{k,cc} = conj(G_{cc,k})
            acc.re += uu.x * gg.re + uu.y * gg.im;
            acc.im += uu.y * gg.re - uu.x * gg.im;
          }
          M[3 * r + cc] = acc;
        }
      cplx<double> F[9];
      double tr_im = 0.0;
#pragma unroll
      for (int r = 0; r < 3; r++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {
          const cplx<double> m1 = M[3 * r + cc], m2 = M[3 * cc + r];
          F[3 * r + cc] = cmake(0.5 * (m1.re - m2.re), 0.5 * (m1.im + m2.im));
        }
      tr_im = F[0].im + F[4].im + F[8].im;
      F[0].im -= tr_im / 3.0;
      F[4].im -= tr_im / 3.0;
      F[8].im -= tr_im / 3.0;
#pragma unroll
      for (int k = 0; k < 9; k++) o[k] = make_double2(F[k].re, F[k].im);
    }
  }
}

}  // namespace

cudaError_t launch_force(const Geom& g, double* out, const void* eta1, const void* xi1,
                         const void* eta2, const void* xi2, const double* bd, const double* bo,
                         const void* g64, size_t gpar, int black, int projected, cudaStream_t s) {
  ForceArgs a;
  a.eta1 = eta1;
  a.xi1 = xi1;
  a.eta2 = eta2;
  a.xi2 = xi2;
  a.bd = bd;
  a.bo = bo;
  a.g64 = g64;
  a.gpar = gpar;
  a.out = out;
  a.black = black;
  a.projected = projected;
  const size_t n = (size_t)g.Vh * 8;
  int blocks = (int)std::min<size_t>((n + 127) / 128, 152 * 32);
  force_kernel<<<blocks, 128, 0, s>>>(g, a);
  return cudaGetLastError();
}

}  // namespace dwf
