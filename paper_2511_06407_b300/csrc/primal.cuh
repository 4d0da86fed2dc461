// Device kernels of the primal (reduced-rank) model of the paper's experiments: features,
// likelihood maps, U / dU / Hessian assembly and the third-derivative contraction. Included once,
// by rmhmc.cu, after model_kernels.cuh.
//
// Model (Sec. 2.1 Eq. Solin_representation; the reduced-rank appendix; Sec. 2.5, 2.6). With J = 2
// (Example 1) two functions F_1, F_2 share the features and the hyperparameters, and
// y_i ~ N(F_1i, delta + exp F_2i); coefficient i of q belongs to function i / P, position i % P.
//   F_i = sum_km a_km phi_m(Xg_ik) + sum_l a_l Xl_il + b,  phi_m(x) = sin(pi m (x + L) / (2L))
//   a_km ~ N(0, c_g V_m(s_g)), V_m(s) = sqrt(pi s) exp(-kappa_m s), kappa_m = pi^2 m^2 / (16 L^2)
//   a_l ~ N(0, c_l), b ~ N(0, Sigma), c_g, s_g, c_l ~ InvGamma, sampled as u = log(theta).
// Per coefficient the prior term is E(a, h) = a^2 e^h / 2 - h / 2 (+ log 2 pi / 2) with
// h = -log(c_g V_m) = -u_cg - log(pi)/2 - u_sg/2 + kappa_m e^{u_sg} (h = -u_cl for a_l), so its
// derivatives follow from E_a = a e^h, E_aa = e^h, E_h = a^2 e^h / 2 - 1/2, E_ah = a e^h,
// E_hh = E_hhh = a^2 e^h / 2, E_aah = e^h, E_ahh = a e^h and those of h:
//   h_cg = -1, h_sg = -1/2 + kappa e^{u_sg}, h_sg,sg = h_sg,sg,sg = kappa e^{u_sg}, others 0.
// The likelihood parts of the Hessian and of the third derivatives are Phi^T diag(tau l'') Phi
// and sum_i tau l'''_i phi_i phi_i phi_i; the contraction with W follows the ordering of Sec. 2.3:
// v = Phi^T [tau l''' o rowsum((Phi W) o Phi)].
#pragma once
#include <math.h>

#include "internal.cuh"

namespace rmhmc {
namespace dev {

// h and its derivatives for feature m (1-based) at (u_cg, u_sg): dh[2], d2h (only sg,sg), d3h.
struct HDerivs {
  double h, eh, h1[2], hss;
};
__device__ __forceinline__ HDerivs h_derivs(const PrimalDev& pd, int m, double u_cg, double u_sg) {
  const double kap = M_PI * M_PI * (double)m * m / (16.0 * pd.L * pd.L);
  const double es = kap * exp(u_sg);
  HDerivs r;
  r.h = -u_cg - 0.5 * log(M_PI) - 0.5 * u_sg + es;
  r.eh = exp(r.h);
  r.h1[0] = -1.0;
  r.h1[1] = -0.5 + es;
  r.hss = es;  // = h_sg,sg = h_sg,sg,sg
  return r;
}

// -sum log p(u) for u = log theta, theta ~ InvGamma(a, b) with the Jacobian, and its derivatives.
__device__ __forceinline__ void hyper_terms(const PrimalDev& pd, const double* u, double& v, double g[3],
                                           double h2[3], double h3[3]) {
  v = 0.0;
  for (int j = 0; j < 3; ++j) {
    const double e = pd.b[j] * exp(-u[j]);
    v += pd.a[j] * u[j] + e - (pd.a[j] * log(pd.b[j]) - lgamma(pd.a[j]));
    g[j] = pd.a[j] - e;
    h2[j] = e;
    h3[j] = -e;
  }
}

// Phi (N x P): feature m of Gaussian column k in column k M + m - 1, then the linear columns,
// then 1 (the bias).
__global__ void k_phi(PrimalDev pd, double* __restrict__ Phi) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)pd.N * pd.P) return;
  const int i = (int)(e / pd.P), col = (int)(e % pd.P);
  const int MG = pd.M * pd.Dg;
  double v = 1.0;
  if (col < MG) {
    const int k = col / pd.M, m = col % pd.M + 1;
    v = sin(M_PI * m * (pd.Xg[(long long)i * pd.Dg + k] + pd.L) / (2.0 * pd.L));
  } else if (col < MG + pd.Dl) {
    v = pd.Xl[(long long)i * pd.Dl + (col - MG)];
  }
  Phi[e] = v;
}

// l, l', l'', l''' (tempered) and the untempered l at F (C x N).
__global__ void k_lik_primal(PrimalDev pd, const double* __restrict__ F, double* __restrict__ l0,
                             double* __restrict__ l1, double* __restrict__ l2, double* __restrict__ l3,
                             double* __restrict__ lraw) {
  const int c = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pd.N) return;
  const long long o = (long long)c * pd.N + i;
  double a0, a1, a2, a3;
  lik_point(pd.lik, pd.y[i], F[o], pd.noise_var, a0, a1, a2, a3);
  const double tau = pd.tau[c];
  lraw[o] = a0;
  l0[o] = tau * a0;
  l1[o] = tau * a1;
  l2[o] = tau * a2;
  l3[o] = tau * a3;
}

// Mean/variance likelihood (J = 2): F is (2, C, N); writes l (tempered) and the untempered l, and
// in ld (9, C, N) the tempered derivatives l_1, l_2, l_11, l_12, l_22, l_111, l_112, l_122, l_222 of
// l = z / 2 + log(2 pi v) / 2 with r = y - F_1, w = e^{F_2}, v = delta + w, rho = w / v,
// z = r^2 / v: l_1 = -r / v, l_2 = rho (1 - z) / 2, l_11 = 1 / v, l_12 = r rho / v,
// l_22 = rho A / 2 with A = (1 - rho)(1 - z) + z rho, l_111 = 0, l_112 = -rho / v,
// l_122 = r rho (1 - 2 rho) / v, l_222 = [rho (1 - rho) A + rho A'] / 2 with
// A' = -rho (1 - rho) + z rho + 2 z rho (1 - 2 rho) (d rho / dF_2 = rho (1 - rho), dz / dF_2 = -z rho).
__global__ void k_lik_meanvar(PrimalDev pd, const double* __restrict__ F, double* __restrict__ l0,
                              double* __restrict__ lraw, double* __restrict__ ld) {
  const int c = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pd.N) return;
  const long long CN = (long long)pd.n_chains * pd.N, o = (long long)c * pd.N + i;
  const double r = pd.y[i] - F[o], w = exp(F[CN + o]);
  const double v = pd.delta + w, rho = w / v, z = r * r / v;
  const double A = (1.0 - rho) * (1.0 - z) + z * rho;
  const double dA = -rho * (1.0 - rho) + z * rho + 2.0 * z * rho * (1.0 - 2.0 * rho);
  const double tau = pd.tau[c];
  const double a0 = 0.5 * z + 0.5 * log(2.0 * M_PI * v);
  lraw[o] = a0;
  l0[o] = tau * a0;
  const double der[9] = {-r / v, 0.5 * rho * (1.0 - z), 1.0 / v, r * rho / v, 0.5 * rho * A, 0.0, -rho / v,
                         r * rho * (1.0 - 2.0 * rho) / v, 0.5 * (rho * (1.0 - rho) * A + rho * dA)};
#pragma unroll
  for (int k = 0; k < 9; ++k) ld[k * CN + o] = tau * der[k];
}

// r_j = sum_{k, l} l_jkl s_kl for the mean/variance model, s_kl = rowsum((Phi W_kl) o Phi) given
// for (k, l) = (0, 0), (0, 1), (1, 1) in s (3, C, N) (s_10 = s_01): r (2, C, N).
__global__ void k_mv_combine(PrimalDev pd, const double* __restrict__ s, const double* __restrict__ ld,
                             double* __restrict__ r) {
  const long long CN = (long long)pd.n_chains * pd.N;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= CN) return;
  const double s00 = s[o], s01 = s[CN + o], s11 = s[2 * CN + o];
  const double t111 = ld[5 * CN + o], t112 = ld[6 * CN + o], t122 = ld[7 * CN + o], t222 = ld[8 * CN + o];
  r[o] = t111 * s00 + 2.0 * t112 * s01 + t122 * s11;
  r[CN + o] = t112 * s00 + 2.0 * t122 * s01 + t222 * s11;
}

// Z_c = diag(l''_c) Phi (C x N x P).
__global__ void k_rowscale(PrimalDev pd, const double* __restrict__ l2, const double* __restrict__ Phi,
                           double* __restrict__ Z) {
  const long long NP = (long long)pd.N * pd.P;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (e >= NP) return;
  Z[c * NP + e] = l2[(long long)c * pd.N + e / pd.P] * Phi[e];
}

// One block per chain. On entry dU[c, :P] = Phi^T l'_c (tempered). Adds the prior gradient of the
// coefficients, writes the hyperparameter gradient, U, the untempered log likelihood LL and the
// 3 x 3 hyperparameter block of the Hessian (ustat[c*9 ...]); zeroes dU's padding.
__global__ void k_primal_udu(PrimalDev pd, const double* __restrict__ q, int dp,
                             const double* __restrict__ l0, const double* __restrict__ lraw,
                             double* __restrict__ U, double* __restrict__ dU, double* __restrict__ LL,
                             double* __restrict__ ustat) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const double* qc = q + (long long)c * dp;
  double* g = dU + (long long)c * dp;
  const int P = pd.P, JP = pd.JP, MG = pd.M * pd.Dg;
  const double u_cg = qc[JP], u_sg = qc[JP + 1], u_cl = qc[JP + 2];
  const double el = exp(-u_cl);
  double sl0 = 0.0, slraw = 0.0;
  for (int i = threadIdx.x; i < pd.N; i += blockDim.x) {
    sl0 += l0[(long long)c * pd.N + i];
    slraw += lraw[(long long)c * pd.N + i];
  }
  double pv = 0.0, gcg = 0.0, gsg = 0.0, gcl = 0.0, hcc = 0.0, hcs = 0.0, hss = 0.0, hll = 0.0;
  for (int i = threadIdx.x; i < JP; i += blockDim.x) {
    const double a = qc[i];
    const int li = i % P;  // position within its function's coefficients
    if (li < MG) {
      const HDerivs r = h_derivs(pd, li % pd.M + 1, u_cg, u_sg);
      const double Eh = 0.5 * a * a * r.eh - 0.5, Ehh = 0.5 * a * a * r.eh;
      pv += 0.5 * a * a * r.eh - 0.5 * r.h;
      g[i] += a * r.eh;
      gcg += Eh * r.h1[0];
      gsg += Eh * r.h1[1];
      hcc += Ehh * r.h1[0] * r.h1[0];
      hcs += Ehh * r.h1[0] * r.h1[1];
      hss += Ehh * r.h1[1] * r.h1[1] + Eh * r.hss;
    } else if (li < MG + pd.Dl) {
      pv += 0.5 * a * a * el + 0.5 * u_cl;
      g[i] += a * el;
      gcl += -0.5 * a * a * el + 0.5;
      hll += 0.5 * a * a * el;
    } else {
      pv += 0.5 * a * a / pd.bias_var + 0.5 * log(pd.bias_var);
      g[i] += a / pd.bias_var;
    }
  }
  sl0 = block_sum(sl0, sh);
  slraw = block_sum(slraw, sh);
  pv = block_sum(pv, sh);
  gcg = block_sum(gcg, sh);
  gsg = block_sum(gsg, sh);
  gcl = block_sum(gcl, sh);
  hcc = block_sum(hcc, sh);
  hcs = block_sum(hcs, sh);
  hss = block_sum(hss, sh);
  hll = block_sum(hll, sh);
  for (int i = pd.d + threadIdx.x; i < dp; i += blockDim.x) g[i] = 0.0;
  if (threadIdx.x == 0) {
    const double u[3] = {u_cg, u_sg, u_cl};
    double hv, hg[3], h2[3], h3[3];
    hyper_terms(pd, u, hv, hg, h2, h3);
    U[c] = sl0 + pv + 0.5 * JP * LOG2PI + hv;
    LL[c] = -slraw;
    g[JP] = gcg + hg[0];
    g[JP + 1] = gsg + hg[1];
    g[JP + 2] = gcl + hg[2];
    double* us = ustat + (long long)c * 9;
    us[0] = hcc + h2[0];
    us[1] = us[3] = hcs;
    us[4] = hss + h2[1];
    us[2] = us[6] = 0.0;
    us[5] = us[7] = 0.0;
    us[8] = hll + h2[2];
  }
}

// On entry H[c, :P, :P] = Phi^T diag(l''_c) Phi. Adds the prior curvature of the coefficients to
// the diagonal and writes every entry in the hyperparameter rows / columns and the padding.
__global__ void k_primal_hess(PrimalDev pd, const double* __restrict__ q, int dp,
                              const double* __restrict__ ustat, double* __restrict__ H) {
  const long long DD = (long long)dp * dp;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (e >= DD) return;
  const int i = (int)(e / dp), j = (int)(e % dp);
  const double* qc = q + (long long)c * dp;
  const int P = pd.P, JP = pd.JP, MG = pd.M * pd.Dg;
  double* Hc = H + c * DD;
  if (i < JP && j < JP) {
    if (i == j) {
      const int li = i % P;
      double v;
      if (li < MG) v = h_derivs(pd, li % pd.M + 1, qc[JP], qc[JP + 1]).eh;
      else if (li < MG + pd.Dl) v = exp(-qc[JP + 2]);
      else v = 1.0 / pd.bias_var;
      Hc[e] += v;
    }
    return;
  }
  double v = 0.0;
  if (i < pd.d && j < pd.d) {
    const int r = min(i, j), s = max(i, j);
    if (r < JP) {
      const int lr = r % P;
      if (lr < MG && s <= JP + 1) {
        const HDerivs hd = h_derivs(pd, lr % pd.M + 1, qc[JP], qc[JP + 1]);
        v = qc[r] * hd.eh * hd.h1[s - JP];
      } else if (lr >= MG && lr < MG + pd.Dl && s == JP + 2) {
        v = -qc[r] * exp(-qc[JP + 2]);
      }
    } else {
      v = ustat[(long long)c * 9 + (r - JP) * 3 + (s - JP)];
    }
  }
  Hc[e] = v;
}

// r_c,i = m_c,i sum_j Y_c,ij Phi_ij (one warp per row; Y = Phi W_block) with m = tau l''' for
// J = 1, or m = 1 (l3 null) for the mean/variance model, whose r are combined afterwards.
__global__ void k_primal_rowdot(PrimalDev pd, const double* __restrict__ Y, const double* __restrict__ Phi,
                                const double* __restrict__ l3, double* __restrict__ r) {
  const int c = blockIdx.y;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= pd.N) return;
  const double* y = Y + ((long long)c * pd.N + i) * pd.P;
  const double* ph = Phi + (long long)i * pd.P;
  double s = 0.0;
  for (int j = lane; j < pd.P; j += 32) s = fma(y[j], ph[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[(long long)c * pd.N + i] = l3 ? l3[(long long)c * pd.N + i] * s : s;
}

// The prior parts of v_i = tr(W dH_i): on entry v[c, :P] holds the likelihood part; adds the
// coefficients' prior parts and writes the hyperparameter entries and the padding. Per Gaussian
// coefficient the third derivatives live on (a, u_cg, u_sg): T[a,a,u_j] = e^h h_j,
// T[a,u_j,u_k] = a e^h (h_j h_k + h_jk), T[u_j,u_k,u_l] = E_hhh h_j h_k h_l
// + E_hh (h_jk h_l + h_jl h_k + h_kl h_j) + E_h h_jkl; per linear coefficient on (a, u_cl) with
// h = -u_cl; the hyperprior adds -b e^{-u} on each (u_j, u_j, u_j).
__global__ void k_primal_contract(PrimalDev pd, const double* __restrict__ q, int dp,
                                  const double* __restrict__ W, double* __restrict__ v) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const long long DD = (long long)dp * dp;
  const double* qc = q + (long long)c * dp;
  const double* Wc = W + c * DD;
  double* vc = v + (long long)c * dp;
  const int P = pd.P, JP = pd.JP, MG = pd.M * pd.Dg;
  const double u_cg = qc[JP], u_sg = qc[JP + 1], u_cl = qc[JP + 2];
  const double el = exp(-u_cl);
  // W on the hyperparameters
  const double Wu[2][2] = {{Wc[(long long)JP * dp + JP], Wc[(long long)JP * dp + JP + 1]},
                           {Wc[(long long)(JP + 1) * dp + JP], Wc[(long long)(JP + 1) * dp + JP + 1]}};
  const double Wll = Wc[(long long)(JP + 2) * dp + JP + 2];
  double vcg = 0.0, vsg = 0.0, vcl = 0.0;
  for (int i = threadIdx.x; i < JP; i += blockDim.x) {
    const double a = qc[i];
    const double Waa = Wc[(long long)i * dp + i];
    const int li = i % P;
    if (li < MG) {
      const HDerivs r = h_derivs(pd, li % pd.M + 1, u_cg, u_sg);
      const double Wau[2] = {Wc[(long long)i * dp + JP], Wc[(long long)i * dp + JP + 1]};
      const double Eh = 0.5 * a * a * r.eh - 0.5, Ehh = 0.5 * a * a * r.eh, Ehhh = Ehh;
      double hjk[2][2] = {{0.0, 0.0}, {0.0, r.hss}};
      double va = 0.0, vu[2] = {0.0, 0.0};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        va += 2.0 * r.eh * r.h1[j] * Wau[j];
#pragma unroll
        for (int k = 0; k < 2; ++k) va += a * r.eh * (r.h1[j] * r.h1[k] + hjk[j][k]) * Wu[j][k];
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        double t = r.eh * r.h1[j] * Waa;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          t += 2.0 * a * r.eh * (r.h1[j] * r.h1[k] + hjk[j][k]) * Wau[k];
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            const double hjkl = (j == 1 && k == 1 && l == 1) ? r.hss : 0.0;
            const double T = Ehhh * r.h1[j] * r.h1[k] * r.h1[l] +
                             Ehh * (hjk[j][k] * r.h1[l] + hjk[j][l] * r.h1[k] + hjk[k][l] * r.h1[j]) +
                             Eh * hjkl;
            t += T * Wu[k][l];
          }
        }
        vu[j] = t;
      }
      vc[i] += va;
      vcg += vu[0];
      vsg += vu[1];
    } else if (li < MG + pd.Dl) {
      const double Wau = Wc[(long long)i * dp + JP + 2];
      vc[i] += -2.0 * el * Wau + a * el * Wll;
      vcl += -el * Waa + 2.0 * a * el * Wau - 0.5 * a * a * el * Wll;
    }
  }
  vcg = block_sum(vcg, sh);
  vsg = block_sum(vsg, sh);
  vcl = block_sum(vcl, sh);
  for (int i = pd.d + threadIdx.x; i < dp; i += blockDim.x) vc[i] = 0.0;
  if (threadIdx.x == 0) {
    const double u[3] = {u_cg, u_sg, u_cl};
    double hv, hg[3], h2[3], h3[3];
    hyper_terms(pd, u, hv, hg, h2, h3);
    vc[JP] = vcg + h3[0] * Wu[0][0];
    vc[JP + 1] = vsg + h3[1] * Wu[1][1];
    vc[JP + 2] = vcl + h3[2] * Wll;
  }
}

}  // namespace dev
}  // namespace rmhmc
