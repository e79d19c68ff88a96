// Off-diagonal self-energy in the band basis: Eqs. (sigc) and (sigx) without the diagonal
// approximation of Sec. III.B (the paper names the full band matrix as future work):
//   Sigma^c_nm(k|tau) += -1/(Omega N_k) sum_j G_j(k - q|tau) sum_IJ conj(M^I_jn) W~_IJ(tau) M^J_jm
//   Sigma^x_nm(k)     += -1/(Omega N_k) sum_j occ_j(k - q) sum_I v_I conj(M^I_jn) M^I_jm
// FP64 on the CUDA cores. Sigma^c: one block per (k, tau); for each j and each chunk of ci rows
// I of W~(tau), the block forms Z = W~(tau)[I chunk, :] a_j (ci x Nb, a_j = M[k][:, j, :]) in
// shared memory and adds G_j a_j[I chunk]^+ Z to the Nb x Nb accumulator, also in shared memory,
// so any NI fits. Sigma^x: one block per k.
#include <cuda_runtime.h>

#include <algorithm>

#include "gw_internal.h"

namespace gwi {
namespace {

constexpr int kOdThreads = 256;

__device__ __forceinline__ double2 cmac(double2 acc, double2 a, double2 b) {  // acc + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cjmac(double2 acc, double2 a, double2 b) {  // acc + conj(a) b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}

__global__ void __launch_bounds__(kOdThreads) k_sigma_offdiag(const double2* __restrict__ M,
                                                              const double2* __restrict__ W,
                                                              const double* __restrict__ G,
                                                              const int* __restrict__ kmq, int nk, int ni, int nb,
                                                              int ntau, int ci, double pref, double2* __restrict__ S) {
  extern __shared__ double2 osm[];
  double2* acc = osm;                  // [nb][nb]
  double2* Z = acc + (size_t)nb * nb;  // [ci][nb]
  const int k = blockIdx.x / ntau, it = blockIdx.x % ntau, t = threadIdx.x;
  const double2* A = M + (size_t)k * ni * nb * nb;  // A[(J nb + j) nb + m]
  const double2* Wt = W + (size_t)it * ni * ni;
  const double* Gk = G + (size_t)kmq[k] * nb * ntau;
  for (int e = t; e < nb * nb; e += kOdThreads) acc[e] = make_double2(0.0, 0.0);
  for (int j = 0; j < nb; ++j) {
    const double g = Gk[(size_t)j * ntau + it];
    for (int I0 = 0; I0 < ni; I0 += ci) {
      const int nr = min(ci, ni - I0);
      for (int e = t; e < nr * nb; e += kOdThreads) {
        const int I = I0 + e / nb, m = e % nb;
        double2 z = make_double2(0.0, 0.0);
        for (int J = 0; J < ni; ++J) z = cmac(z, Wt[(size_t)I * ni + J], A[((size_t)J * nb + j) * nb + m]);
        Z[e] = z;
      }
      __syncthreads();
      for (int e = t; e < nb * nb; e += kOdThreads) {
        const int n = e / nb, m = e % nb;
        double2 s = make_double2(0.0, 0.0);
        for (int r = 0; r < nr; ++r) s = cjmac(s, A[((size_t)(I0 + r) * nb + j) * nb + n], Z[(size_t)r * nb + m]);
        acc[e] = make_double2(fma(g, s.x, acc[e].x), fma(g, s.y, acc[e].y));
      }
      __syncthreads();
    }
  }
  for (int e = t; e < nb * nb; e += kOdThreads) {
    double2* o = S + (((size_t)k * nb * nb + e) * ntau + it);
    *o = make_double2(fma(pref, acc[e].x, o->x), fma(pref, acc[e].y, o->y));
  }
}

__global__ void __launch_bounds__(kOdThreads) k_sigx_offdiag(const double2* __restrict__ M,
                                                             const double* __restrict__ v,
                                                             const double* __restrict__ occ,
                                                             const int* __restrict__ kmq, int ni, int nb,
                                                             double pref, double2* __restrict__ Sx) {
  const int k = blockIdx.x;
  const double2* A = M + (size_t)k * ni * nb * nb;
  const double* f = occ + (size_t)kmq[k] * nb;
  for (int e = threadIdx.x; e < nb * nb; e += kOdThreads) {
    const int n = e / nb, m = e % nb;
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < nb; ++j) {
      double2 u = make_double2(0.0, 0.0);
      for (int I = 0; I < ni; ++I) {
        const double2 a = A[((size_t)I * nb + j) * nb + n], b = A[((size_t)I * nb + j) * nb + m];
        u = cjmac(u, make_double2(v[I] * a.x, v[I] * a.y), b);
      }
      s = make_double2(fma(f[j], u.x, s.x), fma(f[j], u.y, s.y));
    }
    double2* o = Sx + (size_t)k * nb * nb + e;
    *o = make_double2(fma(pref, s.x, o->x), fma(pref, s.y, o->y));
  }
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_selfenergy_offdiag(gw_ctx* c, int iq, const double* G_tau, const double* occ,
                                           const double* W_tau, double* S_tau, double* Sx) {
  if (!c || iq < 0 || iq >= c->nq || !G_tau || !W_tau || !S_tau || (Sx && !occ)) return GW_EINVAL;
  const int ni = c->ni, nb = c->nb, nk = c->nk, nt = c->ntau;
  // rows of W~ per Z chunk: all of them when they fit, else the most that leave room for the
  // Nb x Nb accumulator in 200 KiB of shared memory (a multiple of 8 rows)
  const size_t budget = 200 * 1024, acc_b = (size_t)nb * nb * sizeof(double2), row_b = (size_t)nb * sizeof(double2);
  if (acc_b + 8 * row_b > budget)
    return set_err(c, GW_EINVAL, "gw_selfenergy_offdiag: the nb x nb accumulator and 8 rows of W~ a_j need 16 nb^2 + 128 nb bytes <= 200 KiB (nb <= 109)");
  int ci = (int)std::min<size_t>((size_t)ni, (budget - acc_b) / row_b);
  if (ci < ni) ci &= ~7;
  const size_t smem = acc_b + (size_t)ci * row_b;
  const double2* M = (const double2*)m_block(c, iq);
  if (!M) return GW_ECUDA;
  const int* kmq = c->d_kmq + (size_t)iq * nk;
  const double pref = -1.0 / (c->omega * nk);
  cudaFuncSetAttribute(k_sigma_offdiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_sigma_offdiag<<<(unsigned)(nk * nt), kOdThreads, smem, c->stream>>>(M, (const double2*)W_tau, G_tau, kmq, nk, ni,
                                                                       nb, nt, ci, pref, (double2*)S_tau);
  gw_status st = check_launch(c, "sigma_offdiag");
  if (st != GW_OK || !Sx) return st;
  k_sigx_offdiag<<<(unsigned)nk, kOdThreads, 0, c->stream>>>(M, c->d_v + (size_t)iq * ni, occ, kmq, ni, nb, pref,
                                                              (double2*)Sx);
  return check_launch(c, "sigx_offdiag");
}
