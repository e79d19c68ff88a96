// The paper's tau-domain Dyson equation for the diagonal Green's function (Sec. III.B.5, Eqs.
// dysongf, zxjk, zcjk, dysong): for each state, Sigma^c given on a (uniform power) mesh is
// carried by a natural cubic spline to the uniform mesh t_i = i h, h = tau_1 - tau_0, where
//   sum_r [delta_pr - w_r Z(t_p, t_r)] G(t_r) = G0(t_p),
//   Z(t, t2) = G0(t - t2) s + sum_l w_l G0(t - t_l) Sigma^c(t_l - t2),
// with the trapezoid increments w (h inside, h/2 at the ends) and antiperiodic G0, Sigma^c
// (f(d) = -f(d + beta) for d < 0; a zero difference takes the value at 0+). It is the check of
// the i w Dyson update (gw_green_tau) on small meshes, not a step of the benchmarked iteration.
//
// One block per state: thread 0 solves the spline's tridiagonal system (Thomas algorithm), the
// block evaluates G0 and Sigma^c on the uniform mesh into shared memory, builds the (n + 1) x
// (n + 2) augmented system (the Z^c sum is n + 1 terms per element) in a global scratch, and
// solves it by Gauss-Jordan elimination with partial pivoting (largest modulus, lowest row on
// a tie), all in FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gw_internal.h"

namespace gwi {
namespace {

constexpr int kDyThreads = 256;
constexpr int kDyMaxPts = 1024;  // uniform-mesh points and spline nodes held in shared memory

__device__ double g0_at(double eps, double t, double beta) {  // -e^{-eps t}(1 - n_F(eps)), 0 <= t <= beta
  return eps >= 0.0 ? -exp(-eps * t) / (1.0 + exp(-beta * eps)) : -exp(eps * (beta - t)) / (1.0 + exp(beta * eps));
}

// f(d) at d = (p - r) h on the uniform mesh (n + 1 values, f[0] at 0+): f[p - r] for p >= r,
// -f[p - r + n] below (antiperiodic)
__device__ __forceinline__ double anti(const double* f, int d, int n) { return d >= 0 ? f[d] : -f[d + n]; }

__global__ void __launch_bounds__(kDyThreads) k_dyson_tau(int nu, const double* __restrict__ xu,
                                                          const double* __restrict__ eps,
                                                          const double* __restrict__ sst,
                                                          const double* __restrict__ sigc, int n, double h,
                                                          double* __restrict__ K, double* __restrict__ G,
                                                          int* __restrict__ info) {
  extern __shared__ double dsm[];
  double* sx = dsm;            // [nu] nodes
  double* sM = sx + nu;        // [nu] second derivatives of the spline
  double* sy = sM + nu;        // [nu] Sigma^c at the nodes
  double* g0 = sy + nu;        // [n + 1] G0 on the uniform mesh
  double* sc = g0 + n + 1;     // [n + 1] Sigma^c on the uniform mesh
  double* fc = sc + n + 1;     // [n + 1] column factors of an elimination step
  double* gf = fc + n + 1;     // [2 n + 1] G0(d h), d = -n..n (antiperiodic extension), at gf[d + n]
  double* sf = gf + 2 * n + 1; // [2 n + 1] Sigma^c(d h) likewise
  __shared__ double rv[kDyThreads];
  __shared__ int ri[kDyThreads];
  __shared__ int bad;
  const int b = blockIdx.x, t = threadIdx.x;
  const int np1 = n + 1, L = n + 2;
  const double beta = n * h;
  double* A = K + (size_t)b * np1 * L;
  for (int i = t; i < nu; i += kDyThreads) {
    sx[i] = xu[i];
    sy[i] = sigc[(size_t)b * nu + i];
  }
  if (t == 0) bad = 0;
  __syncthreads();
  if (t == 0) {
    // natural spline: h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1} = 6 (d_i - d_{i-1}),
    // M_0 = M_{nu-1} = 0; forward elimination into sM (as the modified right-hand side) and fc
    // (as the modified super-diagonal), then back substitution
    sM[0] = 0.0;
    fc[0] = 0.0;
    for (int i = 1; i < nu - 1; ++i) {
      const double hl = sx[i] - sx[i - 1], hr = sx[i + 1] - sx[i];
      const double r = 6.0 * ((sy[i + 1] - sy[i]) / hr - (sy[i] - sy[i - 1]) / hl);
      const double den = 2.0 * (hl + hr) - hl * fc[i - 1];
      fc[i] = hr / den;
      sM[i] = (r - hl * sM[i - 1]) / den;
    }
    sM[nu - 1] = 0.0;
    for (int i = nu - 2; i >= 1; --i) sM[i] -= fc[i] * sM[i + 1];
  }
  __syncthreads();
  const double e = eps[b], s = sst[b];
  for (int i = t; i < np1; i += kDyThreads) {
    const double ti = i * h;
    int lo = 0, hi = nu - 1;  // the last node <= ti, clipped to [0, nu - 2]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (sx[mid] <= ti) lo = mid; else hi = mid;
    }
    const int j = min(lo, nu - 2);
    const double hj = sx[j + 1] - sx[j], a0 = ti - sx[j], a1 = sx[j + 1] - ti;
    sc[i] = (sM[j] * a1 * a1 * a1 + sM[j + 1] * a0 * a0 * a0) / (6.0 * hj) + (sy[j] / hj - sM[j] * hj / 6.0) * a1 +
            (sy[j + 1] / hj - sM[j + 1] * hj / 6.0) * a0;
    g0[i] = g0_at(e, ti, beta);
  }
  __syncthreads();
  for (int d = t; d <= 2 * n; d += kDyThreads) {
    gf[d] = anti(g0, d - n, n);
    sf[d] = anti(sc, d - n, n);
  }
  __syncthreads();
  // [I - Z diag(w) | G0]; the trapezoid sum over l as h (sum of all terms - half the two end
  // terms), one multiply-add per term
  for (int idx = t; idx < np1 * np1; idx += kDyThreads) {
    const int p = idx / np1, r = idx % np1;
    const double* gp = gf + p + n;  // gp[-l] = G0(t_p - t_l)
    const double* sr = sf + n - r;  // sr[l] = Sigma^c(t_l - t_r)
    double zc = 0.0;
    for (int l = 0; l <= n; ++l) zc = fma(gp[-l], sr[l], zc);
    zc = h * (zc - 0.5 * (gp[0] * sr[0] + gp[-n] * sr[n]));
    const double wr = (r == 0 || r == n) ? 0.5 * h : h;
    const double z = gp[-r] * s + zc;
    A[(size_t)p * L + r] = (p == r ? 1.0 : 0.0) - wr * z;
  }
  for (int p = t; p < np1; p += kDyThreads) A[(size_t)p * L + np1] = g0[p];
  __syncthreads();
  for (int k = 0; k < np1; ++k) {
    double best = -1.0;
    int bi = np1;
    for (int i = k + t; i < np1; i += kDyThreads) {
      const double m = fabs(A[(size_t)i * L + k]);
      if (m > best) {
        best = m;
        bi = i;
      }
    }
    rv[t] = best;
    ri[t] = bi;
    __syncthreads();
    for (int o = kDyThreads / 2; o > 0; o >>= 1) {
      if (t < o && (rv[t + o] > rv[t] || (rv[t + o] == rv[t] && ri[t + o] < ri[t]))) {
        rv[t] = rv[t + o];
        ri[t] = ri[t + o];
      }
      __syncthreads();
    }
    const int q = ri[0];
    if (!(rv[0] > 0.0)) {
      if (t == 0) bad = k + 1;
      break;  // block-uniform: every thread read the same rv[0]
    }
    if (q != k)
      for (int j = k + t; j < L; j += kDyThreads) {
        const double u = A[(size_t)k * L + j];
        A[(size_t)k * L + j] = A[(size_t)q * L + j];
        A[(size_t)q * L + j] = u;
      }
    __syncthreads();
    const double ip = 1.0 / A[(size_t)k * L + k];
    for (int i = t; i < np1; i += kDyThreads) fc[i] = i == k ? 0.0 : A[(size_t)i * L + k];
    __syncthreads();
    for (int j = k + t; j < L; j += kDyThreads) A[(size_t)k * L + j] *= ip;
    __syncthreads();
    for (int idx = t; idx < np1 * (L - k); idx += kDyThreads) {
      const int i = idx / (L - k), j = k + idx % (L - k);
      if (i != k) A[(size_t)i * L + j] -= fc[i] * A[(size_t)k * L + j];
    }
    __syncthreads();
  }
  if (t == 0) info[b] = bad;
  if (bad) return;
  for (int p = t; p < np1; p += kDyThreads) G[(size_t)b * np1 + p] = A[(size_t)p * L + np1];
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_dyson_tau(gw_ctx* c, int64_t nprob, int n_upm, const double* tau_upm, const double* eps,
                                  const double* s, const double* sigc, double* G, int* info) {
  if (!c || nprob <= 0 || n_upm < 3 || n_upm > kDyMaxPts || !tau_upm || !eps || !s || !sigc || !G || !info)
    return GW_EINVAL;
  if (tau_upm[0] != 0.0) return set_err(c, GW_EINVAL, "gw_dyson_tau: tau_0 must be 0");
  for (int i = 1; i < n_upm; ++i)
    if (!(tau_upm[i] > tau_upm[i - 1])) return set_err(c, GW_EINVAL, "gw_dyson_tau: tau must increase");
  const double h = tau_upm[1] - tau_upm[0], beta = tau_upm[n_upm - 1];
  const double nd = std::round(beta / h);
  if (nd < 2 || nd + 1 > kDyMaxPts) return set_err(c, GW_EINVAL, "gw_dyson_tau: uniform mesh of 3 to 1024 points");
  const int n = (int)nd;
  for (int i = 0; i < n_upm; ++i) {  // every node on the uniform mesh
    const double k = std::round(tau_upm[i] / h);
    if (std::fabs(tau_upm[i] - k * h) > 1e-9 * beta)
      return set_err(c, GW_EINVAL, "gw_dyson_tau: mesh points must be multiples of tau_1 - tau_0");
  }
  const size_t per = (size_t)(n + 1) * (n + 2) * sizeof(double);
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nprob, (int64_t)((1ull << 30) / per)));
  const size_t need = per * chunk + n_upm * sizeof(double);
  if (need > c->dyt_bytes) {
    if (c->d_dyt) cudaFree(c->d_dyt);
    c->d_dyt = nullptr;
    c->dyt_bytes = 0;
    if (cudaMalloc(&c->d_dyt, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "gw_dyson_tau workspace");
    }
    c->dyt_bytes = need;
  }
  double* K = (double*)c->d_dyt;
  double* xu = K + per / sizeof(double) * chunk;
  // the nodes are copied before the call returns
  if (cudaMemcpy(xu, tau_upm, n_upm * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_err(c, GW_ECUDA, "gw_dyson_tau: copy of the mesh");
  const size_t smem = (3 * (size_t)n_upm + 3 * (size_t)(n + 1) + 2 * (size_t)(2 * n + 1)) * sizeof(double);
  cudaFuncSetAttribute(k_dyson_tau, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kt_begin(c, "dyson_tau");
  for (int64_t b0 = 0; b0 < nprob; b0 += chunk) {
    const int64_t nb = std::min(chunk, nprob - b0);
    k_dyson_tau<<<(unsigned)nb, kDyThreads, smem, c->stream>>>(n_upm, xu, eps + b0, s + b0, sigc + b0 * n_upm, n, h,
                                                                K, G + b0 * (n + 1), info + b0);
    gw_status st = check_launch(c, "dyson_tau");
    if (st != GW_OK) return st;
  }
  kt_end(c);
  return GW_OK;
}
