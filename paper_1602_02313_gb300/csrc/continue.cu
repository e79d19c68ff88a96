// Analytic continuation and quasiparticle energies (Sec. III.B.6).
//  * Pade: Vidberg-Serene continued fraction through the first npade Matsubara points.
//  * CPE : continuous-pole expansion (Staar et al. 2014): Im Sigma(w + i0) piecewise linear
//          on a real grid, Sigma(z) = sum_m b_m Phi_m(z), b_m >= 0 (causality, Im Sigma <= 0),
//          Phi_m(z) = int hat_m(x) / (z - x) dx; b from Lawson-Hanson NNLS on the normal
//          equations of the ridge-regularised fit (one thread block per problem).
//  * QP  : root of F(E) = E - eps - sigx + vxc - Re Sigma^c(E + i eta), eta = 1e-4 Ha: the
//          upward crossing nearest eps on a 0.005 Ha scan of eps +- 1 Ha, refined by bisection.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <vector>

#include "gw_internal.h"

namespace gwi {

namespace {

constexpr double kEta = 1e-4;
constexpr int kPadeMax = 64;

struct cd {
  double x, y;
};
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
  const double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ __forceinline__ cd clog_(cd a) { return {log(hypot(a.x, a.y)), atan2(a.y, a.x)}; }

__device__ cd pade_eval(const cd* a, int n, double beta, cd x) {
  cd t = {1.0, 0.0};
  for (int p = n - 1; p >= 1; --p) {
    const cd zp = {0.0, (2.0 * (p - 1) + 1.0) * 3.141592653589793 / beta};
    t = cadd(cd{1.0, 0.0}, cdiv(cmul(a[p], csub(x, zp)), t));
  }
  return cdiv(a[0], t);
}

// CPE basis: hats on interior nodes x[1..ng] of x[0..ng+1].
__device__ cd cpe_phi(const double* x, int m, cd z) {
  const double x0 = x[m], x1 = x[m + 1], x2 = x[m + 2];
  const cd l0 = clog_(csub(z, cd{x0, 0.0})), l1 = clog_(csub(z, cd{x1, 0.0})), l2 = clog_(csub(z, cd{x2, 0.0}));
  const cd rise = csub(cmul(cd{(z.x - x0) / (x1 - x0), z.y / (x1 - x0)}, csub(l0, l1)), cd{1.0, 0.0});
  const cd fall = cadd(cmul(cd{(x2 - z.x) / (x2 - x1), -z.y / (x2 - x1)}, csub(l1, l2)), cd{1.0, 0.0});
  return cadd(rise, fall);
}

__device__ double resig_pade(const cd* a, int n, double beta, double E) { return pade_eval(a, n, beta, {E, kEta}).x; }

// Re sum_m b_m Phi_m(E + i eta); the node logarithms are shared between neighbouring hats.
__device__ double resig_cpe(const double* b, const double* x, int ng, double E) {
  const cd z = {E, kEta};
  double s = 0.0;
  cd l0 = clog_(csub(z, cd{x[0], 0.0})), l1 = clog_(csub(z, cd{x[1], 0.0}));
  for (int m = 0; m < ng; ++m) {
    const cd l2 = clog_(csub(z, cd{x[m + 2], 0.0}));
    if (b[m] != 0.0) {
      const double x0 = x[m], x1 = x[m + 1], x2 = x[m + 2];
      const cd rise = csub(cmul(cd{(z.x - x0) / (x1 - x0), z.y / (x1 - x0)}, csub(l0, l1)), cd{1.0, 0.0});
      const cd fall = cadd(cmul(cd{(x2 - z.x) / (x2 - x1), -z.y / (x2 - x1)}, csub(l1, l2)), cd{1.0, 0.0});
      s += b[m] * (rise.x + fall.x);
    }
    l0 = l1;
    l1 = l2;
  }
  return s;
}

// QP root nearest eps with an upward crossing of F(E) = E - eps - sx + vxc - Re Sigma^c(E):
// scan E_j = eps + (j - 200) 0.005 Ha (j = 0..400), refine the crossing nearest eps by 60
// bisections; without a crossing fall back to Newton from eps (ok = 0).
constexpr int kQpScan = 401;
constexpr double kQpStep = 0.005;

template <class F>
__device__ void qp_solve(F resig, double eps, double sx, double vxc, double* E_out, int* ok_out) {
  auto Ff = [&](double E) { return E - eps - sx + vxc - resig(E); };
  int best = -1;
  double bestd = 0.0;
  double Fprev = Ff(eps - (kQpScan / 2) * kQpStep);
  for (int j = 0; j < kQpScan - 1; ++j) {
    const double E1 = eps + (j + 1 - kQpScan / 2) * kQpStep;
    const double F1 = Ff(E1);
    if (Fprev < 0.0 && F1 >= 0.0) {
      const double E0 = eps + (j - kQpScan / 2) * kQpStep;
      const double d = fabs(0.5 * (E0 + E1) - eps);
      if (best < 0 || d < bestd) {
        best = j;
        bestd = d;
      }
    }
    Fprev = F1;
  }
  if (best >= 0) {
    double lo = eps + (best - kQpScan / 2) * kQpStep, hi = eps + (best + 1 - kQpScan / 2) * kQpStep;
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (Ff(mid) < 0.0)
        lo = mid;
      else
        hi = mid;
    }
    *E_out = 0.5 * (lo + hi);
    *ok_out = 1;
    return;
  }
  double E = eps;
  const double de = 1e-6;
  for (int it = 0; it < 100; ++it) {
    const double Fv = Ff(E);
    const double dF = 1.0 - (resig(E + de) - resig(E - de)) / (2.0 * de);
    if (dF == 0.0 || !isfinite(dF)) break;
    double step = Fv / dF;
    step = fmax(-0.5, fmin(0.5, step));
    E -= step;
    if (fabs(step) < 1e-12 * fmax(1.0, fabs(E))) break;
  }
  *E_out = E;
  *ok_out = 0;
}

// One thread per problem: coefficients, real-axis values, QP root.
__global__ void k_pade(int64_t nprob, const double2* __restrict__ sig, int ncont, int npade, double beta,
                       const double* __restrict__ eps, const double* __restrict__ sigx, const double* __restrict__ vxc,
                       int nreal, const double* __restrict__ wr, double2* __restrict__ sreal, double* __restrict__ eqp,
                       int* __restrict__ info) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  cd g[kPadeMax], a[kPadeMax];
  for (int i = 0; i < npade; ++i) {
    const double2 s = sig[(size_t)p * ncont + i];
    g[i] = {s.x, s.y};
  }
  a[0] = g[0];
  for (int q = 1; q < npade; ++q) {
    const cd prev = g[q - 1];
    const cd zq1 = {0.0, (2.0 * (q - 1) + 1.0) * 3.141592653589793 / beta};
    for (int i = q; i < npade; ++i) {
      const cd zi = {0.0, (2.0 * i + 1.0) * 3.141592653589793 / beta};
      g[i] = cdiv(csub(prev, g[i]), cmul(csub(zi, zq1), g[i]));
    }
    a[q] = g[q];
  }
  for (int r = 0; r < nreal; ++r) {
    const cd v = pade_eval(a, npade, beta, {wr[r], kEta});
    sreal[(size_t)p * nreal + r] = make_double2(v.x, v.y);
  }
  double E;
  int ok;
  qp_solve([&](double e) { return resig_pade(a, npade, beta, e); }, eps[p], sigx[p], vxc[p], &E, &ok);
  eqp[p] = E;
  info[p] = ok ? 0 : 1;
}

// Lawson-Hanson NNLS on the normal equations N b = c (N = A^T A + lambda^2 I, c = A^T y),
// one block per problem; N_PP is factorised by Cholesky in shared memory each solve.
constexpr int kCpeMaxGrid = 128;

__global__ void __launch_bounds__(128) k_cpe_nnls(int64_t nprob, const double2* __restrict__ sig, int ncont,
                                                  const double* __restrict__ A, const double* __restrict__ N, int ng,
                                                  const double* __restrict__ b0, double* __restrict__ bout,
                                                  int* __restrict__ info, int* __restrict__ iters) {
  extern __shared__ double L[];  // [kCpeMaxGrid][kCpeMaxGrid], dynamic
  __shared__ double cvec[kCpeMaxGrid], x[kCpeMaxGrid], z[kCpeMaxGrid], w[kCpeMaxGrid];
  __shared__ int Pset[kCpeMaxGrid], idx[kCpeMaxGrid];
  __shared__ int np_, tbest, done;
  __shared__ double sred[128];
  const int64_t prob = blockIdx.x;
  const int t = threadIdx.x;
  const double2* y = sig + (size_t)prob * ncont;
  // c = A^T y, A = [Re Phi ; Im Phi] (2 ncont x ng)
  for (int m = t; m < ng; m += blockDim.x) {
    double s = 0.0;
    for (int n = 0; n < ncont; ++n) {
      s = fma(A[(size_t)n * ng + m], y[n].x, s);
      s = fma(A[(size_t)(ncont + n) * ng + m], y[n].y, s);
    }
    cvec[m] = s;
    x[m] = 0.0;
    Pset[m] = 0;
  }
  __syncthreads();
  if (b0) {
    // warm start: passive set = support of the seed, then one feasible LS solve below
    for (int m = t; m < ng; m += blockDim.x) {
      const double v = b0[(size_t)prob * ng + m];
      Pset[m] = v > 0.0 ? 1 : 0;
      x[m] = v > 0.0 ? v : 0.0;
    }
  }
  __syncthreads();
  double cmax = 0.0;
  for (int m = 0; m < ng; ++m) cmax = fmax(cmax, fabs(cvec[m]));
  const double tol = 1e-13 * fmax(cmax, 1e-300);
  int outer = 0, status = 0;
  bool need_solve = b0 != nullptr;
  while (true) {
    if (!need_solve) {
      // gradient w = c - N x; pick the most violating inactive index
      for (int m = t; m < ng; m += blockDim.x) {
        double s = cvec[m];
        for (int j = 0; j < ng; ++j)
          if (x[j] != 0.0) s -= N[(size_t)m * ng + j] * x[j];
        w[m] = s;
      }
      __syncthreads();
      if (t == 0) {
        int best = -1;
        double bw = tol;
        for (int m = 0; m < ng; ++m)
          if (!Pset[m] && w[m] > bw) {
            bw = w[m];
            best = m;
          }
        tbest = best;
        if (best >= 0) Pset[best] = 1;
      }
      __syncthreads();
      if (tbest < 0) break;
      if (++outer > 3 * ng) {
        status = 2;
        break;
      }
    }
    need_solve = false;
    // inner loop: solve on the passive set, step back to feasibility if needed
    for (int inner = 0; inner < 3 * ng; ++inner) {
      if (t == 0) {
        int c = 0;
        for (int m = 0; m < ng; ++m)
          if (Pset[m]) idx[c++] = m;
        np_ = c;
      }
      __syncthreads();
      const int p = np_;
      for (int e = t; e < p * p; e += blockDim.x) {
        const int r = e / p, s = e % p;
        L[r * kCpeMaxGrid + s] = N[(size_t)idx[r] * ng + idx[s]];
      }
      __syncthreads();
      // Cholesky N_PP = L L^T (lower triangle, in place)
      for (int j = 0; j < p; ++j) {
        if (t == 0) {
          double d = L[j * kCpeMaxGrid + j];
          for (int k = 0; k < j; ++k) d -= L[j * kCpeMaxGrid + k] * L[j * kCpeMaxGrid + k];
          L[j * kCpeMaxGrid + j] = sqrt(fmax(d, 1e-300));
        }
        __syncthreads();
        for (int i = j + 1 + t; i < p; i += blockDim.x) {
          double s = L[i * kCpeMaxGrid + j];
          for (int k = 0; k < j; ++k) s -= L[i * kCpeMaxGrid + k] * L[j * kCpeMaxGrid + k];
          L[i * kCpeMaxGrid + j] = s / L[j * kCpeMaxGrid + j];
        }
        __syncthreads();
      }
      if (t == 0) {
        // forward / backward substitution into z (compressed), then scatter
        for (int i = 0; i < p; ++i) {
          double s = cvec[idx[i]];
          for (int k = 0; k < i; ++k) s -= L[i * kCpeMaxGrid + k] * sred[k];
          sred[i] = s / L[i * kCpeMaxGrid + i];
        }
        for (int i = p - 1; i >= 0; --i) {
          double s = sred[i];
          for (int k = i + 1; k < p; ++k) s -= L[k * kCpeMaxGrid + i] * sred[k];
          sred[i] = s / L[i * kCpeMaxGrid + i];
        }
        for (int m = 0; m < ng; ++m) z[m] = 0.0;
        for (int i = 0; i < p; ++i) z[idx[i]] = sred[i];
        // feasibility
        double alpha = 2.0;
        for (int i = 0; i < p; ++i) {
          const int m = idx[i];
          if (z[m] <= 0.0) {
            const double a = x[m] / (x[m] - z[m]);
            if (a < alpha) alpha = a;
          }
        }
        if (alpha > 1.0) {
          for (int m = 0; m < ng; ++m) x[m] = z[m];
          done = 1;
        } else {
          for (int m = 0; m < ng; ++m) {
            x[m] += alpha * (z[m] - x[m]);
            if (Pset[m] && x[m] <= 1e-300) {
              x[m] = 0.0;
              Pset[m] = 0;
            }
          }
          done = 0;
        }
      }
      __syncthreads();
      if (done) break;
    }
  }
  for (int m = t; m < ng; m += blockDim.x) bout[(size_t)prob * ng + m] = x[m];
  if (t == 0) {
    info[prob] = status;
    if (iters) iters[prob] = outer;
  }
}

__global__ void k_cpe_qp(int64_t nprob, const double* __restrict__ b, const double* __restrict__ x, int ng,
                         const double* __restrict__ eps, const double* __restrict__ sigx,
                         const double* __restrict__ vxc, int nreal, const double* __restrict__ wr,
                         double2* __restrict__ sreal, double* __restrict__ eqp, int* __restrict__ info) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const double* bp = b + (size_t)p * ng;
  for (int r = 0; r < nreal; ++r) {
    cd s = {0.0, 0.0};
    for (int m = 0; m < ng; ++m)
      if (bp[m] != 0.0) {
        const cd ph = cpe_phi(x, m, {wr[r], kEta});
        s.x += bp[m] * ph.x;
        s.y += bp[m] * ph.y;
      }
    sreal[(size_t)p * nreal + r] = make_double2(s.x, s.y);
  }
  double E;
  int ok;
  qp_solve([&](double e) { return resig_cpe(bp, x, ng, e); }, eps[p], sigx[p], vxc[p], &E, &ok);
  eqp[p] = E;
  if (info[p] == 0 && !ok) info[p] = 1;
}

}  // namespace

gw_status launch_continue(gw_ctx* c, int method, int64_t nprob, const double* sig_iw, const double* eps,
                          const double* sigx, const double* vxc, int nreal, const double* omega_real,
                          double* sig_real, double* e_qp, int* info) {
  if (method == GW_PADE) {
    const int npade = c->ncont < kPadeMax ? c->ncont : kPadeMax;
    k_pade<<<(unsigned)((nprob + 63) / 64), 64, 0, c->stream>>>(nprob, (const double2*)sig_iw, c->ncont, npade,
                                                                 c->beta, eps, sigx, vxc, nreal, omega_real,
                                                                 (double2*)sig_real, e_qp, info);
    return check_launch(c, "pade");
  }
  const size_t need = (size_t)nprob * c->cpe_ngrid * sizeof(double);
  if (need > c->cpe_b_bytes) {
    if (c->d_cpe_b) cudaFree(c->d_cpe_b);
    c->d_cpe_b = nullptr;
    c->cpe_b_bytes = 0;
    if (cudaMalloc((void**)&c->d_cpe_b, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "cpe workspace");
    }
    c->cpe_b_bytes = need;
  }
  const size_t smem = sizeof(double) * kCpeMaxGrid * kCpeMaxGrid;
  cudaFuncSetAttribute(k_cpe_nnls, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  c->cpe_nprob = nprob;
  if ((size_t)nprob * sizeof(int) > c->cpe_iters_bytes) {
    if (c->d_cpe_iters) cudaFree(c->d_cpe_iters);
    c->d_cpe_iters = nullptr;
    c->cpe_iters_bytes = 0;
    if (cudaMalloc((void**)&c->d_cpe_iters, nprob * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "cpe iteration counts");
    }
    c->cpe_iters_bytes = nprob * sizeof(int);
  }
  const double* seed = nullptr;
  if (c->cpe_seed_nprob == nprob) seed = c->d_cpe_seed;  // a seed set by gw_cpe_seed, consumed once
  c->cpe_seed_nprob = 0;
  k_cpe_nnls<<<(unsigned)nprob, 128, smem, c->stream>>>(nprob, (const double2*)sig_iw, c->ncont, c->d_cpe_A, c->d_cpe_N,
                                                     c->cpe_ngrid, seed, c->d_cpe_b, info, c->d_cpe_iters);
  gw_status s = check_launch(c, "cpe_nnls");
  if (s != GW_OK) return s;
  k_cpe_qp<<<(unsigned)((nprob + 63) / 64), 64, 0, c->stream>>>(nprob, c->d_cpe_b, c->d_cpe_x, c->cpe_ngrid, eps,
                                                                 sigx, vxc, nreal, omega_real, (double2*)sig_real,
                                                                 e_qp, info);
  return check_launch(c, "cpe_qp");
}

}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_cpe_setup(gw_ctx* c, int ng, const double* x, double ridge) {
  if (!c || !x || ng < 2 || ng > kCpeMaxGrid || !(ridge >= 0)) return GW_EINVAL;
  for (int i = 1; i < ng + 2; ++i)
    if (!(x[i] > x[i - 1])) return GW_EINVAL;
  const int nc = c->ncont;
  std::vector<double> A((size_t)2 * nc * ng), N((size_t)ng * ng, 0.0);
  for (int n = 0; n < nc; ++n) {
    const std::complex<double> z(0.0, (2.0 * n + 1.0) * M_PI / c->beta);
    for (int m = 0; m < ng; ++m) {
      const double x0 = x[m], x1 = x[m + 1], x2 = x[m + 2];
      const std::complex<double> l0 = std::log(z - x0), l1 = std::log(z - x1), l2 = std::log(z - x2);
      const std::complex<double> ph = (z - x0) / (x1 - x0) * (l0 - l1) - 1.0 + (x2 - z) / (x2 - x1) * (l1 - l2) + 1.0;
      A[(size_t)n * ng + m] = ph.real();
      A[(size_t)(nc + n) * ng + m] = ph.imag();
    }
  }
  double fro = 0.0;
  for (double a : A) fro += a * a;
  const double lam2 = ridge * ridge * fro;
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < ng; ++j) {
      double s = 0.0;
      for (int r = 0; r < 2 * nc; ++r) s += A[(size_t)r * ng + i] * A[(size_t)r * ng + j];
      N[(size_t)i * ng + j] = s + (i == j ? lam2 : 0.0);
    }
  for (double** p : {&c->d_cpe_x, &c->d_cpe_A, &c->d_cpe_N})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  if (cudaMalloc((void**)&c->d_cpe_x, sizeof(double) * (ng + 2)) != cudaSuccess ||
      cudaMalloc((void**)&c->d_cpe_A, sizeof(double) * A.size()) != cudaSuccess ||
      cudaMalloc((void**)&c->d_cpe_N, sizeof(double) * N.size()) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, GW_ENOMEM, "gw_cpe_setup");
  }
  cudaMemcpy(c->d_cpe_x, x, sizeof(double) * (ng + 2), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_cpe_A, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_cpe_N, N.data(), sizeof(double) * N.size(), cudaMemcpyHostToDevice);
  c->cpe_ngrid = ng;
  c->cpe_ridge = ridge;
  c->cpe_x.assign(x, x + ng + 2);
  return GW_OK;
}

extern "C" gw_status gw_cpe_coeffs(gw_ctx* c, double* b) {
  if (!c || !b || !c->d_cpe_b || c->cpe_nprob <= 0) return GW_EINVAL;
  const size_t bytes = (size_t)c->cpe_nprob * c->cpe_ngrid * sizeof(double);
  if (cudaMemcpyAsync(b, c->d_cpe_b, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return set_err(c, GW_ECUDA, "gw_cpe_coeffs");
  return GW_OK;
}

// ---------------------------------------------------------------------------
// Learned-seed support (not in the paper): features and fit matrix for the MLP,
// and the warm start of the next GW_CPE call.
// ---------------------------------------------------------------------------
namespace gwi {
namespace seedk {
// x[p] = [Re s_p(i w_0..nfit-1), Im s_p(...)] / scale_p, scale_p = max |component| (1 if zero)
__global__ void k_cpe_features(int64_t nprob, const double2* __restrict__ sig, int ncont, int nfit,
                               float* __restrict__ x, double* __restrict__ scale) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const double2* s = sig + (size_t)p * ncont;
  double mx = 0.0;
  for (int n = 0; n < nfit; ++n) mx = fmax(mx, fmax(fabs(s[n].x), fabs(s[n].y)));
  const double sc = mx > 0.0 ? mx : 1.0;
  for (int n = 0; n < nfit; ++n) {
    x[(size_t)p * 2 * nfit + n] = (float)(s[n].x / sc);
    x[(size_t)p * 2 * nfit + nfit + n] = (float)(s[n].y / sc);
  }
  scale[p] = sc;
}
__global__ void k_cpe_fitmat(const double* __restrict__ A, int ncont, int ng, int nfit, float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * nfit * ng) return;
  const int r = e / ng, m = e % ng;
  const int src = r < nfit ? r : ncont + (r - nfit);
  out[e] = (float)A[(size_t)src * ng + m];
}
__global__ void k_cpe_seed(int64_t n, int ng, const float* __restrict__ bhat, const double* __restrict__ scale,
                           double* __restrict__ b0) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  b0[e] = (double)bhat[e] * scale[e / ng];
}
}  // namespace seedk
}  // namespace gwi
using namespace gwi::seedk;

extern "C" gw_status gw_cpe_features(gw_ctx* c, int64_t nprob, const double* sig_iw, int nfit, float* x,
                                     double* scale) {
  if (!c || nprob <= 0 || !sig_iw || !x || !scale || nfit < 1 || nfit > c->ncont) return GW_EINVAL;
  k_cpe_features<<<(unsigned)((nprob + 127) / 128), 128, 0, c->stream>>>(nprob, (const double2*)sig_iw, c->ncont,
                                                                         nfit, x, scale);
  return check_launch(c, "cpe_features");
}

extern "C" gw_status gw_cpe_fit_matrix(gw_ctx* c, int nfit, float* A) {
  if (!c || !A || c->cpe_ngrid == 0 || nfit < 1 || nfit > c->ncont) return GW_EINVAL;
  const int n = 2 * nfit * c->cpe_ngrid;
  k_cpe_fitmat<<<(n + 255) / 256, 256, 0, c->stream>>>(c->d_cpe_A, c->ncont, c->cpe_ngrid, nfit, A);
  return check_launch(c, "cpe_fit_matrix");
}

extern "C" gw_status gw_cpe_seed(gw_ctx* c, int64_t nprob, const float* bhat, const double* scale) {
  if (!c || nprob <= 0 || !bhat || !scale || c->cpe_ngrid == 0) return GW_EINVAL;
  const size_t need = (size_t)nprob * c->cpe_ngrid * sizeof(double);
  if (need > c->cpe_seed_bytes) {
    if (c->d_cpe_seed) cudaFree(c->d_cpe_seed);
    c->d_cpe_seed = nullptr;
    c->cpe_seed_bytes = 0;
    if (cudaMalloc((void**)&c->d_cpe_seed, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "cpe seed");
    }
    c->cpe_seed_bytes = need;
  }
  const int64_t n = nprob * c->cpe_ngrid;
  k_cpe_seed<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->cpe_ngrid, bhat, scale, c->d_cpe_seed);
  c->cpe_seed_nprob = nprob;
  return check_launch(c, "cpe_seed");
}

extern "C" gw_status gw_cpe_iterations(gw_ctx* c, int* iters) {
  if (!c || !iters || !c->d_cpe_iters || c->cpe_nprob <= 0) return GW_EINVAL;
  if (cudaMemcpyAsync(iters, c->d_cpe_iters, c->cpe_nprob * sizeof(int), cudaMemcpyDeviceToDevice, c->stream) !=
      cudaSuccess)
    return set_err(c, GW_ECUDA, "gw_cpe_iterations");
  return GW_OK;
}
