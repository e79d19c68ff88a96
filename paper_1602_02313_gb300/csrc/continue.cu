// Analytic continuation and quasiparticle energies (Sec. III.B.6).
//  * Pade: Vidberg-Serene continued fraction through the first npade Matsubara points.
//  * CPE : continuous-pole expansion (Staar et al. 2014): Im Sigma(w + i0) piecewise linear
//          on a real grid, Sigma(z) = sum_m b_m Phi_m(z), b_m >= 0 (causality, Im Sigma <= 0),
//          Phi_m(z) = int hat_m(x) / (z - x) dx; b from Lawson-Hanson NNLS on the normal
//          equations of the ridge-regularised fit (one warp per problem).
//  * QP  : root of F(E) = E - eps - sigx + vxc - Re Sigma^c(E + i eta), eta = 1e-4 Ha: the
//          upward crossing nearest eps on the fixed grid j 0.005 Ha within eps +- 1 Ha, refined
//          by bisection.
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

// QP root nearest eps with an upward crossing of F(E) = E - eps - sx + vxc - Re Sigma^c(E):
// scan the fixed energy grid E_j = j 0.005 Ha for eps - 1 <= E_j <= eps + 1, refine the
// crossing nearest eps by 60 bisections; without a crossing fall back to Newton from eps (ok = 0).
constexpr double kQpStep = 0.005;
constexpr double kQpRange = 1.0;
constexpr int kQpMaxScan = 401;  // points of the scan at most: 2 kQpRange / kQpStep + 1

__device__ __forceinline__ int qp_j0(double eps) { return (int)ceil((eps - kQpRange) / kQpStep); }
__device__ __forceinline__ int qp_j1(double eps) { return (int)floor((eps + kQpRange) / kQpStep); }

template <class F>
__device__ void qp_solve(F resig, double eps, double sx, double vxc, double* E_out, int* ok_out) {
  auto Ff = [&](double E) { return E - eps - sx + vxc - resig(E); };
  const int j0 = qp_j0(eps), j1 = qp_j1(eps);
  bool found = false;
  int best = 0;
  double bestd = 0.0;
  double Fprev = Ff(j0 * kQpStep);
  for (int j = j0; j < j1; ++j) {
    const double E1 = (j + 1) * kQpStep;
    const double F1 = Ff(E1);
    if (Fprev < 0.0 && F1 >= 0.0) {
      const double E0 = j * kQpStep;
      const double d = fabs(0.5 * (E0 + E1) - eps);
      if (!found || d < bestd) {
        found = true;
        best = j;
        bestd = d;
      }
    }
    Fprev = F1;
  }
  if (found) {
    double lo = best * kQpStep, hi = (best + 1) * kQpStep;
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
// one warp per problem. Lane l owns the grid variables m = l + 32 s and the passive-set
// positions k = l + 32 s (s < 4). The Cholesky factor of N_PP lives in shared memory, packed
// by rows in the order the variables joined the passive set, so that adding a variable
// appends one row (a forward substitution, O(p^2)) and removing variables refactors only the
// rows after the first removed one. y = L^-1 c_P is kept alongside and extended the same way.
constexpr int kCpeMaxGrid = 128;
constexpr int kSlots = kCpeMaxGrid / 32;
constexpr double kSeedSupport = 1e-2;  // seed weights above this fraction of the largest start active
constexpr int kWarmSolves = 8;         // solves allowed to turn the seed's support into a feasible point

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_imin(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__host__ __device__ constexpr int tri(int k) { return (k * (k + 1)) >> 1; }

struct NnlsWarp {
  double* L;     // packed lower-triangular factor, row k at tri(k)
  double* dinv;  // 1 / L_kk
  double* cv;    // c = A^T y by variable
  double* xv;    // current iterate by variable
  double* zv;    // passive-set least-squares solution by variable (0 off the set)
  int* idx;      // passive variables in the order they joined
  int* pf;       // passive flag by variable
  int* lst;      // scratch list of variables
};

// Appends variable m as row p: l = L^-1 N_{P,m} (column-oriented forward substitution over
// lane-owned partial sums), pivot sqrt(N_mm - l.l) and the new entry of y. Returns false
// (warp-uniform) when the pivot is not positive.
__device__ bool chol_append(const NnlsWarp& S, const double* __restrict__ N, int ng, int p, int m,
                            double (&yv)[kSlots], int lane) {
  double r[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int k = lane + 32 * s;
    r[s] = k < p ? N[(size_t)m * ng + S.idx[k]] : 0.0;
  }
#pragma unroll
  for (int sk = 0; sk < kSlots; ++sk) {
    if (32 * sk >= p) break;
    const int kend = min(32, p - 32 * sk);
    for (int kk = 0; kk < kend; ++kk) {
      const int k = 32 * sk + kk;
      const double lk = __shfl_sync(0xffffffffu, r[sk], kk) * S.dinv[k];
#pragma unroll
      for (int s = sk; s < kSlots; ++s) {
        const int i = lane + 32 * s;
        if (i > k && i < p) r[s] = fma(-S.L[tri(i) + k], lk, r[s]);
      }
    }
  }
  double ll = 0.0, ly = 0.0;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int k = lane + 32 * s;
    if (k < p) {
      const double l = r[s] * S.dinv[k];
      S.L[tri(p) + k] = l;
      ll = fma(l, l, ll);
      ly = fma(l, yv[s], ly);
    }
  }
  ll = warp_sum(ll);
  ly = warp_sum(ly);
  const double d = N[(size_t)m * ng + m] - ll;
  if (!(d > 0.0)) return false;
  const double piv = sqrt(d);
  const double ynew = (S.cv[m] - ly) / piv;
#pragma unroll
  for (int s = 0; s < kSlots; ++s)
    if (lane + 32 * s == p) yv[s] = ynew;
  if (lane == 0) {
    S.L[tri(p) + p] = piv;
    S.dinv[p] = 1.0 / piv;
    S.idx[p] = m;
    S.pf[m] = 1;
  }
  __syncwarp();
  return true;
}

// z_P = L^-T y (column-oriented backward substitution), scattered into zv by variable.
__device__ void chol_solve(const NnlsWarp& S, int p, const double (&yv)[kSlots], int lane) {
  double t[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) t[s] = yv[s];
#pragma unroll
  for (int sk = kSlots - 1; sk >= 0; --sk) {
    if (32 * sk >= p) continue;
    const int kend = min(32, p - 32 * sk);
    for (int kk = kend - 1; kk >= 0; --kk) {
      const int k = 32 * sk + kk;
      const double zk = __shfl_sync(0xffffffffu, t[sk], kk) * S.dinv[k];
#pragma unroll
      for (int s = 0; s <= sk; ++s) {
        const int j = lane + 32 * s;
        if (j < k) t[s] = fma(-S.L[tri(k) + j], zk, t[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < kSlots; ++s) S.zv[lane + 32 * s] = 0.0;
  __syncwarp();
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int k = lane + 32 * s;
    if (k < p) S.zv[S.idx[k]] = t[s] * S.dinv[k];
  }
  __syncwarp();
}

// After variables left the passive set (pf cleared): compacts the position list, keeps the
// factor rows before the first removed position and re-appends the rest. Returns the new
// size, or -1 if a pivot failed.
__device__ int chol_remove(const NnlsWarp& S, const double* __restrict__ N, int ng, int p, double (&yv)[kSlots],
                           int lane) {
  int kf = p;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int k = lane + 32 * s;
    if (k < p && !S.pf[S.idx[k]]) kf = min(kf, k);
  }
  kf = warp_imin(kf);
  if (kf == p) return p;
  int base = kf;
  for (int k0 = kf; k0 < p; k0 += 32) {
    const int k = k0 + lane;
    const int m = k < p ? S.idx[k] : -1;
    const bool keep = k < p && S.pf[m];
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) S.idx[base + __popc(bal & ((1u << lane) - 1u))] = m;
    base += __popc(bal);
    __syncwarp();
  }
#pragma unroll
  for (int s = 0; s < kSlots; ++s)
    if (lane + 32 * s >= kf) yv[s] = 0.0;
  for (int k = kf; k < base; ++k)
    if (!chol_append(S, N, ng, k, S.idx[k], yv, lane)) return -1;
  return base;
}

__global__ void __launch_bounds__(32) k_cpe_nnls(int64_t nprob, const double2* __restrict__ sig, int ncont,
                                                 const double* __restrict__ A, const double* __restrict__ N, int ng,
                                                 const double* __restrict__ b0, double* __restrict__ bout,
                                                 int* __restrict__ info, int* __restrict__ iters) {
  extern __shared__ double sm[];
  NnlsWarp S;
  S.L = sm;
  S.dinv = S.L + tri(ng);
  S.cv = S.dinv + kCpeMaxGrid;
  S.xv = S.cv + kCpeMaxGrid;
  S.zv = S.xv + kCpeMaxGrid;
  S.idx = reinterpret_cast<int*>(S.zv + kCpeMaxGrid);
  S.pf = S.idx + kCpeMaxGrid;
  S.lst = S.pf + kCpeMaxGrid;
  const int64_t prob = blockIdx.x;
  const int lane = threadIdx.x;
  const double2* yin = sig + (size_t)prob * ncont;
  // c = A^T y, A = [Re Phi ; Im Phi] (2 ncont x ng)
  double cmax = 0.0;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) {
    const int m = lane + 32 * s;
    double c = 0.0;
    if (m < ng)
      for (int n = 0; n < ncont; ++n) {
        c = fma(A[(size_t)n * ng + m], yin[n].x, c);
        c = fma(A[(size_t)(ncont + n) * ng + m], yin[n].y, c);
      }
    S.cv[m] = c;
    S.xv[m] = 0.0;
    S.zv[m] = 0.0;
    S.pf[m] = 0;
    cmax = fmax(cmax, fabs(c));
  }
  for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  __syncwarp();
  const double tol = 1e-13 * fmax(cmax, 1e-300);
  double yv[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; ++s) yv[s] = 0.0;
  int p = 0, outer = 0, status = 0, warm = -1;
  bool need_solve = false;
  if (b0) {
    // warm start: the passive set is the support of the seed (weights above kSeedSupport of
    // the largest), factorised by appends in increasing variable order
    double mx = 0.0;
    for (int m = lane; m < ng; m += 32) mx = fmax(mx, b0[(size_t)prob * ng + m]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int nsel = 0;
    for (int m0 = 0; m0 < ng; m0 += 32) {
      const int m = m0 + lane;
      const bool on = m < ng && mx > 0.0 && b0[(size_t)prob * ng + m] > kSeedSupport * mx;
      const unsigned bal = __ballot_sync(0xffffffffu, on);
      if (on) S.lst[nsel + __popc(bal & ((1u << lane) - 1u))] = m;
      nsel += __popc(bal);
    }
    __syncwarp();
    for (int q = 0; q < nsel; ++q)
      if (chol_append(S, N, ng, p, S.lst[q], yv, lane)) ++p;
    if (p > 0) {
      need_solve = true;
      warm = kWarmSolves;
    }
  }
  while (true) {
    if (!need_solve) {
      // gradient w = c - N x on the inactive variables; the largest positive one joins
      double w[kSlots];
#pragma unroll
      for (int s = 0; s < kSlots; ++s) w[s] = S.cv[lane + 32 * s];
      for (int k = 0; k < p; ++k) {
        const int mk = S.idx[k];
        const double xk = S.xv[mk];
        const double* Nr = N + (size_t)mk * ng;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          const int m = lane + 32 * s;
          if (m < ng) w[s] = fma(-Nr[m], xk, w[s]);
        }
      }
      double bw = tol;
      int best = -1;
#pragma unroll
      for (int s = 0; s < kSlots; ++s) {
        const int m = lane + 32 * s;
        if (m < ng && !S.pf[m] && w[s] > bw) {
          bw = w[s];
          best = m;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, bw, o);
        const int oi = __shfl_xor_sync(0xffffffffu, best, o);
        if (ob > bw || (ob == bw && oi >= 0 && (best < 0 || oi < best))) {
          bw = ob;
          best = oi;
        }
      }
      if (best < 0) break;
      if (++outer > 3 * ng) {
        status = 2;
        break;
      }
      if (!chol_append(S, N, ng, p, best, yv, lane)) {
        status = 3;
        break;
      }
      ++p;
    }
    need_solve = false;
    bool done = false;
    // inner loop: solve on the passive set, step back to feasibility if needed
    for (int inner = 0; inner < 3 * ng; ++inner) {
      chol_solve(S, p, yv, lane);
      // alpha = min over passive z <= 0 of x / (x - z)
      double alpha = 2.0;
#pragma unroll
      for (int s = 0; s < kSlots; ++s) {
        const int m = lane + 32 * s;
        if (m < ng && S.pf[m] && S.zv[m] <= 0.0) alpha = fmin(alpha, S.xv[m] / (S.xv[m] - S.zv[m]));
      }
      alpha = warp_min(alpha);
      if (alpha > 1.0) {
#pragma unroll
        for (int s = 0; s < kSlots; ++s) S.xv[lane + 32 * s] = S.zv[lane + 32 * s];
        __syncwarp();
        done = true;
        break;
      }
#pragma unroll
      for (int s = 0; s < kSlots; ++s) {
        const int m = lane + 32 * s;
        if (warm > 0) {
          // warm start: the seed's support need not be feasible; instead of stepping back
          // one variable at a time, every non-positive variable of the solve leaves and the
          // rest is solved again (at most kWarmSolves times, else a cold restart from x = 0)
          if (S.pf[m] && S.zv[m] <= 0.0) S.pf[m] = 0;
          S.xv[m] = 0.0;
        } else {
          double xm = S.xv[m] + alpha * (S.zv[m] - S.xv[m]);
          if (S.pf[m] && xm <= 1e-300) {
            xm = 0.0;
            S.pf[m] = 0;
          }
          S.xv[m] = xm;
        }
      }
      __syncwarp();
      p = chol_remove(S, N, ng, p, yv, lane);
      if (p < 0) {
        status = 3;
        break;
      }
      if (warm > 0 && --warm == 0) break;
    }
    if (status == 3) break;
    if (warm >= 0) {
      if (!done) {
        // cold restart
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          S.xv[lane + 32 * s] = 0.0;
          S.pf[lane + 32 * s] = 0;
          yv[s] = 0.0;
        }
        p = 0;
        __syncwarp();
      }
      warm = -1;
    }
  }
  for (int m = lane; m < ng; m += 32) bout[(size_t)prob * ng + m] = S.xv[m];
  if (lane == 0) {
    info[prob] = status;
    if (iters) iters[prob] = outer;
  }
}

__host__ __device__ constexpr size_t nnls_smem_bytes(int ng) {
  return sizeof(double) * ((size_t)tri(ng) + 4 * kCpeMaxGrid) + sizeof(int) * 3 * kCpeMaxGrid;
}

// Real-axis values and QP root, one warp per problem: the 401 scan points are split over
// the lanes (each lane sums the active hats at its own energies); the refinement evaluates one
// energy per step with the active hats split over the lanes and a warp sum.
// Re sum_m b_m Phi_m(E + i eta) by one thread over the hats with b_m != 0; the node logarithms
// are computed only for the nodes of those hats, and shared between neighbouring hats (a cache
// of the last three nodes).
__device__ double resig_cpe_lane(const double* b, const double* x, int ng, double E) {
  const cd z = {E, kEta};
  double s = 0.0;
  int i0 = -1, i1 = -1, i2 = -1;
  cd c0{0.0, 0.0}, c1{0.0, 0.0}, c2{0.0, 0.0};
  auto node_log = [&](int n) {
    if (n == i2) return c2;
    if (n == i1) return c1;
    if (n == i0) return c0;
    const cd v = clog_(csub(z, cd{x[n], 0.0}));
    i0 = i1;
    c0 = c1;
    i1 = i2;
    c1 = c2;
    i2 = n;
    c2 = v;
    return v;
  };
  for (int m = 0; m < ng; ++m) {
    if (b[m] == 0.0) continue;
    const cd l0 = node_log(m), l1 = node_log(m + 1), l2 = node_log(m + 2);
    const double x0 = x[m], x1 = x[m + 1], x2 = x[m + 2];
    const cd rise = csub(cmul(cd{(z.x - x0) / (x1 - x0), z.y / (x1 - x0)}, csub(l0, l1)), cd{1.0, 0.0});
    const cd fall = cadd(cmul(cd{(x2 - z.x) / (x2 - x1), -z.y / (x2 - x1)}, csub(l1, l2)), cd{1.0, 0.0});
    s += b[m] * (rise.x + fall.x);
  }
  return s;
}
// The hats with b_m != 0 of one problem, compacted in ascending m into the warp's shared lists
// (one ballot per 32 hats); returns their number.
__device__ int compact_hats(const double* b, int ng, int lane, int* aidx, double* aval) {
  int na = 0;
  for (int m0 = 0; m0 < ng; m0 += 32) {
    const int m = m0 + lane;
    const double v = m < ng ? b[m] : 0.0;
    const unsigned mask = __ballot_sync(0xffffffffu, v != 0.0);
    if (v != 0.0) {
      const int pos = na + __popc(mask & ((1u << lane) - 1u));
      aidx[pos] = m;
      aval[pos] = v;
    }
    na += __popc(mask);
  }
  __syncwarp();
  return na;
}

// Re sum_m b_m Phi_m(E + i eta) over the compacted hats, split evenly over the lanes (one
// hat per lane for up to 32 active hats), and a warp sum.
__device__ double resig_cpe_list(const int* aidx, const double* aval, int na, const double* x, double E,
                                 int lane) {
  const cd z = {E, kEta};
  double s = 0.0;
  for (int a = lane; a < na; a += 32) {
    const int m = aidx[a];
    const double x0 = x[m], x1 = x[m + 1], x2 = x[m + 2];
    const cd l0 = clog_(csub(z, cd{x0, 0.0})), l1 = clog_(csub(z, cd{x1, 0.0})), l2 = clog_(csub(z, cd{x2, 0.0}));
    const cd rise = csub(cmul(cd{(z.x - x0) / (x1 - x0), z.y / (x1 - x0)}, csub(l0, l1)), cd{1.0, 0.0});
    const cd fall = cadd(cmul(cd{(x2 - z.x) / (x2 - x1), -z.y / (x2 - x1)}, csub(l1, l2)), cd{1.0, 0.0});
    s += aval[a] * (rise.x + fall.x);
  }
  return warp_sum(s);
}

// Re Phi_m(E_j + i eta) of every hat m on the scan grid E_j = j kQpStep, j in
// [kTabJ0, kTabJ0 + kTabN), with the same arithmetic as resig_cpe_lane (node logarithms from
// clog_, rise + fall), so that the QP scan from the table gives the same F_j bit for bit.
constexpr int kTabJ0 = -600, kTabN = 1201;  // E in [-3, 3] Ha

__global__ void k_cpe_table(const double* __restrict__ x, int ng, double* __restrict__ tab) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kTabN * ng) return;
  const int m = e % ng, jj = e / ng;
  const cd z = {(kTabJ0 + jj) * kQpStep, kEta};
  const cd l0 = clog_(csub(z, cd{x[m], 0.0})), l1 = clog_(csub(z, cd{x[m + 1], 0.0})),
           l2 = clog_(csub(z, cd{x[m + 2], 0.0}));
  const double x0 = x[m], x1 = x[m + 1], x2 = x[m + 2];
  const cd rise = csub(cmul(cd{(z.x - x0) / (x1 - x0), z.y / (x1 - x0)}, csub(l0, l1)), cd{1.0, 0.0});
  const cd fall = cadd(cmul(cd{(x2 - z.x) / (x2 - x1), -z.y / (x2 - x1)}, csub(l1, l2)), cd{1.0, 0.0});
  tab[e] = rise.x + fall.x;
}

__global__ void k_cpe_qp(int64_t nprob, const double* __restrict__ b, const double* __restrict__ x, int ng,
                         const double* __restrict__ tab, const double* __restrict__ eps, const double* __restrict__ sigx,
                         const double* __restrict__ vxc, int nreal, const double* __restrict__ wr,
                         double2* __restrict__ sreal, double* __restrict__ eqp, int* __restrict__ info) {
  __shared__ int s_idx[4][kCpeMaxGrid];  // the block's 4 warps' active-hat lists
  __shared__ double s_val[4][kCpeMaxGrid];
  const int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= nprob) return;
  const double* bp = b + (size_t)p * ng;
  int* aidx = s_idx[threadIdx.x >> 5];
  double* aval = s_val[threadIdx.x >> 5];
  const int na = compact_hats(bp, ng, lane, aidx, aval);
  for (int r = 0; r < nreal; ++r) {
    double sx_ = 0.0, sy_ = 0.0;
    for (int m = lane; m < ng; m += 32)
      if (bp[m] != 0.0) {
        const cd ph = cpe_phi(x, m, {wr[r], kEta});
        sx_ += bp[m] * ph.x;
        sy_ += bp[m] * ph.y;
      }
    sx_ = warp_sum(sx_);
    sy_ = warp_sum(sy_);
    if (lane == 0) sreal[(size_t)p * nreal + r] = make_double2(sx_, sy_);
  }
  const double e0 = eps[p], s0 = sigx[p], v0 = vxc[p];
  auto F = [&](double E) { return E - e0 - s0 + v0 - resig_cpe_list(aidx, aval, na, x, E, lane); };
  // scan: F at E_j = j kQpStep, j0 <= j <= j1, lanes take consecutive blocks. Inside the range of
  // the table (each hat's Re Phi_m on the grid, built by gw_cpe_setup with the same arithmetic as
  // resig_cpe_lane) Re Sigma^c(E_j) is a dot product over the active hats; outside it each lane
  // evaluates the hats itself.
  const int j0 = qp_j0(e0), j1 = qp_j1(e0), nscan = j1 - j0 + 1;
  const int per = (nscan + 31) / 32;
  const bool use_tab = tab != nullptr && j0 >= kTabJ0 && j1 < kTabJ0 + kTabN;
  double fv[kQpMaxScan / 32 + 2];
  for (int q = 0; q <= per; ++q) {
    const int i = min(lane * per + q, nscan - 1);
    const double E = (j0 + i) * kQpStep;
    double rs = 0.0;
    if (use_tab) {
      const double* T = tab + (size_t)(j0 + i - kTabJ0) * ng;
      for (int a = 0; a < na; ++a) rs += aval[a] * T[aidx[a]];  // ascending m, as over all hats
    } else {
      rs = resig_cpe_lane(bp, x, ng, E);
    }
    fv[q] = E - e0 - s0 + v0 - rs;
  }
  int best = -1;
  double bestd = 0.0;
  for (int q = 0; q < per; ++q) {
    const int i = lane * per + q;
    if (i + 1 >= nscan) break;
    if (fv[q] < 0.0 && fv[q + 1] >= 0.0) {
      const double d = fabs(0.5 * ((j0 + i) * kQpStep + (j0 + i + 1) * kQpStep) - e0);
      if (best < 0 || d < bestd || (d == bestd && i < best)) {
        best = i;
        bestd = d;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const int ob = __shfl_xor_sync(0xffffffffu, best, o);
    const double od = __shfl_xor_sync(0xffffffffu, bestd, o);
    if (ob >= 0 && (best < 0 || od < bestd || (od == bestd && ob < best))) {
      best = ob;
      bestd = od;
    }
  }
  double E;
  int ok;
  if (best >= 0) {
    // the root in [lo, hi] (F(lo) < 0 <= F(hi) from the scan) by the Illinois variant of
    // regula falsi: the secant point of the bracket, with the retained end's value halved when
    // the same end is kept twice in a row, so that both ends converge; it reaches the root the
    // bisection of the oracle reaches in ~6-10 evaluations instead of 60
    const int owner = best / per, qo = best - owner * per;
    double flo = 0.0, fhi = 0.0;
    if (lane == owner) {
      flo = fv[qo];
      fhi = fv[qo + 1];
    }
    flo = __shfl_sync(0xffffffffu, flo, owner);
    fhi = __shfl_sync(0xffffffffu, fhi, owner);
    double lo = (j0 + best) * kQpStep, hi = (j0 + best + 1) * kQpStep;
    int side = 0;
    E = 0.5 * (lo + hi);
    for (int it = 0; it < 60; ++it) {
      double c = fhi != flo ? (lo * fhi - hi * flo) / (fhi - flo) : 0.5 * (lo + hi);
      if (!(c > lo && c < hi)) c = 0.5 * (lo + hi);
      if (!(c > lo && c < hi)) break;  // the bracket is down to adjacent doubles
      E = c;
      const double fc = F(c);
      if (fc == 0.0) break;
      if (fc < 0.0) {
        lo = c;
        flo = fc;
        if (side < 0) fhi *= 0.5;
        side = -1;
      } else {
        hi = c;
        fhi = fc;
        if (side > 0) flo *= 0.5;
        side = 1;
      }
      if (hi - lo <= 4e-16 * fmax(1.0, fabs(c))) break;
    }
    ok = 1;
  } else {
    E = e0;
    ok = 0;
    const double de = 1e-6;
    for (int it = 0; it < 100; ++it) {
      const double Fv = F(E);
      const double dF = 1.0 - (resig_cpe_list(aidx, aval, na, x, E + de, lane) -
                               resig_cpe_list(aidx, aval, na, x, E - de, lane)) /
                                  (2.0 * de);
      if (dF == 0.0 || !isfinite(dF)) break;
      double step = fmax(-0.5, fmin(0.5, Fv / dF));
      E -= step;
      if (fabs(step) < 1e-12 * fmax(1.0, fabs(E))) break;
    }
  }
  if (lane == 0) {
    eqp[p] = E;
    if (info[p] == 0 && !ok) info[p] = 1;
  }
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
  const size_t smem = nnls_smem_bytes(c->cpe_ngrid);
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
  k_cpe_nnls<<<(unsigned)nprob, 32, smem, c->stream>>>(nprob, (const double2*)sig_iw, c->ncont, c->d_cpe_A, c->d_cpe_N,
                                                     c->cpe_ngrid, seed, c->d_cpe_b, info, c->d_cpe_iters);
  gw_status s = check_launch(c, "cpe_nnls");
  if (s != GW_OK) return s;
  k_cpe_qp<<<(unsigned)((nprob + 3) / 4), 128, 0, c->stream>>>(nprob, c->d_cpe_b, c->d_cpe_x, c->cpe_ngrid,
                                                                 c->d_cpe_tab, eps,
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
  for (double** p : {&c->d_cpe_x, &c->d_cpe_A, &c->d_cpe_N, &c->d_cpe_tab})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  if (cudaMalloc((void**)&c->d_cpe_x, sizeof(double) * (ng + 2)) != cudaSuccess ||
      cudaMalloc((void**)&c->d_cpe_A, sizeof(double) * A.size()) != cudaSuccess ||
      cudaMalloc((void**)&c->d_cpe_N, sizeof(double) * N.size()) != cudaSuccess ||
      cudaMalloc((void**)&c->d_cpe_tab, sizeof(double) * kTabN * ng) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, GW_ENOMEM, "gw_cpe_setup");
  }
  cudaMemcpy(c->d_cpe_x, x, sizeof(double) * (ng + 2), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_cpe_A, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_cpe_N, N.data(), sizeof(double) * N.size(), cudaMemcpyHostToDevice);
  k_cpe_table<<<(kTabN * ng + 255) / 256, 256, 0, c->stream>>>(c->d_cpe_x, ng, c->d_cpe_tab);
  if (check_launch(c, "cpe_table") != GW_OK) return GW_ECUDA;
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
