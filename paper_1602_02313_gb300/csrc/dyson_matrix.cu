// Dyson update of the full band matrix of G (Eq. dysonGF of Sec. II without the diagonal
// approximation of Sec. III.B; the paper names off-diagonal G as future work), posed at the
// sparse fermionic Matsubara set like the diagonal update of gw_green_tau:
//   G(k|i w) = [i w - H~ - Sigma^c(k|i w)]^-1,   H~ = diag(eps) + Sigma^x - Sigma_0,
// with the tail (i w - H~)^-1 subtracted in frequency and added back exactly in tau through the
// eigenpairs of H~: U diag(G0(lambda, tau)) U^+. Steps, all FP64 on the CUDA cores:
//   k_dm_fwd   Sigma^c(i w) = sum_t F[w][t] Sigma^c(tau_t) (the fermionic forward map, complex-linear)
//   k_dm_eig   H~ = U diag(lambda) U^+ by cyclic two-sided Jacobi (Forsythe and Henrici's complex
//              rotations, round-robin ordering so that nb/2 disjoint rotations run at once)
//   k_dm_inv   per (k, w): Gauss-Jordan inversion with partial pivoting of i w - H~ - Sigma^c(i w),
//              the remainder R = G(i w) - U (i w - lambda)^-1 U^+ split into the transforms of the
//              real tau-functions Re G_nm and Im G_nm: (R_nm + R_mn) / 2 and (R_nm - R_mn) / 2i
//   k_dm_tau   G(tau) = U diag(G0(lambda, tau)) U^+ + backward maps of the two parts; occupation
//              matrix -G(beta^-) the same way with the map to beta^-.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "gw_internal.h"

namespace gwi {
namespace {

constexpr int kDmThreads = 256;
constexpr int kDmMaxSweeps = 40;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmac(double2 acc, double2 a, double2 b) {  // acc + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cinv(double2 a) {  // 1 / a, scaled against overflow
  const double s = fmax(fabs(a.x), fabs(a.y));
  const double2 b = make_double2(a.x / s, a.y / s);
  const double d = s * (b.x * b.x + b.y * b.y);
  return make_double2(b.x / d, -b.y / d);
}

// G0(eps, tau) = -e^{-eps tau} (1 - n_F(eps)) in the overflow-free form (Sec. III.B.1).
__device__ __forceinline__ double g0_tau(double e, double tau, double beta) {
  const double a = fabs(e);
  const double den = 1.0 + exp(-beta * a);
  return e > 0.0 ? -exp(-a * tau) / den : -exp(-a * (beta - tau)) / den;
}
__device__ __forceinline__ double fermi(double e, double beta) {
  const double x = exp(-beta * fabs(e));
  return e > 0.0 ? x / (1.0 + x) : 1.0 / (1.0 + x);
}

// Sigma^c(i w_j) = sum_t F[j][t] Sigma^c(tau_t) for every matrix element: one thread per output.
__global__ void k_dm_fwd(const double2* __restrict__ S, const double2* __restrict__ F, int64_t nel, int ntau, int nw,
                         double2* __restrict__ Siw) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nel * nw) return;
  const int64_t el = e / nw;
  const int j = (int)(e % nw);
  const double2* s = S + el * ntau;
  const double2* f = F + (size_t)j * ntau;
  double2 acc = make_double2(0.0, 0.0);
  for (int t = 0; t < ntau; ++t) acc = cmac(acc, f[t], s[t]);
  Siw[e] = acc;  // [el][j]
}

// The two players of round r of a round-robin over n (even) players: player 0 stays, the others
// rotate; pair i joins slot i and slot n - 1 - i.
__device__ __forceinline__ void rr_pair(int n, int r, int i, int& p, int& q) {
  auto slot = [&](int s) { return s == 0 ? 0 : 1 + (s - 1 + r) % (n - 1); };
  p = slot(i);
  q = slot(n - 1 - i);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// One block per k: A = H~ (padded to nbp = nb rounded up to even with a decoupled zero), U = 1.
// Sweeps until the off-diagonal Frobenius norm is <= 1e-15 of the matrix's, at most kDmMaxSweeps.
__global__ void __launch_bounds__(kDmThreads) k_dm_eig(const double* __restrict__ eps, const double2* __restrict__ Sx,
                                                       const double2* __restrict__ vxc, int nb, int nbp,
                                                       double2* __restrict__ Aw, double2* __restrict__ Uw,
                                                       double* __restrict__ lam, int* __restrict__ info) {
  __shared__ double red[kDmThreads / 32];
  __shared__ double rot_c[128], rot_s[128];
  __shared__ double2 rot_ph[128];
  __shared__ int stop_flag;
  const int k = blockIdx.x, t = threadIdx.x;
  double2* A = Aw + (size_t)k * nbp * nbp;
  double2* U = Uw + (size_t)k * nbp * nbp;
  for (int e = t; e < nbp * nbp; e += kDmThreads) {
    const int r = e / nbp, c = e % nbp;
    double2 h = make_double2(0.0, 0.0);
    if (r < nb && c < nb) {
      const size_t o = ((size_t)k * nb + r) * nb + c;
      h = csub(Sx ? Sx[o] : make_double2(0.0, 0.0), vxc ? vxc[o] : make_double2(0.0, 0.0));
      if (r == c) h.x += eps[(size_t)k * nb + r];
    }
    A[e] = h;
    U[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // the Hermitian part of the input (Sigma^x - Sigma_0 Hermitian to rounding): average A and A^+
  for (int e = t; e < nbp * nbp; e += kDmThreads) {
    const int r = e / nbp, c = e % nbp;
    if (r < c) {
      const double2 a = A[(size_t)r * nbp + c], b = A[(size_t)c * nbp + r];
      const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      A[(size_t)r * nbp + c] = h;
      A[(size_t)c * nbp + r] = make_double2(h.x, -h.y);
    } else if (r == c) {
      A[e].y = 0.0;
    }
  }
  __syncthreads();
  const int np = nbp / 2;
  int sweep = 0;
  for (; sweep <= kDmMaxSweeps; ++sweep) {
    // off-diagonal and total Frobenius norms
    double off = 0.0, tot = 0.0;
    for (int e = t; e < nbp * nbp; e += kDmThreads) {
      const double2 a = A[e];
      const double m2 = a.x * a.x + a.y * a.y;
      tot += m2;
      if (e / nbp != e % nbp) off += m2;
    }
    for (int s = 16; s; s >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, s);
      tot += __shfl_xor_sync(0xffffffffu, tot, s);
    }
    if ((t & 31) == 0) red[t >> 5] = off;
    __syncthreads();
    if (t == 0) {
      double o = 0.0;
      for (int w = 0; w < kDmThreads / 32; ++w) o += red[w];
      red[0] = o;
    }
    __syncthreads();
    off = red[0];
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = tot;
    __syncthreads();
    if (t == 0) {
      double o = 0.0;
      for (int w = 0; w < kDmThreads / 32; ++w) o += red[w];
      stop_flag = off <= 1e-30 * o;  // |off|_F <= 1e-15 |A|_F
    }
    __syncthreads();
    if (stop_flag || sweep == kDmMaxSweeps) break;
    for (int r = 0; r < nbp - 1; ++r) {
      // rotation of each pair from the current A: zero (A)_pq with J = diag(1, e^{-i phi}) R(theta)
      for (int i = t; i < np; i += kDmThreads) {
        int p, q;
        rr_pair(nbp, r, i, p, q);
        const double a = A[(size_t)p * nbp + p].x, b = A[(size_t)q * nbp + q].x;
        const double2 c = A[(size_t)p * nbp + q];
        const double ac = hypot(c.x, c.y);
        double cs = 1.0, sn = 0.0;
        double2 ph = make_double2(1.0, 0.0);
        if (ac > 0.0) {
          const double z = (b - a) / (2.0 * ac);
          const double tt = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
          cs = 1.0 / sqrt(1.0 + tt * tt);
          sn = tt * cs;
          ph = make_double2(c.x / ac, -c.y / ac);  // e^{-i phi}
        }
        rot_c[i] = cs;
        rot_s[i] = sn;
        rot_ph[i] = ph;
      }
      __syncthreads();
      // columns p, q of A and U: (x_p, x_q) <- (x_p cs - x_q sn e^{-i phi}, x_p sn + x_q cs e^{-i phi})
      for (int e = t; e < np * nbp; e += kDmThreads) {
        const int i = e / nbp, row = e % nbp;
        int p, q;
        rr_pair(nbp, r, i, p, q);
        const double cs = rot_c[i], sn = rot_s[i];
        const double2 ph = rot_ph[i];
        double2* Ar = A + (size_t)row * nbp;
        double2* Ur = U + (size_t)row * nbp;
        const double2 ap = Ar[p], aq = cmul(Ar[q], ph), up = Ur[p], uq = cmul(Ur[q], ph);
        Ar[p] = csub(cscale(cs, ap), cscale(sn, aq));
        Ar[q] = cadd(cscale(sn, ap), cscale(cs, aq));
        Ur[p] = csub(cscale(cs, up), cscale(sn, uq));
        Ur[q] = cadd(cscale(sn, up), cscale(cs, uq));
      }
      __syncthreads();
      // rows p, q of A: (y_p, y_q) <- (cs y_p - sn e^{i phi} y_q, sn y_p + cs e^{i phi} y_q)
      for (int e = t; e < np * nbp; e += kDmThreads) {
        const int i = e / nbp, col = e % nbp;
        int p, q;
        rr_pair(nbp, r, i, p, q);
        const double cs = rot_c[i], sn = rot_s[i];
        const double2 phc = make_double2(rot_ph[i].x, -rot_ph[i].y);
        double2* yp = A + (size_t)p * nbp + col;
        double2* yq = A + (size_t)q * nbp + col;
        const double2 ap = *yp, aq = cmul(*yq, phc);
        *yp = csub(cscale(cs, ap), cscale(sn, aq));
        *yq = cadd(cscale(sn, ap), cscale(cs, aq));
      }
      __syncthreads();
    }
  }
  for (int i = t; i < nbp; i += kDmThreads) lam[(size_t)k * nbp + i] = A[(size_t)i * nbp + i].x;
  if (t == 0) info[k] = stop_flag ? 0 : 1;
}

// One block per (k, w): Gauss-Jordan inversion with partial pivoting of B = i w - H~ - Sigma^c(i w)
// on the augmented [B | 1] (workspace [nb][2 nb]), then the remainder R = B^-1 - U (i w - lambda)^-1 U^+
// as the transforms of the real tau-functions Re G and Im G: ah = (R + R^T) / 2, bh = (R - R^T) / 2i.
__global__ void __launch_bounds__(kDmThreads) k_dm_inv(const double* __restrict__ eps, const double2* __restrict__ Sx,
                                                       const double2* __restrict__ vxc, const double2* __restrict__ Siw,
                                                       const int* __restrict__ widx, double beta, int nb, int nbp,
                                                       int nw, const double2* __restrict__ Uw,
                                                       const double* __restrict__ lam, double2* __restrict__ aug,
                                                       double2* __restrict__ ah, double2* __restrict__ bh,
                                                       int* __restrict__ info) {
  __shared__ double pv[kDmThreads];
  __shared__ int pi[kDmThreads];
  __shared__ int piv_row, fail;
  const int k = blockIdx.x / nw, j = blockIdx.x % nw, t = threadIdx.x;
  const double w = (2.0 * widx[j] + 1.0) * M_PI / beta;
  const int n2 = 2 * nb;
  double2* X = aug + (size_t)blockIdx.x * nb * n2;
  for (int e = t; e < nb * n2; e += kDmThreads) {
    const int r = e / n2, c = e % n2;
    double2 v = make_double2(0.0, 0.0);
    if (c < nb) {
      const size_t o = ((size_t)k * nb + r) * nb + c;
      const double2 h = csub(Sx ? Sx[o] : make_double2(0.0, 0.0), vxc ? vxc[o] : make_double2(0.0, 0.0));
      const double2 s = Siw ? Siw[o * nw + j] : make_double2(0.0, 0.0);
      v = make_double2(-h.x - s.x, -h.y - s.y);
      if (r == c) {
        v.x -= eps[(size_t)k * nb + r];
        v.y += w;
      }
    } else if (c - nb == r) {
      v.x = 1.0;
    }
    X[e] = v;
  }
  if (t == 0) fail = 0;
  __syncthreads();
  for (int col = 0; col < nb; ++col) {
    // pivot: largest |.| in column col among rows >= col (first on ties)
    double best = -1.0;
    int br = col;
    for (int r = col + t; r < nb; r += kDmThreads) {
      const double2 v = X[(size_t)r * n2 + col];
      const double m = v.x * v.x + v.y * v.y;
      if (m > best) {
        best = m;
        br = r;
      }
    }
    pv[t] = best;
    pi[t] = br;
    __syncthreads();
    if (t == 0) {
      double b = -1.0;
      int r0 = col;
      for (int i = 0; i < kDmThreads; ++i)
        if (pv[i] > b || (pv[i] == b && pi[i] < r0)) {
          b = pv[i];
          r0 = pi[i];
        }
      piv_row = r0;
      if (!(b > 0.0) && !fail) {
        fail = 1;
        atomicMax(info + k, 2 + col);
      }
    }
    __syncthreads();
    if (fail) return;  // uniform: the block stops, its output is not written
    const int pr = piv_row;
    if (pr != col)
      for (int c = t; c < n2; c += kDmThreads) {
        const double2 a = X[(size_t)col * n2 + c];
        X[(size_t)col * n2 + c] = X[(size_t)pr * n2 + c];
        X[(size_t)pr * n2 + c] = a;
      }
    __syncthreads();
    const double2 inv = cinv(X[(size_t)col * n2 + col]);
    __syncthreads();
    for (int c = t; c < n2; c += kDmThreads) X[(size_t)col * n2 + c] = cmul(X[(size_t)col * n2 + c], inv);
    __syncthreads();
    for (int e = t; e < nb * n2; e += kDmThreads) {
      const int r = e / n2, c = e % n2;
      if (r == col) continue;
      const double2 f = X[(size_t)r * n2 + col];
      if (c == col) continue;
      X[e] = csub(X[e], cmul(f, X[(size_t)col * n2 + c]));
    }
    __syncthreads();
    for (int r = t; r < nb; r += kDmThreads)
      if (r != col) X[(size_t)r * n2 + col] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  // R = B^-1 - U diag(1 / (i w - lambda)) U^+, split into the two real-function transforms
  const double2* U = Uw + (size_t)k * nbp * nbp;
  const double* lk = lam + (size_t)k * nbp;
  __shared__ double2 gl[256];
  for (int a = t; a < nbp; a += kDmThreads) gl[a] = cinv(make_double2(-lk[a], w));  // 1 / (i w - lambda_a)
  __syncthreads();
  for (int e = t; e < nb * nb; e += kDmThreads) {
    const int n = e / nb, m = e % nb;
    double2 rnm = X[(size_t)n * n2 + nb + m], rmn = X[(size_t)m * n2 + nb + n];
    for (int a = 0; a < nbp; ++a) {
      const double2 g = gl[a];
      const double2 un = U[(size_t)n * nbp + a], um = U[(size_t)m * nbp + a];
      // (U g U^+)_nm = un g conj(um), (U g U^+)_mn = um g conj(un)
      const double2 x = cmul(un, make_double2(um.x, -um.y)), y = cmul(um, make_double2(un.x, -un.y));
      rnm = csub(rnm, cmul(g, x));
      rmn = csub(rmn, cmul(g, y));
    }
    const size_t o = (((size_t)k * nb + n) * nb + m) * nw + j;
    ah[o] = make_double2(0.5 * (rnm.x + rmn.x), 0.5 * (rnm.y + rmn.y));
    const double2 d = csub(rnm, rmn);  // (R_nm - R_mn) / (2 i) = -i d / 2
    bh[o] = make_double2(0.5 * d.y, -0.5 * d.x);
  }
}

// g0t[k][a][t] = G0(lambda_a, tau_t) for t < ntau, n_F(lambda_a) at t = ntau.
__global__ void k_dm_g0tab(const double* __restrict__ lam, const double* __restrict__ tau, double beta, int nk,
                           int nbp, int ntau, double* __restrict__ g0t) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nt1 = ntau + 1;
  if (e >= (int64_t)nk * nbp * nt1) return;
  const int ti = (int)(e % nt1);
  const double l = lam[e / nt1];
  g0t[e] = ti == ntau ? fermi(l, beta) : g0_tau(l, tau[ti], beta);
}

// G[k][n][m][t] = sum_a U_na G0(lambda_a, tau_t) conj(U_ma) + map(ah)[t] + i map(bh)[t], map(x)[t] =
// sum_j Fb[t][j] Re x_j + Fb[t][nw + j] Im x_j; the slot t = ntau gives the occupation matrix
// -G(beta^-) = U diag(n_F(lambda)) U^+ - (mapb(ah) + i mapb(bh)).
__global__ void k_dm_tau(const double2* __restrict__ Uw, const double* __restrict__ g0t,
                         const double2* __restrict__ ah, const double2* __restrict__ bh,
                         const double* __restrict__ Fb, const double* __restrict__ Fbeta, int nk, int nb, int nbp,
                         int nw, int ntau, const int* __restrict__ info, double2* __restrict__ G,
                         double2* __restrict__ occ) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nt1 = ntau + 1;
  if (e >= (int64_t)nk * nb * nb * nt1) return;
  const int ti = (int)(e % nt1);
  const int m = (int)((e / nt1) % nb), n = (int)((e / ((int64_t)nt1 * nb)) % nb);
  const int k = (int)(e / ((int64_t)nt1 * nb * nb));
  if (info[k] >= 2) return;  // a zero pivot: this k is not written
  const double2* U = Uw + (size_t)k * nbp * nbp;
  const double* gk = g0t + (size_t)k * nbp * nt1 + ti;
  const bool at_beta = ti == ntau;
  double2 s = make_double2(0.0, 0.0);
  for (int a = 0; a < nbp; ++a) {
    const double f = gk[(size_t)a * nt1];
    const double2 un = U[(size_t)n * nbp + a], um = U[(size_t)m * nbp + a];
    s = cmac(s, cscale(f, un), make_double2(um.x, -um.y));
  }
  const size_t o = (((size_t)k * nb + n) * nb + m) * nw;
  const double* fr = at_beta ? Fbeta : Fb + (size_t)ti * 2 * nw;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < nw; ++j) {
    const double2 a = ah[o + j], b = bh[o + j];
    re = fma(fr[j], a.x, fma(fr[nw + j], a.y, re));
    im = fma(fr[j], b.x, fma(fr[nw + j], b.y, im));
  }
  const size_t el = ((size_t)k * nb + n) * nb + m;
  if (at_beta)
    occ[el] = make_double2(s.x - re, s.y - im);
  else
    G[el * ntau + ti] = make_double2(s.x + re, s.y + im);
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_dyson_matrix(gw_ctx* c, const double* eps, const double* Sx, const double* vxc,
                                     const double* Sc_tau, double* G_tau, double* occ, int* info) {
  if (!c || !eps || !G_tau || !occ || !info) return GW_EINVAL;
  const int nk = c->nk, nb = c->nb, nw = c->nw, nt = c->ntau;
  if (nb > 256) return set_err(c, GW_EINVAL, "gw_dyson_matrix: nb <= 256");
  const int nbp = nb + (nb & 1);
  const size_t el = (size_t)nk * nb * nb;
  const size_t b_siw = Sc_tau ? el * nw * sizeof(double2) : 0;
  const size_t b_eig = 2 * (size_t)nk * nbp * nbp * sizeof(double2) + (size_t)nk * nbp * sizeof(double);
  const size_t b_aug = (size_t)nk * nw * nb * 2 * nb * sizeof(double2);
  const size_t b_hat = 2 * el * nw * sizeof(double2);
  const size_t b_g0 = (size_t)nk * nbp * (nt + 1) * sizeof(double);
  const size_t need = b_siw + b_eig + b_aug + b_hat + b_g0 + 1024;
  if (need > c->dm_bytes) {
    if (c->d_dm) cudaFree(c->d_dm);
    c->d_dm = nullptr;
    c->dm_bytes = 0;
    if (cudaMalloc(&c->d_dm, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "gw_dyson_matrix: workspace");
    }
    c->dm_bytes = need;
  }
  char* w = (char*)c->d_dm;
  double2* Siw = Sc_tau ? (double2*)w : nullptr;
  w += b_siw;
  double2* A = (double2*)w;
  double2* U = A + (size_t)nk * nbp * nbp;
  double* lam = (double*)(U + (size_t)nk * nbp * nbp);
  w += b_eig;
  double2* aug = (double2*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
  double2* ah = aug + (size_t)nk * nw * nb * 2 * nb;
  double2* bh = ah + el * nw;
  double* g0t = (double*)(bh + el * nw);
  gw_status st;
  if (Sc_tau) {
    const int64_t n = (int64_t)el * nw;
    k_dm_fwd<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const double2*)Sc_tau, (const double2*)c->d_Ffwd,
                                                                 (int64_t)el, nt, nw, Siw);
    if ((st = check_launch(c, "dm_fwd")) != GW_OK) return st;
  }
  k_dm_eig<<<(unsigned)nk, kDmThreads, 0, c->stream>>>(eps, (const double2*)Sx, (const double2*)vxc, nb, nbp, A, U,
                                                       lam, info);
  if ((st = check_launch(c, "dm_eig")) != GW_OK) return st;
  k_dm_inv<<<(unsigned)(nk * nw), kDmThreads, 0, c->stream>>>(eps, (const double2*)Sx, (const double2*)vxc, Siw,
                                                              c->d_widx, c->beta, nb, nbp, nw, U, lam, aug, ah, bh,
                                                              info);
  if ((st = check_launch(c, "dm_inv")) != GW_OK) return st;
  const int64_t ng = (int64_t)nk * nbp * (nt + 1);
  k_dm_g0tab<<<(unsigned)((ng + 255) / 256), 256, 0, c->stream>>>(lam, c->d_tau, c->beta, nk, nbp, nt, g0t);
  if ((st = check_launch(c, "dm_g0tab")) != GW_OK) return st;
  const int64_t n = (int64_t)el * (nt + 1);
  k_dm_tau<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(U, g0t, ah, bh, c->d_Fbwd, c->d_Fbwd_beta, nk, nb, nbp,
                                                                nw, nt, info, (double2*)G_tau, (double2*)occ);
  return check_launch(c, "dm_tau");
}
