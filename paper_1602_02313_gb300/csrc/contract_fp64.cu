// FP64 (CUDA-core) forms of the two product-basis contractions: the parity path.
//
// polarization, Eq. (irpol):  P_II'(q|tau) = 1/(Omega Nk) sum_k sum_ab M^I_ab Q_ab(tau) conj(M^I'_ab)
//   Q_ab(tau) = G_b(k|tau) G_a(k-q|-tau) = -G_b(k|tau) G_a(k-q|beta - tau)   (Sec. II)
// self-energy, Eq. (sigc):    Sigc_n(k|tau) += -1/(Omega Nk) sum_j G_j(k-q|tau) a_jn^H W~(tau) a_jn
#include <cuda_runtime.h>

#include "gw_internal.h"

namespace gwi {

namespace {

constexpr int PT = 32;  // output tile (rows x cols) of the polarization kernel

__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
  // acc += a * conj(b)
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
  return acc;
}

// grid: x = upper-triangle tile index, y = tau; block 256 = 16 x 16 threads, 2 x 2 outputs each.
__global__ void __launch_bounds__(256) k_pol_fp64(const double2* __restrict__ Mq, const double* __restrict__ G,
                                                  const int* __restrict__ kmq, int nk, int ni, int nb, int ntau,
                                                  double pref, double2* __restrict__ P) {
  __shared__ double2 As[PT][PT + 1];
  __shared__ double2 Bs[PT][PT + 1];
  __shared__ double wq[PT];
  const int it = blockIdx.y;
  const int itm = ntau - 1 - it;  // tau_{itm} = beta - tau_it
  const int nt = ni / PT;
  // map linear upper-triangle index -> (ti, tj), ti <= tj
  int t = blockIdx.x, ti = 0;
  while (t >= nt - ti) {
    t -= nt - ti;
    ++ti;
  }
  const int tj = ti + t;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int s = 0; s < 2; ++s) acc[r][s] = make_double2(0.0, 0.0);
  const int np = nb * nb;
  for (int k = 0; k < nk; ++k) {
    const double2* Mk = Mq + (size_t)k * ni * np;
    const int km = kmq[k];
    for (int p0 = 0; p0 < np; p0 += PT) {
      __syncthreads();
      if (threadIdx.x < PT) {
        const int p = p0 + threadIdx.x;
        double w = 0.0;
        if (p < np) {
          const int a = p / nb, b = p - a * nb;
          w = -G[((size_t)k * nb + b) * ntau + it] * G[((size_t)km * nb + a) * ntau + itm];
        }
        wq[threadIdx.x] = w;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < PT * PT; e += 256) {
        const int r = e / PT, cc = e % PT;
        const int p = p0 + cc;
        double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
        if (p < np) {
          va = Mk[(size_t)(ti * PT + r) * np + p];
          vb = Mk[(size_t)(tj * PT + r) * np + p];
        }
        const double w = wq[cc];
        As[r][cc] = make_double2(va.x * w, va.y * w);
        Bs[r][cc] = vb;
      }
      __syncthreads();
#pragma unroll 4
      for (int cc = 0; cc < PT; ++cc) {
        const double2 a0 = As[2 * ty][cc], a1 = As[2 * ty + 1][cc];
        const double2 b0 = Bs[2 * tx][cc], b1 = Bs[2 * tx + 1][cc];
        acc[0][0] = cfma_conj(a0, b0, acc[0][0]);
        acc[0][1] = cfma_conj(a0, b1, acc[0][1]);
        acc[1][0] = cfma_conj(a1, b0, acc[1][0]);
        acc[1][1] = cfma_conj(a1, b1, acc[1][1]);
      }
    }
  }
  double2* Pt = P + (size_t)it * ni * ni;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int I = ti * PT + 2 * ty + r, J = tj * PT + 2 * tx + s;
      const double2 v = make_double2(acc[r][s].x * pref, acc[r][s].y * pref);
      Pt[(size_t)I * ni + J] = v;
      if (ti != tj) Pt[(size_t)J * ni + I] = make_double2(v.x, -v.y);
    }
}

// Self-energy, FP64. grid: x = band tile (32 bands n), y = tau, z = k; block 256 = 32 columns x 8 row groups.
// For each band j at k - q: columns a_jn (n in the tile); d_n = a_jn^H W~ a_jn (real for Hermitian W~),
// accumulated over j with weight G_j(k-q|tau).
constexpr int SC = 32;  // columns (bands n) per block
constexpr int SR = 32;  // rows of W~ per chunk (4 per thread)
constexpr int SJ = 32;  // contraction chunk

__global__ void __launch_bounds__(256) k_sigma_fp64(const double2* __restrict__ Mq, const double* __restrict__ G,
                                                    const double2* __restrict__ W, const int* __restrict__ kmq, int ni,
                                                    int nb, int ntau, double pref, double* __restrict__ S) {
  __shared__ double2 As[SJ][SC + 1];
  __shared__ double2 Ws[SR][SJ + 1];
  __shared__ double red[8][SC];
  const int n0 = blockIdx.x * SC, it = blockIdx.y, k = blockIdx.z;
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int np = nb * nb;
  const double2* Mk = Mq + (size_t)k * ni * np;
  const double2* Wt = W + (size_t)it * ni * ni;
  const int km = kmq[k];
  double sacc = 0.0;  // sum_j G_j d_jn for this thread's column (valid in g == 0)
  for (int j = 0; j < nb; ++j) {
    double dpart = 0.0;
    for (int I0 = 0; I0 < ni; I0 += SR) {
      double2 y[SR / 8];
#pragma unroll
      for (int r = 0; r < SR / 8; ++r) y[r] = make_double2(0.0, 0.0);
      for (int J0 = 0; J0 < ni; J0 += SJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < SJ * SC; e += 256) {
          const int jj = e / SC, cc = e % SC;
          const int n = n0 + cc;
          As[jj][cc] = n < nb ? Mk[(size_t)(J0 + jj) * np + j * nb + n] : make_double2(0.0, 0.0);
        }
        for (int e = threadIdx.x; e < SR * SJ; e += 256) {
          const int rr = e / SJ, jj = e % SJ;
          Ws[rr][jj] = (I0 + rr < ni) ? Wt[(size_t)(I0 + rr) * ni + J0 + jj] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < SJ; ++jj) {
          const double2 a = As[jj][c];
#pragma unroll
          for (int r = 0; r < SR / 8; ++r) {
            const double2 w = Ws[g + 8 * r][jj];
            y[r].x = fma(w.x, a.x, fma(-w.y, a.y, y[r].x));
            y[r].y = fma(w.x, a.y, fma(w.y, a.x, y[r].y));
          }
        }
      }
      // partial d: sum_I conj(A_I) y_I over this thread's rows (real part)
      const int n = n0 + c;
      if (n < nb) {
#pragma unroll
        for (int r = 0; r < SR / 8; ++r) {
          const int I = I0 + g + 8 * r;
          if (I < ni) {
            const double2 a = Mk[(size_t)I * np + j * nb + n];
            dpart = fma(a.x, y[r].x, fma(a.y, y[r].y, dpart));
          }
        }
      }
    }
    __syncthreads();
    red[g][c] = dpart;
    __syncthreads();
    if (g == 0) {
      double d = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) d += red[q][c];
      sacc = fma(G[((size_t)km * nb + j) * ntau + it], d, sacc);
    }
  }
  const int n = n0 + c;
  if (g == 0 && n < nb) S[((size_t)k * nb + n) * ntau + it] += pref * sacc;
}

}  // namespace

gw_status launch_pol_fp64(gw_ctx* c, int iq, const double* G, double* P) {
  if (c->ni % PT) return set_err(c, GW_EUNSUPPORTED, "FP64 polarization needs ni % 32 == 0");
  const int nt = c->ni / PT;
  const double2* Mq = (const double2*)m_block(c, iq);
  if (!Mq) return GW_ECUDA;
  dim3 grid(nt * (nt + 1) / 2, c->ntau);
  k_pol_fp64<<<grid, 256, 0, c->stream>>>(Mq, G, c->d_kmq + (size_t)iq * c->nk, c->nk, c->ni, c->nb, c->ntau,
                                          1.0 / (c->omega * c->nk), (double2*)P);
  return check_launch(c, "pol_fp64");
}

gw_status launch_sigma_fp64(gw_ctx* c, int iq, const double* G, const double* W, double* S) {
  if (c->ni % SJ) return set_err(c, GW_EUNSUPPORTED, "FP64 self-energy needs ni % 32 == 0");
  const double2* Mq = (const double2*)m_block(c, iq);
  if (!Mq) return GW_ECUDA;
  dim3 grid((c->nb + SC - 1) / SC, c->ntau, c->nk);
  k_sigma_fp64<<<grid, 256, 0, c->stream>>>(Mq, G, (const double2*)W, c->d_kmq + (size_t)iq * c->nk, c->ni, c->nb,
                                            c->ntau, -1.0 / (c->omega * c->nk), S);
  return check_launch(c, "sigma_fp64");
}

}  // namespace gwi
