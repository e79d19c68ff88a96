// Screened interaction at bosonic Matsubara frequencies (Sec. III.B.3, Eq. tildeW posed in i nu):
//   Pi = v^1/2 P(i nu) v^1/2,  (1 - Pi) X = Pi,  W~ = W - v = v^1/2 X v^1/2.
// One thread block per (q, nu) system. The augmented matrix [1 - Pi | Pi] (ni x 2 ni,
// complex FP64) lives in a global workspace (L2-resident for typical sizes) and is
// reduced by Gaussian elimination without pivoting, then back-substituted.
// Elimination without pivoting is safe here: P(i nu) has a negative semidefinite
// Hermitian part, so 1 - Pi has Hermitian part >= 1 and every leading principal
// submatrix is nonsingular. A zero pivot is still detected and reported in info.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gw_internal.h"

namespace gwi {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cinv(double2 a) {
  const double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}

__global__ void __launch_bounds__(512) k_screen(const double2* __restrict__ P, const double* __restrict__ sqrtv,
                                                int nnu, int ni, double2* __restrict__ aug_all,
                                                double2* __restrict__ W, int* __restrict__ info) {
  const int sys = blockIdx.x;           // = iqb * nnu + j
  const int iqb = sys / nnu;
  const int n2 = 2 * ni;
  const double* sv = sqrtv + (size_t)iqb * ni;
  const double2* Ps = P + (size_t)sys * ni * ni;
  double2* A = aug_all + (size_t)sys * ni * n2;
  __shared__ int bad;
  __shared__ double2 s_inv;
  if (threadIdx.x == 0) bad = 0;
  // build [1 - Pi | Pi]
  for (int e = threadIdx.x; e < ni * ni; e += blockDim.x) {
    const int I = e / ni, J = e % ni;
    const double s = sv[I] * sv[J];
    const double2 p = Ps[e];
    const double2 pi = make_double2(s * p.x, s * p.y);
    A[(size_t)I * n2 + J] = make_double2((I == J ? 1.0 : 0.0) - pi.x, -pi.y);
    A[(size_t)I * n2 + ni + J] = pi;
  }
  __syncthreads();
  // forward elimination
  for (int kk = 0; kk < ni; ++kk) {
    if (threadIdx.x == 0) {
      const double2 pv = A[(size_t)kk * n2 + kk];
      if (pv.x == 0.0 && pv.y == 0.0) {
        bad = kk + 1;
      } else {
        s_inv = cinv(pv);
      }
    }
    __syncthreads();
    if (bad) break;
    const int rows = ni - kk - 1, cols = n2 - kk - 1;
    const double2 inv = s_inv;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int i = kk + 1 + e / cols, j = kk + 1 + e % cols;
      const double2 l = cmul(A[(size_t)i * n2 + kk], inv);
      const double2 u = A[(size_t)kk * n2 + j];
      double2 a = A[(size_t)i * n2 + j];
      a.x -= l.x * u.x - l.y * u.y;
      a.y -= l.x * u.y + l.y * u.x;
      A[(size_t)i * n2 + j] = a;
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) info[sys] = bad;
    return;
  }
  // back substitution on the right-hand block, in place
  for (int kk = ni - 1; kk >= 0; --kk) {
    const double2 inv = cinv(A[(size_t)kk * n2 + kk]);
    for (int j = threadIdx.x; j < ni; j += blockDim.x) {
      const double2 x = cmul(A[(size_t)kk * n2 + ni + j], inv);
      A[(size_t)kk * n2 + ni + j] = x;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kk * ni; e += blockDim.x) {
      const int i = e / ni, j = e % ni;
      const double2 l = A[(size_t)i * n2 + kk];
      const double2 x = A[(size_t)kk * n2 + ni + j];
      double2 a = A[(size_t)i * n2 + ni + j];
      a.x -= l.x * x.x - l.y * x.y;
      a.y -= l.x * x.y + l.y * x.x;
      A[(size_t)i * n2 + ni + j] = a;
    }
    __syncthreads();
  }
  double2* Ws = W + (size_t)sys * ni * ni;
  for (int e = threadIdx.x; e < ni * ni; e += blockDim.x) {
    const int I = e / ni, J = e % ni;
    const double s = sv[I] * sv[J];
    const double2 x = A[(size_t)I * n2 + ni + J];
    Ws[e] = make_double2(s * x.x, s * x.y);
  }
  if (threadIdx.x == 0) info[sys] = 0;
}

// Blocked Gauss-Jordan form of the same solve, one thread block per system:
// for each 32-column block row R: invert the pivot block A[R][R] in shared memory,
// U = A[R][R]^-1 A[R][c > R] (c running over the remaining left columns and all right-hand
// columns), then A[i][c] -= A[i][R] U for every row i outside R. The rank-32 updates are
// register-tiled FP64 products (8 rows x 4 columns per thread) fed from shared memory, so
// the augmented matrix is read and written once per block row instead of once per column.
// Work 1.5 ni^3 complex multiply-adds.
constexpr int GJ_B = 32;
constexpr int GJ_CH = 32;  // columns per update sub-chunk

__global__ void __launch_bounds__(256, 1) k_screen_gj(const double2* __restrict__ P, const double* __restrict__ sqrtv,
                                                     int nnu, int ni, double2* __restrict__ aug_all,
                                                     double2* __restrict__ W, int* __restrict__ info) {
  extern __shared__ double2 gsm[];
  double2* Pinv = gsm;                    // [32][33]
  double2* L = Pinv + GJ_B * (GJ_B + 1);  // [ni][33]: A[i][R] for all rows (rows of R zeroed)
  double2* U = L + ni * (GJ_B + 1);       // [32][GJ_CH + 1]
  __shared__ int bad;
  __shared__ double2 fcol[GJ_B], rowj[GJ_B];
  const int sys = blockIdx.x;
  const int iqb = sys / nnu;
  const int n2 = 2 * ni;
  const double* sv = sqrtv + (size_t)iqb * ni;
  const double2* Ps = P + (size_t)sys * ni * ni;
  double2* A = aug_all + (size_t)sys * ni * n2;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int e = t; e < ni * ni; e += blockDim.x) {
    const int I = e / ni, J = e % ni;
    const double s = sv[I] * sv[J];
    const double2 p = Ps[e];
    const double2 pi = make_double2(s * p.x, s * p.y);
    A[(size_t)I * n2 + J] = make_double2((I == J ? 1.0 : 0.0) - pi.x, -pi.y);
    A[(size_t)I * n2 + ni + J] = pi;
  }
  __syncthreads();
  const int tr = t & 31, tc = t >> 5;  // row lane, column group (8 groups x 4 columns)
  for (int k0 = 0; k0 < ni; k0 += GJ_B) {
    // pivot block and the left block column of all rows
    for (int e = t; e < GJ_B * GJ_B; e += blockDim.x) {
      const int r = e / GJ_B, c = e % GJ_B;
      Pinv[r * (GJ_B + 1) + c] = A[(size_t)(k0 + r) * n2 + k0 + c];
    }
    for (int e = t; e < ni * GJ_B; e += blockDim.x) {
      const int r = e / GJ_B, c = e % GJ_B;
      L[r * (GJ_B + 1) + c] = (r >= k0 && r < k0 + GJ_B) ? make_double2(0.0, 0.0) : A[(size_t)r * n2 + k0 + c];
    }
    __syncthreads();
    // in-place Gauss-Jordan inversion of the 32 x 32 pivot block (no pivoting):
    // row j <- row j / p (entry j -> 1/p); other rows r: a_rc -= a_rj a_jc / p, a_rj <- -a_rj / p
    for (int j = 0; j < GJ_B; ++j) {
      const double2 p = Pinv[j * (GJ_B + 1) + j];
      if (p.x == 0.0 && p.y == 0.0) {
        if (t == 0) bad = k0 + j + 1;
        break;
      }
      const double2 ip = cinv(p);
      if (t < GJ_B) {
        fcol[t] = Pinv[t * (GJ_B + 1) + j];
        rowj[t] = t == j ? ip : cmul(Pinv[j * (GJ_B + 1) + t], ip);
      }
      __syncthreads();
      for (int e = t; e < GJ_B * GJ_B; e += blockDim.x) {
        const int r = e / GJ_B, c = e % GJ_B;
        if (r == j) {
          Pinv[r * (GJ_B + 1) + c] = rowj[c];
        } else {
          double2 a = c == j ? make_double2(0.0, 0.0) : Pinv[r * (GJ_B + 1) + c];
          const double2 f = fcol[r], u = rowj[c];
          a.x -= f.x * u.x - f.y * u.y;
          a.y -= f.x * u.y + f.y * u.x;
          Pinv[r * (GJ_B + 1) + c] = a;
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (bad) break;
    // remaining columns in sub-chunks: U = Pinv A[R][chunk]; A[i][chunk] -= L[i] U
    for (int c0 = k0 + GJ_B; c0 < n2; c0 += GJ_CH) {
      const int cw = min(GJ_CH, n2 - c0);
      for (int e = t; e < GJ_B * GJ_CH; e += blockDim.x) {
        const int r = e / GJ_CH, c = e % GJ_CH;
        double2 s = make_double2(0.0, 0.0);
        if (c < cw) {
          for (int j = 0; j < GJ_B; ++j) {
            const double2 pv = Pinv[r * (GJ_B + 1) + j];
            const double2 a = A[(size_t)(k0 + j) * n2 + c0 + c];
            s.x += pv.x * a.x - pv.y * a.y;
            s.y += pv.x * a.y + pv.y * a.x;
          }
        }
        U[r * (GJ_CH + 1) + c] = s;
      }
      __syncthreads();
      for (int e = t; e < GJ_B * GJ_CH; e += blockDim.x) {
        const int r = e / GJ_CH, c = e % GJ_CH;
        if (c < cw) A[(size_t)(k0 + r) * n2 + c0 + c] = U[r * (GJ_CH + 1) + c];
      }
      // rank-32 update of all rows outside R: thread (tr, tc) owns rows tr + 32 m, columns 4 tc .. 4 tc + 3
      for (int rbase = 0; rbase < ni; rbase += 256) {
        double2 acc[8][4];
#pragma unroll
        for (int m = 0; m < 8; ++m)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[m][q] = make_double2(0.0, 0.0);
        for (int j = 0; j < GJ_B; ++j) {
          double2 uq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) uq[q] = U[j * (GJ_CH + 1) + 4 * tc + q];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int r = rbase + tr + 32 * m;
            const double2 l = r < ni ? L[r * (GJ_B + 1) + j] : make_double2(0.0, 0.0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[m][q].x = fma(l.x, uq[q].x, fma(-l.y, uq[q].y, acc[m][q].x));
              acc[m][q].y = fma(l.x, uq[q].y, fma(l.y, uq[q].x, acc[m][q].y));
            }
          }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int r = rbase + tr + 32 * m;
          if (r >= ni || (r >= k0 && r < k0 + GJ_B)) continue;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 4 * tc + q;
            if (c < cw) {
              double2* a = &A[(size_t)r * n2 + c0 + c];
              double2 v = *a;
              v.x -= acc[m][q].x;
              v.y -= acc[m][q].y;
              *a = v;
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (bad) {
    if (t == 0) info[sys] = bad;
    return;
  }
  double2* Ws = W + (size_t)sys * ni * ni;
  for (int e = t; e < ni * ni; e += blockDim.x) {
    const int I = e / ni, J = e % ni;
    const double s = sv[I] * sv[J];
    const double2 x = A[(size_t)I * n2 + ni + J];
    Ws[e] = make_double2(s * x.x, s * x.y);
  }
  if (t == 0) info[sys] = 0;
}

}  // namespace

gw_status launch_screen(gw_ctx* c, int iq0, int nqb, const double* P, double* W, int* info, double* aug) {
  const int nsys = nqb * c->nnu;
  const size_t smem = sizeof(double2) * (GJ_B * (GJ_B + 1) + (size_t)c->ni * (GJ_B + 1) + GJ_B * (GJ_CH + 1));
  if (c->ni % GJ_B == 0 && smem <= 200 * 1024) {
    cudaFuncSetAttribute(k_screen_gj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_screen_gj<<<nsys, 256, smem, c->stream>>>((const double2*)P, c->d_sqrtv + (size_t)iq0 * c->ni, c->nnu, c->ni,
                                                 (double2*)aug, (double2*)W, info);
  } else {
    k_screen<<<nsys, 512, 0, c->stream>>>((const double2*)P, c->d_sqrtv + (size_t)iq0 * c->ni, c->nnu, c->ni,
                                          (double2*)aug, (double2*)W, info);
  }
  return check_launch(c, "screen");
}

}  // namespace gwi

// ---------------------------------------------------------------------------
// gw_screen_static: the same solve with its scratch in a file-scope device
// array, for callers that must not allocate device memory. The array is part
// of the library image: every GPU that loads libgw holds it until the process
// exits. Its device address is looked up once per device (cudaGetSymbolAddress
// with that device current) on the first call there.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kScreenStaticBytes = 128ull << 20;  // 128 MiB
static __device__ __align__(256) unsigned char g_screen_scratch[kScreenStaticBytes];
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

extern "C" gw_status gw_screen_static(int nq, int nnu, int ni, const double* sqrt_v, const double* P_iv,
                                      double* Wt_iv, int* info, void* stream) {
  if (nq < 1 || nnu < 1 || ni < 1 || !sqrt_v || !P_iv || !Wt_iv || !info) return GW_EINVAL;
  const size_t per_q = (size_t)nnu * ni * 2 * ni * sizeof(double2);
  if (per_q > kScreenStaticBytes) return GW_EINVAL;  // one q point's systems must fit the scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GW_ECUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_screen_scratch) != cudaSuccess || !p) return GW_ECUDA;
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  const int qpp = (int)(kScreenStaticBytes / per_q);  // q points per pass
  cudaStream_t st = (cudaStream_t)stream;
  for (int q0 = 0; q0 < nq; q0 += qpp) {
    const int cq = nq - q0 < qpp ? nq - q0 : qpp;
    const size_t sys0 = (size_t)q0 * nnu;
    gwi::k_screen<<<cq * nnu, 512, 0, st>>>((const double2*)P_iv + sys0 * ni * ni, sqrt_v + (size_t)q0 * ni, nnu, ni,
                                      (double2*)scratch, (double2*)Wt_iv + sys0 * ni * ni, info + sys0);
    if (cudaGetLastError() != cudaSuccess) return GW_ECUDA;
  }
  return GW_OK;
}
