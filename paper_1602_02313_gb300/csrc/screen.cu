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
#include <type_traits>
#include <string>

#include "arith.cuh"
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

// Blocked in-place Gauss-Jordan inversion, one thread block per system. Since
// Pi = 1 - A with A = 1 - Pi, the solution of A X = Pi is X = A^-1 - 1, so only A^-1 is
// formed (ni^3 complex multiply-adds instead of the 1.5 ni^3 of eliminating [A | Pi]).
// For each 32-row block R: invert the pivot block A_RR in shared memory (no pivoting),
// U_c = A_RR^-1 A_Rc for every column block c != R, A_ic -= A_iR U_c for every row i
// outside R, A_iR <- -A_iR A_RR^-1 and A_RR <- A_RR^-1. The new rows R are written first;
// the other rows follow in passes of 256, each pass holding its 32-column panel A_iR in
// shared memory. The rank-32 updates are register-tiled (8 rows x 4 columns per thread), so
// the matrix is read and written once per block row, for any ni that is a multiple of 32.
//
// The arithmetic is a policy (arith.cuh): native FP64, float-float on the FP32 pipes, or plain
// FP32 (whose scaling by v^1/2 on the way in and out also stays in FP32).
constexpr int GJ_B = 32;
constexpr int GJ_RP = 256;  // rows per update pass (the shared-memory panel)
constexpr int kScreenMaxNi = 1024;  // the largest basis a context accepts

using arith::Fp64;
using arith::Ff32;
using arith::F32;

template <class AR>
__global__ void __launch_bounds__(256, AR::kBlocksPerSm) k_screen_inv(const double2* __restrict__ P, const double* __restrict__ sqrtv,
                                                      int nnu, int ni, typename AR::S* __restrict__ work,
                                                      double2* __restrict__ W, int* __restrict__ info) {
  using S = typename AR::S;
  using Acc = typename AR::Acc;
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  S* Pinv = reinterpret_cast<S*>(gsm_raw);  // [32][33]
  S* L = Pinv + GJ_B * (GJ_B + 1);           // [GJ_RP][33]: A[i][R] of one row pass (rows of R zeroed)
  S* U = L + (size_t)GJ_RP * (GJ_B + 1);     // [32][33]
  __shared__ int bad;
  __shared__ S fcol[GJ_B], rowj[GJ_B];
  const int sys = blockIdx.x;
  const int iqb = sys / nnu;
  const double* sv = sqrtv + (size_t)iqb * ni;
  const double2* Ps = P + (size_t)sys * ni * ni;
  S* A = work + (size_t)sys * ni * ni;
  const int t = threadIdx.x;
  constexpr bool kF32 = std::is_same<AR, F32>::value;
  __shared__ float svf[kF32 ? kScreenMaxNi : 1];  // FP32: v^1/2 as floats
  if (t == 0) bad = 0;
  if constexpr (kF32) {
    // A = 1 - Pi entirely in FP32 (integer-pipe conversions of the inputs; no FP64 operations)
    for (int I = t; I < ni; I += blockDim.x) svf[I] = cvt::d2f(sv[I]);
    __syncthreads();
    for (int e = t; e < ni * ni; e += blockDim.x) {
      const int I = e / ni, J = e % ni;
      const float s = svf[I] * svf[J];
      const double2 p = Ps[e];
      A[e] = make_float2((I == J ? 1.f : 0.f) - s * cvt::d2f(p.x), -s * cvt::d2f(p.y));
    }
  } else {
    for (int e = t; e < ni * ni; e += blockDim.x) {
      const int I = e / ni, J = e % ni;
      const double s = sv[I] * sv[J];
      const double2 p = Ps[e];
      A[e] = AR::from((I == J ? 1.0 : 0.0) - s * p.x, -s * p.y);
    }
  }
  __syncthreads();
  const int tr = t & 31, tc = t >> 5;  // row lane, column group (8 groups x 4 columns)
  for (int k0 = 0; k0 < ni; k0 += GJ_B) {
    for (int e = t; e < GJ_B * GJ_B; e += blockDim.x) {
      const int r = e / GJ_B, c = e % GJ_B;
      Pinv[r * (GJ_B + 1) + c] = A[(size_t)(k0 + r) * ni + k0 + c];
    }
    __syncthreads();
    // in-place Gauss-Jordan inversion of the 32 x 32 pivot block (no pivoting):
    // row j <- row j / p (entry j -> 1/p); other rows r: a_rc -= a_rj a_jc / p, a_rj <- -a_rj / p
    for (int j = 0; j < GJ_B; ++j) {
      const S p = Pinv[j * (GJ_B + 1) + j];
      if (AR::is_zero(p)) {
        if (t == 0) bad = k0 + j + 1;
        break;
      }
      if (t < GJ_B) {
        // one warp: the reciprocal is ~40 FP64-pipe instructions for the FP32-based policies,
        // and only these threads use it
        const S ip = AR::inv(p);
        fcol[t] = Pinv[t * (GJ_B + 1) + j];
        if (t == j) {
          rowj[t] = ip;
        } else {
          Acc a = AR::azero();
          AR::mac(a, Pinv[j * (GJ_B + 1) + t], ip);
          rowj[t] = AR::val(a);
        }
      }
      __syncthreads();
      for (int e = t; e < GJ_B * GJ_B; e += blockDim.x) {
        const int r = e / GJ_B, c = e % GJ_B;
        if (r == j) {
          Pinv[r * (GJ_B + 1) + c] = rowj[c];
        } else {
          Acc a = AR::azero();
          AR::mac(a, fcol[r], rowj[c]);
          Pinv[r * (GJ_B + 1) + c] = AR::sub(c == j ? AR::zero() : Pinv[r * (GJ_B + 1) + c], a);
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (bad) break;
    // rows R: A_Rc <- A_RR^-1 A_Rc for every column block c != R, A_RR <- A_RR^-1; 256 columns
    // per pass, register-tiled: thread t computes rows (t & 3) + 4 m, m = 0 .. 7 (interleaved, so
    // that the four row groups of a warp read Pinv from four different bank groups) and columns
    // 4 (t >> 2) .. + 3 of the pass, reading the old rows R from A; all reads of a pass finish
    // before its writes
    for (int cp = 0; cp < ni; cp += 256) {
      const int rg = t & 3, col = cp + 4 * (t >> 2);
      const bool live = col < ni;
      Acc acc[8][4];
#pragma unroll
      for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = AR::azero();
      if (live) {
        for (int j = 0; j < GJ_B; ++j) {
          S aq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) aq[q] = A[(size_t)(k0 + j) * ni + col + q];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const S pv = Pinv[(rg + 4 * m) * (GJ_B + 1) + j];
#pragma unroll
            for (int q = 0; q < 4; ++q) AR::mac(acc[m][q], pv, aq[q]);
          }
        }
      }
      __syncthreads();
      if (live) {
        const bool isR = col >= k0 && col < k0 + GJ_B;  // a 4-column group lies in one 32-block
#pragma unroll
        for (int m = 0; m < 8; ++m)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            A[(size_t)(k0 + rg + 4 * m) * ni + col + q] =
                isR ? Pinv[(rg + 4 * m) * (GJ_B + 1) + col + q - k0] : AR::val(acc[m][q]);
      }
    }
    __syncthreads();
    // all other rows, in passes of GJ_RP rows: A_ic -= A_iR U_c with U_c the new row block
    // (A_iR <- -A_iR A_RR^-1 for the column block R, which starts from zero); the pass's
    // A_iR are taken into shared memory before its column block R is overwritten
    for (int r0 = 0; r0 < ni; r0 += GJ_RP) {
      for (int e = t; e < GJ_RP * GJ_B; e += blockDim.x) {
        const int r = e / GJ_B, c = e % GJ_B, gr = r0 + r;
        L[r * (GJ_B + 1) + c] = (gr >= ni || (gr >= k0 && gr < k0 + GJ_B)) ? AR::zero() : A[(size_t)gr * ni + k0 + c];
      }
      for (int c0 = 0; c0 < ni; c0 += GJ_B) {
        const bool isR = c0 == k0;
        for (int e = t; e < GJ_B * GJ_B; e += blockDim.x) {
          const int r = e / GJ_B, c = e % GJ_B;
          U[r * (GJ_B + 1) + c] = A[(size_t)(k0 + r) * ni + c0 + c];
        }
        __syncthreads();
        // thread (tr, tc) owns rows r0 + tr + 32 m and columns 4 tc .. 4 tc + 3 of the chunk
        Acc acc[8][4];
#pragma unroll
        for (int m = 0; m < 8; ++m)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[m][q] = AR::azero();
        for (int j = 0; j < GJ_B; ++j) {
          S uq[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) uq[q] = U[j * (GJ_B + 1) + 4 * tc + q];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const S l = L[(tr + 32 * m) * (GJ_B + 1) + j];
#pragma unroll
            for (int q = 0; q < 4; ++q) AR::mac(acc[m][q], l, uq[q]);
          }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int r = r0 + tr + 32 * m;
          if (r >= ni || (r >= k0 && r < k0 + GJ_B)) continue;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            S* a = &A[(size_t)r * ni + c0 + 4 * tc + q];
            *a = AR::sub(isR ? AR::zero() : *a, acc[m][q]);
          }
        }
        __syncthreads();
      }
    }
  }
  if (bad) {
    if (t == 0) info[sys] = bad;
    return;
  }
  // W~ = v^1/2 (A^-1 - 1) v^1/2
  double2* Ws = W + (size_t)sys * ni * ni;
  if constexpr (kF32) {
    for (int e = t; e < ni * ni; e += blockDim.x) {
      const int I = e / ni, J = e % ni;
      const float s = svf[I] * svf[J];
      const float2 x = A[e];
      Ws[e] = make_double2(cvt::f2d(s * (x.x - (I == J ? 1.f : 0.f))), cvt::f2d(s * x.y));
    }
  } else {
    for (int e = t; e < ni * ni; e += blockDim.x) {
      const int I = e / ni, J = e % ni;
      const double s = sv[I] * sv[J];
      const double2 x = AR::to(A[e]);
      Ws[e] = make_double2(s * (x.x - (I == J ? 1.0 : 0.0)), s * x.y);
    }
  }
  if (t == 0) info[sys] = 0;
}

template <class AR>
gw_status launch_inv(gw_ctx* c, int iq0, int nsys, const double* P, double* W, int* info, double* aug) {
  using S = typename AR::S;
  const size_t smem = sizeof(S) * (2 * GJ_B * (GJ_B + 1) + (size_t)GJ_RP * (GJ_B + 1));
  cudaFuncSetAttribute(k_screen_inv<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kt_begin(c, "k_screen_inv");
  k_screen_inv<AR><<<nsys, 256, smem, c->stream>>>((const double2*)P, c->d_sqrtv + (size_t)iq0 * c->ni, c->nnu,
                                                   c->ni, reinterpret_cast<S*>(aug), (double2*)W, info);
  kt_end(c);
  return check_launch(c, "screen");
}

}  // namespace

gw_status launch_screen(gw_ctx* c, int iq0, int nqb, int prec, const double* P, double* W, int* info, double* aug) {
  const int nsys = nqb * c->nnu;
  const bool blocked = c->ni % GJ_B == 0;
  if (prec == GW_F32X2) {
    if (!blocked) return set_err(c, GW_EUNSUPPORTED, "gw_screen: GW_F32X2 needs ni a multiple of 32");
    return launch_inv<Ff32>(c, iq0, nsys, P, W, info, aug);
  }
  if (prec == GW_F32) {
    if (!blocked) return set_err(c, GW_EUNSUPPORTED, "gw_screen: GW_F32 needs ni a multiple of 32");
    return launch_inv<F32>(c, iq0, nsys, P, W, info, aug);
  }
  if (prec != GW_FP64) return set_err(c, GW_EUNSUPPORTED, "gw_screen: precision must be GW_FP64, GW_F32X2 or GW_F32");
  if (blocked) return launch_inv<Fp64>(c, iq0, nsys, P, W, info, aug);
  k_screen<<<nsys, 512, 0, c->stream>>>((const double2*)P, c->d_sqrtv + (size_t)iq0 * c->ni, c->nnu, c->ni,
                                        (double2*)aug, (double2*)W, info);
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
  // an error left by the caller's own earlier work is reported, not cleared
  if (cudaPeekAtLastError() != cudaSuccess) return GW_ECUDA;
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
