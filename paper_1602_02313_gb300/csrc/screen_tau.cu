// The paper's tau-domain form of the screened interaction (Sec. III.B.3, Eq. tildeW), after
// Stan et al.: W~(tau) = v P(tau) v + int_0^beta dtau' v P(tau - tau') W~(tau'), discretised on a
// mesh tau_0 = 0 < ... < tau_M = beta with the paper's trapezoid increments into one dense
// linear system of N = (M + 1) NI unknowns and NI right-hand sides:
//   K[(p, I), (r, J)] = delta_pr delta_IJ - v_I P_IJ(tau_p - tau_r) dtau_r
//   B[(p, I), J']     = v_I P_IJ'(tau_p) v_J'
// It is the cross-check of the i nu route (bosonic transform, algebraic screening, transform
// back) on small meshes, not a step of the benchmarked iteration.
//
// Solver: Gauss-Jordan elimination with partial pivoting on [K | B] in FP64, one launch per
// pivot column (the grid is the rows, so every SM works on every step), reading one copy of
// the augmented matrix and writing the other (rows swap without a race). Every block finds the
// pivot itself (the same reduction in every block, so a step needs no separate launch or
// grid-wide barrier) from FP32 magnitudes |re| + |im| of the pivot column that the previous
// step wrote beside its rows (the modulus of LAPACK's izamax): the largest, the lowest row on
// a tie, as one integer maximum over (magnitude bits, complemented row). The FP64 pipe of this
// GPU is slow (~1/64 of FP32), so each row's factor (its column-k entry over the pivot) is one
// FP64 division by one thread and each element one complex multiply-add. The solution is the
// last NI columns.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gw_internal.h"

namespace gwi {
namespace {

constexpr int kTsThreads = 256;

__device__ __forceinline__ float cabs1f(double2 a) { return (float)(fabs(a.x) + fabs(a.y)); }

__global__ void k_tsys_build(const double2* __restrict__ Pp, const double* __restrict__ v,
                             const double* __restrict__ dtau, int npts, int ni, double2* __restrict__ aug,
                             float* __restrict__ mag) {
  const int64_t N = (int64_t)npts * ni, L = N + ni;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N * L) return;
  const int64_t R = e / L, C = e % L;
  const int p = (int)(R / ni), I = (int)(R % ni);
  double2 val;
  if (C < N) {
    const int r = (int)(C / ni), J = (int)(C % ni);
    const double2 P = Pp[(((size_t)p * npts + r) * ni + I) * ni + J];
    const double s = v[I] * dtau[r];
    val = make_double2((R == C ? 1.0 : 0.0) - s * P.x, -s * P.y);
  } else {
    const int J = (int)(C - N);
    const double2 P = Pp[(((size_t)p * npts + 0) * ni + I) * ni + J];  // tau_p - tau_0 = tau_p
    const double s = v[I] * v[J];
    val = make_double2(s * P.x, s * P.y);
  }
  aug[e] = val;
  if (C == 0) mag[R] = cabs1f(val);  // the first pivot column
}

// Step k: row k <- pivot row q / a_qk; every other row i <- (row i, or row k for i = q)
// - (its column-k entry / a_qk) x pivot row. Columns below k are never read again and are left
// as they are. mag_in holds the pivot column's magnitudes; mag_out receives column k + 1's.
__global__ void __launch_bounds__(kTsThreads) k_tsys_step(const double2* __restrict__ in, double2* __restrict__ out,
                                                          const float* __restrict__ mag_in,
                                                          float* __restrict__ mag_out, int N, int L, int k,
                                                          int* __restrict__ info) {
  __shared__ unsigned long long sk[kTsThreads / 32];
  __shared__ double2 sg;
  if (*info != 0) return;  // an earlier step found no pivot
  const int t = threadIdx.x;
  unsigned long long best = 0ull;
  for (int i = k + t; i < N; i += kTsThreads) {
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(mag_in[i]) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)i);
    best = key > best ? key : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    best = ob > best ? ob : best;
  }
  if ((t & 31) == 0) sk[t >> 5] = best;
  __syncthreads();
  best = sk[0];
  for (int w = 1; w < kTsThreads / 32; ++w) best = sk[w] > best ? sk[w] : best;
  const int q = (int)(0xFFFFFFFFu - (unsigned)(best & 0xFFFFFFFFull));
  const double2 pv = in[(size_t)q * L + k];
  if (pv.x == 0.0 && pv.y == 0.0) {  // also when the FP32 magnitudes all underflowed: checked in FP64
    if (blockIdx.x == 0 && t == 0) atomicCAS(info, 0, k + 1);
    return;
  }
  const int i = blockIdx.x;
  const double2* prow = in + (size_t)q * L;
  const double2* srow = in + (size_t)(i == k ? q : (i == q ? k : i)) * L;
  if (t == 0) {
    const double dn = pv.x * pv.x + pv.y * pv.y;
    const double2 ip = make_double2(pv.x / dn, -pv.y / dn);
    if (i == k) {
      sg = ip;  // row k = pivot row / a_qk
    } else {
      const double2 f = srow[k];
      sg = make_double2(f.x * ip.x - f.y * ip.y, f.x * ip.y + f.y * ip.x);
    }
  }
  __syncthreads();
  const double2 g = sg;
  double2* orow = out + (size_t)i * L;
  for (int j = k + t; j < L; j += kTsThreads) {
    const double2 a = prow[j];
    double2 o;
    if (i == k) {
      o = make_double2(a.x * g.x - a.y * g.y, a.x * g.y + a.y * g.x);
    } else {
      const double2 b = srow[j];
      o = make_double2(b.x - (g.x * a.x - g.y * a.y), b.y - (g.x * a.y + g.y * a.x));
    }
    orow[j] = o;
    if (j == k + 1) mag_out[i] = cabs1f(o);
  }
}

__global__ void k_tsys_out(const double2* __restrict__ aug, int npts, int ni, double2* __restrict__ W) {
  const int64_t N = (int64_t)npts * ni, L = N + ni;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N * ni) return;
  const int64_t R = e / ni;
  const int J = (int)(e % ni);
  W[e] = aug[R * L + N + J];  // W~[r][I][J'] with R = r ni + I
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_screen_tau(gw_ctx* c, int iq, int npts, const double* tau, const double* P_pair,
                                   double* Wt_tau, int* info) {
  if (!c || !tau || !P_pair || !Wt_tau || !info || iq < 0 || iq >= c->nq || npts < 2) return GW_EINVAL;
  for (int r = 1; r < npts; ++r)
    if (!(tau[r] > tau[r - 1])) return set_err(c, GW_EINVAL, "gw_screen_tau: tau must increase");
  const int ni = c->ni;
  const int64_t N = (int64_t)npts * ni, L = N + ni;
  if (N > (1 << 30) / 2) return set_err(c, GW_EINVAL, "gw_screen_tau: system too large");
  // the trapezoid increments of Eq. (tildeW)
  std::vector<double> dt(npts);
  for (int r = 1; r + 1 < npts; ++r) dt[r] = 0.5 * (tau[r + 1] - tau[r - 1]);
  dt[0] = 0.5 * (tau[1] - tau[0]);
  dt[npts - 1] = 0.5 * (tau[npts - 1] - tau[npts - 2]);
  const size_t mat = (size_t)N * L * sizeof(double2);
  const size_t need = 2 * mat + 2 * (size_t)N * sizeof(float) + npts * sizeof(double);
  if (need > c->tsys_bytes) {
    if (c->d_tsys) cudaFree(c->d_tsys);
    c->d_tsys = nullptr;
    c->tsys_bytes = 0;
    if (cudaMalloc(&c->d_tsys, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "gw_screen_tau workspace");
    }
    c->tsys_bytes = need;
  }
  double2* A0 = (double2*)c->d_tsys;
  double2* A1 = (double2*)((char*)c->d_tsys + mat);
  float* M0 = (float*)((char*)c->d_tsys + 2 * mat);
  float* M1 = M0 + N;
  double* d_dt = (double*)(M1 + N);  // 2 N floats after a 16-byte boundary: 8-byte aligned
  // the increments are copied before the call returns (the host vector then goes away)
  if (cudaMemcpy(d_dt, dt.data(), npts * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_err(c, GW_ECUDA, "gw_screen_tau: copy of the increments");
  cudaMemsetAsync(info, 0, sizeof(int), c->stream);
  kt_begin(c, "tau_screen_solve");
  const int64_t ne = N * L;
  k_tsys_build<<<(unsigned)((ne + 255) / 256), 256, 0, c->stream>>>((const double2*)P_pair, c->d_v + (size_t)iq * ni,
                                                                   d_dt, npts, ni, A0, M0);
  gw_status st = check_launch(c, "tsys_build");
  if (st != GW_OK) return st;
  for (int k = 0; k < (int)N; ++k) {
    k_tsys_step<<<(unsigned)N, kTsThreads, 0, c->stream>>>(k % 2 ? A1 : A0, k % 2 ? A0 : A1, k % 2 ? M1 : M0,
                                                          k % 2 ? M0 : M1, (int)N, (int)L, k, info);
    if ((st = check_launch(c, "tsys_step")) != GW_OK) return st;
  }
  const double2* fin = N % 2 ? A1 : A0;
  k_tsys_out<<<(unsigned)((N * ni + 255) / 256), 256, 0, c->stream>>>(fin, npts, ni, (double2*)Wt_tau);
  kt_end(c);
  return check_launch(c, "tsys_out");
}
