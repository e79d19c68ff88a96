// libgw: C ABI entry points, context management and the light kernels
// (matrix-element generator, Green's function, Dyson update, transforms, exchange).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "arith.cuh"
#include "cvt.cuh"
#include "gw_internal.h"

namespace gwi {

gw_status set_err(gw_ctx* c, gw_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

void kt_begin(gw_ctx* c, const char* name) {
  if (!c || !c->ktiming) return;
  gw_ctx::KernelEvents e{name, nullptr, nullptr};
  if (cudaEventCreate(&e.begin) != cudaSuccess || cudaEventCreate(&e.end) != cudaSuccess) {
    cudaGetLastError();
    if (e.begin) cudaEventDestroy(e.begin);
    return;
  }
  cudaEventRecord(e.begin, c->stream);
  c->kev.push_back(e);
}

void kt_end(gw_ctx* c) {
  if (!c || !c->ktiming || c->kev.empty()) return;
  cudaEventRecord(c->kev.back().end, c->stream);
}

static void kt_clear(gw_ctx* c) {
  for (auto& e : c->kev) {
    cudaEventDestroy(e.begin);
    cudaEventDestroy(e.end);
  }
  c->kev.clear();
}

gw_status check_launch(gw_ctx* c, const char* what) {
  if (c) ++c->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(c, GW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return GW_OK;
}

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller: synthetic
// matrix elements M^I_ab(k, q) with E|M|^2 = 1/nb (stand-in for Eq. mmatrix).
// counter = (idx lo, idx hi, 0x4D, 0), key = (seed lo, seed hi), idx the flat
// index of (q, k, I, a, b); 24-bit uniforms u1 = ((x0 >> 8) + 1) 2^-24, u2 = (x1 >> 8) 2^-24.
// Box-Muller in FP32 with the logarithm and the sine / cosine of the generator's definition:
// fixed sequences of explicitly round-to-nearest FP32 operations (no contraction into FMAs), so
// the values are bit-identical to the host generator's.
//   ln u: u = 2^e m, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s), s = (m - 1)/(m + 1), by the
//         odd series to s^11; ln u = e ln 2 + ln m.
//   cos / sin (2 pi u): quadrant o and f = 4 u - o exactly; x = (pi/2) f; Taylor series of sin x
//         to x^13 and of cos x to x^12; the quadrant by exact sign and order changes.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// series coefficients 1/k and (-1)^(k/2) / k! rounded to FP32 (as the host generator rounds them)
__constant__ float c_atanh[5] = {(float)(1.0 / 11), (float)(1.0 / 9), (float)(1.0 / 7), (float)(1.0 / 5),
                                 (float)(1.0 / 3)};
__constant__ float c_sin[6] = {(float)(1.0 / 6227020800.0), (float)(-1.0 / 39916800.0), (float)(1.0 / 362880.0),
                               (float)(-1.0 / 5040.0), (float)(1.0 / 120.0), (float)(-1.0 / 6.0)};
__constant__ float c_cos[6] = {(float)(1.0 / 479001600.0), (float)(-1.0 / 3628800.0), (float)(1.0 / 40320.0),
                               (float)(-1.0 / 720.0), (float)(1.0 / 24.0), (float)(-1.0 / 2.0)};

__device__ __forceinline__ float gen_log(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)((bits >> 23) & 255u) - 126;
  float m = __uint_as_float((bits & 0x7FFFFFu) | (126u << 23));  // u = m 2^e, m in [0.5, 1)
  if (m < (float)0.7071067811865476) {
    m = __fmul_rn(m, 2.0f);
    e -= 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
  const float z = __fmul_rn(s, s);
  float p = __fadd_rn(__fmul_rn(z, c_atanh[0]), c_atanh[1]);
#pragma unroll
  for (int i = 2; i < 5; ++i) p = __fadd_rn(__fmul_rn(p, z), c_atanh[i]);
  p = __fmul_rn(p, z);
  const float s2 = __fadd_rn(s, s);
  const float lm = __fadd_rn(s2, __fmul_rn(s2, p));
  return __fadd_rn(__fmul_rn((float)e, (float)0.6931471805599453), lm);
}

__device__ __forceinline__ void gen_sincos_turn(float u, float& c, float& s) {
  const float t = __fmul_rn(u, 4.0f);
  const float of = floorf(t);
  const float f = __fsub_rn(t, of);
  const int o = (int)of;
  const float x = __fmul_rn(f, (float)1.5707963267948966);
  const float x2 = __fmul_rn(x, x);
  float q = __fadd_rn(__fmul_rn(x2, c_sin[0]), c_sin[1]);
#pragma unroll
  for (int i = 2; i < 6; ++i) q = __fadd_rn(__fmul_rn(q, x2), c_sin[i]);
  q = __fmul_rn(q, x2);
  const float sn = __fadd_rn(x, __fmul_rn(x, q));
  float r = __fadd_rn(__fmul_rn(x2, c_cos[0]), c_cos[1]);
#pragma unroll
  for (int i = 2; i < 6; ++i) r = __fadd_rn(__fmul_rn(r, x2), c_cos[i]);
  r = __fmul_rn(r, x2);
  const float cs = __fadd_rn(1.0f, r);
  c = o == 0 ? cs : (o == 1 ? -sn : (o == 2 ? -cs : sn));
  s = o == 0 ? sn : (o == 1 ? cs : (o == 2 ? -sn : -cs));
}

__global__ void k_gen_m(double2* __restrict__ M, uint64_t n, uint64_t off, uint64_t seed, double scale) {
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t ctr = idx + off;
    uint32_t c0 = (uint32_t)ctr, c1 = (uint32_t)(ctr >> 32), c2 = 0x4Du, c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float u1 = __fmul_rn(__fadd_rn(__uint2float_rn(c0 >> 8), 1.0f), 0x1p-24f);
    const float u2 = __fmul_rn(__uint2float_rn(c1 >> 8), 0x1p-24f);
    const float r = __fsqrt_rn(__fmul_rn(gen_log(u1), -2.0f));
    float co, sn;
    gen_sincos_turn(u2, co, sn);
    M[idx] = make_double2((double)__fmul_rn(r, co) * scale, (double)__fmul_rn(r, sn) * scale);
  }
}

gw_status launch_gen_m(gw_ctx* c, double* M) {
  const uint64_t per_q = (uint64_t)c->nk * c->ni * c->nb * c->nb;
  const uint64_t n = (uint64_t)c->nq * per_q;
  k_gen_m<<<152 * 8, 256, 0, c->stream>>>((double2*)M, n, (uint64_t)c->q0 * per_q, c->seed, std::sqrt(0.5 / c->nb));
  return check_launch(c, "gen_m");
}

// m_lazy: start generating M[iq] on the side stream (once), ordered after nothing else
static bool m_issue(gw_ctx* c, int iq) {
  if (iq >= c->nq || c->m_issued[iq]) return true;
  const uint64_t per_q = (uint64_t)c->nk * c->ni * c->nb * c->nb;
  // many short blocks on a low-priority stream: the contraction kernels' blocks are scheduled
  // first, these fill the room they leave
  const uint64_t nblk = (per_q + 256 * 16 - 1) / (256 * 16);
  k_gen_m<<<(unsigned)nblk, 256, 0, c->m_stream>>>((double2*)c->d_M_own + (size_t)iq * per_q, per_q,
                                                   (uint64_t)(c->q0 + iq) * per_q, c->seed, std::sqrt(0.5 / c->nb));
  if (check_launch(c, "gen_m") != GW_OK) return false;
  if (cudaEventRecord(c->m_done[iq], c->m_stream) != cudaSuccess) return false;
  c->m_issued[iq] = 1;
  return true;
}

const double* m_block(gw_ctx* c, int iq) {
  const uint64_t per_q = (uint64_t)c->nk * c->ni * c->nb * c->nb;
  if (c->m_lazy) {
    // the block of iq must be done before the context's stream uses it; the next q's block is
    // generated meanwhile (FP64-pipe work that runs beside the tensor-core contractions)
    if (!m_issue(c, iq) || cudaStreamWaitEvent(c->stream, c->m_done[iq], 0) != cudaSuccess || !m_issue(c, iq + 1)) {
      set_err(c, GW_ECUDA, "M generation");
      return nullptr;
    }
    return c->d_M + 2 * (size_t)iq * per_q;
  }
  if (!c->m_per_q) return c->d_M + 2 * (size_t)iq * per_q;
  if (c->m_cur != iq) {
    k_gen_m<<<152 * 8, 256, 0, c->stream>>>((double2*)c->d_M_own, per_q, (uint64_t)(c->q0 + iq) * per_q, c->seed,
                                             std::sqrt(0.5 / c->nb));
    if (check_launch(c, "gen_m") != GW_OK) {
      c->m_cur = -1;
      return nullptr;
    }
    c->m_cur = iq;
  }
  return c->d_M_own;
}

// ----------------------------------------------------------------------------
// Reference Green's function G0_j(k|tau) = -exp(-eps tau)[1 - n_F(eps)] (Sec. III.B.1):
// eps > 0: -exp(-eps tau)/(1 + exp(-beta eps)); eps <= 0: -exp(eps(beta - tau))/(1 + exp(beta eps)).
// occ = n_F(eps) = -G(beta^-).
// ----------------------------------------------------------------------------
__device__ __forceinline__ double g0_tau(double e, double t, double beta) {
  const double a = fabs(e);
  const double den = 1.0 + exp(-beta * a);
  return e > 0 ? -exp(-a * t) / den : -exp(-a * (beta - t)) / den;
}
__device__ __forceinline__ double fermi(double e, double beta) {
  const double x = exp(-beta * fabs(e));
  return e > 0 ? x / (1.0 + x) : 1.0 / (1.0 + x);
}

__global__ void k_green0(const double* __restrict__ eps, const double* __restrict__ tau, int nkb, int ntau,
                         double beta, double* __restrict__ G, double* __restrict__ occ) {
  const int64_t n = (int64_t)nkb * ntau;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int kb = (int)(i / ntau), it = (int)(i % ntau);
    const double e = eps[kb];
    G[i] = g0_tau(e, tau[it], beta);
    if (it == 0 && occ) occ[kb] = fermi(e, beta);
  }
}

gw_status launch_green0(gw_ctx* c, const double* eps, double* G, double* occ) {
  const int nkb = c->nk * c->nb;
  const int64_t n = (int64_t)nkb * c->ntau;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_green0<<<blocks, 256, 0, c->stream>>>(eps, c->d_tau, nkb, c->ntau, c->beta, G, occ);
  return check_launch(c, "green0");
}

// ----------------------------------------------------------------------------
// Diagonal Dyson update in i w (Eqs. dysongf, zxjk, zcjk posed at the sparse fermionic set):
// G(i w_j) = 1/(i w_j - eps~ - sigc(i w_j)), eps~ = eps + sigx - vxc;
// R_j = G(i w_j) - 1/(i w_j - eps~);  G(tau_i) = G0(eps~, tau_i) + sum_j A_ij Re R_j + B_ij Im R_j;
// occ = n_F(eps~) - sum_j (Abeta_j Re R_j + Bbeta_j Im R_j).  One thread per (k, band).
// ----------------------------------------------------------------------------
__global__ void k_dyson(const double* __restrict__ eps, const double* __restrict__ sigx,
                        const double* __restrict__ vxc, const double2* __restrict__ sigc, int nkb,
                        const double* __restrict__ tau, int ntau, int nw, const int* __restrict__ widx,
                        double beta, const double* __restrict__ Fbwd,
                        const double* __restrict__ Fbeta, double* __restrict__ G, double* __restrict__ occ) {
  const int kb = blockIdx.x * blockDim.x + threadIdx.x;
  if (kb >= nkb) return;
  const double et = eps[kb] + (sigx ? sigx[kb] : 0.0) - (vxc ? vxc[kb] : 0.0);
  double* g = G + (size_t)kb * ntau;
  for (int i = 0; i < ntau; ++i) g[i] = g0_tau(et, tau[i], beta);
  double ob = 0.0;
  for (int j = 0; j < nw; ++j) {
    const double w = (2.0 * widx[j] + 1.0) * 3.141592653589793 / beta;
    double rr = 0.0, ri = 0.0;
    if (sigc) {
      const double2 s = sigc[(size_t)kb * nw + j];
      // 1/(i w - et - s) - 1/(i w - et)
      const double ar = -et - s.x, ai = w - s.y;
      const double d1 = ar * ar + ai * ai;
      const double br = -et, bi = w;
      const double d2 = br * br + bi * bi;
      rr = ar / d1 - br / d2;
      ri = -ai / d1 + bi / d2;
    }
    for (int i = 0; i < ntau; ++i) g[i] += Fbwd[(size_t)i * 2 * nw + j] * rr + Fbwd[(size_t)i * 2 * nw + nw + j] * ri;
    ob += Fbeta[j] * rr + Fbeta[nw + j] * ri;
  }
  occ[kb] = fermi(et, beta) - ob;
}

gw_status launch_dyson(gw_ctx* c, const double* eps, const double* sigx, const double* vxc,
                       const double* sigc_iw, double* G, double* occ) {
  const int nkb = c->nk * c->nb;
  k_dyson<<<(nkb + 127) / 128, 128, 0, c->stream>>>(eps, sigx, vxc, (const double2*)sigc_iw, nkb, c->d_tau,
                                                   c->ntau, c->nw, c->d_widx, c->beta, c->d_Fbwd, c->d_Fbwd_beta, G,
                                                   occ);
  return check_launch(c, "dyson");
}

// ----------------------------------------------------------------------------
// Transforms: fixed FP64 matrices applied as batched matvecs.
// ----------------------------------------------------------------------------
// BOSE tau -> i nu: out[j][b] = sum_i T[j][i] in[i][b]  (complex T, complex data).
// The arithmetic is a policy: FP64, or float-float (arith.cuh) on the FP32 pipes.
// FP64 complex -> float-float, once per transform call.
__global__ void k_to_ff(const double2* __restrict__ in, arith::Ff32::S* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = arith::Ff32::from(in[i].x, in[i].y);
}

// ghat = (W_IJ + W_JI)/2 and hhat = (W_IJ - W_JI)/(2i) of a Hermitian-matrix function in
// float-float, the same operations as k_bose_bwd's own (one pass over W instead of one per tau block).
__global__ void k_to_ff_sym(const double2* __restrict__ W, int m, int64_t nf, arith::Ff32::S* __restrict__ G,
                            arith::Ff32::S* __restrict__ H) {
  using AR = arith::Ff32;
  const int64_t mm = (int64_t)m * m;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nf * mm) return;
  const int64_t j = i / mm, e = i % mm;
  const int I = (int)(e / m), J = (int)(e % m);
  const double2 ad = W[i], bd = W[j * mm + (int64_t)J * m + I];
  const AR::S a = AR::from(ad.x, ad.y), bv = AR::from(bd.x, bd.y);
  G[i] = AR::half(AR::add(a, bv));
  H[i] = AR::mul_mi(AR::half(AR::dif(a, bv)));
}

static gw_status grow_ws(gw_ctx* c, size_t need) {
  if (need <= c->ff_ws_bytes) return GW_OK;
  if (c->ff_ws) cudaFree(c->ff_ws);
  c->ff_ws = nullptr;
  c->ff_ws_bytes = 0;
  if (cudaMalloc(&c->ff_ws, need) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, GW_ENOMEM, "transform workspace");
  }
  c->ff_ws_bytes = need;
  return GW_OK;
}

// Input values in the policy's storage type (FP64 data as is; float-float data converted once
// beforehand by k_to_ff, so that the FP64-pipe conversions are not repeated per frequency block).
template <int JB, class AR>
__global__ void k_bose_fwd(const double2* __restrict__ T, const typename AR::S* __restrict__ in,
                           double2* __restrict__ out, int64_t batch, int ntau, int nf) {
  // block (x, y, z): 128 batch elements x frequencies j0 .. j0 + JB - 1 (grid.y = ceil(nf / JB))
  // of transform z
  using S = typename AR::S;
  extern __shared__ __align__(16) unsigned char bfsm[];
  S* sT = reinterpret_cast<S*>(bfsm);
  in += (size_t)blockIdx.z * ntau * batch;  // grid.z: consecutive transforms of one call
  out += (size_t)blockIdx.z * nf * batch;
  const int j0 = blockIdx.y * JB, nj = min(JB, nf - j0);
  for (int i = threadIdx.x; i < nj * ntau; i += blockDim.x) {
    const double2 t = T[(size_t)j0 * ntau + i];
    sT[i] = AR::from(t.x, t.y);
  }
  __syncthreads();
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= batch) return;
  typename AR::Acc acc[JB];
#pragma unroll
  for (int q = 0; q < JB; ++q) acc[q] = AR::azero();
  for (int i = 0; i < ntau; ++i) {
    const S x = in[(size_t)i * batch + b];
#pragma unroll
    for (int q = 0; q < JB; ++q)
      if (q < nj) AR::mac(acc[q], sT[q * ntau + i], x);
  }
#pragma unroll
  for (int q = 0; q < JB; ++q)
    if (q < nj) out[(size_t)(j0 + q) * batch + b] = AR::to(AR::val(acc[q]));
}

// BOSE i nu -> tau of a Hermitian-matrix function W[j][I][J]:
// ghat = (W_IJ + W_JI)/2 (transform of Re W(tau)), hhat = (W_IJ - W_JI)/(2i) (of Im W(tau));
// Re W(tau_i) = sum_j A_ij Re ghat_j + B_ij Im ghat_j, Im W(tau_i) likewise with hhat.
// PRE: ghat and hhat come precomputed in float-float (k_to_ff_sym) instead of from W.
template <int IB, class AR, bool PRE>
__global__ void k_bose_bwd(const double* __restrict__ Tb, const double2* __restrict__ W,
                           const typename AR::S* __restrict__ Gh, const typename AR::S* __restrict__ Hh,
                           double2* __restrict__ out, int m, int ntau, int nf) {
  // block (x, y, z): 128 matrix elements x tau points i0 .. i0 + IB - 1 (grid.y = ceil(ntau / IB))
  // of transform z
  using S = typename AR::S;
  using R = typename AR::R;
  extern __shared__ __align__(16) unsigned char bbsm[];
  R* sTb = reinterpret_cast<R*>(bbsm);
  {
    const size_t zq = (size_t)blockIdx.z * m * m;
    if (PRE) {
      Gh += zq * nf;
      Hh += zq * nf;
    } else {
      W += zq * nf;
    }
    out += zq * ntau;
  }
  const int i0 = blockIdx.y * IB, ni = min(IB, ntau - i0);
  for (int i = threadIdx.x; i < ni * 2 * nf; i += blockDim.x) sTb[i] = AR::rfrom(Tb[(size_t)i0 * 2 * nf + i]);
  __syncthreads();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t mm = (int64_t)m * m;
  if (e >= mm) return;
  const int I = (int)(e / m), J = (int)(e % m);
  const int64_t et = (int64_t)J * m + I;
  typename AR::Acc acc[IB];  // re: Re W(tau), im: Im W(tau)
#pragma unroll
  for (int q = 0; q < IB; ++q) acc[q] = AR::azero();
  for (int j = 0; j < nf; ++j) {
    S g, h;
    if (PRE) {
      g = Gh[(size_t)j * mm + e];
      h = Hh[(size_t)j * mm + e];
    } else {
      const double2 ad = W[(size_t)j * mm + e], bd = W[(size_t)j * mm + et];
      const S a = AR::from(ad.x, ad.y), bv = AR::from(bd.x, bd.y);
      g = AR::half(AR::add(a, bv));
      h = AR::mul_mi(AR::half(AR::dif(a, bv)));
    }
#pragma unroll
    for (int q = 0; q < IB; ++q)
      if (q < ni) AR::rmac2(acc[q], sTb[q * 2 * nf + j], sTb[q * 2 * nf + nf + j], g, h);
  }
#pragma unroll
  for (int q = 0; q < IB; ++q)
    if (q < ni) out[(size_t)(i0 + q) * mm + e] = AR::to(AR::val(acc[q]));
}

// FERMI tau -> i w of real rows: out[b][j] = sum_i T[j][i] in[b][i]; one thread per (b, j).
__global__ void k_fermi_fwd(const double2* __restrict__ T, const double* __restrict__ in, double2* __restrict__ out,
                            int64_t batch, int ntau, int nf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= batch * nf) return;
  const int64_t b = e / nf;
  const int j = (int)(e % nf);
  double ar = 0.0, ai = 0.0;
  const double* x = in + (size_t)b * ntau;
  const double2* t = T + (size_t)j * ntau;
  for (int i = 0; i < ntau; ++i) {
    const double xv = x[i];
    const double2 tv = t[i];
    ar = fma(tv.x, xv, ar);
    ai = fma(tv.y, xv, ai);
  }
  out[e] = make_double2(ar, ai);
}

// FERMI i w -> tau of a real function: out[b][i] = sum_j A_ij Re in[b][j] + B_ij Im in[b][j].
__global__ void k_fermi_bwd(const double* __restrict__ Tb, const double2* __restrict__ in, double* __restrict__ out,
                            int64_t batch, int ntau, int nf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= batch * ntau) return;
  const int64_t b = e / ntau;
  const int i = (int)(e % ntau);
  const double* A = Tb + (size_t)i * 2 * nf;
  const double2* x = in + (size_t)b * nf;
  double s = 0.0;
  for (int j = 0; j < nf; ++j) {
    const double2 v = x[j];
    s = fma(A[j], v.x, fma(A[nf + j], v.y, s));
  }
  out[e] = s;
}

// Float-float conversions of a multi-transform call go through the workspace in chunks of
// transforms of at most this many bytes.
constexpr size_t kFfWsCap = 2ull << 30;

gw_status launch_transform(gw_ctx* c, int stat, int dir, int prec, int count, int64_t batch, const double* in,
                           double* out) {
  const int nt = c->ntau;
  if (stat == GW_BOSE && dir == GW_TAU_TO_IW) {
    const int64_t blocks = (batch + 127) / 128;
    if (prec == GW_F32X2) {
      using S = arith::Ff32::S;
      const int64_t per = (int64_t)nt * batch;  // inputs of one transform
      const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(count, kFfWsCap / (sizeof(S) * per)));
      gw_status st;
      if ((st = grow_ws(c, sizeof(S) * per * chunk)) != GW_OK) return st;
      const size_t sm = sizeof(S) * 16 * nt;
      if (sm > 48 * 1024) cudaFuncSetAttribute(k_bose_fwd<16, arith::Ff32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      for (int z0 = 0; z0 < count; z0 += chunk) {
        const int nz = std::min(chunk, count - z0);
        const int64_t n = per * nz;
        k_to_ff<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const double2*)in + per * z0, (S*)c->ff_ws, n);
        if ((st = check_launch(c, "to_ff")) != GW_OK) return st;
        k_bose_fwd<16, arith::Ff32><<<dim3((unsigned)blocks, (c->nnu + 15) / 16, nz), 128, sm, c->stream>>>(
            (const double2*)c->d_Bfwd, (const S*)c->ff_ws, (double2*)out + (int64_t)c->nnu * batch * z0, batch, nt,
            c->nnu);
        if ((st = check_launch(c, "bose_fwd")) != GW_OK) return st;
      }
      return GW_OK;
    }
    const size_t sm = sizeof(double2) * 8 * nt;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_bose_fwd<8, arith::Fp64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_bose_fwd<8, arith::Fp64><<<dim3((unsigned)blocks, (c->nnu + 7) / 8, count), 128, sm, c->stream>>>(
        (const double2*)c->d_Bfwd, (const double2*)in, (double2*)out, batch, nt, c->nnu);
    return check_launch(c, "bose_fwd");
  }
  if (stat == GW_BOSE && dir == GW_IW_TO_TAU) {
    const int m = (int)batch;
    const int64_t mm = (int64_t)m * m;
    const unsigned blocks = (unsigned)((mm + 127) / 128);
    if (prec == GW_F32X2) {
      using S = arith::Ff32::S;
      const int64_t per = (int64_t)c->nnu * mm;  // inputs of one transform
      const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(count, kFfWsCap / (2 * sizeof(S) * per)));
      gw_status st;
      if ((st = grow_ws(c, 2 * sizeof(S) * per * chunk)) != GW_OK) return st;
      const size_t sm = sizeof(arith::Ff32::R) * 16 * 2 * c->nnu;
      if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_bose_bwd<16, arith::Ff32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      for (int z0 = 0; z0 < count; z0 += chunk) {
        const int nz = std::min(chunk, count - z0);
        const int64_t n = per * nz;
        S* Gh = (S*)c->ff_ws;
        S* Hh = Gh + n;
        // nz consecutive transforms are one [nz nnu][m][m] stack for the symmetrisation
        k_to_ff_sym<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const double2*)in + per * z0, m,
                                                                         (int64_t)c->nnu * nz, Gh, Hh);
        if ((st = check_launch(c, "to_ff_sym")) != GW_OK) return st;
        k_bose_bwd<16, arith::Ff32, true><<<dim3(blocks, (nt + 15) / 16, nz), 128, sm, c->stream>>>(
            c->d_Bbwd, nullptr, Gh, Hh, (double2*)out + (int64_t)nt * mm * z0, m, nt, c->nnu);
        if ((st = check_launch(c, "bose_bwd")) != GW_OK) return st;
      }
      return GW_OK;
    }
    const size_t sm = sizeof(double) * 8 * 2 * c->nnu;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_bose_bwd<8, arith::Fp64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_bose_bwd<8, arith::Fp64, false><<<dim3(blocks, (nt + 7) / 8, count), 128, sm, c->stream>>>(
        c->d_Bbwd, (const double2*)in, nullptr, nullptr, (double2*)out, m, nt, c->nnu);
    return check_launch(c, "bose_bwd");
  }
  // FERMI: count consecutive [batch][...] blocks are one batch of count * batch rows
  batch *= count;
  if (stat == GW_FERMI && (dir == GW_TAU_TO_IW || dir == GW_TAU_TO_IW_CONT)) {
    const int nf = dir == GW_TAU_TO_IW ? c->nw : c->ncont;
    const double* T = dir == GW_TAU_TO_IW ? c->d_Ffwd : c->d_Fcont;
    const int64_t n = batch * nf;
    k_fermi_fwd<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>((const double2*)T, in, (double2*)out, batch, nt,
                                                                    nf);
    return check_launch(c, "fermi_fwd");
  }
  if (stat == GW_FERMI && dir == GW_IW_TO_TAU) {
    const int64_t n = batch * nt;
    k_fermi_bwd<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(c->d_Fbwd, (const double2*)in, out, batch, nt,
                                                                    c->nw);
    return check_launch(c, "fermi_bwd");
  }
  return set_err(c, GW_EINVAL, "gw_tau_to_freq: unsupported stat/dir");
}

// ----------------------------------------------------------------------------
// Exchange self-energy, product-basis form of Eq. (sigx) with diagonal v:
// Sigx_n(k) += -1/(Omega Nk) sum_j occ_j(k-q) sum_I v_I |M^I_jn|^2.
// k_vm streams M once, coalesced along the pair index p = j nb + n:
// vm[k][p] = sum_I v_I |M^I_p|^2; k_sigx_occ then contracts with the occupations.
// Deterministic (no atomics).
// ----------------------------------------------------------------------------
__global__ void k_vm(const double2* __restrict__ M, const double* __restrict__ v, int ni, int np,
                     double* __restrict__ vm) {
  const int k = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double2* Mk = M + (size_t)k * ni * np + p;
  // 8 loads in flight per thread, one partial sum per residue of I mod 8
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int I = 0;
  for (; I + 8 <= ni; I += 8) {
    double2 m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = Mk[(size_t)(I + u) * np];
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] = fma(v[I + u], fma(m[u].x, m[u].x, m[u].y * m[u].y), s[u]);
  }
  for (; I < ni; ++I) {
    const double2 m = Mk[(size_t)I * np];
    s[0] = fma(v[I], fma(m.x, m.x, m.y * m.y), s[0]);
  }
  vm[(size_t)k * np + p] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// The same sum in float-float on the FP32 pipes (the mixed chain): M converted on the integer
// pipes (cvt.cuh), |M|^2 = xh^2 + 2 xh xl + yh^2 + 2 yh yl with each product's rounding error
// from an FMA (the xl^2, yl^2 terms lie below 2^-46 relative), times v_I in float-float, summed
// by error-free two-sums into two alternating accumulators; ~1e-12 relative, against the
// FP64 pipe's 3 operations per element, which bound k_vm on GB300.
__device__ __forceinline__ void two_sum_ff(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}

__device__ __forceinline__ void vm_term(double2 m, float vh, float vl, float& ah, float& al) {
  float xh, xl, yh, yl;
  cvt::d2ff(m.x, xh, xl);
  cvt::d2ff(m.y, yh, yl);
  const float p1 = __fmul_rn(xh, xh), p2 = __fmul_rn(yh, yh);  // never contracted into the sums below
  float e1 = fmaf(xh, xh, -p1), e2 = fmaf(yh, yh, -p2);
  e1 = fmaf(2.f * xh, xl, e1);
  e2 = fmaf(2.f * yh, yl, e2);
  float s, t;
  two_sum_ff(p1, p2, s, t);
  t += e1 + e2;
  const float q = __fmul_rn(s, vh);
  float eq = fmaf(s, vh, -q);
  eq = fmaf(s, vl, eq);
  eq = fmaf(t, vh, eq);
  float c, ce;
  two_sum_ff(ah, q, c, ce);
  ah = c;
  al += ce + eq;
}

__global__ void k_vm_ff(const double2* __restrict__ M, const double* __restrict__ v, int ni, int np,
                        double* __restrict__ vm) {
  extern __shared__ float2 svf[];  // v_I as (hi, lo)
  for (int I = threadIdx.x; I < ni; I += blockDim.x) {
    float h, l;
    cvt::d2ff(v[I], h, l);
    svf[I] = make_float2(h, l);
  }
  __syncthreads();
  const int k = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double2* Mk = M + (size_t)k * ni * np + p;
  float ah[2] = {0.f, 0.f}, al[2] = {0.f, 0.f};
  int I = 0;
  for (; I + 8 <= ni; I += 8) {
    double2 m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = Mk[(size_t)(I + u) * np];
#pragma unroll
    for (int u = 0; u < 8; ++u) vm_term(m[u], svf[I + u].x, svf[I + u].y, ah[u & 1], al[u & 1]);
  }
  for (; I < ni; ++I) vm_term(Mk[(size_t)I * np], svf[I].x, svf[I].y, ah[0], al[0]);
  float s, e;
  two_sum_ff(ah[0], ah[1], s, e);
  vm[(size_t)k * np + p] = (double)s + ((double)al[0] + (double)al[1] + (double)e);
}

__global__ void k_sigx_occ(const double* __restrict__ vm, const int* __restrict__ kmq, const double* __restrict__ occ,
                           int nk, int nb, double pref, double* __restrict__ Sx) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nk * nb) return;
  const int k = e / nb, n = e % nb;
  const double* vk = vm + (size_t)k * nb * nb;
  const double* f = occ + (size_t)kmq[k] * nb;
  double s = 0.0;
  for (int j = 0; j < nb; ++j) s = fma(f[j], vk[j * nb + n], s);
  Sx[e] += pref * s;
}

gw_status launch_sigx(gw_ctx* c, int iq, const double* occ, double* Sx, bool ff) {
  const int np = c->nb * c->nb;
  const size_t need = (size_t)c->nk * np * sizeof(double);
  if (need > c->vm_bytes) {
    if (c->d_vm) cudaFree(c->d_vm);
    c->d_vm = nullptr;
    c->vm_bytes = 0;
    if (cudaMalloc((void**)&c->d_vm, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "sigx workspace");
    }
    c->vm_bytes = need;
  }
  const double2* M = (const double2*)m_block(c, iq);
  if (!M) return GW_ECUDA;
  if (ff)
    k_vm_ff<<<dim3((np + 255) / 256, c->nk), 256, sizeof(float2) * c->ni, c->stream>>>(
        M, c->d_v + (size_t)iq * c->ni, c->ni, np, c->d_vm);
  else
    k_vm<<<dim3((np + 255) / 256, c->nk), 256, 0, c->stream>>>(M, c->d_v + (size_t)iq * c->ni, c->ni, np, c->d_vm);
  gw_status s = check_launch(c, "sigx_vm");
  if (s != GW_OK) return s;
  const int n = c->nk * c->nb;
  k_sigx_occ<<<(n + 127) / 128, 128, 0, c->stream>>>(c->d_vm, c->d_kmq + (size_t)iq * c->nk, occ, c->nk, c->nb,
                                                     -1.0 / (c->omega * c->nk), Sx);
  return check_launch(c, "sigx_occ");
}

}  // namespace gwi

using namespace gwi;

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

static bool grid_ok(const gw_grid* g) {
  if (!g || g->ntau <= 0 || g->ntau > 256 || (g->ntau & 1) || !g->tau || g->npole < 1 || g->npole > g->ntau ||
      !g->poles || g->nnu < 1 || !g->nu_idx || g->nw < 1 || !g->w_idx || g->ncont < 1 || g->ncont > 512 ||
      !(g->beta > 0) || 2 * g->nnu < g->npole || 2 * g->nw < g->npole)
    return false;
  for (int i = 0; i < g->ntau; ++i) {
    if (!(g->tau[i] > 0 && g->tau[i] < g->beta)) return false;
    if (i && !(g->tau[i] > g->tau[i - 1])) return false;
    if (std::fabs(g->tau[i] + g->tau[g->ntau - 1 - i] - g->beta) > 1e-12 * g->beta) return false;
  }
  for (int i = 0; i < g->nnu; ++i)
    if (g->nu_idx[i] < 0) return false;
  for (int i = 0; i < g->nw; ++i)
    if (g->w_idx[i] < 0) return false;
  return true;
}

static gw_status upload(gw_ctx* c, double** dst, const std::vector<double>& h) {
  if (cudaMalloc((void**)dst, sizeof(double) * std::max<size_t>(1, h.size())) != cudaSuccess)
    return set_err(c, GW_ENOMEM, "cudaMalloc failed");
  if (!h.empty() && cudaMemcpy(*dst, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return set_err(c, GW_ECUDA, "cudaMemcpy failed");
  return GW_OK;
}

gw_status gw_create(gw_ctx** out, const gw_grid* g, const gw_system* s, int device, void* stream) {
  if (!out || !g || !s) return GW_EINVAL;
  *out = nullptr;
  if (!grid_ok(g)) return GW_EINVAL;
  if (s->m_mode < 0 || s->m_mode > 3 || s->q0 < 0 || s->nk < 1 || s->nq < 1 || s->nb < 1 || s->nb > 256 || s->ni < 16 || s->ni > 1024 || (s->ni % 32) || !s->kmq ||
      !s->v || !(s->omega > 0))
    return GW_EINVAL;
  for (int i = 0; i < s->nq * s->nk; ++i)
    if (s->kmq[i] < 0 || s->kmq[i] >= s->nk) return GW_EINVAL;
  for (int i = 0; i < s->nq * s->ni; ++i)
    if (!(s->v[i] > 0)) return GW_EINVAL;

  gw_ctx* c = new gw_ctx();
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return GW_ECUDA;
  }
  c->stream = (cudaStream_t)stream;
  c->beta = g->beta;
  c->ntau = g->ntau;
  c->npole = g->npole;
  c->nnu = g->nnu;
  c->nw = g->nw;
  c->ncont = g->ncont;
  c->tau.assign(g->tau, g->tau + g->ntau);
  c->poles.assign(g->poles, g->poles + g->npole);
  c->nu_idx.assign(g->nu_idx, g->nu_idx + g->nnu);
  c->w_idx.assign(g->w_idx, g->w_idx + g->nw);
  c->seed = s->seed;
  c->q0 = s->q0;
  c->nk = s->nk;
  c->nq = s->nq;
  c->nb = s->nb;
  c->nocc = s->nocc;
  c->ni = s->ni;
  c->omega = s->omega;
  c->kmq.assign(s->kmq, s->kmq + (size_t)s->nq * s->nk);
  c->v.assign(s->v, s->v + (size_t)s->nq * s->ni);

  build_transforms(c->tau, c->poles, c->beta, c->nu_idx, c->w_idx, c->ncont, &c->T);

  gw_status st = GW_OK;
  std::vector<double> sv(c->v.size());
  for (size_t i = 0; i < sv.size(); ++i) sv[i] = std::sqrt(c->v[i]);
  if ((st = upload(c, &c->d_v, c->v)) || (st = upload(c, &c->d_sqrtv, sv)) ||
      (st = upload(c, &c->d_Bfwd, c->T.B_fwd)) || (st = upload(c, &c->d_Ffwd, c->T.F_fwd)) ||
      (st = upload(c, &c->d_Fcont, c->T.F_cont)) || (st = upload(c, &c->d_Bbwd, c->T.B_bwd)) ||
      (st = upload(c, &c->d_Fbwd, c->T.F_bwd)) || (st = upload(c, &c->d_Fbwd_beta, c->T.F_bwd_beta))) {
    gw_destroy(c);
    return st;
  }
  if (cudaMalloc((void**)&c->d_kmq, sizeof(int) * c->kmq.size()) != cudaSuccess) {
    gw_destroy(c);
    return GW_ENOMEM;
  }
  cudaMemcpy(c->d_kmq, c->kmq.data(), sizeof(int) * c->kmq.size(), cudaMemcpyHostToDevice);
  if ((st = upload(c, &c->d_tau, c->tau)) != GW_OK) {
    gw_destroy(c);
    return st;
  }
  if (cudaMalloc((void**)&c->d_widx, sizeof(int) * c->nw) != cudaSuccess) {
    gw_destroy(c);
    return GW_ENOMEM;
  }
  cudaMemcpy(c->d_widx, c->w_idx.data(), sizeof(int) * c->nw, cudaMemcpyHostToDevice);
  if (cudaMalloc((void**)&c->d_err, 16) != cudaSuccess || cudaMemset(c->d_err, 0, 16) != cudaSuccess) {
    cudaGetLastError();
    gw_destroy(c);
    return GW_ENOMEM;
  }

  if (s->M) {
    c->d_M = s->M;
  } else {
    const size_t per_q = (size_t)c->nk * c->ni * c->nb * c->nb * sizeof(double2);
    const size_t bytes = (size_t)c->nq * per_q;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    c->m_per_q = s->m_mode == 2 || (s->m_mode == 0 && bytes > free_b / 2);
    c->m_lazy = !c->m_per_q && (s->m_mode == 0 || s->m_mode == 3);
    if (cudaMalloc((void**)&c->d_M_own, c->m_per_q ? per_q : bytes) != cudaSuccess) {
      cudaGetLastError();
      gw_destroy(c);
      return GW_ENOMEM;
    }
    c->d_M = c->d_M_own;
    if (c->m_lazy) {
      c->m_done.assign(c->nq, nullptr);
      c->m_issued.assign(c->nq, 0);
      int prio_low = 0, prio_high = 0;
      cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
      bool okc = cudaStreamCreateWithPriority(&c->m_stream, cudaStreamNonBlocking, prio_low) == cudaSuccess;
      for (int q = 0; q < c->nq && okc; ++q)
        okc = cudaEventCreateWithFlags(&c->m_done[q], cudaEventDisableTiming) == cudaSuccess;
      if (!okc) {
        cudaGetLastError();
        gw_destroy(c);
        return GW_ECUDA;
      }
      if (!m_issue(c, 0)) {  // the first block starts at once
        gw_destroy(c);
        return GW_ECUDA;
      }
    } else if (!c->m_per_q && (st = launch_gen_m(c, c->d_M_own)) != GW_OK) {
      gw_destroy(c);
      return st;
    }
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    gw_destroy(c);
    return GW_ECUDA;
  }
  *out = c;
  return GW_OK;
}

gw_status gw_destroy(gw_ctx* c) {
  if (!c) return GW_EINVAL;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaDeviceSynchronize();
  kt_clear(c);
  for (cudaEvent_t e : c->m_done)
    if (e) cudaEventDestroy(e);
  c->m_done.clear();
  if (c->m_stream) cudaStreamDestroy(c->m_stream);
  c->m_stream = nullptr;
  if (c->ff_ws) cudaFree(c->ff_ws);
  if (c->d_tsys) cudaFree(c->d_tsys);
  if (c->d_dyt) cudaFree(c->d_dyt);
  if (c->d_dm) cudaFree(c->d_dm);
  c->ff_ws = nullptr;
  double* bufs[] = {c->d_sqrtv, c->d_v,       c->d_M_own, c->d_Bfwd,  c->d_Ffwd,  c->d_Fcont, c->d_Bbwd,
                    c->d_Fbwd,  c->d_Fbwd_beta, c->d_aug,   c->d_cpe_x, c->d_cpe_A, c->d_cpe_N, c->d_cpe_tab, c->d_cpe_b,
                    c->d_pade,  c->d_vm};
  for (double* p : bufs)
    if (p) cudaFree(p);
  if (c->d_kmq) cudaFree(c->d_kmq);
  if (c->d_cpe_iters) cudaFree(c->d_cpe_iters);
  if (c->d_cpe_seed) cudaFree(c->d_cpe_seed);
  if (c->d_widx) cudaFree(c->d_widx);
  if (c->d_tau) cudaFree(c->d_tau);
  if (c->d_err) cudaFree(c->d_err);
  free_mixed(c);
  delete c;
  return GW_OK;
}

gw_status gw_sync(gw_ctx* c) {
  if (!c) return GW_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return set_err(c, GW_ECUDA, std::string("gw_sync: ") + cudaGetErrorString(e));
  // a bounded wait in a tensor-core contraction that ran out since the last gw_sync
  int h = 0;
  if (cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_err(c, GW_ECUDA, "gw_sync: reading the device error word");
  if (h != 0) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return set_err(c, GW_ETIMEOUT,
                   "gw_sync: a bounded device-side wait ran out in a tensor-core contraction (k_pol_tc / k_sig_tc); "
                   "the outputs of the calls since the last gw_sync are undefined");
  }
  return GW_OK;
}

const char* gw_last_error(gw_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t gw_launch_count(gw_ctx* c) { return c ? c->launches : -1; }

gw_status gw_set_stream(gw_ctx* c, void* stream) {
  if (!c) return GW_EINVAL;
  c->stream = (cudaStream_t)stream;
  return GW_OK;
}

gw_status gw_set_tuning(gw_ctx* c, gw_tune key, int64_t value) {
  if (!c) return GW_EINVAL;
  switch (key) {
    case GW_TUNE_POL_SEG_CHUNKS:
      if (value < 1 || value > 32) return set_err(c, GW_EINVAL, "gw_set_tuning: segment chunks in 1 .. 32");
      c->pol_seg_chunks = (int)value;
      return GW_OK;
    case GW_TUNE_POL_PART_MB:
      if (value < 1 || value > (1ll << 22)) return set_err(c, GW_EINVAL, "gw_set_tuning: partial MiB >= 1");
      c->pol_part_bytes = (size_t)value << 20;
      return GW_OK;
    case GW_TUNE_WAIT_CYCLES:
      if (value < 1000 || value > (1ll << 40)) return set_err(c, GW_EINVAL, "gw_set_tuning: wait cycles in 1e3 .. 2^40");
      c->wait_cycles = value;
      return GW_OK;
    case GW_TUNE_FAULT_STALL:
      if (value != 0 && value != 1) return set_err(c, GW_EINVAL, "gw_set_tuning: stall injection is 0 or 1");
      c->fault_stall = (int)value;
      return GW_OK;
    case GW_TUNE_POL_FORM:
      if (value < 0 || value > 2) return set_err(c, GW_EINVAL, "gw_set_tuning: polarization form is 0, 1 or 2");
      c->pol_form = (int)value;
      return GW_OK;
  }
  return set_err(c, GW_EINVAL, "gw_set_tuning: unknown key");
}

gw_status gw_kernel_timing(gw_ctx* c, int enable) {
  if (!c) return GW_EINVAL;
  kt_clear(c);
  c->ktiming = enable != 0;
  return GW_OK;
}

gw_status gw_kernel_time(gw_ctx* c, const char* kernel, double* total_ms, int64_t* launches) {
  if (!c || !kernel || !total_ms || !launches) return GW_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return set_err(c, GW_ECUDA, "gw_kernel_time: stream");
  double t = 0.0;
  int64_t n = 0;
  for (const auto& e : c->kev) {
    if (std::strcmp(e.name, kernel) != 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.begin, e.end) != cudaSuccess) return set_err(c, GW_ECUDA, "gw_kernel_time: event");
    t += ms;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  return GW_OK;
}

gw_status gw_green_tau(gw_ctx* c, const double* eps, const double* sigx, const double* vxc, const double* sigc_iw,
                       double* G, double* occ) {
  if (!c || !eps || !G || !occ) return GW_EINVAL;
  if (!sigx && !vxc && !sigc_iw) return launch_green0(c, eps, G, occ);
  return launch_dyson(c, eps, sigx, vxc, sigc_iw, G, occ);
}

gw_status gw_polarization(gw_ctx* c, int iq, const double* G, gw_prec prec, double* P) {
  if (!c || !G || !P || iq < 0 || iq >= c->nq) return GW_EINVAL;
  if (prec == GW_FP64) return launch_pol_fp64(c, iq, G, P);
  if (prec == GW_FP16X2) return launch_pol_mixed(c, iq, G, (int)prec, P);
  return GW_EINVAL;
}

gw_status gw_polarization_many(int njobs, gw_ctx* const* ctxs, const int* iqs, const double* const* G_tau,
                               double* const* P_tau, gw_prec prec) {
  if (njobs < 1 || njobs > 16 || !ctxs || !iqs || !G_tau || !P_tau) return GW_EINVAL;
  for (int j = 0; j < njobs; ++j) {
    if (!ctxs[j] || !G_tau[j] || !P_tau[j]) return GW_EINVAL;
    if (iqs[j] < 0 || iqs[j] >= ctxs[j]->nq) return set_err(ctxs[0], GW_EINVAL, "gw_polarization_many: q index");
    if (ctxs[j]->device != ctxs[0]->device)
      return set_err(ctxs[0], GW_EINVAL, "gw_polarization_many: contexts on different devices");
    for (int i = 0; i < j; ++i)
      if (ctxs[i] == ctxs[j]) return set_err(ctxs[0], GW_EINVAL, "gw_polarization_many: a context appears twice");
  }
  if (prec != GW_FP16X2) return set_err(ctxs[0], GW_EUNSUPPORTED, "gw_polarization_many: only GW_FP16X2");
  return launch_pol_many(njobs, ctxs, iqs, G_tau, P_tau);
}

gw_status gw_tau_to_freq_many(gw_ctx* c, gw_stat stat, gw_dir dir, int count, int64_t batch, const double* in,
                              gw_prec prec, double* out) {
  if (!c || !in || !out || batch <= 0 || count <= 0 || count > 65535) return GW_EINVAL;
  if (stat == GW_BOSE && dir == GW_TAU_TO_IW_CONT) return GW_EINVAL;
  if (prec != GW_FP64 && !(prec == GW_F32X2 && stat == GW_BOSE))
    return set_err(c, GW_EUNSUPPORTED, "gw_tau_to_freq: GW_FP64, or GW_F32X2 for the bosonic transforms");
  return launch_transform(c, (int)stat, (int)dir, (int)prec, count, batch, in, out);
}

gw_status gw_tau_to_freq(gw_ctx* c, gw_stat stat, gw_dir dir, int64_t batch, const double* in, gw_prec prec,
                         double* out) {
  return gw_tau_to_freq_many(c, stat, dir, 1, batch, in, prec, out);
}

gw_status gw_screen(gw_ctx* c, int iq0, int nqb, const double* P, gw_prec prec, double* W, int* info) {
  if (!c || !P || !W || !info || iq0 < 0 || nqb < 1 || iq0 + nqb > c->nq) return GW_EINVAL;
  const size_t need = (size_t)nqb * c->nnu * c->ni * 2 * c->ni * sizeof(double2);
  if (need > c->aug_bytes) {
    if (c->d_aug) cudaFree(c->d_aug);
    c->d_aug = nullptr;
    c->aug_bytes = 0;
    if (cudaMalloc((void**)&c->d_aug, need) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, GW_ENOMEM, "gw_screen: workspace");
    }
    c->aug_bytes = need;
  }
  return launch_screen(c, iq0, nqb, (int)prec, P, W, info, c->d_aug);
}

gw_status gw_selfenergy(gw_ctx* c, int iq, const double* G, const double* occ, const double* W, gw_prec prec,
                        double* S, double* Sx) {
  if (!c || !G || !W || !S || iq < 0 || iq >= c->nq || (Sx && !occ)) return GW_EINVAL;
  gw_status st;
  if (prec == GW_FP64)
    st = launch_sigma_fp64(c, iq, G, W, S);
  else if (prec == GW_FP16X2)
    st = launch_sigma_mixed(c, iq, G, W, (int)prec, S);
  else
    return GW_EINVAL;
  if (st != GW_OK) return st;
  if (Sx) return launch_sigx(c, iq, occ, Sx, prec != GW_FP64);  // float-float on the mixed chain
  return GW_OK;
}

gw_status gw_continue(gw_ctx* c, gw_cont_method method, int64_t nprob, const double* sig_iw, const double* eps,
                      const double* sigx, const double* vxc, int nreal, const double* omega_real, double* sig_real,
                      double* e_qp, int* info) {
  if (!c || nprob <= 0 || !sig_iw || !eps || !sigx || !vxc || !e_qp || !info || nreal < 0 ||
      (nreal > 0 && (!omega_real || !sig_real)))
    return GW_EINVAL;
  if (method == GW_CPE && c->cpe_ngrid == 0) return set_err(c, GW_EINVAL, "gw_continue: call gw_cpe_setup first");
  if (method != GW_PADE && method != GW_CPE) return GW_EINVAL;
  return launch_continue(c, (int)method, nprob, sig_iw, eps, sigx, vxc, nreal, omega_real, sig_real, e_qp, info);
}

gw_status gw_copy_m(gw_ctx* c, int iq, int k0, int nkc, double* out) {
  if (!c || !out || iq < 0 || iq >= c->nq || k0 < 0 || nkc < 1 || k0 + nkc > c->nk) return GW_EINVAL;
  const size_t per_k = (size_t)c->ni * c->nb * c->nb * sizeof(double2);
  const double* mq = m_block(c, iq);
  if (!mq) return GW_ECUDA;
  const char* src = (const char*)mq + (size_t)k0 * per_k;
  if (cudaMemcpyAsync(out, src, per_k * nkc, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
    return set_err(c, GW_ECUDA, "gw_copy_m");
  return GW_OK;
}

gw_status gw_transform_matrices(const gw_grid* g, double* B_fwd, double* F_fwd, double* F_cont, double* B_bwd,
                                double* F_bwd) {
  if (!grid_ok(g)) return GW_EINVAL;
  gwi::Transforms T;
  build_transforms(std::vector<double>(g->tau, g->tau + g->ntau), std::vector<double>(g->poles, g->poles + g->npole),
                   g->beta, std::vector<int>(g->nu_idx, g->nu_idx + g->nnu),
                   std::vector<int>(g->w_idx, g->w_idx + g->nw), g->ncont, &T);
  auto cp = [](double* d, const std::vector<double>& s) {
    if (d) std::memcpy(d, s.data(), sizeof(double) * s.size());
  };
  cp(B_fwd, T.B_fwd);
  cp(F_fwd, T.F_fwd);
  cp(F_cont, T.F_cont);
  cp(B_bwd, T.B_bwd);
  cp(F_bwd, T.F_bwd);
  return GW_OK;
}

}  // extern "C"
