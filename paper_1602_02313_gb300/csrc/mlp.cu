// Learned seed of the continuous-pole expansion (not in the paper): a multilayer
// perceptron nin -> nh (x nhidden, GELU) -> nout (softplus) maps the normalised
// Matsubara self-energy of one (k, n) problem to non-negative pole weights on the CPE
// grid. Training minimises L = (1/B) sum_b ||A b_hat_b - x_b||^2 (A = CPE kernel at the
// first nw_fit fermionic frequencies, real-stacked), so no labels are needed.
//
// Every matrix product runs on the tensor cores (tcgen05, fp16 operands from shared
// memory in the 128-byte swizzle layout, FP32 accumulation in TMEM); activations,
// the loss and Adam run in FP32 kernels. Weights are kept in FP32 (master) with fp16
// copies W [out][in] and W^T [in][out] for the two product shapes.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "gw_internal.h"
#include "tc_common.cuh"

using namespace gwi::tc;

struct gw_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nin = 0, nh = 0, nhidden = 0, nout = 0, nlayers = 0;
  std::vector<int> din, dout;  // per layer
  std::vector<float*> W, b, mW, vW, mb, vb, gW, gb;
  std::vector<__half*> Wh, WTh;
  int64_t step = 0;
  // workspaces for batch <= cap
  int64_t cap = 0;
  std::vector<float*> Z;      // pre-activations [B][dout]
  std::vector<__half*> Hh;    // fp16 activations [B][dout] (layer input of the next)
  std::vector<__half*> HT;    // fp16 transposed activations [dout][B] (incl. input at index 0)
  __half* Xh = nullptr;       // fp16 input [B][nin]
  float* out = nullptr;       // [B][nout]
  float* dZ = nullptr;        // [B][max d]
  __half* dZh = nullptr;      // [B][max d]
  __half* dZT = nullptr;      // [max d][B]
  float* dH = nullptr;        // [B][max d]
  float* loss = nullptr;      // [1]
  int* err = nullptr;
  std::string errmsg;
};

namespace gwi {
namespace mlpk {

// ------------------------------------------------------------------ generic GEMM
// C[M][N] (FP32) = A[M][K] * B[N][K]^T, A, B fp16 row-major. M % 128 == 0, N % 16 == 0,
// K % 64 == 0. One block per (128-row tile, 256-column tile); one pipeline stage.
constexpr int GEMM_THREADS = 128;

__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_gemm_tc(const __half* __restrict__ A, const __half* __restrict__ B, float* __restrict__ C, int M, int N, int K,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;          // 128 x 128 B
  unsigned char* sB = base + 16384;  // <= 256 x 128 B
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_g, no_dealloc;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 256;
  const int Nt = min(256, N - n0);
  if (tid == 0) {
    mbar_init(&bar, 1);
    abort_g = 0;
    no_dealloc = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;
  const uint32_t id = idesc_f16(128, Nt, false, false);
  int kc = 0;
  for (; kc < K / 64; ++kc) {
    for (int e = tid; e < 128 * 8; e += GEMM_THREADS) {
      const int r = e >> 3, c = e & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + kc * 64 + 8 * c);
      *reinterpret_cast<uint4*>(sA + sw128_off(r, 8 * c)) = v;
    }
    for (int e = tid; e < Nt * 8; e += GEMM_THREADS) {
      const int r = e >> 3, c = e & 7;
      const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * K + kc * 64 + 8 * c);
      *reinterpret_cast<uint4*>(sB + sw128_off(r, 8 * c)) = v;
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_f16(tbase, sdesc_sw128(smem_u32(sA) + 32 * ks), sdesc_sw128(smem_u32(sB) + 32 * ks), id,
                (kc > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&bar);
    }
    // a thread whose wait runs out stops the whole block after the barrier (abort_g is written
    // only between the two barriers of an iteration, so every thread reads the same value)
    if (!mbar_wait(&bar, kc & 1, err)) abort_g = 1;
    tc_fence_after();
    __syncthreads();
    if (abort_g) break;
  }
  // MMAs still running into TMEM complete before the block frees it; if they do not, it keeps it
  if (abort_g && tid == 0 && !mbar_wait_drain(&bar, kc & 1)) no_dealloc = 1;
  __syncthreads();
  const bool ok = !abort_g;
  const int row = 32 * warp + lane;
  for (int c = 0; c < Nt; c += 16) {
    float v[16];
    if (ok) {
      tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + c, v);
    } else {
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = 0.f;
    }
    float* o = C + (size_t)(m0 + row) * N + n0 + c;
#pragma unroll
    for (int e = 0; e < 16; ++e) o[e] = v[e];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && !no_dealloc) tmem_dealloc(tbase, 256);
}

// ------------------------------------------------------------------ elementwise
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_g(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}
__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + expf(-z)); }

// Z += bias; H = act(Z) (fp16 row-major and transposed copies; FP32 out for the last layer)
__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ bias, int64_t Bn, int d, int last,
                           __half* __restrict__ H, __half* __restrict__ HT, float* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= Bn * d) return;
  const int64_t r = e / d;
  const int c = (int)(e % d);
  const float z = Z[e] + bias[c];
  Z[e] = z;
  const float h = last ? softplus_f(z) : gelu_f(z);
  if (last) out[e] = h;
  if (H) H[e] = __float2half_rn(h);
  if (HT) HT[(size_t)c * Bn + r] = __float2half_rn(h);
}

// residual R = out A^T - x (FP32), loss = (1/B) sum R^2, dOut = (2/B) R A
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ x, const float* __restrict__ Acpe,
                       int64_t Bn, int nout, int nx, float* __restrict__ dOut, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* r = sm;  // [nx]
  const int64_t b = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    float s = -x[b * nx + i];
    for (int m = 0; m < nout; ++m) s = fmaf(Acpe[(size_t)i * nout + m], out[b * nout + m], s);
    r[i] = s;
  }
  __syncthreads();
  float part = 0.f;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) part += r[i] * r[i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part / (float)Bn);
  for (int m = threadIdx.x; m < nout; m += blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < nx; ++i) s = fmaf(r[i], Acpe[(size_t)i * nout + m], s);
    dOut[b * nout + m] = (2.f / (float)Bn) * s;
  }
}

// dZ = dH * act'(Z); fp16 copies (row-major and transposed) of dZ
__global__ void k_act_back(const float* __restrict__ dH, const float* __restrict__ Z, int64_t Bn, int d, int last,
                           float* __restrict__ dZ, __half* __restrict__ dZh, __half* __restrict__ dZT) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= Bn * d) return;
  const int64_t r = e / d;
  const int c = (int)(e % d);
  const float z = Z[e];
  const float g = dH[e] * (last ? sigmoid_f(z) : gelu_g(z));
  dZ[e] = g;
  dZh[e] = __float2half_rn(g);
  dZT[(size_t)c * Bn + r] = __float2half_rn(g);
}

__global__ void k_colsum(const float* __restrict__ dZ, int64_t Bn, int d, float* __restrict__ gb) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  float s = 0.f;
  for (int64_t r = 0; r < Bn; ++r) s += dZ[r * d + c];
  gb[c] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.f - b1) * gg;
  const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// fp16 copies of W [out][in] and W^T [in][out]
__global__ void k_w_half(const float* __restrict__ W, int dout, int din, __half* __restrict__ Wh,
                         __half* __restrict__ WT) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= dout * din) return;
  const int o = e / din, i = e % din;
  const __half h = __float2half_rn(W[e]);
  Wh[e] = h;
  WT[(size_t)i * dout + o] = h;
}

__global__ void k_x_half(const float* __restrict__ x, int64_t Bn, int nin, __half* __restrict__ Xh,
                         __half* __restrict__ XT) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= Bn * nin) return;
  const int64_t r = e / nin;
  const int c = (int)(e % nin);
  const __half h = __float2half_rn(x[e]);
  Xh[e] = h;
  XT[(size_t)c * Bn + r] = h;
}

gw_status mlp_err(gw_mlp* m, gw_status s, const char* what) {
  if (m) m->errmsg = what;
  return s;
}

gw_status mlp_check(gw_mlp* m, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    m->errmsg = std::string(what) + ": " + cudaGetErrorString(e);
    return GW_ECUDA;
  }
  return GW_OK;
}

gw_status gemm(gw_mlp* m, const __half* A, const __half* B, float* C, int M, int N, int K) {
  const size_t smem = 1024 + 16384 + 256 * 128;
  cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(M / 128, (N + 255) / 256);
  k_gemm_tc<<<grid, GEMM_THREADS, smem, m->stream>>>(A, B, C, M, N, K, m->err);
  return mlp_check(m, "mlp gemm");
}

int maxd(const gw_mlp* m) {
  int d = m->nin;
  for (int l = 0; l < m->nlayers; ++l) d = std::max(d, m->dout[l]);
  return d;
}

gw_status ensure_batch(gw_mlp* m, int64_t Bn) {
  if (Bn <= m->cap) return GW_OK;
  auto fr = [](void* p) {
    if (p) cudaFree(p);
  };
  for (float* p : m->Z) fr(p);
  for (__half* p : m->Hh) fr(p);
  for (__half* p : m->HT) fr(p);
  fr(m->Xh);
  fr(m->out);
  fr(m->dZ);
  fr(m->dZh);
  fr(m->dZT);
  fr(m->dH);
  const int L = m->nlayers, D = maxd(m);
  m->Z.assign(L, nullptr);
  m->Hh.assign(L, nullptr);
  m->HT.assign(L + 1, nullptr);
  bool ok = true;
  for (int l = 0; l < L; ++l) {
    ok &= cudaMalloc((void**)&m->Z[l], sizeof(float) * Bn * m->dout[l]) == cudaSuccess;
    ok &= cudaMalloc((void**)&m->Hh[l], sizeof(__half) * Bn * m->dout[l]) == cudaSuccess;
    ok &= cudaMalloc((void**)&m->HT[l + 1], sizeof(__half) * Bn * m->dout[l]) == cudaSuccess;
  }
  ok &= cudaMalloc((void**)&m->HT[0], sizeof(__half) * Bn * m->nin) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->Xh, sizeof(__half) * Bn * m->nin) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->out, sizeof(float) * Bn * m->nout) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->dZ, sizeof(float) * Bn * D) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->dZh, sizeof(__half) * Bn * D) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->dZT, sizeof(__half) * Bn * D) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->dH, sizeof(float) * Bn * D) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    m->cap = 0;
    return mlp_err(m, GW_ENOMEM, "mlp workspace");
  }
  m->cap = Bn;
  return GW_OK;
}

gw_status forward(gw_mlp* m, int64_t Bn, const float* x) {
  gw_status st;
  const int64_t nx = Bn * m->nin;
  k_x_half<<<(unsigned)((nx + 255) / 256), 256, 0, m->stream>>>(x, Bn, m->nin, m->Xh, m->HT[0]);
  if ((st = mlp_check(m, "mlp input")) != GW_OK) return st;
  const __half* h = m->Xh;
  for (int l = 0; l < m->nlayers; ++l) {
    if ((st = gemm(m, h, m->Wh[l], m->Z[l], (int)Bn, m->dout[l], m->din[l])) != GW_OK) return st;
    const int last = l == m->nlayers - 1;
    const int64_t n = Bn * m->dout[l];
    k_bias_act<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->Z[l], m->b[l], Bn, m->dout[l], last, m->Hh[l],
                                                                   m->HT[l + 1], m->out);
    if ((st = mlp_check(m, "mlp act")) != GW_OK) return st;
    h = m->Hh[l];
  }
  return GW_OK;
}

gw_status backward(gw_mlp* m, int64_t Bn, const float* x, const float* Acpe, int nx) {
  gw_status st;
  cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream);
  k_loss<<<(unsigned)Bn, 128, sizeof(float) * nx, m->stream>>>(m->out, x, Acpe, Bn, m->nout, nx, m->dH, m->loss);
  if ((st = mlp_check(m, "mlp loss")) != GW_OK) return st;
  for (int l = m->nlayers - 1; l >= 0; --l) {
    const int d = m->dout[l], di = m->din[l];
    const int64_t n = Bn * d;
    k_act_back<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->dH, m->Z[l], Bn, d, l == m->nlayers - 1, m->dZ,
                                                                   m->dZh, m->dZT);
    if ((st = mlp_check(m, "mlp act back")) != GW_OK) return st;
    // dW = dZ^T H_in : [d][di], K = batch
    if ((st = gemm(m, m->dZT, m->HT[l], m->gW[l], d, di, (int)Bn)) != GW_OK) return st;
    k_colsum<<<(d + 127) / 128, 128, 0, m->stream>>>(m->dZ, Bn, d, m->gb[l]);
    if ((st = mlp_check(m, "mlp colsum")) != GW_OK) return st;
    // dH_in = dZ W : [B][di], K = d
    if (l > 0 && (st = gemm(m, m->dZh, m->WTh[l], m->dH, (int)Bn, di, d)) != GW_OK) return st;
  }
  return GW_OK;
}

gw_status refresh_half(gw_mlp* m) {
  for (int l = 0; l < m->nlayers; ++l) {
    const int n = m->dout[l] * m->din[l];
    k_w_half<<<(n + 255) / 256, 256, 0, m->stream>>>(m->W[l], m->dout[l], m->din[l], m->Wh[l], m->WTh[l]);
    gw_status st = mlp_check(m, "mlp weights fp16");
    if (st != GW_OK) return st;
  }
  return GW_OK;
}

bool shapes_ok(const gw_mlp* m, int64_t Bn) {
  if (Bn <= 0 || Bn % 128) return false;
  for (int l = 0; l < m->nlayers; ++l)
    if (m->din[l] % 64 || m->dout[l] % 128) return false;
  return true;
}

}  // namespace mlpk
}  // namespace gwi

using namespace gwi::mlpk;

extern "C" {

gw_status gw_mlp_create(gw_mlp** out, int nin, int nh, int nhidden, int nout, uint64_t seed, int device,
                        void* stream) {
  if (!out || nin < 64 || nh < 128 || nhidden < 1 || nout < 128 || nin % 64 || nh % 128 || nout % 128)
    return GW_EINVAL;
  gw_mlp* m = new gw_mlp();
  if (cudaSetDevice(device) != cudaSuccess) {
    delete m;
    return GW_ECUDA;
  }
  m->device = device;
  m->stream = (cudaStream_t)stream;
  m->nin = nin;
  m->nh = nh;
  m->nhidden = nhidden;
  m->nout = nout;
  m->nlayers = nhidden + 1;
  for (int l = 0; l < m->nlayers; ++l) {
    m->din.push_back(l == 0 ? nin : nh);
    m->dout.push_back(l == m->nlayers - 1 ? nout : nh);
  }
  // deterministic init: splitmix64-driven Box-Muller normals (He init, small last layer)
  uint64_t s = seed ? seed : 0x9E3779B97F4A7C15ull;
  auto next = [&s]() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto normal = [&]() {
    const double u1 = ((next() >> 11) + 1.0) * 0x1p-53, u2 = (next() >> 11) * 0x1p-53;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  bool ok = true;
  for (int l = 0; l < m->nlayers; ++l) {
    const int din = m->din[l], dout = m->dout[l];
    const double sc = l < m->nlayers - 1 ? std::sqrt(2.0 / din) : 0.1 / std::sqrt((double)din);
    std::vector<float> w((size_t)dout * din);
    for (auto& x : w) x = (float)(normal() * sc);
    float *W, *b, *mW, *vW, *mb, *vb, *gW, *gb;
    __half *Wh, *WTh;
    ok &= cudaMalloc((void**)&W, sizeof(float) * w.size()) == cudaSuccess;
    ok &= cudaMalloc((void**)&mW, sizeof(float) * w.size()) == cudaSuccess;
    ok &= cudaMalloc((void**)&vW, sizeof(float) * w.size()) == cudaSuccess;
    ok &= cudaMalloc((void**)&gW, sizeof(float) * w.size()) == cudaSuccess;
    ok &= cudaMalloc((void**)&b, sizeof(float) * dout) == cudaSuccess;
    ok &= cudaMalloc((void**)&mb, sizeof(float) * dout) == cudaSuccess;
    ok &= cudaMalloc((void**)&vb, sizeof(float) * dout) == cudaSuccess;
    ok &= cudaMalloc((void**)&gb, sizeof(float) * dout) == cudaSuccess;
    ok &= cudaMalloc((void**)&Wh, sizeof(__half) * w.size()) == cudaSuccess;
    ok &= cudaMalloc((void**)&WTh, sizeof(__half) * w.size()) == cudaSuccess;
    if (!ok) break;
    cudaMemcpy(W, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
    cudaMemset(mW, 0, sizeof(float) * w.size());
    cudaMemset(vW, 0, sizeof(float) * w.size());
    cudaMemset(b, 0, sizeof(float) * dout);
    cudaMemset(mb, 0, sizeof(float) * dout);
    cudaMemset(vb, 0, sizeof(float) * dout);
    m->W.push_back(W);
    m->b.push_back(b);
    m->mW.push_back(mW);
    m->vW.push_back(vW);
    m->mb.push_back(mb);
    m->vb.push_back(vb);
    m->gW.push_back(gW);
    m->gb.push_back(gb);
    m->Wh.push_back(Wh);
    m->WTh.push_back(WTh);
  }
  ok &= cudaMalloc((void**)&m->loss, sizeof(float)) == cudaSuccess;
  ok &= cudaMalloc((void**)&m->err, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gw_mlp_destroy(m);
    return GW_ENOMEM;
  }
  cudaMemset(m->err, 0, sizeof(int));
  if (refresh_half(m) != GW_OK || cudaDeviceSynchronize() != cudaSuccess) {
    gw_mlp_destroy(m);
    return GW_ECUDA;
  }
  *out = m;
  return GW_OK;
}

gw_status gw_mlp_destroy(gw_mlp* m) {
  if (!m) return GW_EINVAL;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  auto fr = [](void* p) {
    if (p) cudaFree(p);
  };
  for (auto* v : {&m->W, &m->b, &m->mW, &m->vW, &m->mb, &m->vb, &m->gW, &m->gb, &m->Z})
    for (float* p : *v) fr(p);
  for (auto* v : {&m->Wh, &m->WTh, &m->Hh, &m->HT})
    for (__half* p : *v) fr(p);
  fr(m->Xh);
  fr(m->out);
  fr(m->dZ);
  fr(m->dZh);
  fr(m->dZT);
  fr(m->dH);
  fr(m->loss);
  fr(m->err);
  delete m;
  return GW_OK;
}

const char* gw_mlp_last_error(gw_mlp* m) { return m ? m->errmsg.c_str() : "null handle"; }

gw_status gw_mlp_forward(gw_mlp* m, int64_t batch, const float* x, float* out) {
  if (!m || !x || !out || !shapes_ok(m, batch)) return GW_EINVAL;
  gw_status st;
  if ((st = ensure_batch(m, batch)) != GW_OK) return st;
  if ((st = forward(m, batch, x)) != GW_OK) return st;
  if (cudaMemcpyAsync(out, m->out, sizeof(float) * batch * m->nout, cudaMemcpyDeviceToDevice, m->stream) !=
      cudaSuccess)
    return mlp_err(m, GW_ECUDA, "mlp output copy");
  return GW_OK;
}

gw_status gw_mlp_loss_grad(gw_mlp* m, int64_t batch, const float* x, int nx, const float* Acpe, float* loss,
                           float* grads) {
  if (!m || !x || !Acpe || !shapes_ok(m, batch) || nx <= 0) return GW_EINVAL;
  gw_status st;
  if ((st = ensure_batch(m, batch)) != GW_OK) return st;
  if ((st = forward(m, batch, x)) != GW_OK) return st;
  if ((st = backward(m, batch, x, Acpe, nx)) != GW_OK) return st;
  if (loss) cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, m->stream);
  if (grads) {
    size_t off = 0;
    for (int l = 0; l < m->nlayers; ++l) {
      const size_t nw = (size_t)m->dout[l] * m->din[l];
      cudaMemcpyAsync(grads + off, m->gW[l], sizeof(float) * nw, cudaMemcpyDeviceToDevice, m->stream);
      off += nw;
      cudaMemcpyAsync(grads + off, m->gb[l], sizeof(float) * m->dout[l], cudaMemcpyDeviceToDevice, m->stream);
      off += m->dout[l];
    }
  }
  return mlp_check(m, "mlp loss_grad");
}

gw_status gw_mlp_train_step(gw_mlp* m, int64_t batch, const float* x, int nx, const float* Acpe, float lr,
                            float* loss) {
  gw_status st;
  if ((st = gw_mlp_loss_grad(m, batch, x, nx, Acpe, loss, nullptr)) != GW_OK) return st;
  const float b1 = 0.9f, b2 = 0.999f;
  ++m->step;
  const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
  for (int l = 0; l < m->nlayers; ++l) {
    const int64_t nw = (int64_t)m->dout[l] * m->din[l];
    k_adam<<<(unsigned)((nw + 255) / 256), 256, 0, m->stream>>>(m->W[l], m->gW[l], m->mW[l], m->vW[l], nw, lr, b1, b2,
                                                                1e-8f, c1, c2);
    k_adam<<<(m->dout[l] + 255) / 256, 256, 0, m->stream>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], m->dout[l], lr, b1,
                                                            b2, 1e-8f, c1, c2);
  }
  if ((st = mlp_check(m, "mlp adam")) != GW_OK) return st;
  return refresh_half(m);
}

gw_status gw_mlp_sync(gw_mlp* m) {
  if (!m) return GW_EINVAL;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_err(m, GW_ECUDA, "gw_mlp_sync: stream");
  int h = 0;
  if (cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_err(m, GW_ECUDA, "gw_mlp_sync: reading the device error word");
  if (h != 0) {
    cudaMemset(m->err, 0, sizeof(int));
    return mlp_err(m, GW_ETIMEOUT,
                   "gw_mlp_sync: a bounded wait in the tensor-core GEMM ran out; results since the last sync are undefined");
  }
  return GW_OK;
}

gw_status gw_mlp_get_params(gw_mlp* m, float* params) {
  if (!m || !params) return GW_EINVAL;
  size_t off = 0;
  gw_status st = gw_mlp_sync(m);
  if (st != GW_OK) return st;
  for (int l = 0; l < m->nlayers; ++l) {
    const size_t nw = (size_t)m->dout[l] * m->din[l];
    cudaMemcpy(params + off, m->W[l], sizeof(float) * nw, cudaMemcpyDeviceToHost);
    off += nw;
    cudaMemcpy(params + off, m->b[l], sizeof(float) * m->dout[l], cudaMemcpyDeviceToHost);
    off += m->dout[l];
  }
  return cudaGetLastError() == cudaSuccess ? GW_OK : GW_ECUDA;
}

gw_status gw_mlp_set_params(gw_mlp* m, const float* params) {
  if (!m || !params) return GW_EINVAL;
  size_t off = 0;
  cudaStreamSynchronize(m->stream);
  for (int l = 0; l < m->nlayers; ++l) {
    const size_t nw = (size_t)m->dout[l] * m->din[l];
    cudaMemcpy(m->W[l], params + off, sizeof(float) * nw, cudaMemcpyHostToDevice);
    off += nw;
    cudaMemcpy(m->b[l], params + off, sizeof(float) * m->dout[l], cudaMemcpyHostToDevice);
    off += m->dout[l];
  }
  if (cudaGetLastError() != cudaSuccess) return GW_ECUDA;
  return refresh_half(m);
}

int64_t gw_mlp_num_params(gw_mlp* m) {
  if (!m) return -1;
  int64_t n = 0;
  for (int l = 0; l < m->nlayers; ++l) n += (int64_t)m->dout[l] * m->din[l] + m->dout[l];
  return n;
}

}  // extern "C"
