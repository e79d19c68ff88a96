// Tensor-core (tcgen05, TMEM accumulators) split-precision forms of the two
// product-basis contractions of the GW cycle.
//
// Operands are split into two fp16 slices, x = 2^-s (hi + lo), hi = fp16(2^s x),
// lo = fp16(2^s x - hi) (22 significant bits), and each real product is formed as
// hi*hi + hi*lo + lo*hi on the tensor cores with FP32 accumulation in TMEM.
// Complex arithmetic is written as real GEMMs on stacked real/imaginary parts.
//
// polarization, Eq. (irpol), one q, all tau:
//   P_II'(tau) = pref sum_{k,p} w_p(tau) A_k[I,p] conj(A_k[I',p]),  w_p = -G_b(k|tau) G_a(k-q|beta-tau)
//   Re P = X Y^T, Im P = X' Y^T with rows X_I = [w Re A_I | w Im A_I], Y_I' = [Re A_I' | Im A_I'],
//   X'_I = [w Im A_I | -w Re A_I] (same shared-memory tile, other K halves, negated).
//   Work unit = (K segment, 128 x 128 output tile with ti <= tj, pair of tau); FP32 partial
//   tiles are summed over K segments in FP64 by a second kernel, which also mirrors the
//   Hermitian lower triangle.
//
// self-energy, Eq. (sigc), one q:
//   d_p(tau) = a_p^H W~(tau) a_p = Re a_p^T Wr Re a_p + Im a_p^T Wr Im a_p + 2 Im a_p^T Wi Re a_p
//   (Wr = Re W~ symmetric, Wi = Im W~ antisymmetric), computed as
//   Y1 = Ar Wr, Y2 = Ai Wr + Ar (2 Wi)^T-rows on the tensor cores (rows = pairs p),
//   d_p = <Ar_p, Y1_p> + <Ai_p, Y2_p> in the epilogue (FP32 products, compensated sums);
//   Sigc_n(k|tau) += pref sum_a G_a(k-q|tau) d_(a,n)(tau) in a final kernel.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gw_internal.h"
#include "tc_common.cuh"

namespace gwi {

namespace {

using namespace tc;

constexpr float kScaleA = 256.0f;   // 2^8 on matrix elements (|M| < ~3)
constexpr float kScaleW = 1.0f;     // W~ entries are O(v) <= 4 pi / 0.05
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

// Bounded mbarrier wait shared by all roles of a block: gives up after
// kWaitCycles, or at once if another thread of the block has given up.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      if (err) atomicExch(err, kErrTimeout);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void split2(float x, __half& h, __half& l) {
  h = __float2half_rn(x);
  l = __float2half_rn(x - __half2float(h));
}

// 8 consecutive fp16 values as one 16-byte vector
struct alignas(16) h8 {
  __half v[8];
};

// --------------------------------------------------------------------------- polarization
constexpr int kPolChunksPerSeg = 32;
constexpr int PT_THREADS = 288;  // warps 0-7 produce, warp 8 issues MMAs; warps 0-3 run the epilogue
constexpr int P_STAGE_BYTES = 6 * 16384;  // Yh Yl Xh0 Xl0 Xh1 Xl1, 128 rows x 128 B each

struct PolSmem {
  uint64_t full[2], empty[2], done;
  uint32_t tslot;
  int abort_flag;
};

// Pair weights of Eq. (irpol): wt[k][tau][p] = Q_ab(tau) = -G_b(k|tau) G_a(k-q|beta - tau),
// p = a nb + b, rows padded to npw (multiple of 32) with zeros.
__global__ void k_pol_weights(const double* __restrict__ G, const int* __restrict__ kmq, int nk, int nb, int ntau,
                              int npw, float* __restrict__ wt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nk * ntau * npw) return;
  const int p = (int)(e % npw), it = (int)((e / npw) % ntau), k = (int)(e / ((int64_t)npw * ntau));
  float w = 0.f;
  if (p < nb * nb) {
    const int a = p / nb, b = p - a * nb;
    w = (float)(-G[((size_t)k * nb + b) * ntau + it] * G[((size_t)kmq[k] * nb + a) * ntau + (ntau - 1 - it)]);
  }
  wt[e] = w;
}

__global__ void __launch_bounds__(PT_THREADS, 1)
    k_pol_tc(const double2* __restrict__ Mq, const float* __restrict__ wt, int nk, int ni, int nb, int ntau,
             int npw, int ntiles, const int2* __restrict__ tiles, int nseg, float* __restrict__ part,
             int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  PolSmem& S = *reinterpret_cast<PolSmem*>(base + 2 * P_STAGE_BYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntp = ntau / 2;
  const int u = blockIdx.x;
  const int tp = u % ntp, tile = (u / ntp) % ntiles, seg = u / (ntp * ntiles);
  const int ti = tiles[tile].x, tj = tiles[tile].y;
  const int np = nb * nb, cpk = (np + 31) / 32, total = nk * cpk;
  const int L = (total + nseg - 1) / nseg;
  const int g0 = seg * L, g1 = min(total, g0 + L);
  const int nchunk = max(0, g1 - g0);

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.full[s], 256);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.done, 1);
    S.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 8) tmem_alloc(&S.tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tslot;

  if (warp < 8) {
    // ------------------------------------------------------------ producers
    for (int i = 0; i < nchunk; ++i) {
      const int s = i & 1;
      if (i >= 2 && !wait_bar(&S.empty[s], ((i >> 1) + 1) & 1, &S.abort_flag, err)) break;
      unsigned char* st = base + s * P_STAGE_BYTES;
      const int g = g0 + i, k = g / cpk, p0 = (g % cpk) * 32;
      const double2* Mk = Mq + (size_t)k * ni * np;
      for (int item = tid; item < 512; item += 256) {
        const int r = item >> 2, gq = item & 3;
        const int pb = p0 + 8 * gq;
        // Y rows (block tj)
        float yr[8], yi[8];
        {
          const int I = tj * 128 + r;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            double2 v = make_double2(0.0, 0.0);
            if (I < ni && pb + e < np) v = __ldg(&Mk[(size_t)I * np + pb + e]);
            yr[e] = (float)v.x * kScaleA;
            yi[e] = (float)v.y * kScaleA;
          }
        }
        float xr[8], xi[8];
        if (ti == tj) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            xr[e] = yr[e];
            xi[e] = yi[e];
          }
        } else {
          const int I = ti * 128 + r;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            double2 v = make_double2(0.0, 0.0);
            if (I < ni && pb + e < np) v = __ldg(&Mk[(size_t)I * np + pb + e]);
            xr[e] = (float)v.x * kScaleA;
            xi[e] = (float)v.y * kScaleA;
          }
        }
        const uint32_t oRe = sw128_off(r, 8 * gq), oIm = sw128_off(r, 32 + 8 * gq);
        h8 hr, lr, hi_, li;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          split2(yr[e], hr.v[e], lr.v[e]);
          split2(yi[e], hi_.v[e], li.v[e]);
        }
        *reinterpret_cast<h8*>(st + 0 * 16384 + oRe) = hr;
        *reinterpret_cast<h8*>(st + 0 * 16384 + oIm) = hi_;
        *reinterpret_cast<h8*>(st + 1 * 16384 + oRe) = lr;
        *reinterpret_cast<h8*>(st + 1 * 16384 + oIm) = li;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const float4* wp = reinterpret_cast<const float4*>(wt + ((size_t)k * ntau + 2 * tp + j) * npw + pb);
          const float4 w0 = __ldg(wp), w1 = __ldg(wp + 1);
          const float wv8[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float wv = wv8[e];
            split2(wv * xr[e], hr.v[e], lr.v[e]);
            split2(wv * xi[e], hi_.v[e], li.v[e]);
          }
          *reinterpret_cast<h8*>(st + (2 + 2 * j) * 16384 + oRe) = hr;
          *reinterpret_cast<h8*>(st + (2 + 2 * j) * 16384 + oIm) = hi_;
          *reinterpret_cast<h8*>(st + (3 + 2 * j) * 16384 + oRe) = lr;
          *reinterpret_cast<h8*>(st + (3 + 2 * j) * 16384 + oIm) = li;
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&S.full[s]);
      if (S.abort_flag) break;
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t id = idesc_f16(128, 128, false, false), idn = idesc_f16(128, 128, false, true);
    for (int i = 0; i < nchunk; ++i) {
      const int s = i & 1;
      if (!wait_bar(&S.full[s], (i >> 1) & 1, &S.abort_flag, err)) break;
      tc_fence_after();
      const uint32_t st = smem_u32(base + s * P_STAGE_BYTES);
      const uint32_t yh = st, yl = st + 16384;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t xh = st + (2 + 2 * j) * 16384, xl = st + (3 + 2 * j) * 16384;
        const uint32_t dre = tbase + j * 256, dim = tbase + j * 256 + 128;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
          const uint32_t bo = 32 * ks;
          mma_f16(dre, sdesc_sw128(xh + bo), sdesc_sw128(yh + bo), id, acc);
          mma_f16(dre, sdesc_sw128(xh + bo), sdesc_sw128(yl + bo), id, 1);
          mma_f16(dre, sdesc_sw128(xl + bo), sdesc_sw128(yh + bo), id, 1);
          const uint32_t ao = 32 * ((ks + 2) & 3);
          const uint32_t idx = ks < 2 ? id : idn;
          mma_f16(dim, sdesc_sw128(xh + ao), sdesc_sw128(yh + bo), idx, acc);
          mma_f16(dim, sdesc_sw128(xh + ao), sdesc_sw128(yl + bo), idx, 1);
          mma_f16(dim, sdesc_sw128(xl + ao), sdesc_sw128(yh + bo), idx, 1);
        }
      }
      mma_commit(&S.empty[s]);
    }
    mma_commit(&S.done);
  }

  // ------------------------------------------------------------ epilogue: FP32 partial tiles
  if (warp < 4) {
    const bool ok = nchunk > 0 && wait_bar(&S.done, 0, &S.abort_flag, err);
    tc_fence_after();
    const int row = 32 * warp + lane;
    float* out = part + (size_t)u * 4 * 128 * 128;
    for (int acc = 0; acc < 4; ++acc) {
      for (int c = 0; c < 128; c += 16) {
        float v[16];
        if (ok) {
          tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + acc * 128 + c, v);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0.f;
        }
        float4* o = reinterpret_cast<float4*>(out + ((size_t)acc * 128 + row) * 128 + c);
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) tmem_dealloc(tbase, 512);
}

// Sum the FP32 partial tiles over K segments in FP64 and write the Hermitian P.
__global__ void k_pol_reduce(const float* __restrict__ part, int ni, int ntau, int nt128, const int* __restrict__ tile_of,
                             int ntiles, int nseg, double scale, double2* __restrict__ P) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)ntau * ni * ni;
  if (e >= tot) return;
  const int it = (int)(e / ((int64_t)ni * ni));
  const int I = (int)((e / ni) % ni), J = (int)(e % ni);
  // upper triangle from the tiles; the lower triangle mirrors it (exactly Hermitian)
  int a = I, b = J;
  bool conj = false;
  if (I > J) {
    a = J;
    b = I;
    conj = true;
  }
  const int tile = tile_of[(a / 128) * nt128 + (b / 128)];
  const int ntp = ntau / 2, tp = it / 2, j = it & 1;
  double re = 0.0, im = 0.0;
  for (int s = 0; s < nseg; ++s) {
    const int u = (s * ntiles + tile) * ntp + tp;
    const float* p = part + (size_t)u * 4 * 128 * 128;
    re += (double)p[((size_t)(2 * j) * 128 + (a & 127)) * 128 + (b & 127)];
    im += (double)p[((size_t)(2 * j + 1) * 128 + (a & 127)) * 128 + (b & 127)];
  }
  // Im P_II = 0 exactly for a Hermitian P (the tensor-core sum leaves O(2^-22) residue)
  P[e] = make_double2(re * scale, I == J ? 0.0 : (conj ? -im : im) * scale);
}

// --------------------------------------------------------------------------- self-energy
// Split M[q] into the pair-major fp16 slices XT[slice][k][p][I] (slices: Re hi, Re lo,
// Im hi, Im lo; rows p >= nb^2 zero), via a 32 x 32 shared-memory transpose.
__global__ void k_split_x(const double2* __restrict__ Mq, int nk, int ni, int np, int npp, __half* __restrict__ XT) {
  __shared__ double2 tileS[32][33];
  const int k = blockIdx.z;
  const int p0 = blockIdx.x * 32, I0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int I = I0 + r, p = p0 + tx;
    tileS[r][tx] = (I < ni && p < np) ? Mq[((size_t)k * ni + I) * np + p] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const size_t slice = (size_t)nk * npp * ni;
  for (int r = ty; r < 32; r += 8) {
    const int p = p0 + r, I = I0 + tx;
    if (p >= npp || I >= ni) continue;
    const double2 v = tileS[tx][r];
    __half rh, rl, ih, il;
    split2((float)v.x * kScaleA, rh, rl);
    split2((float)v.y * kScaleA, ih, il);
    const size_t o = ((size_t)k * npp + p) * ni + I;
    XT[o] = rh;
    XT[slice + o] = rl;
    XT[2 * slice + o] = ih;
    XT[3 * slice + o] = il;
  }
}

// Split W~(tau) into BW[slice][tau][I][I'] (slices: Re hi, Re lo, 2 Im hi, 2 Im lo).
__global__ void k_split_w(const double2* __restrict__ W, int ntau, int ni, __half* __restrict__ BW) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)ntau * ni * ni;
  if (e >= n) return;
  const double2 w = W[e];
  __half a, b, c, d;
  split2((float)w.x * kScaleW, a, b);
  split2((float)(2.0 * w.y) * kScaleW, c, d);
  BW[e] = a;
  BW[n + e] = b;
  BW[2 * n + e] = c;
  BW[3 * n + e] = d;
}

constexpr int ST_THREADS = 416;  // warps 0-3 epilogue, 4-11 produce, 12 issues MMAs
constexpr int S_ATILE = 128 * 64;  // 128 rows x 64 B (32 fp16)

struct SigSmem {
  uint64_t full[2], empty[2], tfull, tempty;
  uint32_t tslot;
  int abort_flag;
};

__global__ void __launch_bounds__(ST_THREADS, 1)
    k_sig_tc(const __half* __restrict__ XT, const __half* __restrict__ BW, int nk, int ni, int npp, int ntau,
             double* __restrict__ D, int np, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int BT = ni * 64;                 // one B slice tile: ni rows x 64 B
  const int stage_bytes = 4 * S_ATILE + 4 * BT;
  SigSmem& S = *reinterpret_cast<SigSmem*>(base + 2 * stage_bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pblk = blockIdx.x, k = blockIdx.y;
  const int nkc = ni / 32;
  const int nchunk = ntau * nkc;
  const size_t xslice = (size_t)nk * npp * ni;
  const size_t wslice = (size_t)ntau * ni * ni;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.full[s], 256);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.tfull, 1);
    mbar_init(&S.tempty, 128);
    S.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 12) tmem_alloc(&S.tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tslot;

  if (warp >= 4 && warp < 12) {
    // ------------------------------------------------------------ producers
    const int pt = tid - 128;
    for (int i = 0; i < nchunk; ++i) {
      const int s = i & 1;
      if (i >= 2 && !wait_bar(&S.empty[s], ((i >> 1) + 1) & 1, &S.abort_flag, err)) break;
      unsigned char* st = base + s * stage_bytes;
      const int it = i / nkc, kc = i % nkc;
      // A tiles: 4 slices x 128 rows x 4 chunks of 16 B
      for (int e = pt; e < 4 * 128 * 4; e += 256) {
        const int sl = e >> 9, r = (e >> 2) & 127, c = e & 3;
        const int p = pblk * 128 + r;
        const __half* src = XT + sl * xslice + ((size_t)k * npp + p) * ni + kc * 32 + 8 * c;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
        *reinterpret_cast<uint4*>(st + sl * S_ATILE + sw64_off(r, 8 * c)) = v;
      }
      // B tiles: 4 slices x ni rows x 4 chunks
      for (int e = pt; e < 4 * ni * 4; e += 256) {
        const int sl = e / (ni * 4), rem = e % (ni * 4), r = rem >> 2, c = rem & 3;
        const __half* src = BW + sl * wslice + ((size_t)it * ni + r) * ni + kc * 32 + 8 * c;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
        *reinterpret_cast<uint4*>(st + 4 * S_ATILE + sl * BT + sw64_off(r, 8 * c)) = v;
      }
      fence_proxy_async_smem();
      mbar_arrive(&S.full[s]);
      if (S.abort_flag) break;
    }
  } else if (warp == 12 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t id = idesc_f16(128, ni, false, false);
    const uint32_t y1 = tbase, y2 = tbase + ni;
    for (int i = 0; i < nchunk; ++i) {
      const int s = i & 1, it = i / nkc, kc = i % nkc;
      if (kc == 0 && it > 0 && !wait_bar(&S.tempty, (it - 1) & 1, &S.abort_flag, err)) break;
      if (!wait_bar(&S.full[s], (i >> 1) & 1, &S.abort_flag, err)) break;
      tc_fence_after();
      const uint32_t st = smem_u32(base + s * stage_bytes);
      const uint32_t arh = st, arl = st + S_ATILE, aih = st + 2 * S_ATILE, ail = st + 3 * S_ATILE;
      const uint32_t bb = st + 4 * S_ATILE;
      const uint32_t wrh = bb, wrl = bb + BT, wih = bb + 2 * BT, wil = bb + 3 * BT;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t o = 32 * ks;
        const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
        mma_f16(y1, sdesc_sw64(arh + o), sdesc_sw64(wrh + o), id, acc);
        mma_f16(y1, sdesc_sw64(arh + o), sdesc_sw64(wrl + o), id, 1);
        mma_f16(y1, sdesc_sw64(arl + o), sdesc_sw64(wrh + o), id, 1);
        mma_f16(y2, sdesc_sw64(aih + o), sdesc_sw64(wrh + o), id, acc);
        mma_f16(y2, sdesc_sw64(aih + o), sdesc_sw64(wrl + o), id, 1);
        mma_f16(y2, sdesc_sw64(ail + o), sdesc_sw64(wrh + o), id, 1);
        mma_f16(y2, sdesc_sw64(arh + o), sdesc_sw64(wih + o), id, 1);
        mma_f16(y2, sdesc_sw64(arh + o), sdesc_sw64(wil + o), id, 1);
        mma_f16(y2, sdesc_sw64(arl + o), sdesc_sw64(wih + o), id, 1);
      }
      mma_commit(&S.empty[s]);
      if (kc == nkc - 1) mma_commit(&S.tfull);
    }
  } else if (warp < 4) {
    // ------------------------------------------------------------ epilogue: d_p(tau)
    const int row = 32 * warp + lane;
    const int p = pblk * 128 + row;
    const __half* xr_h = XT + ((size_t)k * npp + p) * ni;
    const __half* xr_l = xr_h + xslice;
    const __half* xi_h = xr_h + 2 * xslice;
    const __half* xi_l = xr_h + 3 * xslice;
    const double dscale = 1.0 / ((double)kScaleA * kScaleA * kScaleW);
    for (int it = 0; it < ntau; ++it) {
      const bool ok = wait_bar(&S.tfull, it & 1, &S.abort_flag, err);
      tc_fence_after();
      float dhi = 0.f, dlo = 0.f;  // compensated (two-sum) accumulator
      if (ok) {
        for (int n0 = 0; n0 < ni; n0 += 16) {
          float v1[16], v2[16];
          tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + n0, v1);
          tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + ni + n0, v2);
          const h8* a0 = reinterpret_cast<const h8*>(xr_h + n0);
          const h8* a1 = reinterpret_cast<const h8*>(xr_l + n0);
          const h8* b0 = reinterpret_cast<const h8*>(xi_h + n0);
          const h8* b1 = reinterpret_cast<const h8*>(xi_l + n0);
          float part = 0.f;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const h8 rh = a0[h], rl = a1[h], ih = b0[h], il = b1[h];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float xr = __half2float(rh.v[e]) + __half2float(rl.v[e]);
              const float xi = __half2float(ih.v[e]) + __half2float(il.v[e]);
              part = fmaf(xr, v1[8 * h + e], part);
              part = fmaf(xi, v2[8 * h + e], part);
            }
          }
          const float s = dhi + part;
          const float bb = s - dhi;
          dlo += (dhi - (s - bb)) + (part - bb);
          dhi = s;
        }
      }
      tc_fence_before();
      mbar_arrive(&S.tempty);
      if (p < np) D[((size_t)k * np + p) * ntau + it] = ((double)dhi + (double)dlo) * dscale;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 12) tmem_dealloc(tbase, 512);
}

// Sigc_n(k|tau) += pref sum_a G_a(k-q|tau) d_(a,n)(tau); deterministic (no atomics).
__global__ void k_sig_reduce(const double* __restrict__ D, const double* __restrict__ G, const int* __restrict__ kmq,
                             int nk, int nb, int ntau, double pref, double* __restrict__ S) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nk * nb * ntau) return;
  const int it = (int)(e % ntau), n = (int)((e / ntau) % nb), k = (int)(e / ((int64_t)ntau * nb));
  const int km = kmq[k];
  const int np = nb * nb;
  double s = 0.0;
  for (int a = 0; a < nb; ++a) s += G[((size_t)km * nb + a) * ntau + it] * D[((size_t)k * np + a * nb + n) * ntau + it];
  S[e] += pref * s;
}

// ------------------------------------------------------------------ workspace helpers
gw_status ensure(gw_ctx* c, void** p, size_t* have, size_t need, const char* what) {
  if (need <= *have) return GW_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, GW_ENOMEM, std::string("tensor-core workspace: ") + what);
  }
  *have = need;
  return GW_OK;
}

int num_sms(gw_ctx* c) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, c->device);
  return n > 0 ? n : 148;
}

}  // namespace

gw_status launch_pol_mixed(gw_ctx* c, int iq, const double* G, int prec, double* P) {
  if (prec != GW_FP16X2) return set_err(c, GW_EUNSUPPORTED, "polarization: only GW_FP16X2 is built on tensor cores");
  if (c->ntau & 1) return set_err(c, GW_EUNSUPPORTED, "polarization: ntau must be even");
  const int nt128 = (c->ni + 127) / 128;
  std::vector<int2> tiles;
  std::vector<int> tile_of(nt128 * nt128, -1);
  for (int a = 0; a < nt128; ++a)
    for (int b = a; b < nt128; ++b) {
      tile_of[a * nt128 + b] = (int)tiles.size();
      tiles.push_back(make_int2(a, b));
    }
  const int ntiles = (int)tiles.size(), ntp = c->ntau / 2;
  const int np = c->nb * c->nb, total = c->nk * ((np + 31) / 32), npw = (np + 31) / 32 * 32;
  // K segments. The tensor cores accumulate in FP32 with an error that grows with the
  // number of MMAs chained into one accumulator (measured ~2^-24 per MMA, biased), so
  // each work unit covers at most kPolChunksPerSeg chunks of 32 pairs (128 MMA steps);
  // the FP32 partial tiles are summed in FP64 afterwards.
  const int sms = num_sms(c);
  const int base_units = ntiles * ntp;
  int nseg = std::max(1, (total + kPolChunksPerSeg - 1) / kPolChunksPerSeg);
  while (base_units * nseg < 2 * sms && (total + nseg) / (nseg + 1) >= 4) ++nseg;
  const int nunits = base_units * nseg;
  const size_t part_bytes = (size_t)nunits * 4 * 128 * 128 * sizeof(float);
  const size_t wt_bytes = (size_t)c->nk * c->ntau * npw * sizeof(float);
  gw_status st;
  if ((st = ensure(c, &c->mw.wslices, &c->mw.wslices_bytes, part_bytes + wt_bytes, "P partials")) != GW_OK) return st;
  float* d_part = (float*)c->mw.wslices;
  float* d_wt = d_part + part_bytes / sizeof(float);
  const size_t meta_bytes = sizeof(int2) * tiles.size() + sizeof(int) * tile_of.size() + sizeof(int);
  if ((st = ensure(c, (void**)&c->mw.dacc, &c->mw.dacc_bytes, meta_bytes + 256, "P tiles")) != GW_OK) return st;
  int2* d_tiles = reinterpret_cast<int2*>(c->mw.dacc);
  int* d_tile_of = reinterpret_cast<int*>(d_tiles + tiles.size());
  int* d_err = d_tile_of + tile_of.size();
  cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(d_tile_of, tile_of.data(), sizeof(int) * tile_of.size(), cudaMemcpyHostToDevice, c->stream);
  cudaMemsetAsync(d_err, 0, sizeof(int), c->stream);
  const size_t smem = 1024 + 2 * P_STAGE_BYTES + sizeof(PolSmem);
  cudaFuncSetAttribute(k_pol_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const double2* Mq = (const double2*)c->d_M + (size_t)iq * c->nk * c->ni * np;
  const int64_t nwt = (int64_t)c->nk * c->ntau * npw;
  k_pol_weights<<<(unsigned)((nwt + 255) / 256), 256, 0, c->stream>>>(G, c->d_kmq + (size_t)iq * c->nk, c->nk, c->nb,
                                                                      c->ntau, npw, d_wt);
  if ((st = check_launch(c, "pol_weights")) != GW_OK) return st;
  k_pol_tc<<<nunits, PT_THREADS, smem, c->stream>>>(Mq, d_wt, c->nk, c->ni, c->nb, c->ntau, npw, ntiles, d_tiles, nseg,
                                                    d_part, d_err);
  if ((st = check_launch(c, "pol_tc")) != GW_OK) return st;
  const int64_t tot = (int64_t)c->ntau * c->ni * c->ni;
  const double scale = 1.0 / ((double)kScaleA * kScaleA * c->omega * c->nk);
  k_pol_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(d_part, c->ni, c->ntau, nt128,
                                                                     d_tile_of, ntiles, nseg, scale, (double2*)P);
  return check_launch(c, "pol_reduce");
}

gw_status launch_sigma_mixed(gw_ctx* c, int iq, const double* G, const double* W, int prec, double* S) {
  if (prec != GW_FP16X2) return set_err(c, GW_EUNSUPPORTED, "self-energy: only GW_FP16X2 is built on tensor cores");
  if (c->ni > 256) return set_err(c, GW_EUNSUPPORTED, "tensor-core self-energy: ni <= 256");
  const int np = c->nb * c->nb, npp = (np + 127) / 128 * 128;
  const size_t xbytes = (size_t)4 * c->nk * npp * c->ni * sizeof(__half);
  const size_t wbytes = (size_t)4 * c->ntau * c->ni * c->ni * sizeof(__half);
  const size_t dbytes = (size_t)c->nk * np * c->ntau * sizeof(double);
  gw_status st;
  if ((st = ensure(c, &c->mw.mslices, &c->mw.mslices_bytes, xbytes + wbytes + dbytes + sizeof(int), "Sigma slices")) !=
      GW_OK)
    return st;
  __half* XT = (__half*)c->mw.mslices;
  __half* BW = XT + xbytes / sizeof(__half);
  double* D = (double*)((char*)c->mw.mslices + xbytes + wbytes);
  int* d_err = (int*)((char*)D + dbytes);
  cudaMemsetAsync(d_err, 0, sizeof(int), c->stream);
  const double2* Mq = (const double2*)c->d_M + (size_t)iq * c->nk * c->ni * np;
  if (c->mw.iq != iq || c->mw.prec != prec) {
    dim3 g((npp + 31) / 32, (c->ni + 31) / 32, c->nk);
    k_split_x<<<g, dim3(32, 8), 0, c->stream>>>(Mq, c->nk, c->ni, np, npp, XT);
    if ((st = check_launch(c, "split_x")) != GW_OK) return st;
    c->mw.iq = iq;
    c->mw.prec = prec;
  }
  const int64_t nw = (int64_t)c->ntau * c->ni * c->ni;
  k_split_w<<<(unsigned)((nw + 255) / 256), 256, 0, c->stream>>>((const double2*)W, c->ntau, c->ni, BW);
  if ((st = check_launch(c, "split_w")) != GW_OK) return st;
  const int stage_bytes = 4 * S_ATILE + 4 * c->ni * 64;
  const size_t smem = 1024 + 2 * stage_bytes + sizeof(SigSmem);
  cudaFuncSetAttribute(k_sig_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(npp / 128, c->nk);
  k_sig_tc<<<grid, ST_THREADS, smem, c->stream>>>(XT, BW, c->nk, c->ni, npp, c->ntau, D, np, d_err);
  if ((st = check_launch(c, "sig_tc")) != GW_OK) return st;
  const int64_t n = (int64_t)c->nk * c->nb * c->ntau;
  k_sig_reduce<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(D, G, c->d_kmq + (size_t)iq * c->nk, c->nk, c->nb,
                                                                   c->ntau, -1.0 / (c->omega * c->nk), S);
  return check_launch(c, "sig_reduce");
}

void free_mixed(gw_ctx* c) {
  if (c->mw.mslices) cudaFree(c->mw.mslices);
  if (c->mw.wslices) cudaFree(c->mw.wslices);
  if (c->mw.dacc) cudaFree(c->mw.dacc);
  c->mw = MixedWork();
}

}  // namespace gwi
