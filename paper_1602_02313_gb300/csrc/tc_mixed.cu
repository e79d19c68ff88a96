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
//   P(tau) is Hermitian (w is real), so the real matrix E = Re P + Im P holds all of it:
//   Re P = (E + E^T) / 2, Im P = (E - E^T) / 2. E is one real GEMM, E = X Y^T with rows
//   X_I = [w (Re A_I + Im A_I) | w (Im A_I - Re A_I)], Y_I' = [Re A_I' | Im A_I']: tiles of E
//   cover NI^2 exactly (the Hermitian half in strips of 128 rows covers 1.5x of it at NI = 256).
//   This E form is used up to NI = 256. Above, the complex form: Re P = X Y^T, Im P = X' Y^T with
//   rows X_I = [w Re A_I | w Im A_I], X'_I = [w Im A_I | -w Re A_I] (the same shared-memory tile,
//   other K halves, negated) over strips of the Hermitian half, two accumulators per X build.
//   Work unit = (K segment, 128-row strip of <= 256 columns, tau); the FP32 partial strips are
//   summed over K segments with float-float accumulators by a second kernel (into E in FP64, and
//   a third forms P; or directly into P, writing the lower triangle too).
//
// self-energy, Eq. (sigc), one q:
//   d_p(tau) = a_p^H W~(tau) a_p = Re a_p^T Wr Re a_p + Im a_p^T Wr Im a_p + 2 Im a_p^T Wi Re a_p
//   (Wr = Re W~ symmetric, Wi = Im W~ antisymmetric). Only the upper triangle enters:
//   with U = upper(Wr) (diagonal halved) and V = strict upper(Wi),
//   d_p = 2 (<Ar_p, Y1_p> + <Ai_p, Y2_p>),  Y1 = Ar U + Ai V,  Y2 = Ai U - Ar V
//   on the tensor cores (rows = pairs p); K chunk I in [32 c, 32 c + 32) only reaches output
//   columns J >= 32 c, so its MMAs start there (~44 % fewer MMA flops than full U, V). The dot
//   products run in the epilogue (FP32 products, compensated sums);
//   Sigc_n(k|tau) += pref sum_a G_a(k-q|tau) d_(a,n)(tau) in a final kernel.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "cvt.cuh"
#include "gw_internal.h"
#include "tc_common.cuh"

namespace gwi {

namespace {

using namespace tc;

constexpr float kScaleA = 256.0f;   // 2^8 on matrix elements (|M| < ~3)
constexpr float kScaleW = 1.0f;     // W~ entries are O(v) <= 4 pi / 0.05
constexpr long long kDrainCycles = 4000000000ll;  // ~2 s at 2 GHz: waits for work already issued

// Bounded mbarrier wait shared by all roles of a block: gives up after `budget` clock cycles
// (the context's wait budget, ~2 s by default), or at once if another thread of the block has
// given up; on giving up it raises the block's abort flag and records kErrTimeout in *err.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > budget) {
      *abort_flag = 1;
      if (err) atomicExch(err, kErrTimeout);
      return false;
    }
  }
  return true;
}

// Wait for work this block has already issued (bulk copies into its shared memory, MMAs into its
// TMEM) before the block gives up its resources; ignores the abort flag, bounded by kDrainCycles.
__device__ __forceinline__ bool drain_bar(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kDrainCycles) return false;
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
// E is covered by "strips": rows [128 i, 128 i + 128) x columns [c0, c0 + N), c0 = 0, 256, ...,
// N <= 256 (the upper triangle of P in the complex form: c0 = 128 i, 128 i + 256, ...). A work
// unit is (K segment, strip, tau). The unscaled
// operand Y (rows of the strip's columns) is bulk-copied from YS, a pre-split,
// pre-swizzled image of M[q]:
//   YS[k][chunk][iblk][slice][128 rows x 128 B], row = [Re A (32 pairs) | Im A (32 pairs)],
// slices hi, lo. The scaled operand X (rows of the strip) is built by the producer warps from the
// same image. TMEM holds E (N columns), or Re P and Im P (N columns each).
constexpr int kPolChunksPerSeg = 32;  // upper bound of the context's K chunks per segment
constexpr int PT_THREADS = 288;                     // warps 0-7 produce / run the epilogue, warp 8 issues MMAs
constexpr int P_XT = 16384;                         // one X slice: 128 rows x 128 B
constexpr int P_STAGE_BYTES = 2 * P_XT + 2 * 256 * 128;  // X hi, lo (128 rows) + Y hi, lo (<= 256 rows)
constexpr int P_TILE = 128 * 256;                   // floats of one unit's partial strip

struct PolSmem {
  uint64_t full[2], empty[2], done, never;  // never: nothing arrives on it (stall injection)
  uint32_t tslot;
  int abort_flag;                           // any role gave up a wait
  int abort_prod[2];                        // producer decision per chunk parity (uniform, see below)
  int no_dealloc;                           // issued work did not drain: keep TMEM, report only
};

__device__ __forceinline__ size_t ys_tile(int k, int c, int iblk, int sl, int cpk, int nib) {
  return ((((size_t)k * cpk + c) * nib + iblk) * 2 + sl) * (size_t)(128 * 64);  // in halves
}

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

// M[q] -> YS (scaled by kScaleA, split into fp16 hi / lo). One thread per (k, I, 8 pairs).
__global__ void k_split_y(const double2* __restrict__ Mq, int nk, int ni, int np, int cpk, int nib,
                          __half* __restrict__ YS) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)nk * ni * cpk * 4;
  if (e >= n) return;
  const int g8 = (int)(e & 3);
  const int c = (int)((e >> 2) % cpk);
  const int I = (int)((e / (4 * cpk)) % ni);
  const int k = (int)(e / ((int64_t)4 * cpk * ni));
  const int pb = c * 32 + 8 * g8;
  h8 rh, rl, ih, il;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double2 v = make_double2(0.0, 0.0);
    if (pb + q < np) v = Mq[((size_t)k * ni + I) * np + pb + q];
    split2(cvt::d2f(v.x) * kScaleA, rh.v[q], rl.v[q]);
    split2(cvt::d2f(v.y) * kScaleA, ih.v[q], il.v[q]);
  }
  const int iblk = I >> 7, r = I & 127;
  __half* hi = YS + ys_tile(k, c, iblk, 0, cpk, nib);
  __half* lo = YS + ys_tile(k, c, iblk, 1, cpk, nib);
  *reinterpret_cast<h8*>(hi + sw128_off(r, 8 * g8) / 2) = rh;
  *reinterpret_cast<h8*>(hi + sw128_off(r, 32 + 8 * g8) / 2) = ih;
  *reinterpret_cast<h8*>(lo + sw128_off(r, 8 * g8) / 2) = rl;
  *reinterpret_cast<h8*>(lo + sw128_off(r, 32 + 8 * g8) / 2) = il;
}

// One polarization job: the operands of one (context, q) and where its partials go.
struct PolJob {
  const __half* YS;
  const float* wt;
  float* part;
  const int4* strips;
  int nk, ni, ntau, cpk, npw, nstrips, nseg, seg0;
  int eform;  // 1: strips of E (one accumulator); 0: strips of the Hermitian half (Re P, Im P)
  int units;  // K segments x strips x tau of this job (this launch's segments)
};

// Barrier phases of a block that runs several work units one after another: the chunk counter
// runs on across units (stage = chunk & 1, phase of that stage = chunk >> 1), and the MMA thread
// commits `done` once per unit.
struct PolPhase {
  int cbase = 0;   // chunks of the units already run by this block
  int units = 0;   // units already run (commits of `done`)
  int last0 = -1;  // (thread 0) last chunk whose copies went to stage 0 / 1
  int last1 = -1;
};

// One work unit u of job J = (K segment, 128 x N strip, tau): the producer warps build
// X = [w (Re A + Im A) | w (Im A - Re A)] (E form) or [w Re A | w Im A] (complex form) and bring Y
// by bulk copy, one thread issues the MMAs, the producer warps then move the FP32 partial strip out
// of TMEM. A wait that runs out raises S.abort_flag.
__device__ __forceinline__ void pol_unit(const PolJob& J, int u, PolSmem& S, unsigned char* base, uint32_t tbase,
                                         int tid, int warp, int lane, PolPhase& ph, int* err, long long wait_cycles,
                                         int stall) {
  const int ntau = J.ntau, nstrips = J.nstrips, cpk = J.cpk, npw = J.npw;
  const int it = u % ntau, strip = (u / ntau) % nstrips, seg = J.seg0 + u / (ntau * nstrips);
  const int4 sd = J.strips[strip];  // (row block, c0, N, -)
  const int xb = sd.x, c0 = sd.y, N = sd.z;
  const int nib = (J.ni + 127) / 128;
  const int total = J.nk * cpk;
  const int L = (total + J.nseg - 1) / J.nseg;
  const int g0 = seg * L, g1 = min(total, g0 + L);
  const int nchunk = max(0, g1 - g0);
  const uint32_t ybytes_slice = (uint32_t)N * 128;
  const __half* YS = J.YS;
  const float* wt = J.wt;

  if (warp < 8) {
    // ------------------------------------------------------------ producers
    // X for the strip's 128 rows: 512 items of (row, 8 pairs), two per thread. Within a
    // warp, the 8 lanes of each quarter take rows r and r + 4 (r < 4 of an 8-row group), so
    // their 16-byte stores land in 8 distinct bank groups of the 128-byte swizzle. The next
    // chunk's operands and weights are loaded while the current chunk is written.
    struct Item {
      h8 rh, rl, ih, il;
      float4 w0, w1;
    };
    int ir[2], ig[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int item = tid + 256 * j, ln = item & 31;
      ir[j] = 8 * (item >> 5) + ((ln & 7) >> 2) * 4 + (ln >> 3);
      ig[j] = ln & 3;
    }
    auto fetch = [&](int i, Item (&it2)[2]) {
      const int g = g0 + i, k = g / cpk, c = g % cpk;
      const __half* xh = YS + ys_tile(k, c, xb, 0, cpk, nib);
      const __half* xl = YS + ys_tile(k, c, xb, 1, cpk, nib);
      const float* wrow = wt + ((size_t)k * ntau + it) * npw + c * 32;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t oRe = sw128_off(ir[j], 8 * ig[j]), oIm = sw128_off(ir[j], 32 + 8 * ig[j]);
        it2[j].rh = *reinterpret_cast<const h8*>(xh + oRe / 2);
        it2[j].rl = *reinterpret_cast<const h8*>(xl + oRe / 2);
        it2[j].ih = *reinterpret_cast<const h8*>(xh + oIm / 2);
        it2[j].il = *reinterpret_cast<const h8*>(xl + oIm / 2);
        it2[j].w0 = __ldg(reinterpret_cast<const float4*>(wrow + 8 * ig[j]));
        it2[j].w1 = __ldg(reinterpret_cast<const float4*>(wrow + 8 * ig[j]) + 1);
      }
    };
    Item cur[2], nxt[2];
    if (nchunk > 0) fetch(0, cur);
    for (int i = 0; i < nchunk; ++i) {
      const int ic = ph.cbase + i, s = ic & 1;
      // All 256 producer threads take the same go / stop decision for chunk ic (their flag slot is
      // written only before this barrier, and slot ic & 1 is not written again before every thread
      // has read it), so every chunk whose copies are issued gets all its arrivals and its full
      // barrier completes once the bytes land: the drain can wait for it.
      if (ic >= 2 && !wait_bar(&S.empty[s], ((ic >> 1) + 1) & 1, &S.abort_flag, err, wait_cycles)) S.abort_prod[s] = 1;
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (S.abort_prod[s]) break;
      unsigned char* st = base + s * P_STAGE_BYTES;
      if (tid == 0) {
        // Y: rows [c0, c0 + N) = whole or leading parts of 128-row blocks, hi and lo slices
        const int g = g0 + i, k = g / cpk, c = g % cpk;
        if (s) ph.last1 = ic; else ph.last0 = ic;
        mbar_arrive_expect_tx(&S.full[s], 2 * ybytes_slice);
        for (int r0 = 0; r0 < N; r0 += 128) {
          const int rows = min(128, N - r0);
          const int yb = (c0 + r0) >> 7;
          for (int sl = 0; sl < 2; ++sl)
            bulk_g2s(st + 2 * P_XT + sl * ybytes_slice + r0 * 128, YS + ys_tile(k, c, yb, sl, cpk, nib),
                     (uint32_t)rows * 128, &S.full[s]);
        }
      }
      if (i + 1 < nchunk) fetch(i + 1, nxt);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint32_t oRe = sw128_off(ir[j], 8 * ig[j]), oIm = sw128_off(ir[j], 32 + 8 * ig[j]);
        const float wv[8] = {cur[j].w0.x, cur[j].w0.y, cur[j].w0.z, cur[j].w0.w,
                             cur[j].w1.x, cur[j].w1.y, cur[j].w1.z, cur[j].w1.w};
        h8 orh, orl, oih, oil;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float re = __half2float(cur[j].rh.v[e]) + __half2float(cur[j].rl.v[e]);
          const float im = __half2float(cur[j].ih.v[e]) + __half2float(cur[j].il.v[e]);
          split2(wv[e] * (J.eform ? re + im : re), orh.v[e], orl.v[e]);
          split2(wv[e] * (J.eform ? im - re : im), oih.v[e], oil.v[e]);
        }
        *reinterpret_cast<h8*>(st + oRe) = orh;
        *reinterpret_cast<h8*>(st + oIm) = oih;
        *reinterpret_cast<h8*>(st + P_XT + oRe) = orl;
        *reinterpret_cast<h8*>(st + P_XT + oIm) = oil;
      }
      fence_proxy_async_smem();
      mbar_arrive(&S.full[s]);
#pragma unroll
      for (int j = 0; j < 2; ++j) cur[j] = nxt[j];
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t id = idesc_f16(128, N, false, false), idn = idesc_f16(128, N, false, true);
    const uint32_t dim = tbase + N;  // Im P (complex form)
    if (stall && ph.units == 0) wait_bar(&S.never, 0, &S.abort_flag, err, wait_cycles);  // injected stall
    for (int i = 0; i < nchunk; ++i) {
      const int ic = ph.cbase + i, s = ic & 1;
      if (S.abort_flag || !wait_bar(&S.full[s], (ic >> 1) & 1, &S.abort_flag, err, wait_cycles)) break;
      tc_fence_after();
      const uint32_t st = smem_u32(base + s * P_STAGE_BYTES);
      const uint32_t xh = st, xl = st + P_XT, yh = st + 2 * P_XT, yl = yh + ybytes_slice;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
        const uint32_t bo = 32 * ks;
        mma_f16(tbase, sdesc_sw128(xh + bo), sdesc_sw128(yh + bo), id, acc);
        mma_f16(tbase, sdesc_sw128(xh + bo), sdesc_sw128(yl + bo), id, 1);
        mma_f16(tbase, sdesc_sw128(xl + bo), sdesc_sw128(yh + bo), id, 1);
        if (!J.eform) {
          // Im P = [w Im A | -w Re A] . [Re A | Im A]: other K half of X, negated for the second half
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

  // ------------------------------------------------------------ epilogue: FP32 partial strip (8 warps)
  // The next unit's MMAs overwrite TMEM only after these threads have armed its first chunk.
  if (warp < 8) {
    const bool ok = nchunk > 0 && wait_bar(&S.done, ph.units & 1, &S.abort_flag, err, wait_cycles) && !S.abort_flag;
    tc_fence_after();
    const int quad = warp & 3, half = warp >> 2;
    const int row = 32 * quad + lane;
    const int nacc = J.eform ? 1 : 2;
    float* out = J.part + (size_t)u * nacc * P_TILE + (size_t)row * 256;
    const int nb16 = N / 16;
    const int ab = 4 * xb + quad;  // the 32-row block of this warp's rows
    for (int acc = 0; acc < nacc; ++acc) {
      for (int bk = half; bk < nb16; bk += 2) {
        if (!J.eform && ((c0 + 16 * bk) >> 5) < ab) continue;  // below the diagonal: never read back
        float v[16];
        if (ok) {
          tmem_ld16(tbase + ((uint32_t)(32 * quad) << 16) + acc * N + 16 * bk, v);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0.f;
        }
        float4* o = reinterpret_cast<float4*>(out + (size_t)acc * P_TILE + 16 * bk);
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      }
    }
    tc_fence_before();
  }
  ph.cbase += nchunk;
  ph.units += 1;
}

__device__ __forceinline__ void pol_block_init(PolSmem& S, int tid, int warp) {
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.full[s], 257);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.done, 1);
    mbar_init(&S.never, 1);
    S.abort_flag = 0;
    S.abort_prod[0] = S.abort_prod[1] = 0;
    S.no_dealloc = 0;
    fence_mbar_init();
  }
  if (warp == 8) tmem_alloc(&S.tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// The block's last act: the copies still in flight into its shared memory land and its MMAs
// complete before it frees the tensor memory (if either does not, it keeps it and only reports).
// Called after a block barrier that follows the last unit's epilogue: every waiter on `done` is
// past its phase when the MMA thread commits `done` once more here.
__device__ __forceinline__ void pol_block_finish(PolSmem& S, uint32_t tbase, int tid, int warp, int lane,
                                                 PolPhase& ph) {
  if (tid == 0) {
    if (ph.last0 >= 0 && !drain_bar(&S.full[0], (ph.last0 >> 1) & 1)) S.no_dealloc = 1;
    if (ph.last1 >= 0 && !drain_bar(&S.full[1], (ph.last1 >> 1) & 1)) S.no_dealloc = 1;
  }
  if (warp == 8 && lane == 0) {
    mma_commit(&S.done);
    if (!drain_bar(&S.done, ph.units & 1)) S.no_dealloc = 1;  // every MMA issued here has completed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8 && !S.no_dealloc) tmem_dealloc(tbase, 512);
}

// One work unit per block: the units of one (context, q).
__global__ void __launch_bounds__(PT_THREADS, 1)
    k_pol_tc(const __half* __restrict__ YS, const float* __restrict__ wt, int nk, int ni, int ntau, int cpk,
             int npw, int nstrips, const int4* __restrict__ strips, int nseg, int seg0, int eform,
             float* __restrict__ part,
             int* __restrict__ err, long long wait_cycles, int stall) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  PolSmem& S = *reinterpret_cast<PolSmem*>(base + 2 * P_STAGE_BYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pol_block_init(S, tid, warp);
  const uint32_t tbase = S.tslot;
  PolJob J{YS, wt, part, strips, nk, ni, ntau, cpk, npw, nstrips, nseg, seg0, eform, 0};
  PolPhase ph;
  pol_unit(J, blockIdx.x, S, base, tbase, tid, warp, lane, ph, err, wait_cycles, stall);
  // the epilogue has seen the unit's `done` phase before the MMA thread commits `done` again in
  // the finish (two commits completing back to back would move the barrier two phases on)
  __syncthreads();
  pol_block_finish(S, tbase, tid, warp, lane, ph);
}

// The batched form: up to kPolQueueJobs (context, q) jobs, their units numbered one after another;
// one block per SM pulls the next unit from a device counter until all are taken (the blocks that
// finish early take more), so that small jobs fill the GPU beside large ones in one launch.
constexpr int kPolQueueJobs = 16;
struct PolQueue {
  PolJob job[kPolQueueJobs];
  int njobs, total;
};

__global__ void __launch_bounds__(PT_THREADS, 1)
    k_pol_tc_queue(const __grid_constant__ PolQueue Q, int* __restrict__ counter, int* __restrict__ err,
                   long long wait_cycles, int stall) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  PolSmem& S = *reinterpret_cast<PolSmem*>(base + 2 * P_STAGE_BYTES);
  __shared__ int item;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  pol_block_init(S, tid, warp);
  const uint32_t tbase = S.tslot;
  PolPhase ph;
  while (true) {
    if (tid == 0) item = S.abort_flag ? Q.total : atomicAdd(counter, 1);
    __syncthreads();
    const int w = item;
    __syncthreads();  // every thread has read `item` before thread 0 writes the next one
    if (w >= Q.total) break;
    int j = 0, u = w;
    while (j + 1 < Q.njobs && u >= Q.job[j].units) u -= Q.job[j++].units;
    pol_unit(Q.job[j], u, S, base, tbase, tid, warp, lane, ph, err, wait_cycles, stall);
    __syncthreads();            // every role is done with the unit: the abort flag no longer changes
    if (S.abort_flag) break;    // the same decision in every thread
  }
  pol_block_finish(S, tbase, tid, warp, lane, ph);
}

// h + l += x with the rounding error of h + x kept exactly in l (Knuth's two-sum)
__device__ __forceinline__ void two_sum_acc(float& h, float& l, float x) {
  const float s = h + x;
  const float v = s - h;
  l += (h - (s - v)) + (x - v);
  h = s;
}

// Complex form: sum the FP32 partial strips of Re P and Im P over K segments and write the
// Hermitian P (FP64).
// One block per (32 x 32 block (ab, bb) with ab <= bb, tau); reads are coalesced along
// the column, the mirrored lower triangle is written through a shared-memory transpose.
__global__ void __launch_bounds__(256) k_pol_reduce(const float* __restrict__ part, int ni, int ntau,
                                                    const int* __restrict__ strip_of, int nstrips,
                                                    const int4* __restrict__ strips, int nseg, double scale,
                                                    int accumulate, double2* __restrict__ P) {
  __shared__ double2 tr[32][33];
  const int nb32 = (ni + 31) / 32;
  int t = blockIdx.x, ab = 0;
  while (t >= nb32 - ab) {
    t -= nb32 - ab;
    ++ab;
  }
  const int bb = ab + t;
  const int it = blockIdx.y;
  const int strip = strip_of[ab * nb32 + bb];
  const int4 sd = strips[strip];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int b = bb * 32 + tx;
  // float-float accumulators (hi + lo, error-free two-sum per addition): as exact as an FP64
  // sum of these FP32 terms to ~2^-44, on the FP32 pipes (GB300's FP64 rate is ~1/64 of FP32)
  float reh[4] = {0, 0, 0, 0}, rel[4] = {0, 0, 0, 0}, imh[4] = {0, 0, 0, 0}, iml[4] = {0, 0, 0, 0};
  size_t o[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) o[r] = (size_t)((ab * 32 + ty + 8 * r) & 127) * 256 + (b - sd.y);
  const size_t ustride = (size_t)nstrips * ntau * 2 * 128 * 256;  // one K segment further
  const float* pre = part + ((size_t)strip * ntau + it) * 2 * 128 * 256;
#pragma unroll 2
  for (int s = 0; s < nseg; ++s, pre += ustride) {
    const float* pim = pre + 128 * 256;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      two_sum_acc(reh[r], rel[r], pre[o[r]]);
      two_sum_acc(imh[r], iml[r], pim[o[r]]);
    }
  }
  double2* Pt = P + (size_t)it * ni * ni;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = ab * 32 + ty + 8 * r;
    double2 v = make_double2(((double)reh[r] + (double)rel[r]) * scale, ((double)imh[r] + (double)iml[r]) * scale);
    if (a == b) v.y = 0.0;  // Im P_II = 0 exactly (the tensor-core sum leaves O(2^-22) residue)
    if (accumulate && a < ni && b < ni) {  // a later pass over K segments: add to the earlier sum
      const double2 o = Pt[(size_t)a * ni + b];
      v.x += o.x;
      v.y += o.y;
    }
    if (a < ni && b < ni && (ab < bb || a <= b)) Pt[(size_t)a * ni + b] = v;
    tr[ty + 8 * r][tx] = make_double2(v.x, -v.y);
  }
  __syncthreads();
  // lower triangle: P[b'][a'] = conj(P[a'][b']) for a' < b'
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int row = bb * 32 + ty + 8 * r;  // b'
    const int col = ab * 32 + tx;          // a'
    if (row < ni && col < ni && col < row) Pt[(size_t)row * ni + col] = tr[tx][ty + 8 * r];
  }
}

// Sum the FP32 partial strips of E over K segments into E (FP64), one block per (strip, 16-row
// band, tau): per segment the block reads the band's 16 KB contiguously (float4 per thread), and
// keeps float-float accumulators (hi + lo, error-free two-sum per addition: as exact as an FP64
// sum of these FP32 terms to ~2^-44, on the FP32 pipes; GB300's FP64 rate is ~1/64 of FP32).
__global__ void __launch_bounds__(256, 2) k_pol_sum_e(const float* __restrict__ part, int ni, int ntau, int nstrips,
                                                      const int4* __restrict__ strips, int nseg,
                                                      double* __restrict__ E) {
  const int strip = blockIdx.x >> 3, band = blockIdx.x & 7, it = blockIdx.y;
  const int4 sd = strips[strip];  // (row block, c0, N, -)
  const size_t ustride = (size_t)nstrips * ntau * P_TILE;  // one K segment further
  const float4* p = reinterpret_cast<const float4*>(part + ((size_t)strip * ntau + it) * P_TILE +
                                                    (size_t)band * 16 * 256) + threadIdx.x;
  float h[16], l[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) h[e] = l[e] = 0.f;
#pragma unroll 2
  for (int sg = 0; sg < nseg; ++sg, p += ustride / 4) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = p[256 * j];
      two_sum_acc(h[4 * j], l[4 * j], v.x);
      two_sum_acc(h[4 * j + 1], l[4 * j + 1], v.y);
      two_sum_acc(h[4 * j + 2], l[4 * j + 2], v.z);
      two_sum_acc(h[4 * j + 3], l[4 * j + 3], v.w);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int f = threadIdx.x + 256 * j;  // float4 of the band: row f / 64, columns 4 (f % 64) + e
    const int row = 128 * sd.x + 16 * band + (f >> 6), cl = 4 * (f & 63);
    if (row < ni && cl < sd.z) {
      double* o = E + ((size_t)it * ni + row) * ni + sd.y + cl;
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = (double)h[4 * j + e] + (double)l[4 * j + e];
    }
  }
}

// P_ab = scale ((E_ab + E_ba) / 2 + i (E_ab - E_ba) / 2), Im P_aa = 0 exactly; one block per
// (32 x 32 block, tau), E_ba through a shared-memory transpose. accumulate: add to P (a later pass
// over K segments).
__global__ void __launch_bounds__(256) k_pol_form(const double* __restrict__ E, int ni, double scale, int accumulate,
                                                  double2* __restrict__ P) {
  __shared__ double tb[32][33];
  const int bx = blockIdx.x, by = blockIdx.y, it = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double* Et = E + (size_t)it * ni * ni;
#pragma unroll
  for (int r = 0; r < 4; ++r) tb[ty + 8 * r][tx] = Et[(size_t)(bx * 32 + ty + 8 * r) * ni + by * 32 + tx];
  __syncthreads();
  double2* Pt = P + (size_t)it * ni * ni;
  const int b = bx * 32 + tx;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = by * 32 + ty + 8 * r;
    const double e1 = Et[(size_t)a * ni + b], e2 = tb[tx][ty + 8 * r];  // E[a][b], E[b][a]
    double2 v = make_double2(0.5 * (e1 + e2) * scale, a == b ? 0.0 : 0.5 * (e1 - e2) * scale);
    if (accumulate) {
      const double2 o = Pt[(size_t)a * ni + b];
      v.x += o.x;
      v.y += o.y;
    }
    Pt[(size_t)a * ni + b] = v;
  }
}

// --------------------------------------------------------------------------- self-energy
// Operand slices live in global memory as ready-made shared-memory images: each 32-wide
// K chunk of a tile is stored in the 64-byte-swizzled K-major layout, so one bulk copy
// per operand and chunk fills a pipeline stage.
//   XS[k][pblk][kc][slice][128 rows x 64 B]   slices: Re hi, Re lo, Im hi, Im lo of M (rows = pairs p)
//   WS[tau][kc][slice][ni rows x 64 B]        slices: U hi, U lo, V hi, V lo; row J, K column I
//                                             holds U[I][J], V[I][J] (zero for I > J)
__device__ __forceinline__ size_t xs_tile(int k, int pblk, int kc, int sl, int npb, int nkc) {
  return ((((size_t)k * npb + pblk) * nkc + kc) * 4 + sl) * (size_t)(128 * 32);  // in halves
}

// Split M[q] into XS and write the epilogue's image XE[k][pblk][I][row] = 2^8 M (FP32 re, im;
// rows contiguous, so that the 32 lanes of a warp, which own 32 consecutive rows, read 256
// contiguous bytes). One block per (k, 32 pairs, 64 I): each thread issues its 8 loads before
// the first use; the scaled FP32 values go through a 64 x 32 shared-memory transpose (rows
// I, padded to 33, columns XOR-swizzled by 2 ((I >> 4) & 3) so that both the row-wise writes
// and the column-wise reads below are free of bank conflicts) and are split into the fp16
// hi / lo slices of XS (rows p >= nb^2 zero).
constexpr int SX_I = 64;
__global__ void __launch_bounds__(256) k_split_x(const double2* __restrict__ Mq, int ni, int np, int npb,
                                                 __half* __restrict__ XS, float2* __restrict__ XE) {
  __shared__ float2 tileF[SX_I][33];
  const int k = blockIdx.z;
  const int p0 = blockIdx.x * 32, I0 = blockIdx.y * SX_I;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int p = p0 + tx;
  double2 v[SX_I / 8];
#pragma unroll
  for (int j = 0; j < SX_I / 8; ++j) {
    const int I = I0 + ty + 8 * j;
    v[j] = (I < ni && p < np) ? Mq[((size_t)k * ni + I) * np + p] : make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int j = 0; j < SX_I / 8; ++j) {
    const int r = ty + 8 * j, I = I0 + r;
    // converted on the integer pipes, then scaled (a power of two: the same value)
    const float2 f = make_float2(cvt::d2f(v[j].x) * kScaleA, cvt::d2f(v[j].y) * kScaleA);
    tileF[r][tx ^ (2 * ((r >> 4) & 3))] = f;
    if (I < ni) XE[(((size_t)k * npb + (p >> 7)) * ni + I) * 128 + (p & 127)] = f;
  }
  __syncthreads();
  // thread t: pair row r = t >> 3, group G = t & 7 of 8 consecutive I (K chunk G >> 2, quarter G & 3)
  const int t = ty * 32 + tx;
  const int r = t >> 3, G = t & 7;
  const int Ib = I0 + 8 * G;
  if (Ib >= ni) return;
  const int nkc = ni / 32;
  h8 rh, rl, ih, il;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int R = 8 * G + e;
    const float2 f = tileF[R][r ^ (2 * ((R >> 4) & 3))];
    split2(f.x, rh.v[e], rl.v[e]);
    split2(f.y, ih.v[e], il.v[e]);
  }
  const int pp = p0 + r;
  const int pblk = pp >> 7, row = pp & 127, kc = Ib >> 5;
  const size_t o = sw64_off(row, Ib & 31) / 2;
  *reinterpret_cast<h8*>(XS + xs_tile(k, pblk, kc, 0, npb, nkc) + o) = rh;
  *reinterpret_cast<h8*>(XS + xs_tile(k, pblk, kc, 1, npb, nkc) + o) = rl;
  *reinterpret_cast<h8*>(XS + xs_tile(k, pblk, kc, 2, npb, nkc) + o) = ih;
  *reinterpret_cast<h8*>(XS + xs_tile(k, pblk, kc, 3, npb, nkc) + o) = il;
}

// Split W~(tau) into WS: image row R, K column C holds U[C][R] and V[C][R]; for C < R these
// are Re W~[R][C] (Wr symmetric) and -Im W~[R][C] (Wi antisymmetric), read along C.
__global__ void k_split_w(const double2* __restrict__ W, int ntau, int ni, __half* __restrict__ WS) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)ntau * ni * ni;
  if (e >= n) return;
  const int it = (int)(e / ((int64_t)ni * ni)), I = (int)((e / ni) % ni), J = (int)(e % ni);  // row I, K column J
  const double2 w = W[e];
  const double u = J < I ? w.x : (J == I ? 0.5 * w.x : 0.0);
  const double v = J < I ? -w.y : 0.0;
  __half a, b, c, d;
  split2((float)u * kScaleW, a, b);
  split2((float)v * kScaleW, c, d);
  const int nkc = ni / 32, kc = J >> 5;
  const size_t tile = (size_t)ni * 32;  // halves per slice tile
  const size_t base = ((size_t)it * nkc + kc) * 4 * tile + sw64_off(I, J & 31) / 2;
  WS[base] = a;
  WS[base + tile] = b;
  WS[base + 2 * tile] = c;
  WS[base + 3 * tile] = d;
}

constexpr int ST_EPI_WARPS = 16;                    // 4 per TMEM lane quadrant
constexpr int ST_THREADS = (ST_EPI_WARPS + 2) * 32;  // + producer warp + MMA warp
constexpr int S_ATILE = 128 * 64;                   // 128 rows x 64 B (32 fp16)

struct SigSmem {
  uint64_t full[2], empty[2], col[32], tempty;  // col[c]: K chunk c of the current unit is done
  uint64_t fin, never;                          // fin: all MMAs done; never: stall injection
  uint32_t tslot;
  int abort_flag;
  int no_dealloc;
  float red[4][128];
};

// The NI output columns are processed in nh parts of NC = NI / nh <= 256 columns (TMEM holds Y1
// and Y2 of one part: 2 NC <= 512 columns). Work units u = (tau, part h); a unit runs the K
// chunks c with 32 c < (h + 1) NC, each over the output columns [max(h NC, 32 c), (h + 1) NC)
// that U and V reach. Output column block j (32 columns) is final once chunk j is done, so the
// epilogue takes each 16-column block as soon as its chunk completes (barrier col[j]) while the
// later chunks still run; only the next unit's first chunk waits for the whole epilogue. The
// epilogue sums d_p over the parts of a tau before writing it.
__global__ void __launch_bounds__(ST_THREADS, 1)
    k_sig_tc(const __half* __restrict__ XS, const float2* __restrict__ XE, const __half* __restrict__ WS, int ni,
             int nh, int npb, int ntau, double* __restrict__ D, int np, int* __restrict__ err, long long wait_cycles,
             int stall) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int NC = ni / nh;  // output columns per part
  const int BT = NC * 64;  // one W slice tile of a part: NC rows x 64 B
  const int a_bytes = 4 * S_ATILE, b_bytes = 4 * BT;
  const int stage_bytes = a_bytes + b_bytes;
  SigSmem& S = *reinterpret_cast<SigSmem*>(base + 2 * stage_bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pblk = blockIdx.x, k = blockIdx.y;
  const int nkc = ni / 32;
  const int nunit = ntau * nh;
  const int PW = ST_EPI_WARPS, MW = ST_EPI_WARPS + 1;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int c = 0; c < 32; ++c) mbar_init(&S.col[c], 1);
    mbar_init(&S.tempty, ST_EPI_WARPS * 32);
    mbar_init(&S.fin, 1);
    mbar_init(&S.never, 1);
    S.abort_flag = 0;
    S.no_dealloc = 0;
    fence_mbar_init();
  }
  if (warp == MW) tmem_alloc(&S.tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = S.tslot;

  if (warp == PW) {
    // ------------------------------------------------------------ producer: bulk copies per chunk
    if (lane == 0) {
      int i = 0;  // running chunk index (stage i & 1)
      int last0 = -1, last1 = -1;  // last chunk whose copies went to stage 0 / 1
      for (int u = 0; u < nunit && !S.abort_flag; ++u) {
        const int it = u / nh, h = u % nh;
        const int kend = min(nkc, ((h + 1) * NC) >> 5);
        for (int kc = 0; kc < kend; ++kc, ++i) {
          const int s = i & 1;
          if (i >= 2 && !wait_bar(&S.empty[s], ((i >> 1) + 1) & 1, &S.abort_flag, err, wait_cycles)) break;
          if (s) last1 = i; else last0 = i;
          const int j0 = max(h * NC, 32 * kc);      // first output column reached
          const int rows = (h + 1) * NC - j0;       // B rows (output columns) copied
          const int roff = j0 - h * NC;             // their offset inside the part
          unsigned char* st = base + s * stage_bytes;
          mbar_arrive_expect_tx(&S.full[s], (uint32_t)(a_bytes + 4 * rows * 64));
          bulk_g2s(st, XS + xs_tile(k, pblk, kc, 0, npb, nkc), (uint32_t)a_bytes, &S.full[s]);
          const __half* w0 = WS + ((size_t)it * nkc + kc) * 4 * ((size_t)ni * 32) + (size_t)j0 * 32;
          for (int sl = 0; sl < 4; ++sl)
            bulk_g2s(st + a_bytes + sl * BT + roff * 64, w0 + (size_t)sl * ni * 32, (uint32_t)rows * 64, &S.full[s]);
        }
      }
      // the copies of every issued chunk land before the block exits (one arrival per chunk,
      // so its full barrier completes once its bytes are in)
      if (last0 >= 0 && !drain_bar(&S.full[0], (last0 >> 1) & 1)) S.no_dealloc = 1;
      if (last1 >= 0 && !drain_bar(&S.full[1], (last1 >> 1) & 1)) S.no_dealloc = 1;
    }
  } else if (warp == MW) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int i = 0;
      bool live = true;
      if (stall) wait_bar(&S.never, 0, &S.abort_flag, err, wait_cycles);  // injected stall: runs out
      for (int u = 0; u < nunit && live && !S.abort_flag; ++u) {
        const int h = u % nh;
        const int kend = min(nkc, ((h + 1) * NC) >> 5);
        if (u > 0 && !wait_bar(&S.tempty, (u - 1) & 1, &S.abort_flag, err, wait_cycles)) break;
        for (int kc = 0; kc < kend; ++kc, ++i) {
          const int s = i & 1;
          if (!wait_bar(&S.full[s], (i >> 1) & 1, &S.abort_flag, err, wait_cycles)) {
            live = false;
            break;
          }
          tc_fence_after();
          const int j0 = max(h * NC, 32 * kc);
          const int roff = j0 - h * NC;
          const uint32_t ncols = (uint32_t)((h + 1) * NC - j0);
          const uint32_t id = idesc_f16(128, ncols, false, false), idn = idesc_f16(128, ncols, false, true);
          const uint32_t y1 = tbase + roff, y2 = tbase + NC + roff;
          const uint32_t st = smem_u32(base + s * stage_bytes);
          const uint32_t arh = st, arl = st + S_ATILE, aih = st + 2 * S_ATILE, ail = st + 3 * S_ATILE;
          const uint32_t bb = st + a_bytes + roff * 64;
          const uint32_t urh = bb, url = bb + BT, vih = bb + 2 * BT, vil = bb + 3 * BT;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t o = 32 * ks;
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            // Y1 = Ar U + Ai V
            mma_f16(y1, sdesc_sw64(arh + o), sdesc_sw64(urh + o), id, acc);
            mma_f16(y1, sdesc_sw64(arh + o), sdesc_sw64(url + o), id, 1);
            mma_f16(y1, sdesc_sw64(arl + o), sdesc_sw64(urh + o), id, 1);
            mma_f16(y1, sdesc_sw64(aih + o), sdesc_sw64(vih + o), id, 1);
            mma_f16(y1, sdesc_sw64(aih + o), sdesc_sw64(vil + o), id, 1);
            mma_f16(y1, sdesc_sw64(ail + o), sdesc_sw64(vih + o), id, 1);
            // Y2 = Ai U - Ar V
            mma_f16(y2, sdesc_sw64(aih + o), sdesc_sw64(urh + o), id, acc);
            mma_f16(y2, sdesc_sw64(aih + o), sdesc_sw64(url + o), id, 1);
            mma_f16(y2, sdesc_sw64(ail + o), sdesc_sw64(urh + o), id, 1);
            mma_f16(y2, sdesc_sw64(arh + o), sdesc_sw64(vih + o), idn, 1);
            mma_f16(y2, sdesc_sw64(arh + o), sdesc_sw64(vil + o), idn, 1);
            mma_f16(y2, sdesc_sw64(arl + o), sdesc_sw64(vih + o), idn, 1);
          }
          mma_commit(&S.empty[s]);
          mma_commit(&S.col[kc]);
        }
      }
      mma_commit(&S.fin);
      if (!drain_bar(&S.fin, 0)) S.no_dealloc = 1;  // every MMA issued here has completed
    }
  } else {
    // ------------------------------------------------------------ epilogue: d_p(tau), 16 warps
    // Thread (quad, grp, lane) owns row 32 quad + lane and the 16-column blocks grp, grp + 4, ...
    // of each part, taken in column order as their K chunks complete. Its XE values do not
    // depend on tau: each block's are fetched before the wait for its chunk.
    const int quad = warp & 3, grp = warp >> 2;  // lane quadrant, column group
    const int row = 32 * quad + lane;
    const int p = pblk * 128 + row;
    const int nblk = NC / 16;  // 16-column blocks of a part, dealt round-robin to the 4 column groups
    const double dscale = 2.0 / ((double)kScaleA * kScaleA * kScaleW);  // d_p = 2 (<Ar, Y1> + <Ai, Y2>)
    const float2* xe = XE + ((size_t)k * npb + pblk) * ni * 128 + row;
    float dhi = 0.f, dlo = 0.f;  // compensated (two-sum) accumulator over the parts of one tau
    for (int u = 0; u < nunit; ++u) {
      const int it = u / nh, h = u % nh;
      const float2* xh = xe + (size_t)h * NC * 128;
      if (h == 0) dhi = dlo = 0.f;
      float2 xa[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) xa[c] = grp < nblk ? __ldg(xh + (size_t)(16 * grp + c) * 128) : make_float2(0.f, 0.f);
      bool ok = true;
      {
        for (int bk = grp; bk < nblk && ok; bk += 4) {
          const int n0 = 16 * bk;
          if (bk != grp) {  // in flight while this block's chunk completes
#pragma unroll
            for (int c = 0; c < 16; ++c) xa[c] = __ldg(xh + (size_t)(n0 + c) * 128);
          }
          // the K chunk c that finishes this block's columns runs in parts h' >= h of every tau
          // (32 c < (h' + 1) NC), so before this unit it has completed tau (nh - h) times
          ok = wait_bar(&S.col[(h * NC + n0) >> 5], (it * (nh - h)) & 1, &S.abort_flag, err, wait_cycles);
          tc_fence_after();
          if (!ok) break;
          float v1[16], v2[16];
          tmem_ld16(tbase + ((uint32_t)(32 * quad) << 16) + n0, v1);
          tmem_ld16(tbase + ((uint32_t)(32 * quad) << 16) + NC + n0, v2);
          float part = 0.f;
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            part = fmaf(xa[c].x, v1[c], part);
            part = fmaf(xa[c].y, v2[c], part);
          }
          const float s2 = dhi + part;
          const float bb = s2 - dhi;
          dlo += (dhi - (s2 - bb)) + (part - bb);
          dhi = s2;
        }
      }
      tc_fence_before();
      mbar_arrive(&S.tempty);
      if (h != nh - 1) continue;
      // combine the four column groups of each row
      S.red[grp][row] = dhi + dlo;  // dlo is the two-sum error term of dhi
      asm volatile("bar.sync 1, %0;" ::"r"(ST_EPI_WARPS * 32) : "memory");
      if (grp == 0 && p < np) {
        const double d = (double)S.red[0][row] + (double)S.red[1][row] + (double)S.red[2][row] +
                         (double)S.red[3][row];
        D[((size_t)k * np + p) * ntau + it] = d * dscale;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(ST_EPI_WARPS * 32) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MW && !S.no_dealloc) tmem_dealloc(tbase, 512);
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

// Host plan of one polarization job: strips, K segments, workspace, and the operand image and
// pair weights of its q, built on the context's stream.
struct PolPrep {
  int nstrips = 0, nseg = 0, seg_pass = 0, base_units = 0, nb32 = 0, cpk = 0, npw = 0, eform = 1;
  float* d_part = nullptr;
  float* d_wt = nullptr;
  __half* d_ys = nullptr;
  double* d_e = nullptr;
  int4* d_strips = nullptr;
  int* d_strip_of = nullptr;
  double scale = 0.0;
};

static gw_status pol_prepare(gw_ctx* c, int iq, const double* G, PolPrep* pp) {
  const int ni = c->ni, nib = (ni + 127) / 128, nb32 = (ni + 31) / 32;
  // Which form: the producers' X builds pace the E form (one accumulator per build) and the MMAs
  // the complex form (Re P and Im P from one build). Per (k, tau, chunk), E needs nib ceil(ni / 256)
  // builds and 3 ni (128 nib) MMA columns, the complex form one build per strip of the Hermitian
  // half and 6 x its columns; E is the faster one up to ni = 256 (2 builds either way at 256, a
  // third less MMA work), the complex one above (at 512: 8 builds against 6).
  const int eform = c->pol_form == 1 ? 1 : c->pol_form == 2 ? 0 : (ni <= 256 ? 1 : 0);
  // strips covering E: rows of block i, columns [0, ni) in pieces <= 256; or covering the upper
  // triangle of P: rows of block i, columns [128 i, ni) in pieces <= 256
  std::vector<int4> strips;
  std::vector<int> strip_of(eform ? 0 : nb32 * nb32, -1);
  for (int i = 0; i < nib; ++i)
    for (int c0 = eform ? 0 : 128 * i; c0 < ni; c0 += 256) {
      const int N = std::min(256, ni - c0);
      if (!eform)
        for (int ab = 4 * i; ab < std::min(4 * i + 4, nb32); ++ab)
          for (int bb = c0 / 32; bb < (c0 + N) / 32; ++bb) strip_of[ab * nb32 + bb] = (int)strips.size();
      strips.push_back(make_int4(i, c0, N, 0));
    }
  const int nstrips = (int)strips.size();
  const int np = c->nb * c->nb, cpk = (np + 31) / 32, total = c->nk * cpk, npw = cpk * 32;
  // K segments. The tensor cores accumulate in FP32 with an error that grows with the
  // number of MMAs chained into one accumulator (measured ~2^-24 per MMA, biased), so
  // each work unit covers at most the context's pol_seg_chunks <= kPolChunksPerSeg chunks of
  // 32 pairs (384 chained MMAs at 32);
  // the FP32 partial strips are summed afterwards with float-float accumulators.
  const int sms = num_sms(c);
  const int base_units = nstrips * c->ntau;
  const int seg_chunks = std::max(1, std::min(c->pol_seg_chunks, kPolChunksPerSeg));
  int nseg = std::max(1, (total + seg_chunks - 1) / seg_chunks);
  while (base_units * nseg < 2 * sms && (total + nseg) / (nseg + 1) >= 4) ++nseg;
  // the partials of at most pol_part_bytes are held at once: segments run in passes, each
  // reduced into P (the first pass writes, later ones add)
  const size_t seg_bytes = (size_t)base_units * (eform ? 1 : 2) * P_TILE * sizeof(float);
  const int seg_pass = (int)std::max<size_t>(1, std::min<size_t>(nseg, c->pol_part_bytes / seg_bytes));
  const size_t part_bytes = seg_bytes * seg_pass;
  const size_t wt_bytes = (size_t)c->nk * c->ntau * npw * sizeof(float);
  const size_t ys_bytes = (size_t)c->nk * cpk * nib * 2 * 128 * 64 * sizeof(__half);
  const size_t e_bytes = eform ? (size_t)c->ntau * ni * ni * sizeof(double) : 0;
  gw_status st;
  if ((st = ensure(c, &c->mw.wslices, &c->mw.wslices_bytes, part_bytes + wt_bytes + ys_bytes + e_bytes,
                   "P workspace")) != GW_OK)
    return st;
  float* d_part = (float*)c->mw.wslices;
  float* d_wt = d_part + part_bytes / sizeof(float);
  __half* d_ys = (__half*)((char*)d_wt + wt_bytes);
  double* d_e = (double*)((char*)d_ys + ys_bytes);
  const size_t meta_bytes = sizeof(int4) * strips.size() + sizeof(int) * strip_of.size();
  const void* meta_before = c->mw.dacc;
  if ((st = ensure(c, (void**)&c->mw.dacc, &c->mw.dacc_bytes, meta_bytes + 256, "P strips")) != GW_OK) return st;
  if (c->mw.dacc != meta_before || c->mw.strips_form != eform) c->mw.strips_ready = false;
  int4* d_strips = reinterpret_cast<int4*>(c->mw.dacc);
  int* d_strip_of = reinterpret_cast<int*>(d_strips + strips.size());
  if (!c->mw.strips_ready) {  // depends on ni and the form: uploaded on the first call of each
    if (cudaMemcpy(d_strips, strips.data(), sizeof(int4) * strips.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!strip_of.empty() && cudaMemcpy(d_strip_of, strip_of.data(), sizeof(int) * strip_of.size(),
                                         cudaMemcpyHostToDevice) != cudaSuccess))
      return set_err(c, GW_ECUDA, "P strips upload");
    c->mw.strips_ready = true;
    c->mw.strips_form = eform;
  }
  if (ni % 128) cudaMemsetAsync(d_ys, 0, ys_bytes, c->stream);  // rows >= ni of the last block stay zero
  const double2* Mq = (const double2*)m_block(c, iq);
  if (!Mq) return GW_ECUDA;
  const int64_t nsp = (int64_t)c->nk * ni * cpk * 4;
  k_split_y<<<(unsigned)((nsp + 255) / 256), 256, 0, c->stream>>>(Mq, c->nk, ni, np, cpk, nib, d_ys);
  if ((st = check_launch(c, "split_y")) != GW_OK) return st;
  const int64_t nwt = (int64_t)c->nk * c->ntau * npw;
  k_pol_weights<<<(unsigned)((nwt + 255) / 256), 256, 0, c->stream>>>(G, c->d_kmq + (size_t)iq * c->nk, c->nk, c->nb,
                                                                      c->ntau, npw, d_wt);
  if ((st = check_launch(c, "pol_weights")) != GW_OK) return st;
  pp->nstrips = nstrips;
  pp->nseg = nseg;
  pp->seg_pass = seg_pass;
  pp->base_units = base_units;
  pp->nb32 = nb32;
  pp->cpk = cpk;
  pp->npw = npw;
  pp->d_part = d_part;
  pp->d_wt = d_wt;
  pp->d_ys = d_ys;
  pp->d_e = d_e;
  pp->d_strips = d_strips;
  pp->d_strip_of = d_strip_of;
  pp->eform = eform;
  pp->scale = 1.0 / ((double)kScaleA * kScaleA * c->omega * c->nk);
  return GW_OK;
}

// Sum the partials of the segments [s0, s0 + ns) into E, then form P from E (the first pass writes
// P, later ones add).
static gw_status pol_reduce(gw_ctx* c, const PolPrep& pp, int s0, int ns, double* P) {
  if (!pp.eform) {
    k_pol_reduce<<<dim3(pp.nb32 * (pp.nb32 + 1) / 2, c->ntau), 256, 0, c->stream>>>(
        pp.d_part, c->ni, c->ntau, pp.d_strip_of, pp.nstrips, pp.d_strips, ns, pp.scale, s0 > 0 ? 1 : 0,
        (double2*)P);
    return check_launch(c, "pol_reduce");
  }
  k_pol_sum_e<<<dim3(pp.nstrips * 8, c->ntau), 256, 0, c->stream>>>(pp.d_part, c->ni, c->ntau, pp.nstrips,
                                                                     pp.d_strips, ns, pp.d_e);
  gw_status st = check_launch(c, "pol_sum_e");
  if (st != GW_OK) return st;
  k_pol_form<<<dim3(pp.nb32, pp.nb32, c->ntau), 256, 0, c->stream>>>(pp.d_e, c->ni, pp.scale, s0 > 0 ? 1 : 0,
                                                                       (double2*)P);
  return check_launch(c, "pol_form");
}

static size_t pol_smem() { return 1024 + 2 * P_STAGE_BYTES + sizeof(PolSmem); }

gw_status launch_pol_mixed(gw_ctx* c, int iq, const double* G, int prec, double* P) {
  if (prec != GW_FP16X2) return set_err(c, GW_EUNSUPPORTED, "polarization: only GW_FP16X2 is built on tensor cores");
  PolPrep pp;
  gw_status st;
  if ((st = pol_prepare(c, iq, G, &pp)) != GW_OK) return st;
  const size_t smem = pol_smem();
  cudaFuncSetAttribute(k_pol_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int s0 = 0; s0 < pp.nseg; s0 += pp.seg_pass) {
    const int ns = std::min(pp.seg_pass, pp.nseg - s0);
    kt_begin(c, "k_pol_tc");
    k_pol_tc<<<pp.base_units * ns, PT_THREADS, smem, c->stream>>>(pp.d_ys, pp.d_wt, c->nk, c->ni, c->ntau, pp.cpk,
                                                                  pp.npw, pp.nstrips, pp.d_strips, pp.nseg, s0,
                                                                  pp.eform, pp.d_part, c->d_err, c->wait_cycles,
                                                                  c->fault_stall);
    kt_end(c);
    if ((st = check_launch(c, "pol_tc")) != GW_OK) return st;
    if ((st = pol_reduce(c, pp, s0, ns, P)) != GW_OK) return st;
  }
  return GW_OK;
}

// Several (context, q) polarizations in one persistent launch per pass over K segments, on the
// first context's stream: each job's operand image and weights are built on that stream, then
// one block per SM pulls (job, K segment, strip, tau) units from a device counter.
gw_status launch_pol_many(int njobs, gw_ctx* const* ctxs, const int* iqs, const double* const* G, double* const* P) {
  gw_ctx* c0 = ctxs[0];
  std::vector<PolPrep> pp(njobs);
  std::vector<cudaStream_t> saved(njobs);
  gw_status st = GW_OK;
  for (int j = 0; j < njobs; ++j) {
    saved[j] = ctxs[j]->stream;
    ctxs[j]->stream = c0->stream;
  }
  for (int j = 0; j < njobs && st == GW_OK; ++j) st = pol_prepare(ctxs[j], iqs[j], G[j], &pp[j]);
  std::vector<int> s0(njobs, 0);
  const size_t smem = pol_smem();
  cudaFuncSetAttribute(k_pol_tc_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int* counter = c0->d_err + 1;
  while (st == GW_OK) {
    PolQueue Q{};
    Q.njobs = 0;
    Q.total = 0;
    std::vector<int> jid, nsj;
    for (int j = 0; j < njobs; ++j) {
      if (s0[j] >= pp[j].nseg) continue;
      const int ns = std::min(pp[j].seg_pass, pp[j].nseg - s0[j]);
      gw_ctx* c = ctxs[j];
      PolJob& J = Q.job[Q.njobs++];
      J = PolJob{pp[j].d_ys, pp[j].d_wt, pp[j].d_part, pp[j].d_strips, c->nk, c->ni, c->ntau, pp[j].cpk,
                 pp[j].npw, pp[j].nstrips, pp[j].nseg, s0[j], pp[j].eform, pp[j].base_units * ns};
      Q.total += J.units;
      jid.push_back(j);
      nsj.push_back(ns);
    }
    if (Q.njobs == 0) break;
    cudaMemsetAsync(counter, 0, sizeof(int), c0->stream);
    kt_begin(c0, "k_pol_tc");
    k_pol_tc_queue<<<num_sms(c0), PT_THREADS, smem, c0->stream>>>(Q, counter, c0->d_err, c0->wait_cycles,
                                                                  c0->fault_stall);
    kt_end(c0);
    if ((st = check_launch(c0, "pol_tc_queue")) != GW_OK) break;
    for (size_t q = 0; q < jid.size() && st == GW_OK; ++q) {
      const int j = jid[q];
      st = pol_reduce(ctxs[j], pp[j], s0[j], nsj[q], P[j]);
      s0[j] += nsj[q];
    }
  }
  for (int j = 0; j < njobs; ++j) ctxs[j]->stream = saved[j];
  return st;
}

gw_status launch_sigma_mixed(gw_ctx* c, int iq, const double* G, const double* W, int prec, double* S) {
  if (prec != GW_FP16X2) return set_err(c, GW_EUNSUPPORTED, "self-energy: only GW_FP16X2 is built on tensor cores");
  const int nh = (c->ni + 255) / 256;  // output-column parts of <= 256 columns
  if (c->ni % 32 || c->ni % (16 * nh))
    return set_err(c, GW_EUNSUPPORTED, "tensor-core self-energy: ni a multiple of 32 that splits into parts of 16k columns");
  const int np = c->nb * c->nb, npb = (np + 127) / 128, npp = npb * 128;
  const size_t xbytes = (size_t)4 * c->nk * npp * c->ni * sizeof(__half);
  const size_t wbytes = (size_t)4 * c->ntau * c->ni * c->ni * sizeof(__half);
  const size_t dbytes = (size_t)c->nk * np * c->ntau * sizeof(double);
  const size_t ebytes = (size_t)c->nk * npp * c->ni * sizeof(float2);
  gw_status st;
  if ((st = ensure(c, &c->mw.mslices, &c->mw.mslices_bytes, xbytes + wbytes + dbytes + ebytes + 256,
                   "Sigma slices")) != GW_OK)
    return st;
  __half* XS = (__half*)c->mw.mslices;
  __half* WS = XS + xbytes / sizeof(__half);
  double* D = (double*)((char*)c->mw.mslices + xbytes + wbytes);
  float2* XE = (float2*)((char*)D + dbytes);
  if (c->mw.iq != iq || c->mw.prec != prec) {
    const double2* Mq = (const double2*)m_block(c, iq);
    if (!Mq) return GW_ECUDA;
    dim3 g(npp / 32, (c->ni + SX_I - 1) / SX_I, c->nk);
    k_split_x<<<g, dim3(32, 8), 0, c->stream>>>(Mq, c->ni, np, npb, XS, XE);
    if ((st = check_launch(c, "split_x")) != GW_OK) return st;
    c->mw.iq = iq;
    c->mw.prec = prec;
  }
  const int64_t nw = (int64_t)c->ntau * c->ni * c->ni;
  k_split_w<<<(unsigned)((nw + 255) / 256), 256, 0, c->stream>>>((const double2*)W, c->ntau, c->ni, WS);
  if ((st = check_launch(c, "split_w")) != GW_OK) return st;
  const int stage_bytes = 4 * S_ATILE + 4 * (c->ni / nh) * 64;
  const size_t smem = 1024 + 2 * stage_bytes + sizeof(SigSmem);
  cudaFuncSetAttribute(k_sig_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(npb, c->nk);
  kt_begin(c, "k_sig_tc");
  k_sig_tc<<<grid, ST_THREADS, smem, c->stream>>>(XS, XE, WS, c->ni, nh, npb, c->ntau, D, np, c->d_err,
                                                  c->wait_cycles, c->fault_stall);
  kt_end(c);
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
