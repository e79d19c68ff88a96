// Complex arithmetic policies shared by the FP64-bound kernels (screening, transforms).
//  * Fp64 : double2 values, FP64 fused multiply-adds.
//  * F32  : float2 values, FP32 fused multiply-adds (rounding error ~6e-8 per operation; for
//           the dielectric inverse of the mixed chain, whose input P already carries the
//           ~1e-6 error of the fp16-split tensor-core contraction).
//  * Ff32 : float-float values (hi + lo, two FP32 each, ~44-bit significand). A product
//           is hi*hi with its exact rounding error from an FMA plus the two cross terms;
//           it joins the accumulator through an error-free two-sum (Knuth), the errors
//           collect in the accumulator's low word. All of it runs on the FP32 pipes, which
//           on GB300 issue about 64 times more operations per clock than the FP64 ones.
// Both expose: S (stored value), Acc (accumulator), from/to double, zero, azero, is_zero,
// mac (acc += l u, complex), rmac (real parts: acc.re += a x, acc.im += a y for real a),
// val (accumulator -> value), sub (b - acc), inv (complex reciprocal).
#pragma once
#include <cuda_runtime.h>

#include "cvt.cuh"

namespace gwi {
namespace arith {

__device__ __forceinline__ double2 cinv_d(double2 a) {
  const double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}

struct Fp64 {
  static constexpr int kBlocksPerSm = 1;  // occupancy target of the register-tiled screening kernel
  using S = double2;    // stored value (workspace, shared memory)
  using Acc = double2;  // accumulator
  __device__ static S from(double re, double im) { return make_double2(re, im); }
  __device__ static double2 to(S v) { return v; }
  __device__ static S zero() { return make_double2(0.0, 0.0); }
  __device__ static Acc azero() { return make_double2(0.0, 0.0); }
  __device__ static bool is_zero(S v) { return v.x == 0.0 && v.y == 0.0; }
  __device__ static void mac(Acc& a, S l, S u) {  // a += l u
    a.x = fma(l.x, u.x, fma(-l.y, u.y, a.x));
    a.y = fma(l.x, u.y, fma(l.y, u.x, a.y));
  }
  __device__ static S val(Acc a) { return a; }
  __device__ static S sub(S b, Acc a) { return make_double2(b.x - a.x, b.y - a.y); }  // b - a
  __device__ static S inv(S v) { return cinv_d(v); }
  using R = double;  // stored real coefficient
  __device__ static R rfrom(double x) { return x; }
  __device__ static S add(S a, S b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static S dif(S a, S b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ static S half(S a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
  __device__ static S mul_mi(S a) { return make_double2(a.y, -a.x); }  // -i a
  // acc.re += A g.re + B g.im, acc.im += A h.re + B h.im
  __device__ static void rmac2(Acc& acc, R A, R B, S g, S h) {
    acc.x = fma(A, g.x, fma(B, g.y, acc.x));
    acc.y = fma(A, h.x, fma(B, h.y, acc.y));
  }
};

struct F32 {
  static constexpr int kBlocksPerSm = 2;
  using S = float2;
  using Acc = float2;
  __device__ static S from(double re, double im) { return make_float2(cvt::d2f(re), cvt::d2f(im)); }
  __device__ static double2 to(S v) { return make_double2((double)v.x, (double)v.y); }
  __device__ static S zero() { return make_float2(0.f, 0.f); }
  __device__ static Acc azero() { return make_float2(0.f, 0.f); }
  __device__ static bool is_zero(S v) { return v.x == 0.f && v.y == 0.f; }
  __device__ static void mac(Acc& a, S l, S u) {  // a += l u
    a.x = fmaf(l.x, u.x, fmaf(-l.y, u.y, a.x));
    a.y = fmaf(l.x, u.y, fmaf(l.y, u.x, a.y));
  }
  __device__ static S val(Acc a) { return a; }
  __device__ static S sub(S b, Acc a) { return make_float2(b.x - a.x, b.y - a.y); }  // b - a
  __device__ static S inv(S v) {  // one reciprocal per pivot: in FP64
    const double2 r = cinv_d(to(v));
    return from(r.x, r.y);
  }
};

struct Ff32 {
  static constexpr int kBlocksPerSm = 1;
  struct __align__(16) S {
    float rh, rl, ih, il;
  };
  using Acc = S;
  __device__ static S from(double re, double im) {  // hi = RN(x), lo = RN(x - hi), on the integer pipes
    S v;
    cvt::d2ff(re, v.rh, v.rl);
    cvt::d2ff(im, v.ih, v.il);
    return v;
  }
  __device__ static double2 to(S v) {
    return make_double2((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
  }
  __device__ static S zero() { return {0.f, 0.f, 0.f, 0.f}; }
  __device__ static Acc azero() { return {0.f, 0.f, 0.f, 0.f}; }
  __device__ static bool is_zero(S v) { return v.rh == 0.f && v.ih == 0.f; }
  // h + l += (xh + xl)(yh + yl), dropping xl yl
  __device__ __forceinline__ static void ffmac(float& h, float& l, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);  // never contracted into an FMA with the sum below
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    const float s = h + p;
    const float v = s - h;
    const float err = (h - (s - v)) + (p - v);
    h = s;
    l += err + e;
  }
  __device__ static void mac(Acc& a, S x, S y) {
    ffmac(a.rh, a.rl, x.rh, x.rl, y.rh, y.rl);
    ffmac(a.rh, a.rl, -x.ih, -x.il, y.ih, y.il);
    ffmac(a.ih, a.il, x.rh, x.rl, y.ih, y.il);
    ffmac(a.ih, a.il, x.ih, x.il, y.rh, y.rl);
  }
  __device__ __forceinline__ static void renorm(float& h, float& l) {
    const float s = h + l;
    l = l - (s - h);
    h = s;
  }
  __device__ static S val(Acc a) {
    renorm(a.rh, a.rl);
    renorm(a.ih, a.il);
    return a;
  }
  __device__ __forceinline__ static void ffsub(float bh, float bl, float ah, float al, float& h, float& l) {
    const float s = bh - ah;
    const float v = s - bh;
    const float err = (bh - (s - v)) + (-ah - v);
    h = s;
    l = err + (bl - al);
    renorm(h, l);
  }
  __device__ static S sub(S b, Acc a) {
    S r;
    ffsub(b.rh, b.rl, a.rh, a.rl, r.rh, r.rl);
    ffsub(b.ih, b.il, a.ih, a.il, r.ih, r.il);
    return r;
  }
  __device__ static S inv(S v) {  // one reciprocal per pivot: in FP64
    const double2 d = to(v);
    const double2 r = cinv_d(d);
    return from(r.x, r.y);
  }
  struct __align__(8) R {
    float h, l;
  };
  __device__ static R rfrom(double x) {
    R r;
    cvt::d2ff(x, r.h, r.l);
    return r;
  }
  __device__ __forceinline__ static void ffadd(float ah, float al, float bh, float bl, float& h, float& l) {
    const float s = ah + bh;
    const float v = s - ah;
    const float err = (ah - (s - v)) + (bh - v);
    h = s;
    l = err + (al + bl);
    renorm(h, l);
  }
  __device__ static S add(S a, S b) {
    S r;
    ffadd(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
    ffadd(a.ih, a.il, b.ih, b.il, r.ih, r.il);
    return r;
  }
  __device__ static S dif(S a, S b) {
    S r;
    ffadd(a.rh, a.rl, -b.rh, -b.rl, r.rh, r.rl);
    ffadd(a.ih, a.il, -b.ih, -b.il, r.ih, r.il);
    return r;
  }
  __device__ static S half(S a) { return {0.5f * a.rh, 0.5f * a.rl, 0.5f * a.ih, 0.5f * a.il}; }
  __device__ static S mul_mi(S a) { return {a.ih, a.il, -a.rh, -a.rl}; }
  __device__ static void rmac2(Acc& acc, R A, R B, S g, S h) {
    ffmac(acc.rh, acc.rl, A.h, A.l, g.rh, g.rl);
    ffmac(acc.rh, acc.rl, B.h, B.l, g.ih, g.il);
    ffmac(acc.ih, acc.il, A.h, A.l, h.rh, h.rl);
    ffmac(acc.ih, acc.il, B.h, B.l, h.ih, h.il);
  }
};

}  // namespace arith
}  // namespace gwi
