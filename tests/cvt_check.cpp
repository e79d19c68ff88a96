// Host check of the integer-pipe conversions in cvt.cuh against the host's IEEE 754
// conversions (round to nearest, ties to even): every class of input, both words, bit for bit.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "cvt.cuh"

using gwi::cvt::d2f;
using gwi::cvt::d2ff;

static uint32_t fb(float f) {
  uint32_t u;
  std::memcpy(&u, &f, sizeof u);
  return u;
}
static double mk(uint64_t sign, uint64_t E, uint64_t mant) {
  const uint64_t u = (sign << 63) | (E << 52) | (mant & ((1ull << 52) - 1));
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
}

static long n_checked = 0, n_bad = 0;

static bool same(float a, float b) { return (std::isnan(a) && std::isnan(b)) || fb(a) == fb(b); }

static void check(double x) {
  ++n_checked;
  const float h_ref = (float)x;
  const float l_ref = std::isfinite(x) && std::isfinite(h_ref) ? (float)(x - (double)h_ref) : 0.f;
  const float h1 = d2f(x);
  float h2, l2;
  d2ff(x, h2, l2);
  bool ok = same(h1, h_ref) && same(h2, h_ref);
  if (std::isfinite(x) && std::isfinite(h_ref)) ok = ok && same(l2, l_ref);
  if (!ok && n_bad++ < 10)
    std::printf("mismatch x=%a: d2f %a d2ff (%a, %a), expected (%a, %a)\n", x, h1, h2, l2, h_ref, l_ref);
}

int main() {
  std::mt19937_64 rng(12345);
  // random bit patterns over every exponent, both signs
  for (uint64_t E = 0; E < 2048; ++E)
    for (int i = 0; i < 2000; ++i) check(mk(rng() & 1, E, rng()));
  // the rounding boundaries of the 29 dropped bits, with even and odd kept significands,
  // including the all-ones significand whose rounding carries into the exponent
  const uint64_t tails[] = {0x0000000ull, 0x0000001ull, 0x0FFFFFFFull, 0x10000000ull, 0x10000001ull,
                            0x1FFFFFFFull};
  const uint64_t heads[] = {0ull, 1ull, 2ull, 3ull, (1ull << 23) - 2, (1ull << 23) - 1, 0x2AAAAAull};
  for (uint64_t E = 890; E < 1160; ++E)
    for (uint64_t s = 0; s < 2; ++s)
      for (uint64_t hd : heads)
        for (uint64_t tl : tails) check(mk(s, E, (hd << 29) | tl));
  // zeros, subnormals, the largest finite doubles, infinities, nan
  check(0.0);
  check(-0.0);
  check(mk(0, 0, 1));
  check(mk(1, 0, 12345));
  check(mk(0, 2046, ~0ull));
  check(INFINITY);
  check(-INFINITY);
  check(NAN);
  // values of the workload's magnitudes
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int i = 0; i < 1000000; ++i) check(nd(rng) * std::pow(10.0, (double)(i % 17) - 8.0));
  // float -> double widening, bit for bit against the host's conversion, every float exponent
  for (uint32_t e = 0; e < 256; ++e)
    for (int i = 0; i < 4000; ++i) {
      const uint32_t u = ((uint32_t)(rng() & 1) << 31) | (e << 23) | (uint32_t)(rng() & 0x7FFFFFu);
      float f;
      std::memcpy(&f, &u, sizeof f);
      const double a = gwi::cvt::f2d(f), b = (double)f;
      ++n_checked;
      uint64_t ua, ub;
      std::memcpy(&ua, &a, sizeof ua);
      std::memcpy(&ub, &b, sizeof ub);
      if (!(ua == ub || (std::isnan(a) && std::isnan(b))) && n_bad++ < 10) std::printf("f2d mismatch %a\n", (double)f);
    }
  std::printf("checked %ld values, %ld mismatches\n", n_checked, n_bad);
  return n_bad ? 1 : 0;
}
