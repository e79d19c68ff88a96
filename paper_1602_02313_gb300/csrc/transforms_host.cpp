// Host construction of the imaginary-time <-> Matsubara transform matrices.
//
// The paper transforms Sigma(tau) -> Sigma(i w_n) = int_0^beta e^{i w_n tau} Sigma(tau) dtau
// (Eq. trans). With the screening posed at bosonic Matsubara frequencies, the GPU
// path also needs tau -> i nu, i nu -> tau and i w -> tau. All maps come from one
// model: a real tau-function on [0, beta] is a sum of Lehmann kernels
//     K(tau, E) = exp(-E tau) / (1 + exp(-beta E))      (E >= 0)
//               = exp(E (beta - tau)) / (1 + exp(beta E)) (E < 0)
// whose Matsubara transforms are closed form:
//     fermionic  -1 / (i w - E)
//     bosonic    -tanh(beta E / 2) / (i nu - E)     (beta/2 at nu = E = 0).
// forward : least-squares fit of the tau samples, evaluated at the frequencies;
// backward: least-squares fit (real coefficients) of Re/Im of the frequency
//           samples, evaluated at the tau nodes.
// The fits are ill-conditioned (cond ~ 1e9 on Gauss-Legendre-in-log grids), so
// everything is formed in double-double arithmetic (Dekker 1971; Knuth TwoSum;
// FMA-based TwoProd) with Householder QR, and rounded to FP64 once at the end.
#include <cmath>
#include <vector>

#include "gw_internal.h"

namespace gwi {
namespace {

struct dd {
  double hi, lo;
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline dd mk(double a) { return {a, 0.0}; }
inline dd add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline dd neg(dd a) { return {-a.hi, -a.lo}; }
inline dd sub(dd a, dd b) { return add(a, neg(b)); }
inline dd mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
inline dd mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
inline dd div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = sub(a, mul_d(b, q1));
  double q2 = r.hi / b.hi;
  r = sub(r, mul_d(b, q2));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return add(q, mk(q3));
}
inline dd sqrt_dd(dd a) {
  if (a.hi <= 0.0) return mk(0.0);
  double x = std::sqrt(a.hi);
  dd x2 = two_prod(x, x);
  dd r = sub(a, x2);
  return add(mk(x), mk(r.hi / (2.0 * x)));
}
inline double to_d(dd a) { return a.hi + a.lo; }

const dd kLn2 = {0.6931471805599453, 2.3190468138462996e-17};
const dd kPi = {3.141592653589793, 1.2246467991473532e-16};

// exp in double-double: x = k ln2 + r, exp(r) = (exp(r / 1024))^1024, with a
// 14-term Taylor series (exact division by n) for the reduced argument.
dd exp_dd_exact(dd x) {
  if (x.hi < -740.0) return mk(0.0);
  double k = std::nearbyint(x.hi / kLn2.hi);
  dd r = sub(x, mul_d(kLn2, k));
  r = mul_d(r, 1.0 / 1024.0);
  dd term = mk(1.0), sum = mk(1.0);
  for (int n = 1; n <= 14; ++n) {
    term = div(mul(term, r), mk((double)n));
    sum = add(sum, term);
  }
  for (int i = 0; i < 10; ++i) sum = mul(sum, sum);
  return {std::ldexp(sum.hi, (int)k), std::ldexp(sum.lo, (int)k)};
}

dd kernel_tau(dd tau, dd E, dd beta) {
  dd one = mk(1.0);
  if (E.hi >= 0) return div(exp_dd_exact(neg(mul(E, tau))), add(one, exp_dd_exact(neg(mul(beta, E)))));
  return div(exp_dd_exact(mul(E, sub(beta, tau))), add(one, exp_dd_exact(mul(beta, E))));
}

// (re, im) of the Matsubara transform of K(., E) at index n.
void kernel_hat(int n, dd E, dd beta, bool fermionic, dd* re, dd* im) {
  dd z = div(mul_d(kPi, (double)(fermionic ? 2 * n + 1 : 2 * n)), beta);
  dd den = add(mul(z, z), mul(E, E));
  if (fermionic) {
    *re = div(E, den);
    *im = div(z, den);
    return;
  }
  if (n == 0 && E.hi == 0.0) {
    *re = mul_d(beta, 0.5);
    *im = mk(0.0);
    return;
  }
  dd one = mk(1.0), th;
  if (E.hi >= 0) {
    dd x = exp_dd_exact(neg(mul(beta, E)));
    th = div(sub(one, x), add(one, x));
  } else {
    dd x = exp_dd_exact(mul(beta, E));
    th = neg(div(sub(one, x), add(one, x)));
  }
  *re = div(mul(th, E), den);
  *im = div(mul(th, z), den);
}

// Pseudo-inverse (p x m, row-major) of the m x p matrix A (row-major, m >= p)
// by Householder QR: A = Q R, pinv = R^{-1} Q^T.
std::vector<dd> pinv(const std::vector<dd>& Ain, int m, int p) {
  std::vector<dd> A = Ain;                       // m x p, overwritten by R
  std::vector<dd> QT(m * (size_t)m, mk(0.0));    // accumulates Q^T applied to I
  for (int i = 0; i < m; ++i) QT[i * (size_t)m + i] = mk(1.0);
  std::vector<dd> v(m);
  for (int j = 0; j < p; ++j) {
    dd nrm2 = mk(0.0);
    for (int i = j; i < m; ++i) nrm2 = add(nrm2, mul(A[i * (size_t)p + j], A[i * (size_t)p + j]));
    dd nrm = sqrt_dd(nrm2);
    if (nrm.hi == 0.0) continue;
    dd alpha = A[j * (size_t)p + j].hi >= 0 ? neg(nrm) : nrm;
    for (int i = 0; i < m; ++i) v[i] = mk(0.0);
    v[j] = sub(A[j * (size_t)p + j], alpha);
    for (int i = j + 1; i < m; ++i) v[i] = A[i * (size_t)p + j];
    dd vv = mk(0.0);
    for (int i = j; i < m; ++i) vv = add(vv, mul(v[i], v[i]));
    if (vv.hi == 0.0) continue;
    dd two_over = div(mk(2.0), vv);
    for (int c = j; c < p; ++c) {
      dd s = mk(0.0);
      for (int i = j; i < m; ++i) s = add(s, mul(v[i], A[i * (size_t)p + c]));
      s = mul(s, two_over);
      for (int i = j; i < m; ++i) A[i * (size_t)p + c] = sub(A[i * (size_t)p + c], mul(s, v[i]));
    }
    for (int c = 0; c < m; ++c) {
      dd s = mk(0.0);
      for (int i = j; i < m; ++i) s = add(s, mul(v[i], QT[i * (size_t)m + c]));
      s = mul(s, two_over);
      for (int i = j; i < m; ++i) QT[i * (size_t)m + c] = sub(QT[i * (size_t)m + c], mul(s, v[i]));
    }
  }
  // solve R X = (Q^T)[0:p, :] by back substitution
  std::vector<dd> X(p * (size_t)m);
  for (int c = 0; c < m; ++c) {
    for (int r = p - 1; r >= 0; --r) {
      dd s = QT[r * (size_t)m + c];
      for (int t = r + 1; t < p; ++t) s = sub(s, mul(A[r * (size_t)p + t], X[t * (size_t)m + c]));
      X[r * (size_t)m + c] = div(s, A[r * (size_t)p + r]);
    }
  }
  return X;
}

}  // namespace

void build_transforms(const std::vector<double>& tau_d, const std::vector<double>& poles_d, double beta_d,
                      const std::vector<int>& nu_idx, const std::vector<int>& w_idx, int ncont,
                      Transforms* out) {
  const int nt = (int)tau_d.size(), np = (int)poles_d.size();
  const dd beta = mk(beta_d);
  std::vector<dd> E(np), tau(nt);
  for (int l = 0; l < np; ++l) E[l] = mk(poles_d[l]);
  for (int i = 0; i < nt; ++i) tau[i] = mk(tau_d[i]);
  std::vector<dd> Kt(nt * (size_t)np);
  for (int i = 0; i < nt; ++i)
    for (int l = 0; l < np; ++l) Kt[i * (size_t)np + l] = kernel_tau(tau[i], E[l], beta);
  std::vector<dd> Kbeta(np);
  for (int l = 0; l < np; ++l) Kbeta[l] = kernel_tau(beta, E[l], beta);
  std::vector<dd> Ktp = pinv(Kt, nt, np);  // np x nt

  auto fwd = [&](const std::vector<int>& idx, bool ferm, std::vector<double>* o) {
    const int nf = (int)idx.size();
    o->assign(2 * (size_t)nf * nt, 0.0);
    std::vector<dd> hre(np), him(np);
    for (int j = 0; j < nf; ++j) {
      for (int l = 0; l < np; ++l) kernel_hat(idx[j], E[l], beta, ferm, &hre[l], &him[l]);
      for (int i = 0; i < nt; ++i) {
        dd sr = mk(0.0), si = mk(0.0);
        for (int l = 0; l < np; ++l) {
          sr = add(sr, mul(hre[l], Ktp[l * (size_t)nt + i]));
          si = add(si, mul(him[l], Ktp[l * (size_t)nt + i]));
        }
        (*o)[2 * ((size_t)j * nt + i)] = to_d(sr);
        (*o)[2 * ((size_t)j * nt + i) + 1] = to_d(si);
      }
    }
  };
  auto bwd = [&](const std::vector<int>& idx, bool ferm, std::vector<double>* o, std::vector<double>* obeta) {
    const int nf = (int)idx.size();
    const int m = 2 * nf;
    std::vector<dd> H(m * (size_t)np);
    for (int j = 0; j < nf; ++j)
      for (int l = 0; l < np; ++l) {
        dd re, im;
        kernel_hat(idx[j], E[l], beta, ferm, &re, &im);
        H[j * (size_t)np + l] = re;
        H[(nf + j) * (size_t)np + l] = im;
      }
    std::vector<dd> Hp = pinv(H, m, np);  // np x m
    o->assign((size_t)nt * m, 0.0);
    for (int i = 0; i < nt; ++i)
      for (int c = 0; c < m; ++c) {
        dd s = mk(0.0);
        for (int l = 0; l < np; ++l) s = add(s, mul(Kt[i * (size_t)np + l], Hp[l * (size_t)m + c]));
        (*o)[(size_t)i * m + c] = to_d(s);
      }
    if (obeta) {
      obeta->assign(m, 0.0);
      for (int c = 0; c < m; ++c) {
        dd s = mk(0.0);
        for (int l = 0; l < np; ++l) s = add(s, mul(Kbeta[l], Hp[l * (size_t)m + c]));
        (*obeta)[c] = to_d(s);
      }
    }
  };
  fwd(nu_idx, false, &out->B_fwd);
  fwd(w_idx, true, &out->F_fwd);
  std::vector<int> cont(ncont);
  for (int n = 0; n < ncont; ++n) cont[n] = n;
  fwd(cont, true, &out->F_cont);
  bwd(nu_idx, false, &out->B_bwd, nullptr);
  bwd(w_idx, true, &out->F_bwd, &out->F_bwd_beta);
}

}  // namespace gwi
