// Crystal-symmetry reduction of the self-energy (Sec. III.C): the contribution of q' = R q to
// Sigma_n(k) is the contribution of q at R^-1 k, so with P, W~ and the self-energy computed for
// the irreducible q points only, each one's contribution T[k'] (all k' of the mesh) is carried to
// the members of its star:  S[k] += sum_r T[kinv_r(k)],  kinv_r(k) = index of R_r^-1 k.
// One thread per (k, column); the sum over r in the given order (deterministic).
#include <cuda_runtime.h>

#include "gw_internal.h"

namespace gwi {
namespace {

__global__ void k_sigma_star(int nrep, const int* __restrict__ kinv, int nk, int64_t ncol,
                             const double* __restrict__ T, double* __restrict__ S) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nk * ncol) return;
  const int k = (int)(e / ncol);
  const int64_t col = e % ncol;
  double s = 0.0;
  for (int r = 0; r < nrep; ++r) {
    const int src = kinv[(size_t)r * nk + k];
    if ((unsigned)src < (unsigned)nk) s += T[(size_t)src * ncol + col];  // out-of-range entries are skipped
  }
  S[e] += s;
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" gw_status gw_sigma_star(gw_ctx* c, int nrep, const int* kinv, int64_t ncol, const double* T, double* S) {
  if (!c || nrep < 1 || !kinv || ncol < 1 || !T || !S) return GW_EINVAL;
  const int64_t n = (int64_t)c->nk * ncol;
  k_sigma_star<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(nrep, kinv, c->nk, ncol, T, S);
  return check_launch(c, "sigma_star");
}
