// Tensor-core (tcgen05) split-precision contractions. Placeholder until the
// kernels land: the mixed precisions report GW_EUNSUPPORTED.
#include <cuda_runtime.h>

#include "gw_internal.h"

namespace gwi {

gw_status launch_pol_mixed(gw_ctx* c, int, const double*, int, double*) {
  return set_err(c, GW_EUNSUPPORTED, "mixed-precision polarization not built");
}
gw_status launch_sigma_mixed(gw_ctx* c, int, const double*, const double*, int, double*) {
  return set_err(c, GW_EUNSUPPORTED, "mixed-precision self-energy not built");
}
void free_mixed(gw_ctx* c) {
  if (c->mw.mslices) cudaFree(c->mw.mslices);
  if (c->mw.wslices) cudaFree(c->mw.wslices);
  if (c->mw.dacc) cudaFree(c->mw.dacc);
  c->mw = MixedWork();
}

}  // namespace gwi
