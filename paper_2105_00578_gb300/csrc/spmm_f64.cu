// spmm_f64.cu -- instantiations of the Laplacian SpMM for double blocks.
#include "spmm_kernels.cuh"

namespace sphynx {
void spmm_dispatch_f64(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d) {
  if (a.mode == 0) spmm_lapw<double, double, 0>(g, d, a.lap, a.bp);
  else spmm_lapw<double, double, 1>(g, d, a.lap, a.bp);
}
}  // namespace sphynx
