// spmm_f32.cu -- instantiations of the Laplacian SpMM for float blocks
// (the polynomial chain may hand its next vector on in bfloat16).
#include "spmm_kernels.cuh"

namespace sphynx {
void spmm_dispatch_f32(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d) {
  if (a.mode == 0) spmm_lapw<float, float, 0>(g, d, a.lap, a.bp);
  else if (a.tout == DT::BF16) spmm_lapw<float, __nv_bfloat16, 1>(g, d, a.lap, a.bp);
  else spmm_lapw<float, float, 1>(g, d, a.lap, a.bp);
}
}  // namespace sphynx
