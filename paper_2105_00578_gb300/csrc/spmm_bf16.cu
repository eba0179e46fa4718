// spmm_bf16.cu -- instantiations of the Laplacian SpMM for bfloat16 blocks
// (products accumulate in float).
#include "spmm_kernels.cuh"

namespace sphynx {
void spmm_dispatch_bf16(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d) {
  if (a.mode == 0) spmm_lapw<__nv_bfloat16, __nv_bfloat16, 0>(g, d, a.lap, a.bp);
  else spmm_lapw<__nv_bfloat16, __nv_bfloat16, 1>(g, d, a.lap, a.bp);
}
}  // namespace sphynx
