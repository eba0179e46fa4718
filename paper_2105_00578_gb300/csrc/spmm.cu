// spmm.cu -- host entry of the Laplacian SpMM: argument checks, byte and
// time accounting, dispatch to the per-type instantiations.
#include "spmm_kernels.cuh"

namespace sphynx {

void spmm(sphynx_graph *g, const SpmmArgs &a) {
  if (!(a.bp == 1 || a.bp == 4 || a.bp == 8 || a.bp == 12 || a.bp == 16))
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: block width %d", a.bp);
  if (a.ld_x < a.bp || (a.mode == 0 && a.ld_y < a.bp) || (a.mode == 1 && a.ld_y < a.bp))
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: leading dimension smaller than block width");
  if (a.mode == 1 && a.tin == DT::F64 && a.tout != DT::F64)
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: double chain must stay double");
  SpmmDev d{a.x, a.ld_x, a.ld_y, a.y, a.t_out, a.yacc, a.first, a.inv, a.i_cur, a.done};

  // algorithmic bytes: row pointers, column indices (+ weights), X once,
  // the diagonal / D^{-1/2} vector, and the outputs
  const double n = static_cast<double>(g->n), nnz = static_cast<double>(g->nnz);
  const double si = static_cast<double>(dt_size(a.tin));
  const double sa = a.tin == DT::F64 ? 8.0 : 4.0;
  const double b = static_cast<double>(a.b_true);
  double bytes = 8.0 * (n + 1) + nnz * (g->weighted ? 8.0 : 4.0) + n * b * si + n * sa;
  if (a.mode == 0) {
    bytes += n * b * sa;
  } else {
    bytes += n * b * static_cast<double>(dt_size(a.tout)) + n * b * sa * (a.first ? 1.0 : 2.0);
  }
  g->ctr.spmm_bytes += bytes;
  g->ctr.spmm_launches += 1;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g->ctr.timing) {
    if (g->ctr.ev_used + 2 > g->ctr.ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        SPX_CUDA(cudaEventCreate(&e));
        g->ctr.ev_pool.push_back(e);
      }
    }
    e0 = g->ctr.ev_pool[g->ctr.ev_used++];
    e1 = g->ctr.ev_pool[g->ctr.ev_used++];
    SPX_CUDA(cudaEventRecord(e0, g->stream));
  }
  switch (a.tin) {
    case DT::F64: spmm_dispatch_f64(g, a, d); break;
    case DT::F32: spmm_dispatch_f32(g, a, d); break;
    case DT::BF16: spmm_dispatch_bf16(g, a, d); break;
  }
  if (g->ctr.timing) SPX_CUDA(cudaEventRecord(e1, g->stream));
}

}  // namespace sphynx
