// spmm.cu -- host entry of the Laplacian SpMM: argument checks, the
// per-shape autotuner, byte and time accounting, dispatch to the per-type
// instantiations.
#include "spmm_kernels.cuh"

namespace sphynx {

namespace {

// z = D^{-1/2} x for the normalized product's gathers: rows of bp values
// (bp a multiple of 4, or 1), one 16-byte quarter-row (float) or 16-byte pair
// (double) a thread
template <typename T, int V>
__global__ void k_prescale(const T *__restrict__ x, const T *__restrict__ dinv, int64_t n, int bp, T *__restrict__ z) {
  const int per_row = bp / V;   // vectors a row
  const int64_t total = n * per_row;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < total;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = k / per_row;
    const T s = __ldg(dinv + row);
    if constexpr (V == 4) {
      float4 v = __ldg(reinterpret_cast<const float4 *>(x) + k);
      v.x *= s; v.y *= s; v.z *= s; v.w *= s;
      reinterpret_cast<float4 *>(z)[k] = v;
    } else if constexpr (V == 2) {
      double2 v = __ldg(reinterpret_cast<const double2 *>(x) + k);
      v.x *= s; v.y *= s;
      reinterpret_cast<double2 *>(z)[k] = v;
    } else {
      z[k] = s * x[k];
    }
  }
}

// c_k = (w_k or 1) * dinv[col_k] in float, the kernels' own rounding of the
// normalized coefficient
__global__ void k_ncoef_csr(const int32_t *__restrict__ col, const float *__restrict__ w,
                            const float *__restrict__ dinvf, int64_t nnz, float *__restrict__ c) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < nnz;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float wk = w ? w[k] : 1.f;
    c[k] = wk * dinvf[col[k]];
  }
}

// the short rows' coefficients into SELL slot order (the layout of sell_w)
__global__ void k_ncoef_sell(const int64_t *__restrict__ rp, const float *__restrict__ c, int64_t n,
                             const uint8_t *__restrict__ sdeg, const int64_t *__restrict__ sptr, float *__restrict__ cs) {
  const int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (row >= n) return;
  const int d = sdeg[row];
  if (d == 0xFF) return;
  const int64_t b = sptr[row >> 5] + (row & 31), src = rp[row];
  for (int t = 0; t < d; ++t) cs[b + 32 * t] = c[src + t];
}

void ensure_ncoef(sphynx_graph *g) {
  SpmmPlan &p = g->plan;
  if (p.ncoef_csr.p) return;
  p.ncoef_csr.alloc(static_cast<size_t>(g->nnz > 0 ? g->nnz : 1) * sizeof(float));
  p.ncoef_sell.alloc(static_cast<size_t>(p.sell_entries > 0 ? p.sell_entries : 1) * sizeof(float));
  const unsigned gc = static_cast<unsigned>(std::min<int64_t>((g->nnz + 255) / 256, 16 * kSmCount));
  if (g->nnz > 0) {
    k_ncoef_csr<<<gc, 256, 0, g->stream>>>(g->col, g->w, g->dinvf.as<float>(), g->nnz, p.ncoef_csr.as<float>());
    SPX_LAUNCHED();
  }
  k_ncoef_sell<<<static_cast<unsigned>((g->n + 255) / 256), 256, 0, g->stream>>>(
      g->rowptr, p.ncoef_csr.as<float>(), g->n, p.sell_deg.as<uint8_t>(), p.sell_ptr.as<int64_t>(),
      p.ncoef_sell.as<float>());
  SPX_LAUNCHED();
  g->ctr.launches += 2;
}

void dispatch(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d) {
  switch (a.tin) {
    case DT::F64: spmm_dispatch_f64(g, a, d); break;
    case DT::F32: spmm_dispatch_f32(g, a, d); break;
    case DT::BF16: spmm_dispatch_bf16(g, a, d); break;
  }
}

// The caller's product redirected to scratch outputs (a polynomial step's
// accumulator is read and written, so the real one must not be touched).
SpmmDev tune_args(sphynx_graph *g, const SpmmArgs &a) {
  const size_t out_bytes = static_cast<size_t>(g->n) * a.ld_y * 8 + 256;
  const size_t t_bytes = static_cast<size_t>(g->n) * a.ld_x * 8 + 256;
  if (g->plan.tune_scratch.bytes < out_bytes + t_bytes) g->plan.tune_scratch.alloc(out_bytes + t_bytes);
  char *base = g->plan.tune_scratch.as<char>();
  SPX_CUDA(cudaMemsetAsync(base, 0, out_bytes + t_bytes, g->stream));
  SpmmArgs s = a;
  if (a.mode == 0) {
    s.y = base;
  } else {
    s.yacc = base;
    s.t_out = base + out_bytes;
  }
  return SpmmDev{s.x,      s.ld_x, s.ld_y, s.y,     s.t_out,      s.yacc,       s.first,   s.yterms,
                 s.inv,    s.invf, s.i_cur, nullptr, s.row_graph, s.inv_stride, nullptr, nullptr, s.x, nullptr, nullptr};
}

}  // namespace

// Time both short-row schedules for this product with the caller's input
// and scratch outputs, alternating them over five rounds, and return the
// faster.
SpmmTuning spmm_tune(sphynx_graph *g, const SpmmArgs &a) {
  const SpmmArgs &s = a;
  const SpmmDev d = tune_args(g, a);
  cudaEvent_t e0, e1;
  SPX_CUDA(cudaEventCreate(&e0));
  SPX_CUDA(cudaEventCreate(&e1));
  SpmmTuning t{kCsrStaged, {1e30f, 1e30f, 1e30f}};
  const int64_t launches = g->ctr.launches;
  const int nv = g->plan.pat_slices > 0 ? 3 : 2;   // the shared-pattern layout exists on some graphs only
  for (int v = 0; v < nv; ++v) {   // warm-up of each
    g->plan.variant = v;
    dispatch(g, s, d);
  }
  // alternate the schedules so that neither always runs on a warmer L2
  for (int round = 0; round < 5; ++round) {
    for (int k = 0; k < nv; ++k) {
      const int v = (round + k) % nv;
      g->plan.variant = v;
      SPX_CUDA(cudaEventRecord(e0, g->stream));
      dispatch(g, s, d);
      SPX_CUDA(cudaEventRecord(e1, g->stream));
      SPX_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      SPX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      t.us[v] = ms * 1000.f < t.us[v] ? ms * 1000.f : t.us[v];
    }
  }
  g->ctr.launches = launches;   // tuning launches are not part of the caller's work
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  t.variant = kCsrStaged;
  for (int v = 1; v < nv; ++v)
    if (t.us[v] < t.us[t.variant]) t.variant = v;
  return t;
}

// Time the SELL schedule under every slice stride 2^ls (ls < kSellLsCount),
// rotating the order over five rounds, and keep the fastest in plan.sell_ls.
// Strides change only which block runs a slice, never a product's value.
void spmm_tune_sell_stride(sphynx_graph *g, const SpmmArgs &a) {
  const SpmmDev d = tune_args(g, a);
  cudaEvent_t e0, e1;
  SPX_CUDA(cudaEventCreate(&e0));
  SPX_CUDA(cudaEventCreate(&e1));
  const int64_t launches = g->ctr.launches;
  const int variant = g->plan.variant;
  // the SELL schedule in force (pinned, else tuned); plain SELL-32 when that is CSR
  const int sv = g->plan.forced > 0 ? g->plan.forced : g->plan.tuned_variant;
  g->plan.variant = sv == kSellPattern ? kSellPattern : kSell32;
  float us[kSellLsCount];
  for (int k = 0; k < kSellLsCount; ++k) {   // warm-up of each
    us[k] = 1e30f;
    g->plan.sell_ls = k;
    dispatch(g, a, d);
  }
  for (int round = 0; round < 5; ++round) {
    for (int k = 0; k < kSellLsCount; ++k) {
      const int ls = (round + k) % kSellLsCount;
      g->plan.sell_ls = ls;
      SPX_CUDA(cudaEventRecord(e0, g->stream));
      dispatch(g, a, d);
      SPX_CUDA(cudaEventRecord(e1, g->stream));
      SPX_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      SPX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      us[ls] = ms * 1000.f < us[ls] ? ms * 1000.f : us[ls];
    }
  }
  g->ctr.launches = launches;
  g->plan.variant = variant;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int best = 0;
  for (int k = 0; k < kSellLsCount; ++k) {
    g->plan.tuned_ls_us[k] = us[k];
    if (us[k] < us[best]) best = k;
  }
  g->plan.sell_ls = best;
}

void spmm(sphynx_graph *g, const SpmmArgs &a) {
  if (!(a.bp == 1 || a.bp == 4 || a.bp == 8 || a.bp == 12 || a.bp == 16))
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: block width %d", a.bp);
  // the kernels index X (and the chain's output) with the compile-time width:
  // a runtime stride costs a 64-bit multiply per gather (about a third of the
  // chain step's time)
  if (a.ld_x != a.bp) fail(SPHYNX_ERR_INVALID_ARG, "spmm: input rows must be exactly the block width apart");
  if ((a.mode == 0 && a.ld_y < a.bp) || (a.mode == 1 && a.ld_y < a.bp))
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: leading dimension smaller than block width");
  if (a.mode == 1 && a.tin == DT::F64 && a.tout != DT::F64)
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: double chain must stay double");
  // gathers are 16-byte vector loads (8-byte for bfloat16 rows of 4 or 12)
  if (a.bp > 1) {
    const size_t row_bytes = static_cast<size_t>(a.ld_x) * dt_size(a.tin);
    const size_t need = (a.tin == DT::BF16 && a.bp % 8 != 0) ? 8 : 16;
    if (row_bytes % need || reinterpret_cast<uintptr_t>(a.x) % need)
      fail(SPHYNX_ERR_INVALID_ARG, "spmm: input rows must be %zu-byte aligned", need);
  }
  if (a.mode == 1 && (a.yterms < 0 || a.yterms > 2 || (a.first && a.yterms != 2)))
    fail(SPHYNX_ERR_INVALID_ARG, "spmm: polynomial step adds 0, 1 or 2 terms (2 on the first step)");
  SpmmDev d{a.x,   a.ld_x, a.ld_y, a.y,      a.t_out,    a.yacc,        a.first,  a.yterms,
            a.inv, a.invf, a.i_cur, a.done, a.row_graph, a.inv_stride, a.act_blocks, a.n_act, a.x, nullptr, nullptr};
  const bool prescaled = g->plan.prescale && a.lap == SPHYNX_NORMALIZED && a.tin != DT::BF16 && g->n > 0;
  const bool coefs = g->plan.prescale && a.lap == SPHYNX_NORMALIZED && a.tin == DT::BF16 && g->n > 0;
  if (coefs) {
    ensure_ncoef(g);
    d.coef_csr = g->plan.ncoef_csr.as<float>();
    d.coef_sell = g->plan.ncoef_sell.as<float>();
  }

  // schedule: forced, or the one the autotuner chose for this graph at create
  g->plan.variant = g->plan.forced >= 0 ? g->plan.forced : g->plan.tuned_variant;

  // algorithmic bytes: the graph in the layout the schedule reads (CSR row
  // pointers and indices, or the SELL-32 slices plus the long rows' CSR
  // entries; weights when present), X once, the diagonal / D^{-1/2} vector,
  // and the outputs
  const double n = static_cast<double>(g->n), nnz = static_cast<double>(g->nnz);
  const double si = static_cast<double>(dt_size(a.tin));
  const double sa = a.tin == DT::F64 ? 8.0 : 4.0;
  const double b = static_cast<double>(a.b_true);
  const double graph_bytes =
      (g->plan.variant == kSell32
           ? g->plan.sell_bytes
           : g->plan.variant == kSellPattern ? g->plan.pat_bytes
                                             : 8.0 * (n + 1) + g->plan.short_entries * (g->weighted ? 8.0 : 4.0)) +
      g->plan.med_bytes + g->plan.long_bytes;
  double bytes = graph_bytes + n * b * si + n * sa;
  if (prescaled) bytes += 3.0 * n * b * si;   // the pass reads X and writes Z; the epilogue reads X again
  if (coefs && !g->weighted) bytes += 4.0 * nnz;   // the coefficient stream (weighted graphs: in place of the weights)
  if (a.mode == 0) {
    bytes += n * b * sa;
  } else {
    bytes += n * b * static_cast<double>(dt_size(a.tout)) + n * b * sa * (a.first ? 1.0 : (a.yterms ? 2.0 : 0.0));
  }
  const int dti = static_cast<int>(a.tin);
  g->ctr.spmm_bytes += bytes;
  g->ctr.spmm_launches += 1;
  g->ctr.spmm_bytes_dt[dti] += bytes;
  g->ctr.spmm_launches_dt[dti] += 1;

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g->ctr.timing) {
    if (g->ctr.ev_used + 2 > g->ctr.ev_pool.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        SPX_CUDA(cudaEventCreate(&e));
        g->ctr.ev_pool.push_back(e);
      }
    }
    if (g->ctr.ev_dt.size() < g->ctr.ev_pool.size() / 2) g->ctr.ev_dt.resize(g->ctr.ev_pool.size() / 2);
    g->ctr.ev_dt[g->ctr.ev_used / 2] = dti;
    e0 = g->ctr.ev_pool[g->ctr.ev_used++];
    e1 = g->ctr.ev_pool[g->ctr.ev_used++];
    SPX_CUDA(cudaEventRecord(e0, g->stream));
  }
  if (prescaled) {
    // sized for double rows of the widest block, so that a graph captured
    // around this product never sees the buffer move
    void *z = g->workspace("spmm_prescaled", static_cast<size_t>(g->n) * 16 * 8 + 256, false);
    const bool vec = a.bp % 4 == 0;   // rows of 4, 8, 12 or 16 values, 16-byte aligned
    const int64_t total = g->n * (vec ? a.bp / (a.tin == DT::F64 ? 2 : 4) : a.bp);
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 16 * kSmCount));
    if (a.tin == DT::F64) {
      if (vec)
        k_prescale<double, 2><<<grid, 256, 0, g->stream>>>(static_cast<const double *>(a.x), g->dinv.as<double>(),
                                                            g->n, a.bp, static_cast<double *>(z));
      else
        k_prescale<double, 1><<<grid, 256, 0, g->stream>>>(static_cast<const double *>(a.x), g->dinv.as<double>(),
                                                            g->n, a.bp, static_cast<double *>(z));
    } else {
      if (vec)
        k_prescale<float, 4><<<grid, 256, 0, g->stream>>>(static_cast<const float *>(a.x), g->dinvf.as<float>(), g->n,
                                                           a.bp, static_cast<float *>(z));
      else
        k_prescale<float, 1><<<grid, 256, 0, g->stream>>>(static_cast<const float *>(a.x), g->dinvf.as<float>(), g->n,
                                                           a.bp, static_cast<float *>(z));
    }
    SPX_LAUNCHED();
    g->ctr.launches++;
    d.xe = a.x;
    d.x = z;
  }
  dispatch(g, a, d);
  if (g->ctr.timing) SPX_CUDA(cudaEventRecord(e1, g->stream));
}

}  // namespace sphynx
