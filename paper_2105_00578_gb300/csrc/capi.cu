// capi.cu -- step-level entry points that work on caller buffers without a
// graph handle: the Rayleigh-Ritz Gram products and the FP64 Rayleigh-Ritz
// solve (Sec. 3.3, the Rayleigh-Ritz step of Algorithm 1).
#include "internal.cuh"

#include <cstring>

using namespace sphynx;

extern "C" {

int sphynx_gram(int32_t dtype, const void *const *s_blocks, const void *const *ls_blocks, int32_t nblk, int32_t ld,
                int64_t n, const double *bdiag, double *ga_out, double *gb_out, void *stream) {
  return guarded([&]() -> int {
    if (dtype != SPHYNX_DT_F32 && dtype != SPHYNX_DT_F64) fail(SPHYNX_ERR_INVALID_ARG, "dtype %d", dtype);
    if (nblk < 1 || nblk > 3) fail(SPHYNX_ERR_INVALID_ARG, "nblk %d", nblk);
    if (ld != 4 && ld != 8 && ld != 12 && ld != 16) fail(SPHYNX_ERR_INVALID_ARG, "ld %d", ld);
    if (n < 1) fail(SPHYNX_ERR_INVALID_ARG, "n %lld", static_cast<long long>(n));
    if (!s_blocks || !ls_blocks || !ga_out || !gb_out) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < nblk; ++k)
      if (!s_blocks[k] || !ls_blocks[k]) fail(SPHYNX_ERR_INVALID_ARG, "NULL block %d", k);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int M = nblk * ld;
    const int grid = gram_grid(n);
    const size_t npart = gram_partials_size(nblk, ld, grid);
    const size_t bytes = npart * 8 + 2 * static_cast<size_t>(M) * M * 8 + (bdiag ? static_cast<size_t>(n) * 4 : 0) + 512;
    void *scratch = nullptr;
    SPX_CUDA(cudaMallocAsync(&scratch, bytes, st));
    char *p = static_cast<char *>(scratch);
    double *part = reinterpret_cast<double *>(p);
    double *ga = part + npart;
    double *gb = ga + M * M;
    // the float copy of diag(B) starts on a 16-byte boundary (staged copies)
    float *bf = bdiag ? reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(gb + M * M) + 15) & ~uintptr_t(15))
                      : nullptr;
    try {
      SPX_CUDA(cudaMemsetAsync(ga, 0, 2 * static_cast<size_t>(M) * M * 8, st));
      if (bdiag && dtype == SPHYNX_DT_F32) launch_d2f(st, bdiag, bf, n);
      GramArgs a{static_cast<DT>(dtype), nblk, ld, n, {}, {}, bdiag, bf, part, ga, gb, nullptr};
      for (int k = 0; k < 3; ++k) {
        a.s[k] = k < nblk ? s_blocks[k] : nullptr;
        a.ls[k] = k < nblk ? ls_blocks[k] : nullptr;
      }
      const int pg = launch_gram(st, a, grid);
      launch_gram_reduce(st, part, nblk, ld, pg, ga, gb, nullptr);
      SPX_CUDA(cudaMemcpyAsync(ga_out, ga, static_cast<size_t>(M) * M * 8, cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaMemcpyAsync(gb_out, gb, static_cast<size_t>(M) * M * 8, cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaFreeAsync(scratch, st);
      throw;
    }
    SPX_CUDA(cudaFreeAsync(scratch, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    return SPHYNX_OK;
  });
}

int sphynx_rayleigh_ritz(const double *ga, const double *gb, const int32_t *active, int32_t m, int32_t nev,
                         double u_work, double *theta_out, double *y_out, int32_t *used_svqb, void *stream) {
  return guarded([&]() -> int {
    if (!ga || !gb || !active || !theta_out || !y_out) fail(SPHYNX_ERR_INVALID_ARG, "NULL argument");
    if (m < 1 || m > 3 * SPHYNX_MAX_NEV) fail(SPHYNX_ERR_INVALID_ARG, "m %d", m);
    if (nev < 1 || nev > m || nev > SPHYNX_MAX_NEV) fail(SPHYNX_ERR_INVALID_ARG, "nev %d", nev);
    if (!(u_work > 0.0)) fail(SPHYNX_ERR_INVALID_ARG, "u_work");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t mm = static_cast<size_t>(m) * m;
    const size_t bytes = (2 * mm + static_cast<size_t>(m) * nev + nev + 8) * 8 + static_cast<size_t>(m) * 4 + 64;
    void *scratch = nullptr;
    SPX_CUDA(cudaMallocAsync(&scratch, bytes, st));
    double *dga = static_cast<double *>(scratch);
    double *dgb = dga + mm;
    double *dy = dgb + mm;
    double *dth = dy + static_cast<size_t>(m) * nev;
    int *dsv = reinterpret_cast<int *>(dth + nev + 4);
    int *dact = dsv + 4;
    int sv = 0;
    try {
      SPX_CUDA(cudaMemcpyAsync(dga, ga, mm * 8, cudaMemcpyHostToDevice, st));
      SPX_CUDA(cudaMemcpyAsync(dgb, gb, mm * 8, cudaMemcpyHostToDevice, st));
      SPX_CUDA(cudaMemcpyAsync(dact, active, static_cast<size_t>(m) * 4, cudaMemcpyHostToDevice, st));
      SPX_CUDA(cudaMemsetAsync(dsv, 0, 16, st));
      launch_rayleigh_ritz(st, dga, dgb, m, nev, nev, u_work, nullptr, dy, nullptr, DT::F64, dact, dth, dsv, 0);
      SPX_CUDA(cudaMemcpyAsync(y_out, dy, static_cast<size_t>(m) * nev * 8, cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaMemcpyAsync(theta_out, dth, static_cast<size_t>(nev) * 8, cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaMemcpyAsync(&sv, dsv, 4, cudaMemcpyDeviceToHost, st));
      SPX_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaFreeAsync(scratch, st);
      throw;
    }
    SPX_CUDA(cudaFreeAsync(scratch, st));
    SPX_CUDA(cudaStreamSynchronize(st));
    if (used_svqb) *used_svqb = sv < 0 ? 0 : sv;
    if (sv < 0) fail(SPHYNX_ERR_BREAKDOWN, "Rayleigh-Ritz basis has fewer than nev independent columns");
    return SPHYNX_OK;
  });
}

}  // extern "C"
