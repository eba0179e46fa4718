// gram.cu -- Gram matrices of the Rayleigh-Ritz step (Sec. 3.3, Algorithm 1
// line 7): G_A = S^T (L S) and G_B = S^T B S for the tall-skinny block
// S = [S_0 | S_1 | S_2] (n x M, M = nblk * ld <= 48) and its L-image.
//
// Both matrices are symmetric (L and B are), so only their upper triangles
// are formed, in 4 x 4 output tiles: NB = mb (mb + 1) tiles with mb = M / 4.
// A CTA streams slabs of TR rows of S, LS and diag(B) into shared memory with
// cp.async 16-byte copies, double-buffered so that the next slab is in flight
// while the current one is multiplied.  Its 256 threads form
// floor(256 / NB) groups of NB threads, thread t of a group owning tile t and
// the group owning rows grp, grp + ngroups, ...  Per row a thread does two
// 16-byte shared loads and 16 FMAs (B applied on the fly for G_B tiles).
// float: products and short sums in float, folded every 64 rows into a float
// (hi, lo) pair with Knuth's TwoSum (about 48 significant bits); double:
// plain double FMAs.  Per-CTA partials are written in double and a second
// kernel adds them in a fixed order, so results do not depend on scheduling.
// Every element of S and LS is read once: the kernel is bound by those bytes.
#include "internal.cuh"

namespace sphynx {

namespace {

constexpr int kThreads = 256;

template <typename T> struct Tile {
  static constexpr int rows = 64;
  static constexpr int stages = 4;   // slabs in flight: enough bytes to cover DRAM latency
};
template <> struct Tile<double> {
  static constexpr int rows = 32;
  static constexpr int stages = 3;
};

// four consecutive elements, moved with 16-byte accesses
template <typename T> struct Q4 { T x, y, z, w; };
__device__ __forceinline__ Q4<float> ld4(const float *p) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q4<double> ld4(const double *p) {
  const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
  return {a.x, a.y, b.x, b.y};
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// packed float pairs (fma.rn.f32x2, sm_100 and later)
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// 4 x 4 tile accumulator: a_i c_j for i, j < 4
template <typename T> struct Acc44 {
  T v[16];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = T(0);
  }
  __device__ __forceinline__ void add(const Q4<T> &a, const Q4<T> &c) {
    const T av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) v[i * 4 + j] += av[i] * cv[j];
  }
  __device__ __forceinline__ T get(int q) const { return v[q]; }
  __device__ __forceinline__ void set(int q, T x) { v[q] = x; }
};
template <> struct Acc44<float> {
  unsigned long long v[8];   // pairs (i, j), (i, j + 1)
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = 0ull;
  }
  __device__ __forceinline__ void add(const Q4<float> &a, const Q4<float> &c) {
    const unsigned long long c01 = pk2(c.x, c.y), c23 = pk2(c.z, c.w);
    const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const unsigned long long ai = pk2(av[i], av[i]);
      v[2 * i] = fma2(ai, c01, v[2 * i]);
      v[2 * i + 1] = fma2(ai, c23, v[2 * i + 1]);
    }
  }
  __device__ __forceinline__ float get(int q) const {
    const float2 f = upk2(v[q >> 1]);
    return (q & 1) ? f.y : f.x;
  }
  __device__ __forceinline__ void set(int q, float x) {
    float2 f = upk2(v[q >> 1]);
    if (q & 1) f.y = x; else f.x = x;
    v[q >> 1] = pk2(f.x, f.y);
  }
};

__device__ __forceinline__ void two_sum_fold(float &hi, float &lo, float &acc) {
  const float s = hi + acc;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (acc - bp);
  hi = s;
  lo += e;
  acc = 0.f;
}

// nbu = upper tiles of one matrix; nb = 2 nbu tiles per row group; a group
// is a whole number of warps (tpg threads) so that every warp reads one row
// at a time and its shared loads of that row are broadcasts
struct Shape {
  int mb, nbu, nb, tpg, ngroups;
};

__host__ __device__ constexpr Shape shape_of(int M) {
  return Shape{M / 4, (M / 4) * (M / 4 + 1) / 2, (M / 4) * (M / 4 + 1), ((M / 4) * (M / 4 + 1) + 31) / 32 * 32,
               kThreads / (((M / 4) * (M / 4 + 1) + 31) / 32 * 32)};
}

// tile index u in [0, nbu) -> (bi, bj) with bi <= bj (row-major upper triangle)
__device__ __forceinline__ void upper_tile(int u, int mb, int &bi, int &bj) {
  bi = 0;
  while (u >= mb - bi) {
    u -= mb - bi;
    ++bi;
  }
  bj = bi + u;
}

// shared layout of one slab: per block, TR rows of LD values, S then LS, then
// the TR diagonal entries of B
template <typename T, int LD, int NBLK>
struct Slab {
  static constexpr int TR = Tile<T>::rows;
  // elements of one block, padded by 16 bytes so that the same column of
  // different blocks falls in different shared-memory banks
  static constexpr int blk = TR * LD + 16 / static_cast<int>(sizeof(T));
  static constexpr int elems = 2 * NBLK * blk + TR;   // S, LS, diag(B)
};

template <typename T, int LD, int NBLK>
__device__ __forceinline__ void stage(T *buf, int64_t r0, int64_t n, const T *const (&srcS)[3],
                                      const T *const (&srcL)[3], const T *bdiag) {
  using SL = Slab<T, LD, NBLK>;
  constexpr int TR = SL::TR;
  constexpr int per = 16 / static_cast<int>(sizeof(T));   // elements per 16-byte copy
  constexpr int chunks = TR * LD / per;                    // per block and array
#pragma unroll
  for (int blk = 0; blk < NBLK; ++blk) {
    for (int i = threadIdx.x; i < 2 * chunks; i += kThreads) {
      const int arr = i / chunks, c = i - arr * chunks;
      const int r = c * per / LD;
      const bool ok = r0 + r < n;
      const T *src = (arr == 0 ? srcS[blk] : srcL[blk]) + (ok ? r0 * LD + c * per : 0);
      cp16(buf + (arr * NBLK + blk) * SL::blk + c * per, src, ok ? 16 : 0);
    }
  }
  if (bdiag) {
    for (int c = threadIdx.x; c < TR / per; c += kThreads) {
      const int r = c * per;
      const int64_t left = n - r0 - r;
      const int bytes = left >= per ? 16 : (left > 0 ? static_cast<int>(left) * static_cast<int>(sizeof(T)) : 0);
      cp16(buf + 2 * NBLK * SL::blk + r, bdiag + (bytes ? r0 + r : 0), bytes);
    }
  }
}

template <typename T, int LD, int NBLK>
__global__ void __launch_bounds__(kThreads)
k_gram(int64_t n, const T *s0, const T *s1, const T *s2, const T *l0, const T *l1, const T *l2,
       const T *bdiag, double *partials, const int *done) {
  using SL = Slab<T, LD, NBLK>;
  constexpr int M = LD * NBLK;
  constexpr int TR = SL::TR;
  constexpr Shape sh = shape_of(M);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (done && *done) return;
  constexpr int NS = Tile<T>::stages;
  T *const base = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x;
  const int grp = tid / sh.tpg, t = tid - (tid / sh.tpg) * sh.tpg;
  const bool active = grp < sh.ngroups && t < sh.nb;
  int bi = 0, bj = 0;
  const int tt = t < sh.nb ? t : 0;   // padding threads of a group take tile 0 and stay idle
  const bool isA = tt < sh.nbu;
  upper_tile(isA ? tt : tt - sh.nbu, sh.mb, bi, bj);
  // offsets of the thread's two column groups inside a slab
  const int offA = (bi * 4 / LD) * SL::blk + (bi * 4) % LD;                        // S, rows x LD
  const int offC = ((isA ? NBLK : 0) + bj * 4 / LD) * SL::blk + (bj * 4) % LD;    // LS or S
  const T *const srcS[3] = {s0, s1, s2};
  const T *const srcL[3] = {l0, l1, l2};
  Acc44<T> acc;
  acc.zero();
  float hi[16], lo[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) { hi[q] = 0.f; lo[q] = 0.f; }
  const int64_t ntile = (n + TR - 1) / TR;
  const bool useB = !isA && bdiag != nullptr;
  int since_flush = 0;
  // ring of NS slabs: slab it % NS holds this CTA's it-th row slab; NS - 1
  // slabs are in flight while one is multiplied
  int64_t tile = blockIdx.x;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) {
    const int64_t tl = tile + static_cast<int64_t>(s) * gridDim.x;
    if (tl < ntile) stage<T, LD, NBLK>(base + s * SL::elems, tl * TR, n, srcS, srcL, bdiag);
    cp_commit();
  }
  for (int it = 0; tile < ntile; tile += gridDim.x, ++it) {
    const int64_t ahead = tile + static_cast<int64_t>(NS - 1) * gridDim.x;
    if (ahead < ntile) stage<T, LD, NBLK>(base + ((it + NS - 1) % NS) * SL::elems, ahead * TR, n, srcS, srcL, bdiag);
    cp_commit();
    cp_wait<NS - 1>();     // this slab's group has landed; the NS - 1 later ones may be in flight
    __syncthreads();
    const T *buf = base + (it % NS) * SL::elems;
    if (active) {
      const T *bd = buf + 2 * NBLK * SL::blk;
#pragma unroll 4
      for (int r = grp; r < TR; r += sh.ngroups) {
        const Q4<T> av = ld4(buf + offA + r * LD);
        Q4<T> cv = ld4(buf + offC + r * LD);
        if (useB) {
          const T b = bd[r];
          cv = {cv.x * b, cv.y * b, cv.z * b, cv.w * b};
        }
        acc.add(av, cv);
      }
      if constexpr (std::is_same<T, float>::value) {
        since_flush += (TR + sh.ngroups - 1) / sh.ngroups;
        if (since_flush >= 64) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            float a = acc.get(q);
            two_sum_fold(hi[q], lo[q], a);
          }
          acc.zero();
          since_flush = 0;
        }
      }
    }
    __syncthreads();       // the slab may be refilled by the next stage
  }
  cp_wait<0>();
  __syncthreads();
  double *red = reinterpret_cast<double *>(smem_raw);  // [ngroups][nb * 16]
  if (active) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      double v;
      if constexpr (std::is_same<T, float>::value) {
        float a = acc.get(q);
        two_sum_fold(hi[q], lo[q], a);
        v = static_cast<double>(hi[q]) + static_cast<double>(lo[q]);
      } else {
        v = acc.get(q);
      }
      red[(grp * sh.nb + t) * 16 + q] = v;
    }
  }
  __syncthreads();
  for (int o = tid; o < sh.nb * 16; o += kThreads) {
    double s = 0.0;
    for (int g = 0; g < sh.ngroups; ++g) s += red[g * sh.nb * 16 + o];
    partials[static_cast<int64_t>(blockIdx.x) * sh.nb * 16 + o] = s;
  }
}

// partials [grid][nb * 16] -> symmetric G_A and G_B (M x M); 8 threads per entry
__global__ void k_gram_reduce(const double *partials, int M, int grid, double *ga, double *gb, const int *done) {
  __shared__ double red[32][9];
  if (done && *done) return;
  const Shape sh = shape_of(M);
  const int lo = threadIdx.x & 7, oi = threadIdx.x >> 3;
  const int o = blockIdx.x * 32 + oi;
  double s = 0.0;
  if (o < sh.nb * 16)
    for (int g = lo; g < grid; g += 8) s += partials[static_cast<int64_t>(g) * sh.nb * 16 + o];
  red[oi][lo] = s;
  __syncthreads();
  if (lo == 0 && o < sh.nb * 16) {
    double tot = 0.0;
    for (int k = 0; k < 8; ++k) tot += red[oi][k];
    const int tile = o / 16, q = o % 16, i = q / 4, j = q % 4;
    const bool isA = tile < sh.nbu;
    int bi, bj;
    upper_tile(isA ? tile : tile - sh.nbu, sh.mb, bi, bj);
    double *g = isA ? ga : gb;
    const int r = 4 * bi + i, c = 4 * bj + j;
    if (bi < bj || i <= j) {
      g[r * M + c] = tot;
      g[c * M + r] = tot;
    }
  }
}

template <typename T, int LD, int NBLK>
void launch_t(cudaStream_t st, const GramArgs &a, const T *bd, int grid) {
  constexpr int M = LD * NBLK;
  const Shape sh = shape_of(M);
  const size_t slabs = static_cast<size_t>(Tile<T>::stages) * Slab<T, LD, NBLK>::elems * sizeof(T);
  const size_t red = static_cast<size_t>(sh.ngroups) * sh.nb * 16 * sizeof(double);
  const size_t sm = slabs > red ? slabs : red;
  if (sm > 48 * 1024)
    SPX_CUDA(cudaFuncSetAttribute(k_gram<T, LD, NBLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sm)));
  auto p = [&](int k) { return k < NBLK ? static_cast<const T *>(a.s[k]) : nullptr; };
  auto q = [&](int k) { return k < NBLK ? static_cast<const T *>(a.ls[k]) : nullptr; };
  k_gram<T, LD, NBLK><<<grid, kThreads, sm, st>>>(a.n, p(0), p(1), p(2), q(0), q(1), q(2), bd, a.partials, a.done);
  SPX_LAUNCHED();
}

template <typename T, int NBLK>
void launch_ld(cudaStream_t st, const GramArgs &a, const T *bd, int grid) {
  switch (a.ld) {
    case 4: launch_t<T, 4, NBLK>(st, a, bd, grid); break;
    case 8: launch_t<T, 8, NBLK>(st, a, bd, grid); break;
    case 12: launch_t<T, 12, NBLK>(st, a, bd, grid); break;
    case 16: launch_t<T, 16, NBLK>(st, a, bd, grid); break;
    default: fail(SPHYNX_ERR_INVALID_ARG, "gram: ld %d", a.ld);
  }
}

template <typename T>
void launch_typed(cudaStream_t st, const GramArgs &a, const T *bd, int grid) {
  // 16-byte copies need 16-byte aligned blocks and diagonal
  for (int k = 0; k < a.nblk; ++k)
    if (reinterpret_cast<uintptr_t>(a.s[k]) % 16 || reinterpret_cast<uintptr_t>(a.ls[k]) % 16)
      fail(SPHYNX_ERR_INVALID_ARG, "gram: blocks must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(bd) % 16) fail(SPHYNX_ERR_INVALID_ARG, "gram: B diagonal must be 16-byte aligned");
  switch (a.nblk) {
    case 1: launch_ld<T, 1>(st, a, bd, grid); break;
    case 2: launch_ld<T, 2>(st, a, bd, grid); break;
    case 3: launch_ld<T, 3>(st, a, bd, grid); break;
    default: fail(SPHYNX_ERR_INVALID_ARG, "gram: nblk %d", a.nblk);
  }
}

}  // namespace

int gram_grid(int64_t n) {
  int64_t g = (n + 63) / 64;
  if (g > 4 * kSmCount) g = 4 * kSmCount;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

size_t gram_partials_size(int nblk, int ld, int grid) {
  return static_cast<size_t>(grid) * shape_of(nblk * ld).nb * 16;
}

void launch_gram(cudaStream_t st, const GramArgs &a, int grid) {
  if (a.dt == DT::F64) launch_typed<double>(st, a, a.bdiag, grid);
  else launch_typed<float>(st, a, a.bdiagf, grid);
}

void launch_gram_reduce(cudaStream_t st, const double *partials, int nblk, int ld, int grid, double *ga,
                        double *gb, const int *done) {
  const int M = nblk * ld;
  const int blocks = (shape_of(M).nb * 16 + 31) / 32;
  k_gram_reduce<<<blocks, 256, 0, st>>>(partials, M, grid, ga, gb, done);
  SPX_LAUNCHED();
}

}  // namespace sphynx
