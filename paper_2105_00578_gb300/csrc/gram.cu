// gram.cu -- Gram matrices of the Rayleigh-Ritz step (Sec. 3.3, Algorithm
// 1): G_A = S^T (L S) and G_B = S^T B S for the tall-skinny block
// S = [S_0 | S_1 | S_2] (n x M, M = nblk * ld <= 48) and its L-image.
//
// Both matrices are symmetric (L and B are), so only their upper triangles
// are formed.  Float blocks use k_gram8 below (8 x 8 tiles per thread); the
// double path uses k_gram, in 4 x 4 output tiles: NB = mb (mb + 1) tiles with
// mb = M / 4.  A CTA streams slabs of TR rows of S, LS and diag(B) into shared
// memory with cp.async 16-byte copies, multi-buffered so that the next slabs
// are in flight while the current one is multiplied.  Its 256 threads form
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
constexpr int kFoldRows = 4096;   // rows a thread of the 8 x 8 kernel adds into one float running sum

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

// ---- float blocks: 8 x 8 register tiles ------------------------------------
//
// The 4 x 4 tiles above cost two 16-byte shared loads (eight quarter-warp
// wavefronts per warp) for 16 FMAs, which leaves the kernel bound by shared
// memory at about half the FMA rate.  Here a thread owns an 8 x 8 tile: four
// 16-byte loads for 64 FMAs.  The columns are cut into 4-wide chunks (MC =
// M / 4); tile row bi covers chunks 2 bi and 2 bi + 1, the second one absent
// (zero) when MC is odd.  A row group is nb = 2 nbu threads (nbu upper tiles
// per matrix), groups are contiguous in the thread index, and G groups take
// the rows of a slab in turn.  Block k of a slab starts at a 16-byte slot
// chosen so that the chunks one quarter warp reads (two adjacent rows when a
// group straddles it) fall in different banks; for b = 7 (ld 8, three
// blocks) the placement (slots 0, 1, 4, 3, 4, 5 modulo 8) was found by
// exhaustive search over the thread-to-tile map below.
//
// Summation: a thread adds the products of up to 64 of its rows in float,
// then adds that sum into a float running sum.  The launch gives every thread
// at most kFoldRows = 4096 rows (64 such folds), so each entry of a thread's
// running sum is within (64 + 64) u of the exact sum of its |terms| (u = 2^-24);
// threads are then added in double.  (A TwoSum-compensated running sum would
// cost 64 more registers or shared floats per thread; that halved the resident
// warps and made the kernel slower than the 4 x 4 one.)  The result is written
// in the 4 x 4 kernel's partial layout, so one reduction serves both.
template <int LD, int NBLK>
struct G8 {
  static constexpr int M = LD * NBLK;
  static constexpr int MC = M / 4;
  static constexpr int mb = (MC + 1) / 2;
  static constexpr int nbu = mb * (mb + 1) / 2;
  static constexpr int nb = 2 * nbu;
  static constexpr int G = nb >= 96 ? 1 : 96 / nb;
  static constexpr int threads = nb * G;
  static constexpr int TR = 64;
  static constexpr int stages = 2;                     // two slabs: more resident CTAs beat a deeper ring
  static constexpr int blkw = TR * LD + 32;            // floats per block, with room for the slot shift
  static constexpr int elems = 2 * NBLK * blkw + TR;   // S blocks, LS blocks, diag(B)
  static constexpr int nbu4 = MC * (MC + 1) / 2;       // upper 4 x 4 tiles of one matrix
  // shared bytes: the slab ring, reused at the end for the nb x 64 tile sums
  static constexpr size_t smem_bytes = static_cast<size_t>(stages) * elems * 4 > static_cast<size_t>(nb) * 64 * 8
                                           ? static_cast<size_t>(stages) * elems * 4
                                           : static_cast<size_t>(nb) * 64 * 8;
  __host__ __device__ static constexpr int slot(int k) {
    return (LD == 8 && NBLK == 3) ? (k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 4 : k == 3 ? 3 : k == 4 ? 4 : 5) : k;
  }
  __host__ __device__ static constexpr int block_off(int k) { return k * blkw + 4 * slot(k); }
  // offset of 4-column chunk q (q < MC) of S (ls = false) or LS in a slab row 0
  __host__ __device__ static constexpr int chunk_off(int q, bool ls) {
    return block_off((ls ? NBLK : 0) + (4 * q) / LD) + (4 * q) % LD;
  }
};

template <int LD, int NBLK>
__device__ __forceinline__ void stage8(float *buf, int64_t r0, int64_t n, const float *const (&srcS)[3],
                                       const float *const (&srcL)[3], const float *bdiag) {
  using C = G8<LD, NBLK>;
  constexpr int chunks = C::TR * LD / 4;   // 16-byte copies per block
#pragma unroll
  for (int blk = 0; blk < NBLK; ++blk) {
    for (int i = threadIdx.x; i < 2 * chunks; i += C::threads) {
      const int arr = i / chunks, c = i - arr * chunks;
      const int r = c * 4 / LD;
      const bool ok = r0 + r < n;
      const float *src = (arr == 0 ? srcS[blk] : srcL[blk]) + (ok ? r0 * LD + c * 4 : 0);
      cp16(buf + C::block_off(arr * NBLK + blk) + c * 4, src, ok ? 16 : 0);
    }
  }
  if (bdiag) {
    for (int c = threadIdx.x; c < C::TR / 4; c += C::threads) {
      const int r = c * 4;
      const int64_t left = n - r0 - r;
      const int bytes = left >= 4 ? 16 : (left > 0 ? static_cast<int>(left) * 4 : 0);
      cp16(buf + 2 * NBLK * C::blkw + r, bdiag + (bytes ? r0 + r : 0), bytes);
    }
  }
}

__device__ __forceinline__ Q4<float> ld4z(const float *p, bool ok) {
  return ok ? ld4(p) : Q4<float>{0.f, 0.f, 0.f, 0.f};
}

// u-th upper 4 x 4 tile (row-major upper triangle of an mc x mc tile grid)
__device__ __forceinline__ int upper_index(int bi, int bj, int mc) { return bi * mc - bi * (bi - 1) / 2 + (bj - bi); }

template <int LD, int NBLK>
__global__ void __launch_bounds__(G8<LD, NBLK>::threads, 3)
k_gram8(int64_t n, const float *s0, const float *s1, const float *s2, const float *l0, const float *l1,
        const float *l2, const float *bdiag, double *partials, const int *done) {
  using C = G8<LD, NBLK>;
  constexpr int TR = C::TR, NS = C::stages;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (done && *done) return;
  float *const base = reinterpret_cast<float *>(smem_raw);
  const int tid = threadIdx.x;
  const int grp = tid / C::nb, t = tid - (tid / C::nb) * C::nb;
  const bool isA = t < C::nbu;
  int bi, bj;
  upper_tile(isA ? t : t - C::nbu, C::mb, bi, bj);
  const bool a1 = 2 * bi + 1 < C::MC, c1 = 2 * bj + 1 < C::MC;
  const int oa0 = C::chunk_off(2 * bi, false), oa1 = a1 ? C::chunk_off(2 * bi + 1, false) : oa0;
  const int oc0 = C::chunk_off(2 * bj, isA), oc1 = c1 ? C::chunk_off(2 * bj + 1, isA) : oc0;
  const float *const srcS[3] = {s0, s1, s2};
  const float *const srcL[3] = {l0, l1, l2};
  const bool useB = !isA && bdiag != nullptr;
  unsigned long long acc[8][4];   // (a_i c_2p, a_i c_2p+1), up to 64 rows
  float hi[64];                   // running sums of the folded blocks
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[i][p] = 0ull;
#pragma unroll
  for (int q = 0; q < 64; ++q) hi[q] = 0.f;
  const int64_t ntile = (n + TR - 1) / TR;
  int since_flush = 0;
  int64_t tile = blockIdx.x;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) {
    const int64_t tl = tile + static_cast<int64_t>(s) * gridDim.x;
    if (tl < ntile) stage8<LD, NBLK>(base + s * C::elems, tl * TR, n, srcS, srcL, bdiag);
    cp_commit();
  }
  for (int it = 0; tile < ntile; tile += gridDim.x, ++it) {
    const int64_t ahead = tile + static_cast<int64_t>(NS - 1) * gridDim.x;
    if (ahead < ntile) stage8<LD, NBLK>(base + ((it + NS - 1) % NS) * C::elems, ahead * TR, n, srcS, srcL, bdiag);
    cp_commit();
    cp_wait<NS - 1>();
    __syncthreads();
    const float *buf = base + (it % NS) * C::elems;
    const float *bd = buf + 2 * NBLK * C::blkw;
#pragma unroll 1
    for (int r = grp; r < TR; r += C::G) {
      const Q4<float> x0 = ld4(buf + oa0 + r * LD), x1 = ld4z(buf + oa1 + r * LD, a1);
      const Q4<float> y0 = ld4(buf + oc0 + r * LD), y1 = ld4z(buf + oc1 + r * LD, c1);
      float av[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      if (useB) {
        const float b = bd[r];
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] *= b;
      }
      const unsigned long long cp[4] = {pk2(y0.x, y0.y), pk2(y0.z, y0.w), pk2(y1.x, y1.y), pk2(y1.z, y1.w)};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const unsigned long long ai = pk2(av[i], av[i]);
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[i][p] = fma2(ai, cp[p], acc[i][p]);
      }
    }
    since_flush += (TR - grp + C::G - 1) / C::G;
    if (since_flush >= 64) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 f = upk2(acc[i][p]);
          hi[8 * i + 2 * p] += f.x;
          hi[8 * i + 2 * p + 1] += f.y;
          acc[i][p] = 0ull;
        }
      since_flush = 0;
    }
    __syncthreads();
  }
  cp_wait<0>();
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float2 f = upk2(acc[i][p]);
      hi[8 * i + 2 * p] += f.x;
      hi[8 * i + 2 * p + 1] += f.y;
    }
  // groups add their tile sums into red [nb][64] one after another
  double *red = reinterpret_cast<double *>(smem_raw);
  for (int g = 0; g < C::G; ++g) {
    if (grp == g) {
#pragma unroll
      for (int q = 0; q < 64; ++q) {
        const double v = static_cast<double>(hi[q]);
        red[t * 64 + q] = g ? red[t * 64 + q] + v : v;
      }
    }
    __syncthreads();
  }
  double *out = partials + static_cast<int64_t>(blockIdx.x) * 2 * C::nbu4 * 16;
  for (int o = tid; o < C::nb * 64; o += C::threads) {
    const int tt = o / 64, e = o % 64, i = e / 8, j = e % 8;
    const bool tA = tt < C::nbu;
    int ti, tj;
    upper_tile(tA ? tt : tt - C::nbu, C::mb, ti, tj);
    const int bi4 = 2 * ti + i / 4, bj4 = 2 * tj + j / 4;
    if (bi4 >= C::MC || bj4 >= C::MC || bi4 > bj4) continue;
    out[((tA ? 0 : C::nbu4) + upper_index(bi4, bj4, C::MC)) * 16 + (i % 4) * 4 + j % 4] = red[tt * 64 + e];
  }
}

// partials [grid][nb * 16] -> symmetric G_A and G_B (M x M).  A block takes
// 32 entries; its eight warps add every eighth partial row with four
// independent sums each (so the loads overlap), and warp 0 adds the eight
// warp sums in a fixed order.
__global__ void __launch_bounds__(256) k_gram_reduce(const double *partials, int M, int grid, double *ga, double *gb,
                                                     const int *done) {
  __shared__ double red[8][33];
  if (done && *done) return;
  const Shape sh = shape_of(M);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  const int64_t stride = static_cast<int64_t>(sh.nb) * 16;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (o < sh.nb * 16) {
    int g = w;
    for (; g + 24 < grid; g += 32) {
      s0 += partials[g * stride + o];
      s1 += partials[(g + 8) * stride + o];
      s2 += partials[(g + 16) * stride + o];
      s3 += partials[(g + 24) * stride + o];
    }
    for (; g < grid; g += 8) s0 += partials[g * stride + o];
  }
  red[w][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (w == 0 && o < sh.nb * 16) {
    double tot = 0.0;
    for (int k = 0; k < 8; ++k) tot += red[k][lane];
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
int launch_t(cudaStream_t st, const GramArgs &a, const T *bd, int grid) {
  auto p = [&](int k) { return k < NBLK ? static_cast<const T *>(a.s[k]) : nullptr; };
  auto q = [&](int k) { return k < NBLK ? static_cast<const T *>(a.ls[k]) : nullptr; };
  if constexpr (std::is_same<T, float>::value) {
    using C = G8<LD, NBLK>;
    const size_t sm = C::smem_bytes;
    // one wave of resident CTAs: each walks the slabs with a grid stride
    SPX_CUDA(cudaFuncSetAttribute(k_gram8<LD, NBLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sm)));
    static int per_sm = 0;
    if (per_sm == 0) {
      int b = 0;
      SPX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_gram8<LD, NBLK>, C::threads, sm));
      per_sm = b > 0 ? b : 1;
    }
    // whole waves of resident CTAs, enough of them that no thread takes more
    // than kFoldRows rows
    const int64_t wave = static_cast<int64_t>(per_sm) * kSmCount;
    const int64_t need = (a.n + static_cast<int64_t>(kFoldRows) * C::G - 1) / (static_cast<int64_t>(kFoldRows) * C::G);
    int64_t g64 = (need + wave - 1) / wave * wave;
    if (g64 > grid) g64 = grid;
    const int g = static_cast<int>(g64);
    k_gram8<LD, NBLK><<<g, C::threads, sm, st>>>(a.n, p(0), p(1), p(2), q(0), q(1), q(2), bd, a.partials, a.done);
    SPX_LAUNCHED();
    return g;
  } else {
    constexpr int M = LD * NBLK;
    const Shape sh = shape_of(M);
    const size_t slabs = static_cast<size_t>(Tile<T>::stages) * Slab<T, LD, NBLK>::elems * sizeof(T);
    const size_t red = static_cast<size_t>(sh.ngroups) * sh.nb * 16 * sizeof(double);
    const size_t sm = slabs > red ? slabs : red;
    if (sm > 48 * 1024)
      SPX_CUDA(cudaFuncSetAttribute(k_gram<T, LD, NBLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(sm)));
    // two waves of the 2 resident CTAs per SM; the compensated sums take any row count
    const int g = grid < 4 * kSmCount ? grid : 4 * kSmCount;
    k_gram<T, LD, NBLK><<<g, kThreads, sm, st>>>(a.n, p(0), p(1), p(2), q(0), q(1), q(2), bd, a.partials, a.done);
    SPX_LAUNCHED();
    return g;
  }
}

template <typename T, int NBLK>
int launch_ld(cudaStream_t st, const GramArgs &a, const T *bd, int grid) {
  switch (a.ld) {
    case 4: return launch_t<T, 4, NBLK>(st, a, bd, grid);
    case 8: return launch_t<T, 8, NBLK>(st, a, bd, grid);
    case 12: return launch_t<T, 12, NBLK>(st, a, bd, grid);
    case 16: return launch_t<T, 16, NBLK>(st, a, bd, grid);
    default: fail(SPHYNX_ERR_INVALID_ARG, "gram: ld %d", a.ld);
  }
  return 0;
}

template <typename T>
int launch_typed(cudaStream_t st, const GramArgs &a, const T *bd, int grid) {
  // 16-byte copies need 16-byte aligned blocks and diagonal
  for (int k = 0; k < a.nblk; ++k)
    if (reinterpret_cast<uintptr_t>(a.s[k]) % 16 || reinterpret_cast<uintptr_t>(a.ls[k]) % 16)
      fail(SPHYNX_ERR_INVALID_ARG, "gram: blocks must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(bd) % 16) fail(SPHYNX_ERR_INVALID_ARG, "gram: B diagonal must be 16-byte aligned");
  switch (a.nblk) {
    case 1: return launch_ld<T, 1>(st, a, bd, grid);
    case 2: return launch_ld<T, 2>(st, a, bd, grid);
    case 3: return launch_ld<T, 3>(st, a, bd, grid);
    default: fail(SPHYNX_ERR_INVALID_ARG, "gram: nblk %d", a.nblk);
  }
  return 0;
}

}  // namespace

int gram_grid(int64_t n) {
  // enough CTAs for both kernels: two waves of the 4 x 4 kernel, and for the
  // 8 x 8 kernel (at least two row groups a CTA) at most kFoldRows rows a thread
  int64_t g = (n + 2 * kFoldRows - 1) / (2 * kFoldRows) + 8 * kSmCount;
  if (g > (n + 63) / 64) g = (n + 63) / 64;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

size_t gram_partials_size(int nblk, int ld, int grid) {
  return static_cast<size_t>(grid) * shape_of(nblk * ld).nb * 16;
}

int launch_gram(cudaStream_t st, const GramArgs &a, int grid) {
  if (a.dt == DT::F64) return launch_typed<double>(st, a, a.bdiag, grid);
  return launch_typed<float>(st, a, a.bdiagf, grid);
}

void launch_gram_reduce(cudaStream_t st, const double *partials, int nblk, int ld, int grid, double *ga,
                        double *gb, const int *done) {
  const int M = nblk * ld;
  const int blocks = (shape_of(M).nb * 16 + 31) / 32;
  k_gram_reduce<<<blocks, 256, 0, st>>>(partials, M, grid, ga, gb, done);
  SPX_LAUNCHED();
}

}  // namespace sphynx
