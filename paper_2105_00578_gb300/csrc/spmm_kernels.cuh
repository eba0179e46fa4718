// spmm_kernels.cuh -- the Laplacian block product Y = L X without forming L.
//
// L is one of (Sec. 3.2, Eqs. 2-3, weighted rule):
//   combinatorial  (L_C X)_i = deg_i X_i - sum_j w_ij X_j
//   normalized     (L_N X)_i = X_i - s_i sum_j w_ij s_j X_j,   s = D^{-1/2}
// (the generalized problem applies L_C; its B = D is applied elsewhere).
//
// Schedules.  Rows with at most kShortDeg neighbours go to the short-row
// kernel: a warp owns 32 consecutive rows, stages their column indices (and
// weights) with coalesced loads into shared memory, and each lane then walks
// its own row, gathering X rows with 16-byte vector loads.  Longer rows are
// cut into work items of kLongChunk entries; a warp per item reduces its
// entries with shuffles into a partial row, and a finalise kernel adds the
// partials of each long row in a fixed order (deterministic results) and
// applies the epilogue.
//
// Epilogues.  Mode 0 stores L X.  Mode 1 is one step of the product-form
// polynomial preconditioner (Sec. 5.2): with t the input block,
//   t' = t - (L t) / theta_i   (stored in type TT),
// and y = sum_i t_i / theta_i is gathered two terms at a time, so that the
// accumulator is read and written only every other step:
//   yterms 2:  y = (first ? 0 : y) + t / theta_i + t' / theta_{i+1}
//   yterms 1:  y = y + t' / theta_{i+1}            (last step, t already in y)
//   yterms 0:  y untouched (t' is added by the next step as its input)
// The terms use the stored (rounded) chain vectors, so the sum is the same
// whichever step adds them.
#pragma once

#include "internal.cuh"

namespace sphynx {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerCta = 4;
constexpr int kStageCap = 32 * kShortDeg;

template <typename TI> struct AccOf { using T = float; };
template <> struct AccOf<double> { using T = double; };

__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---- row loads / stores (rows are 16-byte aligned for bp >= 4) --------------
template <int BP>
__device__ __forceinline__ void load_row(const double *__restrict__ p, double (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = __ldg(p);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 2) {
      double2 v = __ldg(reinterpret_cast<const double2 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y;
    }
  }
}
template <int BP>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = __ldg(p);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      float4 v = __ldg(reinterpret_cast<const float4 *>(p + c));
      o[c] = v.x; o[c + 1] = v.y; o[c + 2] = v.z; o[c + 3] = v.w;
    }
  }
}
template <int BP>
__device__ __forceinline__ void load_row(const __nv_bfloat16 *__restrict__ p, float (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = __bfloat162float(p[0]);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      uint2 v = __ldg(reinterpret_cast<const uint2 *>(p + c));
      __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&v.x);
      __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&v.y);
      float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      o[c] = fa.x; o[c + 1] = fa.y; o[c + 2] = fb.x; o[c + 3] = fb.y;
    }
  }
}
// plain (coherent) loads for buffers written by the same launch sequence
template <int BP>
__device__ __forceinline__ void load_row_rw(const double *p, double (&o)[BP]) {
#pragma unroll
  for (int c = 0; c < BP; ++c) o[c] = p[c];
}
template <int BP>
__device__ __forceinline__ void load_row_rw(const float *p, float (&o)[BP]) {
  if constexpr (BP == 1) {
    o[0] = p[0];
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      float4 v = *reinterpret_cast<const float4 *>(p + c);
      o[c] = v.x; o[c + 1] = v.y; o[c + 2] = v.z; o[c + 3] = v.w;
    }
  }
}

template <int BP>
__device__ __forceinline__ void store_row(double *p, const double (&v)[BP]) {
  if constexpr (BP == 1) {
    p[0] = v[0];
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 2) *reinterpret_cast<double2 *>(p + c) = make_double2(v[c], v[c + 1]);
  }
}
template <int BP>
__device__ __forceinline__ void store_row(float *p, const float (&v)[BP]) {
  if constexpr (BP == 1) {
    p[0] = v[0];
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4)
      *reinterpret_cast<float4 *>(p + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
  }
}
// bf16 store rounds to nearest-even and returns the stored values in v
template <int BP>
__device__ __forceinline__ void store_row(__nv_bfloat16 *p, float (&v)[BP]) {
  if constexpr (BP == 1) {
    p[0] = __float2bfloat16_rn(v[0]);
    v[0] = __bfloat162float(p[0]);
  } else {
#pragma unroll
    for (int c = 0; c < BP; c += 4) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v[c], v[c + 1]);
      __nv_bfloat162 b = __floats2bfloat162_rn(v[c + 2], v[c + 3]);
      uint2 u;
      u.x = *reinterpret_cast<unsigned *>(&a);
      u.y = *reinterpret_cast<unsigned *>(&b);
      *reinterpret_cast<uint2 *>(p + c) = u;
      float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      v[c] = fa.x; v[c + 1] = fa.y; v[c + 2] = fb.x; v[c + 3] = fb.y;
    }
  }
}

template <typename TA> __device__ __forceinline__ TA deg_of(const LapView &L, int64_t i);
template <> __device__ __forceinline__ double deg_of<double>(const LapView &L, int64_t i) { return L.deg[i]; }
template <> __device__ __forceinline__ float deg_of<float>(const LapView &L, int64_t i) { return L.degf[i]; }
template <typename TA> __device__ __forceinline__ TA dinv_of(const LapView &L, int64_t i);
template <> __device__ __forceinline__ double dinv_of<double>(const LapView &L, int64_t i) { return __ldg(L.dinv + i); }
template <> __device__ __forceinline__ float dinv_of<float>(const LapView &L, int64_t i) { return __ldg(L.dinvf + i); }

struct SpmmDev {              // kernel-side view of SpmmArgs
  const void *x;
  int ldx, ldy;
  void *y;
  void *tout;
  void *yacc;
  int first;
  int yterms;          // mode 1: terms this step adds to y (2, 1 or 0)
  const double *inv;
  const float *invf;   // float copy of inv (the float path never touches FP64)
  int icur;
  const int *done;
  const int32_t *row_graph;  // batches: graph of every row, whose roots start at
  int inv_stride;            // inv[row_graph[row] * inv_stride] (NULL: one graph)
  const int32_t *act_blocks; // batches: the 1024-row blocks (row >> 10) that hold a row of a graph
  const int *n_act;          // still iterating, and their count; a fixed grid walks the list
  const void *xe;            // the epilogue's own rows X_i (x itself, or X when x holds D^{-1/2} X)
  const float *coef_csr;     // normalized: per-entry (w_ij or 1) D^{-1/2}_j in CSR order (NULL: gather D^{-1/2}_j)
  const float *coef_sell;    // the same in SELL slot order
};

constexpr int kListGrid = kSmCount * 16;   // CTAs of a launch that walks an active-block list

// acc = sum_j w_ij (s_j) X_j of row `row`; epilogue applies the diagonal part.
template <int LAP, typename TI, typename TT, int BP, int MODE>
__device__ __forceinline__ void spmm_epilogue(const LapView &L, const SpmmDev &a, int64_t row,
                                              const typename AccOf<TI>::T (&acc)[BP]) {
  using TA = typename AccOf<TI>::T;
  const TI *x = static_cast<const TI *>(a.xe);
  TA xi[BP];
  load_row<BP>(x + row * BP, xi);
  TA out[BP];
  if constexpr (LAP == SPHYNX_NORMALIZED) {
    const TA s = dinv_of<TA>(L, row);
#pragma unroll
    for (int c = 0; c < BP; ++c) out[c] = xi[c] - s * acc[c];
  } else {
    const TA d = deg_of<TA>(L, row);
#pragma unroll
    for (int c = 0; c < BP; ++c) out[c] = d * xi[c] - acc[c];
  }
  if constexpr (MODE == 0) {
    store_row<BP>(static_cast<TA *>(a.y) + row * a.ldy, out);
  } else {
    TA ic, inx;
    const int64_t ib = a.icur + (a.row_graph ? static_cast<int64_t>(__ldg(a.row_graph + row)) * a.inv_stride : 0);
    if constexpr (std::is_same<TA, double>::value) {
      ic = a.inv[ib];
      inx = a.inv[ib + 1];
    } else {
      ic = a.invf[ib];
      inx = a.invf[ib + 1];
    }
    TA tn[BP];
#pragma unroll
    for (int c = 0; c < BP; ++c) tn[c] = xi[c] - out[c] * ic;
    store_row<BP>(static_cast<TT *>(a.tout) + row * BP, tn);  // tn now holds the stored values
    if (a.yterms != 0) {
      TA *yp = static_cast<TA *>(a.yacc) + row * a.ldy;
      TA ya[BP];
      if (a.first) {
#pragma unroll
        for (int c = 0; c < BP; ++c) ya[c] = xi[c] * ic;
      } else {
        load_row_rw<BP>(yp, ya);
        if (a.yterms == 2) {
#pragma unroll
          for (int c = 0; c < BP; ++c) ya[c] += xi[c] * ic;
        }
      }
#pragma unroll
      for (int c = 0; c < BP; ++c) ya[c] += tn[c] * inx;
      store_row<BP>(yp, ya);
    }
  }
}

// ---- packed float pairs: add.rn.f32x2 / fma.rn.f32x2 (sm_100 and later) ----
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
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// two bfloat16 in one 32-bit word -> the float pair (low, high), exactly
__device__ __forceinline__ unsigned long long bf2_to_f2(unsigned w) {
  return pk2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// The raw bits of one gathered row of X (loaded first, converted later, so
// that a batch of gathers is in flight at once).
template <typename TI, int BP> struct RawRow;
template <int BP> struct RawRow<float, BP> {
  static constexpr int N = BP == 1 ? 1 : BP / 4;
  float4 q[N];
  __device__ __forceinline__ void load(const float *__restrict__ p) {
    if constexpr (BP == 1) {
      q[0].x = __ldg(p);
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) q[k] = __ldg(reinterpret_cast<const float4 *>(p + 4 * k));
    }
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < N; ++k) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
};
template <int BP> struct RawRow<__nv_bfloat16, BP> {
  // rows of a multiple of 8 values are 16-byte aligned, rows of 4 or 12 only 8-byte
  static constexpr bool kWide = BP % 8 == 0;
  static constexpr int N = kWide ? BP / 8 : BP / 4;
  uint4 q[kWide ? N : 1];
  uint2 h[kWide ? 1 : N];
  __device__ __forceinline__ void load(const __nv_bfloat16 *__restrict__ p) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if constexpr (kWide) q[k] = __ldg(reinterpret_cast<const uint4 *>(p + 8 * k));
      else h[k] = __ldg(reinterpret_cast<const uint2 *>(p + 4 * k));
    }
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if constexpr (kWide) q[k] = make_uint4(0u, 0u, 0u, 0u);
      else h[k] = make_uint2(0u, 0u);
    }
  }
};
template <int BP> struct RawRow<double, BP> {
  double v[BP];
  __device__ __forceinline__ void load(const double *__restrict__ p) { load_row<BP>(p, v); }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < BP; ++c) v[c] = 0.0;
  }
};

// gathers kept in flight per lane: about 128 bytes of X rows
template <typename TI, int BP> struct GatherBatch {
  static constexpr int bytes = BP * static_cast<int>(sizeof(TI));
  static constexpr int U = bytes <= 16 ? 8 : (bytes <= 32 ? 4 : 2);
};

// Running sum of coef * X_j over a row's neighbours j.
template <typename TI, int BP> struct RowAcc {
  // float and bfloat16 inputs: packed float pairs (a scalar for BP == 1)
  static constexpr int NP = BP >= 2 ? BP / 2 : 1;
  unsigned long long v[NP];
  float s;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q] = 0ull;
    s = 0.f;
  }
  template <bool COEF>
  __device__ __forceinline__ void add(const TI *__restrict__ p, float coef) {
    const unsigned long long cc = COEF ? pk2(coef, coef) : 0ull;
    if constexpr (BP == 1) {
      const float xv = to_acc(p[0]);
      s = COEF ? fmaf(coef, xv, s) : s + xv;
    } else if constexpr (std::is_same<TI, float>::value) {
#pragma unroll
      for (int c = 0; c < BP; c += 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p + c));
        const unsigned long long a0 = pk2(q.x, q.y), a1 = pk2(q.z, q.w);
        v[c / 2] = COEF ? fma2(cc, a0, v[c / 2]) : add2(v[c / 2], a0);
        v[c / 2 + 1] = COEF ? fma2(cc, a1, v[c / 2 + 1]) : add2(v[c / 2 + 1], a1);
      }
    } else if constexpr (BP % 8 == 0) {
      // bfloat16 rows of a multiple of 8 values (leading dimension a multiple
      // of 8, so rows are 16-byte aligned): 16-byte gathers
#pragma unroll
      for (int c = 0; c < BP; c += 8) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p + c));
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const unsigned long long f = bf2_to_f2(w[i]);
          v[c / 2 + i] = COEF ? fma2(cc, f, v[c / 2 + i]) : add2(v[c / 2 + i], f);
        }
      }
    } else {
      // bfloat16 rows of 4 or 12 values: rows are only 8-byte aligned
#pragma unroll
      for (int c = 0; c < BP; c += 4) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p + c));
        const unsigned long long f0 = bf2_to_f2(q.x), f1 = bf2_to_f2(q.y);
        v[c / 2] = COEF ? fma2(cc, f0, v[c / 2]) : add2(v[c / 2], f0);
        v[c / 2 + 1] = COEF ? fma2(cc, f1, v[c / 2 + 1]) : add2(v[c / 2 + 1], f1);
      }
    }
  }
  template <bool COEF, bool MIX = false>
  __device__ __forceinline__ void accum(const RawRow<TI, BP> &r, float coef) {
    const unsigned long long cc = COEF ? pk2(coef, coef) : 0ull;
    if constexpr (BP == 1) {
      const float xv = r.q[0].x;
      s = COEF ? fmaf(coef, xv, s) : s + xv;
    } else if constexpr (std::is_same<TI, float>::value) {
#pragma unroll
      for (int k = 0; k < BP / 4; ++k) {
        const float4 q = r.q[k];
        const unsigned long long a0 = pk2(q.x, q.y), a1 = pk2(q.z, q.w);
        v[2 * k] = COEF ? fma2(cc, a0, v[2 * k]) : add2(v[2 * k], a0);
        v[2 * k + 1] = COEF ? fma2(cc, a1, v[2 * k + 1]) : add2(v[2 * k + 1], a1);
      }
    } else if constexpr (RawRow<TI, BP>::kWide) {
#pragma unroll
      for (int k = 0; k < BP / 8; ++k) {
        const unsigned w[4] = {r.q[k].x, r.q[k].y, r.q[k].z, r.q[k].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const unsigned long long f = bf2_to_f2(w[i]);
          v[4 * k + i] = COEF ? fma2(cc, f, v[4 * k + i]) : add2(v[4 * k + i], f);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < BP / 4; ++k) {
        const unsigned long long f0 = bf2_to_f2(r.h[k].x), f1 = bf2_to_f2(r.h[k].y);
        v[2 * k] = COEF ? fma2(cc, f0, v[2 * k]) : add2(v[2 * k], f0);
        v[2 * k + 1] = COEF ? fma2(cc, f1, v[2 * k + 1]) : add2(v[2 * k + 1], f1);
      }
    }
  }
  __device__ __forceinline__ void merge(const RowAcc &o) {
#pragma unroll
    for (int q = 0; q < NP; ++q) v[q] = add2(v[q], o.v[q]);
    s += o.s;
  }
  __device__ __forceinline__ void get(float (&o)[BP]) const {
    if constexpr (BP == 1) {
      o[0] = s;
    } else {
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float2 f = upk2(v[q]);
        o[2 * q] = f.x;
        o[2 * q + 1] = f.y;
      }
    }
  }
};
// the sm_100 mixed-precision add: acc + (the bfloat16 half of w), rounded
// once in float -- the exact widening of bfloat16 makes it the unpack-and-add
// result bit for bit, in one instruction instead of two
__device__ __forceinline__ void add_bf16_pair(float &lo_acc, float &hi_acc, unsigned w) {
  asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
      "add.rn.f32.bf16 %0, lo, %0;\n\tadd.rn.f32.bf16 %1, hi, %1;\n\t}"
      : "+f"(lo_acc), "+f"(hi_acc)
      : "r"(w));
}
__device__ __forceinline__ void add_bf16_lo(float &lo_acc, unsigned w) {
  asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %1;\n\tadd.rn.f32.bf16 %0, lo, %0;\n\t}"
      : "+f"(lo_acc)
      : "r"(w));
}

// bfloat16 inputs: plain float accumulators.  With MIX, unit coefficients (the
// combinatorial Laplacian of an unweighted graph) add each value with the
// mixed-precision add, one instruction instead of two: the shared-pattern
// rows take it, being issue-bound (the chain step on the 27-point mesh: 57
// instead of 64 us); the explicit-slice rows, bound by load latency, ran
// slower with it (80 instead of 74 us) and unpack and add.
template <int BP> struct RowAcc<__nv_bfloat16, BP> {
  float a[BP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < BP; ++c) a[c] = 0.f;
  }
  // NW words of 2 values each (low half first) into columns c0, c0 + 1, ...
  template <bool COEF, int NW, bool MIX = false>
  __device__ __forceinline__ void add_words(const unsigned *w, int c0, float coef) {
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      if (c0 + 2 * i >= BP) break;
      if constexpr (COEF || !MIX) {
        const float lo = __uint_as_float(w[i] << 16), hi = __uint_as_float(w[i] & 0xffff0000u);
        a[c0 + 2 * i] = COEF ? fmaf(coef, lo, a[c0 + 2 * i]) : a[c0 + 2 * i] + lo;
        a[c0 + 2 * i + 1] = COEF ? fmaf(coef, hi, a[c0 + 2 * i + 1]) : a[c0 + 2 * i + 1] + hi;
      } else {
        add_bf16_pair(a[c0 + 2 * i], a[c0 + 2 * i + 1], w[i]);
      }
    }
  }
  template <bool COEF>
  __device__ __forceinline__ void add(const __nv_bfloat16 *__restrict__ p, float coef) {
    if constexpr (BP % 8 == 0) {
#pragma unroll
      for (int c = 0; c < BP; c += 8) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p + c));
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
        add_words<COEF, 4>(w, c, coef);
      }
    } else {
#pragma unroll
      for (int c = 0; c < BP; c += 4) {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p + c));
        const unsigned w[2] = {q.x, q.y};
        add_words<COEF, 2>(w, c, coef);
      }
    }
  }
  template <bool COEF, bool MIX = false>
  __device__ __forceinline__ void accum(const RawRow<__nv_bfloat16, BP> &r, float coef) {
    if constexpr (RawRow<__nv_bfloat16, BP>::kWide) {
#pragma unroll
      for (int k = 0; k < BP / 8; ++k) {
        const unsigned w[4] = {r.q[k].x, r.q[k].y, r.q[k].z, r.q[k].w};
        add_words<COEF, 4, MIX>(w, 8 * k, coef);
      }
    } else {
#pragma unroll
      for (int k = 0; k < BP / 4; ++k) {
        const unsigned w[2] = {r.h[k].x, r.h[k].y};
        add_words<COEF, 2, MIX>(w, 4 * k, coef);
      }
    }
  }
  __device__ __forceinline__ void merge(const RowAcc &o) {
#pragma unroll
    for (int c = 0; c < BP; ++c) a[c] += o.a[c];
  }
  __device__ __forceinline__ void get(float (&o)[BP]) const {
#pragma unroll
    for (int c = 0; c < BP; ++c) o[c] = a[c];
  }
};

template <int BP> struct RowAcc<double, BP> {
  double v[BP];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < BP; ++c) v[c] = 0.0;
  }
  template <bool COEF>
  __device__ __forceinline__ void add(const double *__restrict__ p, double coef) {
    double xj[BP];
    load_row<BP>(p, xj);
#pragma unroll
    for (int c = 0; c < BP; ++c) v[c] = COEF ? fma(coef, xj[c], v[c]) : v[c] + xj[c];
  }
  template <bool COEF, bool MIX = false>
  __device__ __forceinline__ void accum(const RawRow<double, BP> &r, double coef) {
#pragma unroll
    for (int c = 0; c < BP; ++c) v[c] = COEF ? fma(coef, r.v[c], v[c]) : v[c] + r.v[c];
  }
  __device__ __forceinline__ void merge(const RowAcc &o) {
#pragma unroll
    for (int c = 0; c < BP; ++c) v[c] += o.v[c];
  }
  __device__ __forceinline__ void get(double (&o)[BP]) const {
#pragma unroll
    for (int c = 0; c < BP; ++c) o[c] = v[c];
  }
};

template <int LAP, typename TI, int BP, bool W>
__device__ __forceinline__ void spmm_accumulate(const LapView &L, const TI *__restrict__ x,
                                                int j, float wv, RowAcc<TI, BP> &acc) {
  using TA = typename AccOf<TI>::T;
  const TI *p = x + static_cast<int64_t>(j) * BP;   // rows exactly BP wide
  if constexpr (LAP == SPHYNX_NORMALIZED || W) {
    TA coef = W ? static_cast<TA>(wv) : TA(1);
    if constexpr (LAP == SPHYNX_NORMALIZED) {
      if (L.gather_scale) coef *= dinv_of<TA>(L, j);
    }
    acc.template add<true>(p, coef);
  } else {
    acc.template add<false>(p, TA(1));
  }
}

// N consecutive entries t0 .. t0 + N - 1 of a row: N column indices, then N
// gathers in flight together, then N accumulations in entry order.
template <int N, int LAP, typename TI, int BP, bool W, class ColAt, class WAt>
__device__ __forceinline__ void spmm_batch(const LapView &L, const TI *__restrict__ x, int t0, ColAt col_at,
                                           WAt w_at, RowAcc<TI, BP> &acc) {
  using TA = typename AccOf<TI>::T;
  int jj[N];
#pragma unroll
  for (int u = 0; u < N; ++u) jj[u] = col_at(t0 + u);
  RawRow<TI, BP> rr[N];
#pragma unroll
  for (int u = 0; u < N; ++u) rr[u].load(x + static_cast<int64_t>(jj[u]) * BP);
#pragma unroll
  for (int u = 0; u < N; ++u) {
    if constexpr (LAP == SPHYNX_NORMALIZED || W) {
      TA coef = W ? static_cast<TA>(w_at(t0 + u)) : TA(1);
      if constexpr (LAP == SPHYNX_NORMALIZED) {
        if (L.gather_scale) coef *= dinv_of<TA>(L, jj[u]);
      }
      acc.template accum<true>(rr[u], coef);
    } else {
      acc.template accum<false>(rr[u], TA(1));
    }
  }
}

// The last rem <= R entries of a row as one batch of exactly rem (selected
// among 1 .. R at run time), so that no gather slot is padded with zeros.
template <int R, int LAP, typename TI, int BP, bool W, class ColAt, class WAt>
__device__ __forceinline__ void spmm_tail(const LapView &L, const TI *__restrict__ x, int t0, int rem,
                                          ColAt col_at, WAt w_at, RowAcc<TI, BP> &acc) {
  if constexpr (R > 0) {
    if (rem == R) {
      spmm_batch<R, LAP, TI, BP, W>(L, x, t0, col_at, w_at, acc);
      return;
    }
    spmm_tail<R - 1, LAP, TI, BP, W>(L, x, t0, rem, col_at, w_at, acc);
  }
}

// One row's d entries in batches of U (see spmm_batch); col_at(t) / w_at(t)
// read entry t < d.
template <int LAP, typename TI, int BP, bool W, class ColAt, class WAt>
__device__ __forceinline__ void spmm_row(const LapView &L, const TI *__restrict__ x, int d,
                                         ColAt col_at, WAt w_at, RowAcc<TI, BP> &acc) {
  using TA = typename AccOf<TI>::T;
  constexpr int U = GatherBatch<TI, BP>::U;
  if constexpr (U > 4) {
    // narrow rows (16 bytes or less): plain batches keep the register count,
    // hence the number of resident warps, high
    int t0 = 0;
    for (; t0 + U <= d; t0 += U) spmm_batch<U, LAP, TI, BP, W>(L, x, t0, col_at, w_at, acc);
    // the remainder (< U entries): a batch of 4 if at least 4 are left, then
    // one batch of exactly what is left
    if (d - t0 >= 4) {
      spmm_batch<4, LAP, TI, BP, W>(L, x, t0, col_at, w_at, acc);
      t0 += 4;
    }
    spmm_tail<3, LAP, TI, BP, W>(L, x, t0, d - t0, col_at, w_at, acc);
    return;
  }
  // wide rows: software pipeline -- the next batch's column indices (and
  // weights) are requested before this batch's gathers, so their latencies overlap
  int jn[U];
  float wn[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    jn[u] = u < d ? col_at(u) : -1;
    if constexpr (W) wn[u] = u < d ? w_at(u) : 0.f;
  }
  for (int t0 = 0; t0 < d; t0 += U) {
    int jj[U];
    float wv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      jj[u] = jn[u];
      if constexpr (W) wv[u] = wn[u];
    }
    const int t1 = t0 + U;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      jn[u] = t1 + u < d ? col_at(t1 + u) : -1;
      if constexpr (W) wn[u] = t1 + u < d ? w_at(t1 + u) : 0.f;
    }
    RawRow<TI, BP> rr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (jj[u] >= 0) rr[u].load(x + static_cast<int64_t>(jj[u]) * BP);
      else rr[u].zero();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if constexpr (LAP == SPHYNX_NORMALIZED || W) {
        TA coef = TA(0);
        if (jj[u] >= 0) {
          coef = W ? static_cast<TA>(wv[u]) : TA(1);
          if constexpr (LAP == SPHYNX_NORMALIZED) {
            if (L.gather_scale) coef *= dinv_of<TA>(L, jj[u]);
          }
        }
        acc.template accum<true>(rr[u], coef);
      } else {
        acc.template accum<false>(rr[u], TA(1));
      }
    }
  }
}

// A row of a shared-pattern slice: entry k of the slice's union U is the
// column row + U[k], present where bit k of the row's mask is set.  Lane k
// holds U[k] (myoff), so each offset reaches the warp by one shuffle and the
// gathers of a batch depend on no load.  Absent entries gather nothing and add
// zero, so the row's sum is the explicit layout's sum, term for term.
template <int R, int LAP, typename TI, int BP>
__device__ __forceinline__ void pattern_batch(const LapView &L, const TI *__restrict__ x, int row, int myoff,
                                              unsigned mk, int k0, RowAcc<TI, BP> &acc) {
  using TA = typename AccOf<TI>::T;
  int jj[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int k = k0 + u;
    const int off = __shfl_sync(kFull, myoff, k);
    jj[u] = ((mk >> k) & 1u) ? row + off : -1;
  }
  RawRow<TI, BP> rr[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if (jj[u] >= 0) rr[u].load(x + static_cast<int64_t>(jj[u]) * BP);
    else rr[u].zero();
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    if constexpr (LAP == SPHYNX_NORMALIZED) {
      const TA coef = jj[u] >= 0 ? (L.gather_scale ? dinv_of<TA>(L, jj[u]) : TA(1)) : TA(0);
      acc.template accum<true>(rr[u], coef);
    } else {
      acc.template accum<false, true>(rr[u], TA(1));
    }
  }
}

template <int R, int LAP, typename TI, int BP>
__device__ __forceinline__ void pattern_tail(const LapView &L, const TI *__restrict__ x, int row, int myoff,
                                             unsigned mk, int k0, int rem, RowAcc<TI, BP> &acc) {
  if constexpr (R > 0) {
    if (rem == R) {
      pattern_batch<R, LAP, TI, BP>(L, x, row, myoff, mk, k0, acc);
      return;
    }
    pattern_tail<R - 1, LAP, TI, BP>(L, x, row, myoff, mk, k0, rem, acc);
  }
}

// nu (<= 31, warp-uniform) union entries in batches of the gather width, the
// last batch exactly as long as what is left
template <int LAP, typename TI, int BP>
__device__ __forceinline__ void spmm_pattern_row(const LapView &L, const TI *__restrict__ x, int row, int myoff,
                                                 unsigned mk, int nu, RowAcc<TI, BP> &acc) {
  constexpr int U = GatherBatch<TI, BP>::U;
  int k0 = 0;
  for (; k0 + U <= nu; k0 += U) pattern_batch<U, LAP, TI, BP>(L, x, row, myoff, mk, k0, acc);
  pattern_tail<U - 1, LAP, TI, BP>(L, x, row, myoff, mk, k0, nu - k0, acc);
}

// the warp's 32 rows row0 .. row0 + 31 of the CSR-staged schedule; s_col and
// s_w are the warp's shared staging areas
template <int LAP, typename TI, typename TT, int BP, bool W, int MODE>
__device__ __forceinline__ void short_rows(const LapView &L, const SpmmDev &a, int64_t row0, int lane, int *s_colw,
                                           float *s_ww) {
  using TA = typename AccOf<TI>::T;
  if (row0 >= L.n) return;  // uniform per warp
  const int64_t row = row0 + lane;
  const bool valid = row < L.n;
  int64_t rb = 0, re = 0;
  if (valid) {
    rb = __ldcs(L.rowptr + row);
    re = __ldcs(L.rowptr + row + 1);
  }
  const int nvalid = L.n - row0 < 32 ? static_cast<int>(L.n - row0) : 32;
  const int64_t wb = __shfl_sync(kFull, rb, 0);
  const int64_t we = __shfl_sync(kFull, re, nvalid - 1);
  const int64_t base = wb & ~static_cast<int64_t>(3);
  const bool staged = we - base <= kStageCap + 4;
  if (staged) {
    // whole 16-byte chunks inside [base, we), then the tail one by one; the
    // column stream is read once, so it is loaded evict-first
    const int64_t vend = we & ~static_cast<int64_t>(3);
    const int nvec = static_cast<int>((vend - base) >> 2);
    const int4 *gc = reinterpret_cast<const int4 *>(L.col + base);
    for (int v = lane; v < nvec; v += 32) *reinterpret_cast<int4 *>(&s_colw[4 * v]) = __ldcs(gc + v);
    for (int64_t gidx = vend + lane; gidx < we; gidx += 32) s_colw[gidx - base] = __ldcs(L.col + gidx);
    if constexpr (W) {
      const float4 *gw = reinterpret_cast<const float4 *>(L.w + base);
      for (int v = lane; v < nvec; v += 32) *reinterpret_cast<float4 *>(&s_ww[4 * v]) = __ldcs(gw + v);
      for (int64_t gidx = vend + lane; gidx < we; gidx += 32) s_ww[gidx - base] = __ldcs(L.w + gidx);
    }
  }
  __syncwarp();
  if (!valid || re - rb > kShortDeg) return;
  const TI *__restrict__ x = static_cast<const TI *>(a.x);
  RowAcc<TI, BP> acc;
  acc.zero();
  const int len = static_cast<int>(re - rb);
  if (staged) {
    const int *sc = &s_colw[rb - base];
    const float *sw = W ? &s_ww[rb - base] : nullptr;
    spmm_row<LAP, TI, BP, W>(
        L, x, len, [&](int t) { return sc[t]; }, [&](int t) { return sw[t]; }, acc);
  } else {
    const int32_t *gc = L.col + rb;
    const float *gw = W ? L.w + rb : nullptr;
    spmm_row<LAP, TI, BP, W>(
        L, x, len, [&](int t) { return __ldg(gc + t); }, [&](int t) { return __ldg(gw + t); }, acc);
  }
  TA sum[BP];
  acc.get(sum);
  spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, sum);
}

template <int LAP, typename TI, typename TT, int BP, bool W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_spmm_short(const LapView L, const SpmmDev a) {
  // column indices (and weights) of each warp's 32 rows, staged from the
  // 16-byte-aligned position at or below the window start
  __shared__ __align__(16) int s_col[kWarpsPerCta][kStageCap + 8];
  __shared__ __align__(16) float s_w[kWarpsPerCta][W ? kStageCap + 8 : 4];
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (a.act_blocks) {
    // a batch's active 1024-row blocks, 128 rows to a CTA item
    const int64_t items = 8 * static_cast<int64_t>(*a.n_act);
    for (int64_t i = blockIdx.x; i < items; i += gridDim.x) {
      const int64_t row0 = static_cast<int64_t>(a.act_blocks[i >> 3]) * 1024 + (i & 7) * 128 + wid * 32;
      short_rows<LAP, TI, TT, BP, W, MODE>(L, a, row0, lane, s_col[wid], s_w[wid]);
      __syncwarp();
    }
    return;
  }
  const int64_t row0 = (static_cast<int64_t>(blockIdx.x) * kWarpsPerCta + wid) * 32;
  short_rows<LAP, TI, TT, BP, W, MODE>(L, a, row0, lane, s_col[wid], s_w[wid]);
}

// SELL-32 schedule: a warp per slice of 32 rows, lane = row.  Entry t of all
// 32 rows is one contiguous segment (64 bytes of 16-bit offsets col - row, or
// 128 bytes of 32-bit indices), so column reads are coalesced without shared
// memory and all of L1 is left to the X gathers.  The slice's format is
// uniform over the warp.
// Slice order: the four warps of a block take slices 2^ls apart, and 2^ls
// consecutive blocks cover a group of 4 * 2^ls slices.  On a mesh whose grid
// lines are 32 * 2^ls rows long, a block's 128 rows then lie on four
// neighbouring lines instead of one, so the X rows its gathers touch overlap
// far more and L1 serves more of them.  The autotuner picks ls per graph.
// Resident 128-thread blocks the gather-latency-bound SELL kernel asks for:
// 16 (32 registers a thread, every warp slot of the SM) for rows of at most
// 16 bytes, 8 (64 registers) for 32-byte float rows.
template <typename TI, int BP> struct SellOccupancy {
  static constexpr bool f32 = std::is_same<TI, float>::value;
  // float rows of 12 and 16 values: without a bound the explicit-slice path
  // took 134-180 registers, three resident blocks, and its gathers waited
  static constexpr int blocks =
      ((std::is_same<TI, __nv_bfloat16>::value && BP <= 8) || (f32 && BP <= 4))
          ? 16
          : (f32 && BP == 8 ? 8 : (f32 && BP == 12 ? 6 : (f32 && BP == 16 ? 4 : 1)));
};

// Slice kinds a launch may meet.  KIND 0: explicit slices of 16- or 32-bit
// indices; 1: only 16-bit ones; 2: shared-pattern slices (kPatternTag in the
// slice offset, block in pcol) besides explicit ones; 3: only shared-pattern
// slices.
template <int LAP, typename TI, typename TT, int BP, bool W, int MODE, int KIND>
__device__ __forceinline__ void sell_slice(const LapView &L, const SpmmDev &a, const int16_t *__restrict__ scol,
                                           const float *__restrict__ sw, const int64_t *__restrict__ sptr,
                                           const int64_t *__restrict__ cptr, const uint8_t *__restrict__ sdeg,
                                           const int16_t *__restrict__ pcol, int64_t slice, int lane) {
  using TA = typename AccOf<TI>::T;
  if (slice * 32 >= L.n) return;  // uniform per warp
  const int64_t row = slice * 32 + lane;
  const int64_t cbase = __ldg(cptr + slice);
  const TI *__restrict__ x = static_cast<const TI *>(a.x);
  RowAcc<TI, BP> acc;
  acc.zero();
  if constexpr (KIND >= 2 && !W) {
    if (KIND == 3 || cbase >= kPatternTag) {
      // one 64-byte offset list and one mask per lane: no per-entry index stream
      const int16_t *pb = pcol + (cbase - kPatternTag);
      const int myoff = __ldg(pb + lane);
      const unsigned mk = __ldg(reinterpret_cast<const unsigned *>(pb + 32) + lane);
      const unsigned any = __reduce_or_sync(kFull, mk & 0x7fffffffu);
      const int nu = 32 - __clz(any);
      spmm_pattern_row<LAP, TI, BP>(L, x, static_cast<int>(row), myoff, mk, nu, acc);
      if (mk >> 31) return;   // long row or padding lane
      TA sum[BP];
      acc.get(sum);
      spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, sum);
      return;
    }
  }
  if constexpr (KIND != 3) {
    const bool valid = row < L.n;
    const int sd = valid ? sdeg[row] : 0xFF;
    const int d = sd == 0xFF ? 0 : sd;
    const float *wp = W ? sw + __ldg(sptr + slice) + lane : nullptr;
    {
      // One bulk L2 prefetch of the slice's whole index block (dmax segments of
      // 64 or 128 bytes, contiguous, 64-byte aligned).  Without it every batch
      // of the row loop waits on DRAM for its segments before it can gather;
      // with it only the first batch does (9 % off the mesh's chain step).
      const int dmax = __reduce_max_sync(kFull, d);
      if (dmax > 0 && lane == 0) {
        const bool nar = KIND == 1 || cbase < 0;
        const void *blkp = nar ? static_cast<const void *>(scol + (~cbase)) : static_cast<const void *>(scol + cbase);
        const unsigned bytes = static_cast<unsigned>(dmax) * (nar ? 64u : 128u);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(blkp), "r"(bytes) : "memory");
      }
    }
    if (KIND == 1 || cbase < 0) {
      const int16_t *cp = scol + (~cbase) + lane;
      const int r = static_cast<int>(row);
      spmm_row<LAP, TI, BP, W>(
          L, x, d, [&](int t) { return r + static_cast<int>(__ldcs(cp + 32 * t)); },
          [&](int t) { return __ldcs(wp + 32 * t); }, acc);
    } else {
      const int32_t *cp = reinterpret_cast<const int32_t *>(scol + cbase) + lane;
      spmm_row<LAP, TI, BP, W>(
          L, x, d, [&](int t) { return __ldcs(cp + 32 * t); }, [&](int t) { return __ldcs(wp + 32 * t); },
          acc);
    }
    if (sd == 0xFF) return;   // padding lane or a long row
    TA sum[BP];
    acc.get(sum);
    spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, sum);
  }
}

template <int LAP, typename TI, typename TT, int BP, bool W, int MODE, int KIND>
__global__ void __launch_bounds__(128, SellOccupancy<TI, BP>::blocks)
k_spmm_sell(const LapView L, const SpmmDev a, const int16_t *__restrict__ scol, const float *__restrict__ sw,
            const int64_t *__restrict__ sptr, const int64_t *__restrict__ cptr, const uint8_t *__restrict__ sdeg,
            const int16_t *__restrict__ pcol, int ls) {
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (a.act_blocks) {
    // a batch's active 1024-row blocks: 32 slices each, four to a CTA item
    const int64_t items = 8 * static_cast<int64_t>(*a.n_act);
    for (int64_t i = blockIdx.x; i < items; i += gridDim.x) {
      const int64_t slice = static_cast<int64_t>(a.act_blocks[i >> 3]) * 32 + (i & 7) * 4 + wid;
      sell_slice<LAP, TI, TT, BP, W, MODE, KIND>(L, a, scol, sw, sptr, cptr, sdeg, pcol, slice, lane);
    }
    return;
  }
  const int64_t blk = blockIdx.x;
  const int64_t slice = ((blk >> ls) << (ls + 2)) + (blk & ((1 << ls) - 1)) + (static_cast<int64_t>(wid) << ls);
  sell_slice<LAP, TI, TT, BP, W, MODE, KIND>(L, a, scol, sw, sptr, cptr, sdeg, pcol, slice, lane);
}

// Medium rows (kShortDeg < degree <= med_max), sorted by degree at create: a
// group of G lanes per row, G the smallest power of two that leaves each lane
// at most kGroupPerLane entries (G = 32 above 32 kGroupPerLane entries), and
// 32 / G rows to a warp.  Lane l of a
// group takes entries l, l + G, l + 2G, ... of its row from the CSR arrays in
// batches of gathers (spmm_row), and a butterfly of shuffles adds the G
// partial sums.  A lane's chain of dependent gathers is thus at most
// kGroupPerLane / U batches long instead of d / U: on a power-law graph one
// lane walking a row of thousands of neighbours set the launch's duration.
// Rounding grows with d / G + log2 G.
template <int LAP, typename TI, typename TT, int BP, bool W, int MODE>
__global__ void __launch_bounds__(128)
k_spmm_group(const LapView L, const SpmmDev a, const int32_t *__restrict__ grow, const int2 *__restrict__ units,
             int64_t n_units) {
  using TA = typename AccOf<TI>::T;
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t unit = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (unit >= n_units) return;  // uniform per warp
  const int2 u = __ldg(units + unit);   // {first sorted row, log2 G | (rows << 8)}
  const int lg = u.y & 0xff, rows = u.y >> 8;
  const int r = lane >> lg, gl = lane & ((1 << lg) - 1);
  int row = -1;
  int64_t beg = 0;
  int d = 0;
  if (r < rows) {
    row = __ldg(grow + u.x + r);
    beg = __ldg(L.rowptr + row);
    d = static_cast<int>(__ldg(L.rowptr + row + 1) - beg);
  }
  const int nl = d > gl ? ((d - gl - 1) >> lg) + 1 : 0;   // this lane's entries
  const int32_t *cp = L.col + beg + gl;
  const float *wp = W ? L.w + beg + gl : nullptr;
  const TI *__restrict__ x = static_cast<const TI *>(a.x);
  RowAcc<TI, BP> acc;
  acc.zero();
  spmm_row<LAP, TI, BP, W>(
      L, x, nl, [&](int t) { return __ldcs(cp + (static_cast<int64_t>(t) << lg)); },
      [&](int t) { return __ldcs(wp + (static_cast<int64_t>(t) << lg)); }, acc);
  TA sum[BP];
  acc.get(sum);
  for (int off = (1 << lg) >> 1; off > 0; off >>= 1) {   // lg is uniform per warp
#pragma unroll
    for (int c = 0; c < BP; ++c) sum[c] += __shfl_xor_sync(kFull, sum[c], off);
  }
  if (row < 0 || gl != 0) return;
  spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, sum);
}

// One warp per long-row work item: partial[item] = sum over the item's entries.
template <int LAP, typename TI, int BP, bool W>
__global__ void __launch_bounds__(256)
k_spmm_long(const LapView L, const SpmmDev a, const int64_t *__restrict__ items, int64_t n_items,
            typename AccOf<TI>::T *__restrict__ partials) {
  using TA = typename AccOf<TI>::T;
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t item = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (item >= n_items) return;
  const int64_t b = items[item * 4 + 1], e = items[item * 4 + 2];
  const TI *__restrict__ x = static_cast<const TI *>(a.x);
  RowAcc<TI, BP> racc;
  racc.zero();
  // lane l: entries b + l, b + l + 32, ... in order, in batches of gathers
  const int nl = e - b > lane ? static_cast<int>((e - b - lane - 1) / 32) + 1 : 0;
  const int32_t *cp = L.col + b + lane;
  const float *wp = W ? L.w + b + lane : nullptr;
  spmm_row<LAP, TI, BP, W>(
      L, x, nl, [&](int t) { return __ldcs(cp + 32 * static_cast<int64_t>(t)); },
      [&](int t) { return __ldcs(wp + 32 * static_cast<int64_t>(t)); }, racc);
  TA acc[BP];
  racc.get(acc);
#pragma unroll
  for (int c = 0; c < BP; ++c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(kFull, acc[c], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < BP; ++c) partials[item * BP + c] = acc[c];
  }
}

// One warp per long row: lane l adds the row's partials l, l + 32, ... in
// item order, a butterfly of shuffles adds the lanes' sums (a fixed order,
// so results repeat exactly), and lane 0 applies the epilogue.
template <int LAP, typename TI, typename TT, int BP, int MODE>
__global__ void __launch_bounds__(128)
k_spmm_finalize(const LapView L, const SpmmDev a, const int64_t *__restrict__ split, int64_t n_long,
                const typename AccOf<TI>::T *__restrict__ partials) {
  using TA = typename AccOf<TI>::T;
  if (a.done && *a.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t t = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (t >= n_long) return;   // uniform per warp
  const int64_t row = split[t * 3], first = split[t * 3 + 1], cnt = split[t * 3 + 2];
  TA acc[BP];
#pragma unroll
  for (int c = 0; c < BP; ++c) acc[c] = TA(0);
  for (int64_t s = first + lane; s < first + cnt; s += 32) {
#pragma unroll
    for (int c = 0; c < BP; ++c) acc[c] += partials[s * BP + c];
  }
#pragma unroll
  for (int c = 0; c < BP; ++c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(kFull, acc[c], off);
  }
  if (lane == 0) spmm_epilogue<LAP, TI, TT, BP, MODE>(L, a, row, acc);
}

template <int LAP, typename TI, typename TT, int BP, bool W, int MODE>
void spmm_launch_t(sphynx_graph *g, const SpmmDev &a) {
  using TA = typename AccOf<TI>::T;
  LapView L = g->view();
  if (a.xe != a.x) L.gather_scale = 0;   // x holds D^{-1/2} X
  if (a.coef_csr) {                      // the coefficients already hold D^{-1/2}_j
    L.w = a.coef_csr;
    L.gather_scale = 0;
  }
  cudaStream_t st = g->stream;
  const int64_t warps = (g->n + 31) / 32;
  const int64_t grid = (warps + kWarpsPerCta - 1) / kWarpsPerCta;
  if (grid > 0) {
    const SpmmPlan &p = g->plan;
    if (p.variant == kSell32 || (p.variant == kSellPattern && !W)) {
      // whole groups of 4 * 2^ls slices, 2^ls blocks each
      const int ls = p.sell_ls;
      const unsigned gs = a.act_blocks ? static_cast<unsigned>(kListGrid)
                                       : static_cast<unsigned>(((warps + (int64_t{4} << ls) - 1) >> (ls + 2)) << ls);
      const int16_t *sc = p.sell_col.as<int16_t>();
      const float *swp = a.coef_sell ? a.coef_sell : p.sell_w.as<float>();
      const int64_t *sp = p.sell_ptr.as<int64_t>();
      const uint8_t *sd = p.sell_deg.as<uint8_t>();
      bool launched = false;
      if constexpr (!W) {
        if (p.variant == kSellPattern) {
          const int64_t *pc = p.pat_cptr.as<int64_t>();
          const int16_t *pcl = p.pat_col.as<int16_t>();
          if (p.pat_all)
            k_spmm_sell<LAP, TI, TT, BP, W, MODE, 3><<<gs, 128, 0, st>>>(L, a, sc, swp, sp, pc, sd, pcl, ls);
          else
            k_spmm_sell<LAP, TI, TT, BP, W, MODE, 2><<<gs, 128, 0, st>>>(L, a, sc, swp, sp, pc, sd, pcl, ls);
          launched = true;
        }
      }
      if (!launched) {
        if (p.sell_narrow == (g->n + 31) / 32)
          k_spmm_sell<LAP, TI, TT, BP, W, MODE, 1><<<gs, 128, 0, st>>>(L, a, sc, swp, sp, p.sell_cptr.as<int64_t>(),
                                                                       sd, nullptr, ls);
        else
          k_spmm_sell<LAP, TI, TT, BP, W, MODE, 0><<<gs, 128, 0, st>>>(L, a, sc, swp, sp, p.sell_cptr.as<int64_t>(),
                                                                       sd, nullptr, ls);
      }
    } else {
      const unsigned gsh = a.act_blocks ? static_cast<unsigned>(kListGrid) : static_cast<unsigned>(grid);
      k_spmm_short<LAP, TI, TT, BP, W, MODE><<<gsh, 32 * kWarpsPerCta, 0, st>>>(L, a);
    }
    SPX_LAUNCHED();
    g->ctr.launches++;
  }
  if (g->plan.n_units > 0) {
    const int64_t gm = (g->plan.n_units * 32 + 127) / 128;
    k_spmm_group<LAP, TI, TT, BP, W, MODE><<<static_cast<unsigned>(gm), 128, 0, st>>>(
        L, a, g->plan.grp_row.as<int32_t>(), g->plan.grp_unit.as<int2>(), g->plan.n_units);
    SPX_LAUNCHED();
    g->ctr.launches++;
  }
  if (g->plan.n_long > 0) {
    TA *part = g->plan.partials.as<TA>();
    const int64_t gl = (g->plan.n_items * 32 + 255) / 256;
    k_spmm_long<LAP, TI, BP, W><<<static_cast<unsigned>(gl), 256, 0, st>>>(
        L, a, g->plan.items.as<int64_t>(), g->plan.n_items, part);
    SPX_LAUNCHED();
    const int64_t gf = (g->plan.n_long * 32 + 127) / 128;
    k_spmm_finalize<LAP, TI, TT, BP, MODE><<<static_cast<unsigned>(gf), 128, 0, st>>>(
        L, a, g->plan.split.as<int64_t>(), g->plan.n_long, part);
    SPX_LAUNCHED();
    g->ctr.launches += 2;
  }
}

template <int LAP, typename TI, typename TT, bool W, int MODE>
void spmm_bp(sphynx_graph *g, const SpmmDev &a, int bp) {
  switch (bp) {
    case 4: spmm_launch_t<LAP, TI, TT, 4, W, MODE>(g, a); break;
    case 8: spmm_launch_t<LAP, TI, TT, 8, W, MODE>(g, a); break;
    case 12: spmm_launch_t<LAP, TI, TT, 12, W, MODE>(g, a); break;
    case 16: spmm_launch_t<LAP, TI, TT, 16, W, MODE>(g, a); break;
    default: fail(SPHYNX_ERR_INVALID_ARG, "block width %d not supported", bp);
  }
}

template <typename TI, typename TT, int MODE>
void spmm_lapw(sphynx_graph *g, const SpmmDev &a, int lap, int bp) {
  const bool w = g->weighted || a.coef_csr != nullptr;
  if (bp == 1) {
    if constexpr (MODE == 0 && !std::is_same<TI, __nv_bfloat16>::value) {
      if (lap == SPHYNX_NORMALIZED) {
        if (w) spmm_launch_t<SPHYNX_NORMALIZED, TI, TT, 1, true, 0>(g, a);
        else spmm_launch_t<SPHYNX_NORMALIZED, TI, TT, 1, false, 0>(g, a);
      } else {
        if (w) spmm_launch_t<SPHYNX_COMBINATORIAL, TI, TT, 1, true, 0>(g, a);
        else spmm_launch_t<SPHYNX_COMBINATORIAL, TI, TT, 1, false, 0>(g, a);
      }
      return;
    }
    fail(SPHYNX_ERR_INVALID_ARG, "single-column product only in plain mode for float/double");
  }
  if (lap == SPHYNX_NORMALIZED) {
    if (w) spmm_bp<SPHYNX_NORMALIZED, TI, TT, true, MODE>(g, a, bp);
    else spmm_bp<SPHYNX_NORMALIZED, TI, TT, false, MODE>(g, a, bp);
  } else {
    if (w) spmm_bp<SPHYNX_COMBINATORIAL, TI, TT, true, MODE>(g, a, bp);
    else spmm_bp<SPHYNX_COMBINATORIAL, TI, TT, false, MODE>(g, a, bp);
  }
}

void spmm_dispatch_f64(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d);
void spmm_dispatch_f32(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d);
void spmm_dispatch_bf16(sphynx_graph *g, const SpmmArgs &a, const SpmmDev &d);

}  // namespace sphynx
