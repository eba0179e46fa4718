/* Native fast paths of the seeded graph generators in graphs.py.
 *
 * Same definitions, same draws: the numpy code in graphs.py is the reference
 * and a CPU test checks that both produce the same graph bit for bit.  These
 * routines only build inputs (edge draws, sorting, deduplication, the largest
 * connected component, edge weights); none of the partitioning method's
 * arithmetic lives here.  Built with -ffp-contract=off so that the few
 * floating-point expressions round exactly as numpy's do on every machine.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a
 * counter-based generator, exactly as graphs.uniform01 defines it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL
#define MIX1 0xBF58476D1CE4E5B9ULL
#define MIX2 0x94D049BB133111EBULL

static inline uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= MIX1;
  z ^= z >> 27;
  z *= MIX2;
  z ^= z >> 31;
  return z;
}

static uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed * 0x632BE59BD9B4E019ULL + stream * GOLDEN + 0x5851F42D4C957F2DULL);
}

/* the ctr-th draw (ctr >= 1) of a stream, in [0, 1) with 53 bits */
static inline double u01(uint64_t key, uint64_t ctr) {
  return (double)(mix64(key + ctr * GOLDEN) >> 11) * (1.0 / 9007199254740992.0);
}

/* R-MAT edge draws e = 0..m-1 as undirected keys min * n + max (n = 2^scale);
 * a self-loop gets UINT64_MAX.  Level l of edge e uses draw e + 1 of stream
 * 100 + l, as graphs.rmat does. */
void gen_rmat_keys(int scale, int64_t m, double a, double ab, double abc, uint64_t seed, uint64_t *keys) {
  uint64_t lk[64];
  for (int l = 0; l < scale; ++l) lk[l] = stream_key(seed, 100 + (uint64_t)l);
  const uint64_t n = 1ULL << scale;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    uint64_t s = 0, d = 0;
    for (int l = 0; l < scale; ++l) {
      const double u = u01(lk[l], (uint64_t)e + 1);
      const uint64_t bit = 1ULL << (scale - 1 - l);
      if (u >= ab) s |= bit;
      if ((u >= a && u < ab) || u >= abc) d |= bit;
    }
    keys[e] = s == d ? UINT64_MAX : (s < d ? s * n + d : d * n + s);
  }
}

/* Sort keys[0..m) ascending (least significant digit first, 16-bit digits over
 * the low `bits` bits; UINT64_MAX entries are moved to the end first) and drop
 * duplicates and UINT64_MAX.  Returns the number of distinct keys, left at the
 * front of keys; tmp holds m entries.  Returns -1 if memory runs out. */
int64_t gen_sort_unique(uint64_t *keys, uint64_t *tmp, int64_t m, int bits) {
  int64_t live = 0;
  for (int64_t i = 0; i < m; ++i)
    if (keys[i] != UINT64_MAX) keys[live++] = keys[i];
  int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536);
  if (!cnt) return -1;
  uint64_t *src = keys, *dst = tmp;
  for (int shift = 0; shift < bits; shift += 16) {
    memset(cnt, 0, sizeof(int64_t) * 65536);
    for (int64_t i = 0; i < live; ++i) cnt[(src[i] >> shift) & 0xFFFF]++;
    int64_t run = 0;
    for (int d = 0; d < 65536; ++d) {
      const int64_t c = cnt[d];
      cnt[d] = run;
      run += c;
    }
    for (int64_t i = 0; i < live; ++i) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
    uint64_t *t = src;
    src = dst;
    dst = t;
  }
  free(cnt);
  if (src != keys) memcpy(keys, src, sizeof(uint64_t) * (size_t)live);
  int64_t u = 0;
  for (int64_t i = 0; i < live; ++i)
    if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
  return u;
}

/* CSR of the simple undirected graph whose distinct sorted keys a * n + b
 * (a < b) are given: row_ptr[n + 1], col[2u], columns sorted within each row.
 * For row r the entries with a column below r (from keys (c, r)) are written
 * first, in ascending c, then those above r (from keys (r, c)), ascending. */
int gen_csr_from_keys(int64_t n, const uint64_t *keys, int64_t u, int64_t *row_ptr, int32_t *col) {
  memset(row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < u; ++i) {
    row_ptr[keys[i] / (uint64_t)n + 1]++;
    row_ptr[keys[i] % (uint64_t)n + 1]++;
  }
  for (int64_t r = 0; r < n; ++r) row_ptr[r + 1] += row_ptr[r];
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!cur) return -1;
  memcpy(cur, row_ptr, sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < u; ++i) {
    const uint64_t a = keys[i] / (uint64_t)n, b = keys[i] % (uint64_t)n;
    col[cur[b]++] = (int32_t)a;
  }
  for (int64_t i = 0; i < u; ++i) {
    const uint64_t a = keys[i] / (uint64_t)n, b = keys[i] % (uint64_t)n;
    col[cur[a]++] = (int32_t)b;
  }
  free(cur);
  return 0;
}

static int64_t uf_find(int64_t *p, int64_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

/* Connected components: label[v] in 0..ncomp-1, numbered in the order of each
 * component's smallest vertex (the order a search from vertex 0 upwards finds
 * them).  Returns ncomp, or -1 if memory runs out. */
int64_t gen_components(int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t *label) {
  int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!p) return -1;
  for (int64_t v = 0; v < n; ++v) p[v] = v;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
      int64_t x = uf_find(p, v), y = uf_find(p, col[k]);
      if (x == y) continue;
      if (x < y) p[y] = x;
      else p[x] = y;
    }
  int64_t ncomp = 0;
  for (int64_t v = 0; v < n; ++v) label[v] = -1;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t r = uf_find(p, v);
    if (label[r] < 0) label[r] = ncomp++;
    label[v] = label[r];
  }
  free(p);
  return ncomp;
}

/* The induced subgraph on the vertices labelled `keep`, renumbered in their
 * original order.  out_row_ptr[n_keep + 1], out_col and out_w (if w) sized by
 * the caller (the kept rows' entries).  Returns the kept entry count. */
int64_t gen_induced(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w, const int64_t *label,
                    int64_t keep, int64_t *out_row_ptr, int32_t *out_col, float *out_w) {
  int64_t *newid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!newid) return -1;
  int64_t nk = 0;
  for (int64_t v = 0; v < n; ++v) newid[v] = label[v] == keep ? nk++ : -1;
  int64_t e = 0;
  out_row_ptr[0] = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (label[v] != keep) continue;
    for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
      out_col[e] = (int32_t)newid[col[k]];
      if (w) out_w[e] = w[k];
      ++e;
    }
    out_row_ptr[newid[v] + 1] = e;
  }
  free(newid);
  return e;
}

/* FP32 weights uniform in [lo, hi), one draw per unordered pair {r, c}:
 * draw a * n + b + 1 (a = min, b = max) of stream 31, as
 * graphs.random_edge_weights defines it. */
void gen_edge_weights(int64_t n, const int64_t *row_ptr, const int32_t *col, double lo, double hi, uint64_t seed,
                      float *w) {
  const uint64_t key = stream_key(seed, 31);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t r = 0; r < n; ++r)
    for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
      const uint64_t c = (uint64_t)col[k];
      const uint64_t a = (uint64_t)r < c ? (uint64_t)r : c, b = (uint64_t)r < c ? c : (uint64_t)r;
      const double u = u01(key, a * (uint64_t)n + b + 1);
      w[k] = (float)(lo + (hi - lo) * u);
    }
}

/* Random geometric graph: points (x_i, y_i) = draw i + 1 of streams 21 and 22
 * (as graphs.rgg draws them), joined when their distance is at most r.
 * Pairs are found through a uniform grid of cells of side >= r and written as
 * keys min * n + max (each pair once, unsorted).  Returns the number of keys,
 * or -1 if more than cap would be written (or memory runs out). */
int64_t gen_rgg_keys(int64_t n, double r, uint64_t seed, uint64_t *keys, int64_t cap) {
  if (n < 1) return 0;
  const uint64_t kx = stream_key(seed, 21), ky = stream_key(seed, 22);
  double *x = (double *)malloc(sizeof(double) * (size_t)n), *y = (double *)malloc(sizeof(double) * (size_t)n);
  int64_t nc = (int64_t)(1.0 / r);
  if (nc < 1) nc = 1;
  if (nc > 65536) nc = 65536;
  const int64_t ncell = nc * nc;
  int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n), *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!x || !y || !start || !order || !cell) {
    free(x); free(y); free(start); free(order); free(cell);
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    x[i] = u01(kx, (uint64_t)i + 1);
    y[i] = u01(ky, (uint64_t)i + 1);
    int64_t cx = (int64_t)(x[i] * (double)nc), cy = (int64_t)(y[i] * (double)nc);
    if (cx >= nc) cx = nc - 1;
    if (cy >= nc) cy = nc - 1;
    cell[i] = cy * nc + cx;
    start[cell[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  {
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    if (!cur) {
      free(x); free(y); free(start); free(order); free(cell);
      return -1;
    }
    memcpy(cur, start, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) order[cur[cell[i]]++] = i;
    free(cur);
  }
  const double r2 = r * r;
  int64_t m = 0;
  for (int64_t i = 0; i < n && m >= 0; ++i) {
    const int64_t cx = cell[i] % nc, cy = cell[i] / nc;
    for (int64_t dy = -1; dy <= 1 && m >= 0; ++dy)
      for (int64_t dx = -1; dx <= 1; ++dx) {
        const int64_t ax = cx + dx, ay = cy + dy;
        if (ax < 0 || ay < 0 || ax >= nc || ay >= nc) continue;
        const int64_t c = ay * nc + ax;
        for (int64_t k = start[c]; k < start[c + 1]; ++k) {
          const int64_t j = order[k];
          if (j <= i) continue;
          const double ddx = x[i] - x[j], ddy = y[i] - y[j];
          if (ddx * ddx + ddy * ddy <= r2) {
            if (m >= cap) {
              m = -1;
              break;
            }
            keys[m++] = (uint64_t)i * (uint64_t)n + (uint64_t)j;
          }
        }
        if (m < 0) break;
      }
  }
  free(x); free(y); free(start); free(order); free(cell);
  return m;
}
