/*
 * sz3o.c -- serial CPU oracle of the SZ3-Interp hot path.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark.  The CUDA library never includes, links or calls
 * anything here.  See sz3o.h for what is computed and where the paper defines
 * it.  Parity status of each function (what pins it) is listed in the header
 * comment of every function below and in the test files tests/test_oracle_*.py.
 */
#include "sz3o.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs FLT_EVAL_METHOD == 0 (every operation rounded in its own type)"
#endif

/* ---------------------------------------------------------------------------
 * Geometry and parameter checks.
 * ------------------------------------------------------------------------- */
typedef struct {
  uint32_t ndim, L;
  uint64_t n[4];      /* extents, slowest first */
  uint64_t stride[4]; /* row-major element strides */
  uint64_t N;
  const sz3o_params* p;
} walk_geom;

static int level_interp(const walk_geom* g, uint32_t l) {
  return g->p->per_level ? g->p->level_interp[l] : (int)g->p->interp;
}

static const uint8_t* level_order(const walk_geom* g, uint32_t l) {
  return g->p->per_level ? g->p->level_order[l] : g->p->dim_order;
}

/* Is axis d one of order[0..k-1]? */
static int earlier_in_order(const uint8_t* order, uint32_t k, uint32_t d) {
  uint32_t j;
  for (j = 0; j < k; ++j)
    if (order[j] == d) return 1;
  return 0;
}

static int is_permutation(const uint8_t* o, uint32_t ndim) {
  uint32_t seen = 0, k;
  for (k = 0; k < ndim; ++k) {
    if (o[k] >= ndim) return 0;
    if (seen & (1u << o[k])) return 0;
    seen |= 1u << o[k];
  }
  return 1;
}

static int geom_of(const sz3o_params* p, walk_geom* g) {
  uint32_t d, l;
  uint64_t maxn = 1;
  if (!p) return SZ3O_E_INVAL;
  if (p->dtype != SZ3O_F32 && p->dtype != SZ3O_F64) return SZ3O_E_INVAL;
  if (p->ndim < 1 || p->ndim > 4) return SZ3O_E_INVAL;
  if (p->eb_mode != SZ3O_EB_ABS && p->eb_mode != SZ3O_EB_REL) return SZ3O_E_INVAL;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return SZ3O_E_INVAL;
  if (p->radius < 2 || p->radius > 32768) return SZ3O_E_INVAL;
  if (p->chunk_codes < 8 || p->chunk_codes > 65536 || (p->chunk_codes % 8) != 0) return SZ3O_E_INVAL;
  if (p->per_level > 1) return SZ3O_E_INVAL;
  g->ndim = p->ndim;
  g->N = 1;
  g->p = p;
  for (d = 0; d < p->ndim; ++d) {
    if (p->dims[d] < 1 || p->dims[d] > ((uint64_t)1 << 31)) return SZ3O_E_INVAL;
    g->n[d] = p->dims[d];
    if (g->n[d] > maxn) maxn = g->n[d];
    if (g->N > (((uint64_t)1 << 31) / g->n[d])) return SZ3O_E_INVAL; /* N <= 2^31 */
    g->N *= g->n[d];
  }
  for (d = p->ndim; d < 4; ++d) g->n[d] = 1;
  g->stride[p->ndim - 1] = 1;
  for (d = p->ndim - 1; d > 0; --d) g->stride[d - 1] = g->stride[d] * g->n[d];
  g->L = 0;
  while (((uint64_t)1 << g->L) < maxn) ++g->L;
  if (!p->per_level) {
    if (p->interp > SZ3O_CUBIC) return SZ3O_E_INVAL;
    if (!is_permutation(p->dim_order, p->ndim)) return SZ3O_E_INVAL;
  } else {
    for (l = 1; l <= g->L; ++l) {
      if (p->level_interp[l] > SZ3O_CUBIC) return SZ3O_E_INVAL;
      if (!is_permutation(p->level_order[l], p->ndim)) return SZ3O_E_INVAL;
    }
  }
  return SZ3O_OK;
}

int sz3o_shape(const sz3o_params* p, uint64_t* n_points, uint32_t* n_levels) {
  walk_geom g;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  if (n_points) *n_points = g.N;
  if (n_levels) *n_levels = g.L;
  return SZ3O_OK;
}

/* ---------------------------------------------------------------------------
 * Selection helpers (type independent): candidates, sample blocks.
 * Candidate c = 2 o + interp: interp 0 linear / 1 cubic, o an axis order of
 * the list below (3-D: (0,1,2), (1,2,0), (2,0,1), (2,1,0); 2-D: (0,1), (1,0)
 * listed twice, so the later copies never win a tie; 1-D: (0)).
 * Sample blocks of level l: up to 16 points per axis of G_{l-1} (the grid of
 * stride 2^(l-1)); block b starts on axis d at splitmix64(key) mod
 * (m_d - span_d + 1), key = seed ^ (l << 48) ^ (b << 8) ^ d, with splitmix64
 * the published SplitMix64 output function applied to key.
 * ------------------------------------------------------------------------- */
#define SZ3O_SEL_MAX_BLOCKS 1024

typedef struct {
  uint32_t n;  /* 0: the whole grid */
  uint64_t lo[SZ3O_SEL_MAX_BLOCKS][4], hi[SZ3O_SEL_MAX_BLOCKS][4];
} sel_blocks;

static const uint8_t* sel_order(uint32_t ndim, uint32_t o) {
  static const uint8_t o3[4][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const uint8_t o2[4][2] = {{0, 1}, {1, 0}, {0, 1}, {1, 0}};
  static const uint8_t o1[1] = {0};
  if (ndim == 3) return o3[o];
  if (ndim == 2) return o2[o];
  return o1;
}

static uint64_t splitmix64(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void sel_make_blocks(const walk_geom* g, uint32_t l, uint32_t nblocks, uint64_t seed, sel_blocks* blk) {
  const uint64_t s = (uint64_t)1 << (l - 1);
  uint32_t b, d;
  blk->n = nblocks > SZ3O_SEL_MAX_BLOCKS ? SZ3O_SEL_MAX_BLOCKS : nblocks;
  for (b = 0; b < blk->n; ++b)
    for (d = 0; d < g->ndim; ++d) {
      const uint64_t m = (g->n[d] + s - 1) / s;
      const uint64_t span = m < 16 ? m : 16;
      const uint64_t key = seed ^ ((uint64_t)l << 48) ^ ((uint64_t)b << 8) ^ (uint64_t)d;
      const uint64_t o = splitmix64(key) % (m - span + 1);
      blk->lo[b][d] = o;
      blk->hi[b][d] = o + span;
    }
}

/* Is grid point gc inside one of blocks 0..b-1? */
static int sel_in_earlier(const sel_blocks* blk, uint32_t b, const uint64_t* gc, uint32_t ndim) {
  uint32_t e, d;
  for (e = 0; e < b; ++e) {
    int in = 1;
    for (d = 0; d < ndim && in; ++d) in = gc[d] >= blk->lo[e][d] && gc[d] < blk->hi[e][d];
    if (in) return 1;
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * The two type instantiations.
 * ------------------------------------------------------------------------- */
#define T float
#define SFX _f32
#define FABS fabsf
#define NEXTAFTER nextafterf
#include "sz3o_typed.inc"
#undef T
#undef SFX
#undef FABS
#undef NEXTAFTER

#define T double
#define SFX _f64
#define FABS fabs
#define NEXTAFTER nextafter
#include "sz3o_typed.inc"
#undef T
#undef SFX
#undef FABS
#undef NEXTAFTER

/* ---------------------------------------------------------------------------
 * Traversal order (the reading of the interpolation schedule): spatial index
 * of the point behind every code.  Uses the same walk as quantize, with a
 * visitor that records indices instead of values.
 * ------------------------------------------------------------------------- */
int sz3o_traversal(const sz3o_params* p, uint64_t* spatial, uint64_t n) {
  walk_geom g;
  uint64_t pos = 0;
  uint32_t l;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  if (n < g.N) return SZ3O_E_CAPACITY;
  spatial[pos++] = 0;
  for (l = g.L; l >= 1; --l) {
    uint64_t s = (uint64_t)1 << (l - 1);
    const uint8_t* order = level_order(&g, l);
    uint32_t k;
    for (k = 0; k < g.ndim; ++k) {
      uint32_t a = order[k], d;
      uint64_t start[4], step[4], c[4];
      int done = 0;
      for (d = 0; d < g.ndim; ++d) {
        start[d] = (d == a) ? s : 0;
        step[d] = (d == a) ? 2 * s : (earlier_in_order(order, k, d) ? s : 2 * s);
        if (start[d] >= g.n[d]) done = 1;
        c[d] = start[d];
      }
      while (!done) {
        uint64_t idx = 0;
        int dd;
        for (d = 0; d < g.ndim; ++d) idx += c[d] * g.stride[d];
        spatial[pos++] = idx;
        for (dd = (int)g.ndim - 1; dd >= 0; --dd) {
          c[dd] += step[dd];
          if (c[dd] < g.n[dd]) break;
          c[dd] = start[dd];
          if (dd == 0) done = 1;
        }
      }
    }
  }
  return pos == g.N ? SZ3O_OK : SZ3O_E_INVAL;
}

int sz3o_error_bound(const sz3o_params* p, const void* x, double* eb_abs, void* eb_T) {
  walk_geom g;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  if (p->dtype == SZ3O_F32) return eb_of_f32(p, (const float*)x, g.N, eb_abs, (float*)eb_T);
  return eb_of_f64(p, (const double*)x, g.N, eb_abs, (double*)eb_T);
}

int sz3o_quantize1(uint32_t dtype, const void* x, const void* pred, const void* eb_T,
                   uint32_t radius, uint32_t* code, void* recon) {
  if (radius < 2 || radius > 32768) return SZ3O_E_INVAL;
  if (dtype == SZ3O_F32) {
    float e = *(const float*)eb_T;
    if (!isnormal(e) || !(e > 0)) return SZ3O_E_INVAL;
    *code = quantize_f32(*(const float*)x, *(const float*)pred, e, 1.0f / e, radius, (float*)recon);
  } else if (dtype == SZ3O_F64) {
    double e = *(const double*)eb_T;
    if (!isnormal(e) || !(e > 0)) return SZ3O_E_INVAL;
    *code = quantize_f64(*(const double*)x, *(const double*)pred, e, 1.0 / e, radius, (double*)recon);
  } else {
    return SZ3O_E_INVAL;
  }
  return SZ3O_OK;
}

int sz3o_quantize(const sz3o_params* p, const void* x, uint16_t* codes, void* unpred,
                  uint64_t* n_unpred, void* recon, void* eb_T) {
  walk_geom g;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  if (p->dtype == SZ3O_F32)
    return quantize_field_f32(p, &g, (const float*)x, codes, (float*)unpred, n_unpred,
                              (float*)recon, (float*)eb_T, NULL);
  return quantize_field_f64(p, &g, (const double*)x, codes, (double*)unpred, n_unpred,
                            (double*)recon, (double*)eb_T, NULL);
}

int sz3o_recover(const sz3o_params* p, const void* eb_T, const uint16_t* codes,
                 const void* unpred, uint64_t n_unpred, void* out) {
  walk_geom g;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  if (p->dtype == SZ3O_F32)
    return recover_field_f32(p, &g, *(const float*)eb_T, codes, (const float*)unpred, n_unpred,
                             (float*)out);
  return recover_field_f64(p, &g, *(const double*)eb_T, codes, (const double*)unpred, n_unpred,
                           (double*)out);
}

/* ---------------------------------------------------------------------------
 * Histogram (the frequencies the Huffman tree is built from, Sec. 3.2 Encoder).
 * ------------------------------------------------------------------------- */
int sz3o_histogram(const uint16_t* codes, uint64_t n, uint64_t* hist) {
  uint64_t i;
  memset(hist, 0, 65536 * sizeof(uint64_t));
  for (i = 0; i < n; ++i) hist[codes[i]]++;
  return SZ3O_OK;
}

/* ---------------------------------------------------------------------------
 * Huffman code lengths (Sec. 3.2 Encoder: tree built greedily from the
 * frequencies).  Two-queue construction over the used symbols sorted by
 * (frequency, symbol): each step joins the two lightest fronts; on equal
 * weight the leaf queue is taken first; the internal queue is FIFO.  A code
 * length is the depth of the leaf; a single used symbol gets length 1.  If the
 * longest code exceeds lmax, every used frequency f becomes max(1, f >> 1) and
 * the tree is rebuilt.
 * ------------------------------------------------------------------------- */
typedef struct {
  uint64_t f;
  uint32_t s;
} leaf_t;

static int leaf_cmp(const void* A, const void* B) {
  const leaf_t* a = (const leaf_t*)A;
  const leaf_t* b = (const leaf_t*)B;
  if (a->f != b->f) return a->f < b->f ? -1 : 1;
  return a->s < b->s ? -1 : (a->s > b->s ? 1 : 0);
}

/* Returns the longest length, or 0 on allocation failure. */
static uint32_t build_lengths(const uint64_t* freq, uint32_t nsym, uint8_t* len, uint32_t* nused) {
  leaf_t* leaves;
  uint64_t* nodef;     /* internal node weights, creation order        */
  uint32_t* parent;    /* parent of node j (leaves: j < K; internal: K + i) */
  uint32_t* depth;
  uint32_t K = 0, i, li = 0, ni = 0, nn = 0, maxlen = 0;
  for (i = 0; i < nsym; ++i) len[i] = 0;
  for (i = 0; i < nsym; ++i)
    if (freq[i]) ++K;
  *nused = K;
  if (K == 0) return 1;
  if (K == 1) {
    for (i = 0; i < nsym; ++i)
      if (freq[i]) len[i] = 1;
    return 1;
  }
  leaves = (leaf_t*)malloc(sizeof(leaf_t) * K);
  nodef = (uint64_t*)malloc(sizeof(uint64_t) * K);
  parent = (uint32_t*)malloc(sizeof(uint32_t) * 2 * K);
  depth = (uint32_t*)malloc(sizeof(uint32_t) * 2 * K);
  if (!leaves || !nodef || !parent || !depth) {
    free(leaves);
    free(nodef);
    free(parent);
    free(depth);
    return 0;
  }
  K = 0;
  for (i = 0; i < nsym; ++i)
    if (freq[i]) {
      leaves[K].f = freq[i];
      leaves[K].s = i;
      ++K;
    }
  qsort(leaves, K, sizeof(leaf_t), leaf_cmp);
  /* K - 1 merges.  Node ids: leaf j -> j, internal i -> K + i. */
  while (nn < K - 1) {
    uint32_t pick[2];
    uint64_t w[2];
    int t;
    for (t = 0; t < 2; ++t) {
      if (li < K && (ni >= nn || leaves[li].f <= nodef[ni])) {
        pick[t] = li;
        w[t] = leaves[li].f;
        ++li;
      } else {
        pick[t] = K + ni;
        w[t] = nodef[ni];
        ++ni;
      }
    }
    nodef[nn] = w[0] + w[1];
    parent[pick[0]] = K + nn;
    parent[pick[1]] = K + nn;
    ++nn;
  }
  /* Depths: the root is the last internal node; parents are created after
   * their children, so walking internal nodes from last to first sees every
   * parent before its children. */
  depth[K + nn - 1] = 0;
  for (i = nn - 1; i-- > 0;) depth[K + i] = depth[parent[K + i]] + 1;
  for (i = 0; i < K; ++i) {
    uint32_t dl = depth[parent[i]] + 1;
    len[leaves[i].s] = (uint8_t)(dl > 255 ? 255 : dl);
    if (dl > maxlen) maxlen = dl;
  }
  free(leaves);
  free(nodef);
  free(parent);
  free(depth);
  return maxlen;
}

int sz3o_huffman_lengths(const uint64_t* freq, uint32_t nsym, uint32_t lmax, uint8_t* len) {
  uint64_t* f;
  uint32_t i, nused, maxlen;
  if (nsym == 0 || lmax < 1 || lmax > 32) return SZ3O_E_INVAL;
  f = (uint64_t*)malloc(sizeof(uint64_t) * nsym);
  if (!f) return SZ3O_E_NOMEM;
  memcpy(f, freq, sizeof(uint64_t) * nsym);
  for (;;) {
    maxlen = build_lengths(f, nsym, len, &nused);
    if (maxlen == 0) {
      free(f);
      return SZ3O_E_NOMEM;
    }
    if (nused > ((uint64_t)1 << lmax)) {
      free(f);
      return SZ3O_E_INVAL;
    }
    if (maxlen <= lmax) break;
    for (i = 0; i < nsym; ++i)
      if (f[i]) f[i] = (f[i] >> 1) ? (f[i] >> 1) : 1;
  }
  free(f);
  return SZ3O_OK;
}

/* Canonical codes: symbols ordered by (length, symbol); the first gets the
 * all-zero code, each next one the previous code plus one, shifted left by the
 * growth in length. */
int sz3o_canonical_codes(const uint8_t* len, uint32_t nsym, uint32_t* code) {
  uint32_t L, s, have = 0, prev_len = 0;
  uint64_t c = 0;
  for (s = 0; s < nsym; ++s) code[s] = 0;
  for (L = 1; L <= 32; ++L) {
    for (s = 0; s < nsym; ++s) {
      if (len[s] != L) continue;
      if (have) c = (c + 1) << (L - prev_len);
      if (c >> L) return SZ3O_E_INVAL; /* lengths violate Kraft */
      code[s] = (uint32_t)c;
      prev_len = L;
      have = 1;
    }
  }
  return SZ3O_OK;
}

/* Chunked encode: every chunk starts on a fresh 32-bit word; bits are packed
 * most significant first; the tail of a chunk's last word is zero.  For every
 * chunk the bit lengths of its first ceil(chunk/512) - 1 sub-blocks of 512
 * codes are recorded as well (sub_bits, may be NULL): they let a decoder
 * start inside a chunk. */
int sz3o_huffman_encode(const uint16_t* codes, uint64_t n, const uint8_t* len,
                        const uint32_t* code, uint32_t chunk, uint32_t* words,
                        uint64_t cap_words, uint32_t* chunk_words, uint16_t* sub_bits,
                        uint64_t* n_words) {
  uint64_t nchunks, j, w = 0;
  uint32_t nsb;
  if (chunk == 0) return SZ3O_E_INVAL;
  nchunks = (n + chunk - 1) / chunk;
  nsb = (chunk + SZ3O_SUBBLOCK - 1) / SZ3O_SUBBLOCK;
  for (j = 0; j < nchunks; ++j) {
    uint64_t i0 = j * chunk, i1 = i0 + chunk < n ? i0 + chunk : n, i;
    uint64_t w0 = w;
    uint32_t acc = 0, nacc = 0; /* bits held in acc (MSB-aligned count) */
    uint32_t sb_bits = 0;
    for (i = i0; i < i1; ++i) {
      uint32_t L = len[codes[i]], b;
      uint32_t v = code[codes[i]];
      if (L == 0) return SZ3O_E_INVAL;
      for (b = L; b-- > 0;) {
        acc = (acc << 1) | ((v >> b) & 1u);
        if (++nacc == 32) {
          if (w >= cap_words) return SZ3O_E_CAPACITY;
          words[w++] = acc;
          acc = 0;
          nacc = 0;
        }
      }
      sb_bits += L;
      if ((i - i0 + 1) % SZ3O_SUBBLOCK == 0) {
        uint64_t sb = (i - i0) / SZ3O_SUBBLOCK;
        if (sub_bits && sb + 1 < nsb) sub_bits[j * (nsb - 1) + sb] = (uint16_t)sb_bits;
        sb_bits = 0;
      }
    }
    if (sub_bits) { /* sub-blocks past the end of a short last chunk are empty */
      uint64_t sb;
      for (sb = (i1 - i0 + SZ3O_SUBBLOCK - 1) / SZ3O_SUBBLOCK; sb + 1 < nsb; ++sb) {
        if (sb * SZ3O_SUBBLOCK >= i1 - i0) sub_bits[j * (nsb - 1) + sb] = 0;
      }
      if ((i1 - i0) % SZ3O_SUBBLOCK != 0) {
        uint64_t sb = (i1 - i0) / SZ3O_SUBBLOCK;
        if (sb + 1 < nsb) sub_bits[j * (nsb - 1) + sb] = (uint16_t)sb_bits;
      }
    }
    if (nacc) {
      if (w >= cap_words) return SZ3O_E_CAPACITY;
      words[w++] = acc << (32 - nacc);
    }
    chunk_words[j] = (uint32_t)(w - w0);
  }
  *n_words = w;
  return SZ3O_OK;
}

/* Chunked decode with the canonical code: read one bit at a time until the
 * prefix read so far is a code of its length.  With sub_bits, every sub-block
 * boundary must fall where the recorded lengths put it. */
int sz3o_huffman_decode(const uint32_t* words, uint64_t n_words, const uint32_t* chunk_words,
                        const uint16_t* sub_bits, uint32_t chunk, const uint8_t* len,
                        uint32_t nsym, uint16_t* codes, uint64_t n) {
  uint64_t first[33], count[33], offs[33];
  uint32_t* sorted;
  uint64_t nchunks, j, w = 0;
  uint32_t L, s, k = 0, nsb;
  uint64_t c = 0;
  int have = 0;
  uint32_t prev_len = 0;
  if (chunk == 0) return SZ3O_E_INVAL;
  nsb = (chunk + SZ3O_SUBBLOCK - 1) / SZ3O_SUBBLOCK;
  sorted = (uint32_t*)malloc(sizeof(uint32_t) * (nsym ? nsym : 1));
  if (!sorted) return SZ3O_E_NOMEM;
  for (L = 0; L <= 32; ++L) {
    first[L] = 0;
    count[L] = 0;
    offs[L] = 0;
  }
  for (L = 1; L <= 32; ++L) {
    offs[L] = k;
    for (s = 0; s < nsym; ++s) {
      if (len[s] != L) continue;
      if (have) c = (c + 1) << (L - prev_len);
      if (count[L] == 0) first[L] = c;
      count[L]++;
      sorted[k++] = s;
      prev_len = L;
      have = 1;
    }
  }
  nchunks = (n + chunk - 1) / chunk;
  for (j = 0; j < nchunks; ++j) {
    uint64_t i0 = j * chunk, i1 = i0 + chunk < n ? i0 + chunk : n, i;
    uint64_t wend = w + chunk_words[j], bit = 0, expect = 0;
    if (wend > n_words) {
      free(sorted);
      return SZ3O_E_CORRUPT;
    }
    for (i = i0; i < i1; ++i) {
      uint64_t v = 0;
      int found = 0;
      if (sub_bits && i > i0 && (i - i0) % SZ3O_SUBBLOCK == 0) {
        expect += sub_bits[j * (nsb - 1) + (i - i0) / SZ3O_SUBBLOCK - 1];
        if (bit != expect) {
          free(sorted);
          return SZ3O_E_CORRUPT;
        }
      }
      for (L = 1; L <= 32 && !found; ++L) {
        uint64_t wi = w + bit / 32;
        if (wi >= wend) break;
        v = (v << 1) | ((words[wi] >> (31 - bit % 32)) & 1u);
        ++bit;
        if (count[L] && v >= first[L] && v - first[L] < count[L]) {
          codes[i] = (uint16_t)sorted[offs[L] + (v - first[L])];
          found = 1;
        }
      }
      if (!found) {
        free(sorted);
        return SZ3O_E_CORRUPT;
      }
    }
    if (sub_bits) { /* recorded lengths of empty sub-blocks must be zero */
      uint64_t sb;
      for (sb = (i1 - i0 + SZ3O_SUBBLOCK - 1) / SZ3O_SUBBLOCK; sb + 1 < nsb; ++sb)
        if (sub_bits[j * (nsb - 1) + sb] != 0) {
          free(sorted);
          return SZ3O_E_CORRUPT;
        }
    }
    w = wend;
  }
  free(sorted);
  return SZ3O_OK;
}

/* ---------------------------------------------------------------------------
 * Stream (Alg. 1 lines 5-9: allocate, save predictor (nothing to save: the
 * interpolation has constant coefficients), save quantizer (unpredictables),
 * encode, save encoder (code lengths)).  Little-endian, written byte by byte.
 *
 *   off  size  field
 *     0     4  magic "SZ3G"
 *     4     2  version (1)
 *     6     1  dtype          7   1  ndim
 *     8    32  dims[4] (u64)
 *    40     1  eb_mode       41   1  interp     42  1  per_level   43  1  L
 *    44     4  radius
 *    48     8  eb (as given, f64)        56  8  eb_abs (f64)
 *    64     8  eb_T bit pattern (u32 for f32, zero-extended)
 *    72     4  chunk_codes   76   4  n_used_syms
 *    80     8  n_codes       88   8  n_unpred     96  8  n_chunks  104 8 payload words
 *   112    32  level_interp[32]   (entries 1..L when per_level, else zero)
 *   144   128  level_order[32][4] (entries 1..L when per_level, else zero)
 *   272     4  dim_order[4]
 *   276    12  zero
 *   288        sections, each starting on an 8-byte boundary, zero padded:
 *              unpredictable values  T[n_unpred]
 *              code-length table     n_used x (u16 symbol, u8 length), by symbol
 *              chunk table           u32[n_chunks] (words per chunk)
 *              sub-block table       u16[n_chunks x (ceil(chunk/512) - 1)]: bit
 *                                    lengths of each chunk's 512-code sub-blocks
 *                                    but the last (0 past a short chunk's end)
 *              payload               u32[payload words]
 * ------------------------------------------------------------------------- */
static uint64_t pad8(uint64_t x) { return (x + 7) & ~(uint64_t)7; }

static uint64_t nsb_of(uint32_t chunk) { return (chunk + SZ3O_SUBBLOCK - 1) / SZ3O_SUBBLOCK; }

static void put_le(uint8_t* b, uint64_t v, int nbytes) {
  int i;
  for (i = 0; i < nbytes; ++i) b[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t get_le(const uint8_t* b, int nbytes) {
  uint64_t v = 0;
  int i;
  for (i = nbytes; i-- > 0;) v = (v << 8) | b[i];
  return v;
}

static uint64_t f64_bits(double d) {
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
}

static double f64_of(uint64_t u) {
  double d;
  memcpy(&d, &u, 8);
  return d;
}

int sz3o_compress_bound(const sz3o_params* p, uint64_t* max_bytes) {
  walk_geom g;
  uint64_t esz, nchunks, maxbits_chunk;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  esz = p->dtype == SZ3O_F32 ? 4 : 8;
  nchunks = (g.N + p->chunk_codes - 1) / p->chunk_codes;
  maxbits_chunk = (uint64_t)p->chunk_codes * SZ3O_LMAX;
  *max_bytes = SZ3O_HEADER_BYTES + pad8(g.N * esz) + pad8((uint64_t)2 * p->radius * 3) +
               pad8(nchunks * 4) + pad8(nchunks * (nsb_of(p->chunk_codes) - 1) * 2) +
               pad8(nchunks * ((maxbits_chunk + 31) / 32) * 4);
  return SZ3O_OK;
}

int sz3o_compress(const sz3o_params* p, const void* x, void* out, uint64_t capacity,
                  uint64_t* out_bytes) {
  walk_geom g;
  uint64_t esz, n_unpred = 0, nchunks, n_words = 0, off, i, cap_words;
  uint64_t* hist = NULL;
  uint16_t* codes = NULL;
  void* unpred = NULL;
  void* recon = NULL;
  uint8_t* len = NULL;
  uint32_t* code = NULL;
  uint32_t* chunk_words = NULL;
  uint16_t* sub_bits = NULL;
  uint32_t* words = NULL;
  uint32_t nsym, n_used = 0, l;
  uint64_t nsub_entries;
  double eb_abs = 0;
  uint8_t ebT[8];
  uint8_t* o = (uint8_t*)out;
  int rc = geom_of(p, &g);
  if (rc) return rc;
  esz = p->dtype == SZ3O_F32 ? 4 : 8;
  nsym = 2 * p->radius;
  nchunks = (g.N + p->chunk_codes - 1) / p->chunk_codes;
  cap_words = nchunks * (((uint64_t)p->chunk_codes * SZ3O_LMAX + 31) / 32);
  codes = (uint16_t*)malloc(g.N * 2);
  unpred = malloc(g.N * esz);
  recon = malloc(g.N * esz);
  hist = (uint64_t*)malloc(65536 * sizeof(uint64_t));
  len = (uint8_t*)malloc(nsym);
  code = (uint32_t*)malloc(nsym * 4);
  chunk_words = (uint32_t*)malloc(nchunks * 4);
  nsub_entries = nchunks * (nsb_of(p->chunk_codes) - 1);
  sub_bits = (uint16_t*)malloc(nsub_entries ? nsub_entries * 2 : 2);
  words = (uint32_t*)malloc(cap_words * 4);
  if (!codes || !unpred || !recon || !hist || !len || !code || !chunk_words || !sub_bits || !words) {
    rc = SZ3O_E_NOMEM;
    goto done;
  }
  memset(ebT, 0, sizeof ebT);
  if (p->dtype == SZ3O_F32)
    rc = quantize_field_f32(p, &g, (const float*)x, codes, (float*)unpred, &n_unpred,
                            (float*)recon, (float*)ebT, &eb_abs);
  else
    rc = quantize_field_f64(p, &g, (const double*)x, codes, (double*)unpred, &n_unpred,
                            (double*)recon, (double*)ebT, &eb_abs);
  if (rc) goto done;
  sz3o_histogram(codes, g.N, hist);
  rc = sz3o_huffman_lengths(hist, nsym, SZ3O_LMAX, len);
  if (rc) goto done;
  rc = sz3o_canonical_codes(len, nsym, code);
  if (rc) goto done;
  rc = sz3o_huffman_encode(codes, g.N, len, code, p->chunk_codes, words, cap_words, chunk_words,
                           sub_bits, &n_words);
  if (rc) goto done;
  for (i = 0; i < nsym; ++i)
    if (len[i]) ++n_used;
  off = SZ3O_HEADER_BYTES + pad8(n_unpred * esz) + pad8((uint64_t)n_used * 3) + pad8(nchunks * 4) +
        pad8(nsub_entries * 2) + pad8(n_words * 4);
  if (off > capacity) {
    rc = SZ3O_E_CAPACITY;
    goto done;
  }
  memset(o, 0, off);
  o[0] = 'S';
  o[1] = 'Z';
  o[2] = '3';
  o[3] = 'G';
  put_le(o + 4, 1, 2);
  o[6] = (uint8_t)p->dtype;
  o[7] = (uint8_t)p->ndim;
  for (i = 0; i < 4; ++i) put_le(o + 8 + 8 * i, i < p->ndim ? p->dims[i] : 1, 8);
  o[40] = (uint8_t)p->eb_mode;
  o[41] = (uint8_t)p->interp;
  o[42] = p->per_level;
  o[43] = (uint8_t)g.L;
  put_le(o + 44, p->radius, 4);
  put_le(o + 48, f64_bits(p->eb), 8);
  put_le(o + 56, f64_bits(eb_abs), 8);
  put_le(o + 64, esz == 4 ? get_le(ebT, 4) : get_le(ebT, 8), 8);
  put_le(o + 72, p->chunk_codes, 4);
  put_le(o + 76, n_used, 4);
  put_le(o + 80, g.N, 8);
  put_le(o + 88, n_unpred, 8);
  put_le(o + 96, nchunks, 8);
  put_le(o + 104, n_words, 8);
  if (p->per_level) {
    for (l = 1; l <= g.L; ++l) {
      o[112 + l] = p->level_interp[l];
      for (i = 0; i < 4; ++i) o[144 + 4 * l + i] = i < p->ndim ? p->level_order[l][i] : 0;
    }
  }
  for (i = 0; i < 4; ++i) o[272 + i] = i < p->ndim ? p->dim_order[i] : 0;
  off = SZ3O_HEADER_BYTES;
  for (i = 0; i < n_unpred; ++i) {
    uint8_t tmp[8];
    memcpy(tmp, (uint8_t*)unpred + i * esz, esz);
    put_le(o + off + i * esz, get_le(tmp, (int)esz), (int)esz);
  }
  off += pad8(n_unpred * esz);
  {
    uint64_t k = 0;
    for (i = 0; i < nsym; ++i)
      if (len[i]) {
        put_le(o + off + 3 * k, i, 2);
        o[off + 3 * k + 2] = len[i];
        ++k;
      }
  }
  off += pad8((uint64_t)n_used * 3);
  for (i = 0; i < nchunks; ++i) put_le(o + off + 4 * i, chunk_words[i], 4);
  off += pad8(nchunks * 4);
  for (i = 0; i < nsub_entries; ++i) put_le(o + off + 2 * i, sub_bits[i], 2);
  off += pad8(nsub_entries * 2);
  for (i = 0; i < n_words; ++i) put_le(o + off + 4 * i, words[i], 4);
  off += pad8(n_words * 4);
  *out_bytes = off;
  rc = SZ3O_OK;
done:
  free(codes);
  free(unpred);
  free(recon);
  free(hist);
  free(len);
  free(code);
  free(chunk_words);
  free(sub_bits);
  free(words);
  return rc;
}

typedef struct {
  sz3o_params p;
  uint64_t N, n_unpred, n_chunks, n_words;
  uint32_t n_used, L;
  uint8_t ebT[8];
  uint64_t off_unpred, off_table, off_chunks, off_sub, off_payload, end;
} parsed_t;

static int parse(const uint8_t* s, uint64_t bytes, parsed_t* h) {
  walk_geom g;
  uint64_t esz, i, l;
  int rc;
  memset(h, 0, sizeof *h);
  if (bytes < SZ3O_HEADER_BYTES) return SZ3O_E_CORRUPT;
  if (s[0] != 'S' || s[1] != 'Z' || s[2] != '3' || s[3] != 'G') return SZ3O_E_CORRUPT;
  if (get_le(s + 4, 2) != 1) return SZ3O_E_CORRUPT;
  h->p.dtype = s[6];
  h->p.ndim = s[7];
  if (h->p.ndim < 1 || h->p.ndim > 4) return SZ3O_E_CORRUPT;
  for (i = 0; i < 4; ++i) h->p.dims[i] = get_le(s + 8 + 8 * i, 8);
  h->p.eb_mode = s[40];
  h->p.interp = s[41];
  h->p.per_level = s[42];
  h->L = s[43];
  h->p.radius = (uint32_t)get_le(s + 44, 4);
  h->p.eb = f64_of(get_le(s + 48, 8));
  h->p.chunk_codes = (uint32_t)get_le(s + 72, 4);
  for (l = 0; l < SZ3O_MAX_LEVELS; ++l) {
    h->p.level_interp[l] = s[112 + l];
    for (i = 0; i < 4; ++i) h->p.level_order[l][i] = s[144 + 4 * l + i];
  }
  for (i = 0; i < 4; ++i) h->p.dim_order[i] = s[272 + i];
  rc = geom_of(&h->p, &g);
  if (rc) return SZ3O_E_CORRUPT;
  if (g.L != h->L) return SZ3O_E_CORRUPT;
  h->N = g.N;
  esz = h->p.dtype == SZ3O_F32 ? 4 : 8;
  put_le(h->ebT, get_le(s + 64, 8), 8);
  if (esz == 4) {
    float e;
    uint32_t u = (uint32_t)get_le(s + 64, 4);
    if (get_le(s + 68, 4) != 0) return SZ3O_E_CORRUPT;
    memcpy(&e, &u, 4);
    if (!isnormal(e) || !(e > 0) || !isnormal(1.0f / e)) return SZ3O_E_CORRUPT;
    memcpy(h->ebT, &e, 4);
  } else {
    double e = f64_of(get_le(s + 64, 8));
    if (!isnormal(e) || !(e > 0) || !isnormal(1.0 / e)) return SZ3O_E_CORRUPT;
    memcpy(h->ebT, &e, 8);
  }
  h->n_used = (uint32_t)get_le(s + 76, 4);
  if (get_le(s + 80, 8) != g.N) return SZ3O_E_CORRUPT;
  h->n_unpred = get_le(s + 88, 8);
  h->n_chunks = get_le(s + 96, 8);
  h->n_words = get_le(s + 104, 8);
  if (h->n_unpred > g.N) return SZ3O_E_CORRUPT;
  if (h->n_chunks != (g.N + h->p.chunk_codes - 1) / h->p.chunk_codes) return SZ3O_E_CORRUPT;
  if (h->n_used < 1 || h->n_used > 2 * h->p.radius) return SZ3O_E_CORRUPT;
  if (h->n_words > h->n_chunks * (((uint64_t)h->p.chunk_codes * SZ3O_LMAX + 31) / 32))
    return SZ3O_E_CORRUPT;
  h->off_unpred = SZ3O_HEADER_BYTES;
  h->off_table = h->off_unpred + pad8(h->n_unpred * esz);
  h->off_chunks = h->off_table + pad8((uint64_t)h->n_used * 3);
  h->off_sub = h->off_chunks + pad8(h->n_chunks * 4);
  h->off_payload = h->off_sub + pad8(h->n_chunks * (nsb_of(h->p.chunk_codes) - 1) * 2);
  h->end = h->off_payload + pad8(h->n_words * 4);
  if (h->end > bytes) return SZ3O_E_CORRUPT;
  return SZ3O_OK;
}

int sz3o_read_header(const void* stream, uint64_t bytes, sz3o_params* p, uint64_t* n_points) {
  parsed_t h;
  int rc = parse((const uint8_t*)stream, bytes, &h);
  if (rc) return rc;
  if (p) *p = h.p;
  if (n_points) *n_points = h.N;
  return SZ3O_OK;
}

int sz3o_decompress(const void* stream, uint64_t bytes, void* out, uint64_t capacity) {
  const uint8_t* s = (const uint8_t*)stream;
  parsed_t h;
  uint64_t esz, i, sum = 0, maxw;
  uint32_t nsym;
  uint8_t* len = NULL;
  uint32_t* chunk_words = NULL;
  uint16_t* sub_bits = NULL;
  uint32_t* words = NULL;
  uint16_t* codes = NULL;
  uint8_t* unpred = NULL;
  double kraft = 0;
  uint64_t nsub_entries;
  int rc = parse(s, bytes, &h);
  if (rc) return rc;
  esz = h.p.dtype == SZ3O_F32 ? 4 : 8;
  if (capacity < h.N * esz) return SZ3O_E_CAPACITY;
  nsym = 2 * h.p.radius;
  len = (uint8_t*)calloc(nsym, 1);
  chunk_words = (uint32_t*)malloc(h.n_chunks * 4);
  nsub_entries = h.n_chunks * (nsb_of(h.p.chunk_codes) - 1);
  sub_bits = (uint16_t*)malloc(nsub_entries ? nsub_entries * 2 : 2);
  words = (uint32_t*)malloc((h.n_words ? h.n_words : 1) * 4);
  codes = (uint16_t*)malloc(h.N * 2);
  unpred = (uint8_t*)malloc((h.n_unpred ? h.n_unpred : 1) * esz);
  if (!len || !chunk_words || !sub_bits || !words || !codes || !unpred) {
    rc = SZ3O_E_NOMEM;
    goto done;
  }
  /* Code-length table: symbols strictly increasing, lengths 1..LMAX, Kraft
   * sum 1 (or a single symbol of length 1). */
  for (i = 0; i < h.n_used; ++i) {
    uint64_t sym = get_le(s + h.off_table + 3 * i, 2);
    uint32_t L = s[h.off_table + 3 * i + 2];
    if (sym >= nsym || L < 1 || L > SZ3O_LMAX) {
      rc = SZ3O_E_CORRUPT;
      goto done;
    }
    if (i > 0 && sym <= get_le(s + h.off_table + 3 * (i - 1), 2)) {
      rc = SZ3O_E_CORRUPT;
      goto done;
    }
    len[sym] = (uint8_t)L;
    kraft += ldexp(1.0, -(int)L);
  }
  if (h.n_used == 1 ? kraft != 0.5 : kraft != 1.0) {
    rc = SZ3O_E_CORRUPT;
    goto done;
  }
  maxw = ((uint64_t)h.p.chunk_codes * SZ3O_LMAX + 31) / 32;
  for (i = 0; i < h.n_chunks; ++i) {
    chunk_words[i] = (uint32_t)get_le(s + h.off_chunks + 4 * i, 4);
    if (chunk_words[i] > maxw) {
      rc = SZ3O_E_CORRUPT;
      goto done;
    }
    sum += chunk_words[i];
  }
  if (sum != h.n_words) {
    rc = SZ3O_E_CORRUPT;
    goto done;
  }
  for (i = 0; i < nsub_entries; ++i) sub_bits[i] = (uint16_t)get_le(s + h.off_sub + 2 * i, 2);
  for (i = 0; i < h.n_words; ++i) words[i] = (uint32_t)get_le(s + h.off_payload + 4 * i, 4);
  rc = sz3o_huffman_decode(words, h.n_words, chunk_words, sub_bits, h.p.chunk_codes, len, nsym, codes,
                           h.N);
  if (rc) goto done;
  for (i = 0; i < h.n_unpred; ++i) {
    uint64_t v = get_le(s + h.off_unpred + i * esz, (int)esz);
    memcpy(unpred + i * esz, &v, esz); /* little-endian host assumed by memcpy of the low bytes */
  }
  {
    walk_geom g;
    geom_of(&h.p, &g);
    if (esz == 4) {
      float e;
      memcpy(&e, h.ebT, 4);
      rc = recover_field_f32(&h.p, &g, e, codes, (const float*)unpred, h.n_unpred, (float*)out);
    } else {
      double e;
      memcpy(&e, h.ebT, 8);
      rc = recover_field_f64(&h.p, &g, e, codes, (const double*)unpred, h.n_unpred, (double*)out);
    }
  }
done:
  free(len);
  free(chunk_words);
  free(sub_bits);
  free(words);
  free(codes);
  free(unpred);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Per-level selection (see sel_hist in sz3o_typed.inc).
 * ------------------------------------------------------------------------- */
static int sel_geom(const sz3o_params* p, uint32_t level, walk_geom* g) {
  int rc = geom_of(p, g);
  if (rc) return rc;
  if (p->ndim > 3 || level < 1 || level > g->L) return SZ3O_E_INVAL;
  return SZ3O_OK;
}

int sz3o_select_costs(const sz3o_params* p, const void* x, uint32_t level, uint32_t nblocks, uint64_t seed,
                      double* cost) {
  walk_geom g;
  int rc = sel_geom(p, level, &g);
  if (rc) return rc;
  if (!x || !cost) return SZ3O_E_INVAL;
  return p->dtype == SZ3O_F32 ? select_costs_f32(p, &g, (const float*)x, level, nblocks, seed, cost)
                              : select_costs_f64(p, &g, (const double*)x, level, nblocks, seed, cost);
}

uint64_t sz3o_splitmix64(uint64_t key) { return splitmix64(key); }

uint32_t sz3o_select_blocks(const sz3o_params* p, uint32_t level, uint32_t nblocks, uint64_t seed, uint64_t* lo,
                            uint64_t* hi) {
  walk_geom g;
  sel_blocks* blk;
  uint32_t b, d, n;
  if (geom_of(p, &g) != SZ3O_OK || level < 1 || level > g.L) return 0;
  blk = (sel_blocks*)malloc(sizeof(sel_blocks));
  if (!blk) return 0;
  sel_make_blocks(&g, level, nblocks, seed, blk);
  for (b = 0; b < blk->n; ++b)
    for (d = 0; d < g.ndim; ++d) {
      lo[4 * b + d] = blk->lo[b][d];
      hi[4 * b + d] = blk->hi[b][d];
    }
  n = blk->n;
  free(blk);
  return n;
}

int sz3o_select_features(const sz3o_params* p, const void* x, uint32_t level, uint32_t nblocks, uint64_t seed,
                         double* feat) {
  walk_geom g;
  int rc = sel_geom(p, level, &g);
  if (rc) return rc;
  if (!x || !feat) return SZ3O_E_INVAL;
  return p->dtype == SZ3O_F32 ? select_features_f32(p, &g, (const float*)x, level, nblocks, seed, feat)
                              : select_features_f64(p, &g, (const double*)x, level, nblocks, seed, feat);
}
