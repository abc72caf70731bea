// k_huffman.cu -- the encoder module of the pipeline (SZ3 paper Sec. 3.2
// Encoder): Huffman code lengths built greedily from the code histogram,
// canonical codewords, chunk-parallel encode and decode, and the stream
// sections that go with them.
//
//  * codebook_kernel  one CTA: used symbols sorted by (frequency, symbol),
//    two-queue merge (leaf first on equal weight), depths by a bounded walk to
//    the root, frequency halving while a code is longer than 24 bits, then
//    canonical codewords ordered by (length, symbol).
//  * count_kernel / emit_kernel  one warp per chunk of the code stream: chunk
//    bit counts and their prefix (a scan, or decoupled look-back over the
//    chunks for the payload word offset and the unpredictable-value offset),
//    then packing through a shared-memory word ring (MSB first) and the
//    gather of the chunk's unpredictable values.
//  * decode_kernel    one thread per 512-code sub-block: 12-bit direct table,
//    canonical comparison for longer codes; counts zero codes for the
//    recover step.
#include <algorithm>

#include "internal.cuh"

namespace sz3g {

constexpr int kCbThreads = 1024;
constexpr int kSmemLeaves = 8192;  // leaf count handled in shared memory
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kValMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;

// ---------------------------------------------------------------------------
// Block primitives (1024 threads).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v,
                                                                   unsigned long long* s_warp,
                                                                   unsigned long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = lane < nw ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) s_warp[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  const unsigned long long before = (w ? s_warp[w - 1] : 0) + x - v;
  if (total) *total = s_warp[nw - 1];
  __syncthreads();
  return before;
}

// cnt[d] += 1 for every lane with `valid`, one atomic per distinct d in the
// warp (all 32 lanes call it).
__device__ __forceinline__ void warp_count(uint32_t* cnt, uint32_t d, bool valid) {
  const unsigned m = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu);
  if (valid && (int)(threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&cnt[d], (uint32_t)__popc(m));
}

// One stable counting pass over K items on the whole block (32 warps): item
// i has digit dig(i) in [0, NB) and emit(i, r) receives its rank r in the
// order (digit, input position).  Tiles of one item per thread: the rank is
// the digit's start, plus the items of that digit in earlier tiles, earlier
// warps of the tile and earlier lanes of the warp.
template <int NB, typename DigFn, typename EmitFn>
__device__ __forceinline__ void block_counting_pass(int K, DigFn dig, EmitFn emit) {
  static_assert(NB <= 32, "one warp per digit");
  __shared__ uint32_t s_first[NB], s_run[NB], s_wc[32][NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < NB) {
    s_first[tid] = 0;
    s_run[tid] = 0;
  }
  __syncthreads();
  for (int i0 = 0; i0 < K; i0 += kCbThreads) {
    const int i = i0 + tid;
    warp_count(s_first, i < K ? dig(i) : 0u, i < K);
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t acc = 0;
    for (int d = 0; d < NB; ++d) {
      const uint32_t c = s_first[d];
      s_first[d] = acc;
      acc += c;
    }
  }
  for (int t0 = 0; t0 < K; t0 += kCbThreads) {
    for (int i = tid; i < 32 * NB; i += kCbThreads) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const int i = t0 + tid;
    const uint32_t d = i < K ? dig(i) : (uint32_t)NB;  // NB: no item
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d < (uint32_t)NB && lane == __ffs(peers) - 1) s_wc[warp][d] = (uint32_t)__popc(peers);
    __syncthreads();
    if (warp < NB) {  // warp w: offsets of digit w in the tile's warps
      const uint32_t c = s_wc[lane][warp], base = s_run[warp];
      uint32_t x = c;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      s_wc[lane][warp] = base + x - c;
      __syncwarp();
      if (lane == 31) s_run[warp] = base + x;
    }
    __syncthreads();
    if (d < (uint32_t)NB) emit(i, s_first[d] + s_wc[warp][d] + (uint32_t)__popc(peers & ((1u << lane) - 1u)));
    __syncthreads();
  }
}

// Keys (weight << 16 | position in symbol order) sorted by weight, ties in
// input order: least-significant-digit radix passes of 4 bits over the
// weight, as many as its largest value needs.  a and b alternate; returns
// the array holding the result.
__device__ unsigned long long* block_radix_sort_w(unsigned long long* a, unsigned long long* b, int K) {
  __shared__ uint32_t s_max;
  if (threadIdx.x == 0) s_max = 1;
  __syncthreads();
  uint32_t m = 1;
  for (int i = threadIdx.x; i < K; i += kCbThreads) m = max(m, (uint32_t)(a[i] >> 16));
  atomicMax(&s_max, m);
  __syncthreads();
  const int passes = (32 - __clz((int)s_max) + 3) / 4;
  for (int p = 0; p < passes; ++p) {
    const int sh = 16 + 4 * p;
    block_counting_pass<16>(
        K, [&](int i) { return (uint32_t)(a[i] >> sh) & 15u; }, [&](int i, uint32_t r) { b[r] = a[i]; });
    __syncthreads();
    unsigned long long* t = a;
    a = b;
    b = t;
  }
  return a;
}

// Sorts nseg arrays seg(0) .. seg(nseg - 1) of n distinct keys each,
// ascending and in place, by a bitonic network on the whole block.  Each
// array must hold the next power of two >= n keys (npad): the tail is padded
// with ~0, above every key.  Element e of the concatenated arrays lives in
// slot e / blockDim of thread e % blockDim, so the compare-exchanges at
// distances below 32 stay inside a warp and run on registers by shuffles;
// only the longer distances go through shared memory, with a barrier each.
// Requires nseg * npad <= SLOTS * blockDim.
template <int SLOTS, typename SegFn>
__device__ void block_bitonic_sort(SegFn seg, int nseg, int n) {
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  const int npad = 1 << lg, total = nseg * npad, NT = (int)blockDim.x, tid = (int)threadIdx.x;
  __syncthreads();  // the keys are written
  unsigned long long x[SLOTS];
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    const int e = q * NT + tid, i = e & (npad - 1);
    x[q] = (e < total && i < n) ? seg(e >> lg)[i] : ~0ull;
  }
  // compare-exchange at distance j < 32 on registers (every lane of a warp
  // with any element takes part)
  auto warp_stages = [&](int k, int j0) {
    for (int j = j0; j > 0; j >>= 1)
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        if (q * NT >= total) break;
        const int e = q * NT + tid, i = e & (npad - 1);
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[q], j);
        const bool lower = (i & j) == 0, asc = (i & k) == 0;
        x[q] = (lower == asc) ? (x[q] < y ? x[q] : y) : (x[q] < y ? y : x[q]);
      }
  };
  for (int k = 2; k <= npad; k <<= 1) {
    if (k > 32) {  // distances k/2 .. 32 in shared memory
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        const int e = q * NT + tid;
        if (e < total) seg(e >> lg)[e & (npad - 1)] = x[q];
      }
      __syncthreads();
      for (int j = k >> 1; j >= 32; j >>= 1) {
        for (int it = tid; it < total >> 1; it += NT) {
          const int s = it >> (lg - 1), u = it & ((npad >> 1) - 1);
          const int i = ((u & ~(j - 1)) << 1) | (u & (j - 1));  // pair (i, i + j)
          unsigned long long* A = seg(s);
          const unsigned long long a0 = A[i], a1 = A[i + j];
          if ((a0 > a1) == ((i & k) == 0)) {
            A[i] = a1;
            A[i + j] = a0;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < SLOTS; ++q) {
        const int e = q * NT + tid;
        if (e < total) x[q] = seg(e >> lg)[e & (npad - 1)];
      }
      warp_stages(k, 16);
    } else {
      warp_stages(k, k >> 1);
    }
  }
  __syncthreads();  // every read of the arrays above is done
#pragma unroll
  for (int q = 0; q < SLOTS; ++q) {
    const int e = q * NT + tid;
    if (e < total) seg(e >> lg)[e & (npad - 1)] = x[q];
  }
  __syncthreads();
}

// First index in [lo, hi) of the ascending array a whose value exceeds w
// (hi if none), the same in every lane: a 32-way search by the whole warp,
// two probe rounds for up to 1024 values.  Lane l probes the last value of
// block l; the blocks whose last value is not above w form a prefix.
__device__ __forceinline__ uint32_t warp_upper_bound(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t w) {
  const uint32_t lane = threadIdx.x & 31;
  while (lo < hi) {
    const uint32_t s = (hi - lo + 31) >> 5, b = lo + s * lane;
    const bool le = b < hi && a[min(b + s, hi) - 1] <= w;
    const uint32_t nlo = lo + s * (uint32_t)__popc(__ballot_sync(0xffffffffu, le));
    if (nlo >= hi) return hi;
    hi = min(nlo + s, hi) - 1;  // the last value of the first such block exceeds w
    lo = nlo;
  }
  return lo;
}

// The items at positions d and d + 1 of the merge of leaves [a, cL) and
// internal nodes [m, je) (a leaf before an internal node of equal weight);
// both exist.  Returns the sum of their weights and their ids (leaf x,
// internal node Ku + y) in ia / ib.  One merge-path search inside the
// segment, then the two fronts.
__device__ __forceinline__ uint32_t seg_pair(const uint32_t* lw, const uint32_t* W, uint32_t Ku, uint32_t a,
                                             uint32_t cL, uint32_t m, uint32_t je, uint32_t d, uint32_t* ia,
                                             uint32_t* ib) {
  const uint32_t nI = je - m;
  uint32_t lo = d > nI ? d - nI : 0u, hi = min(d, cL - a);  // leaves among the first d items
  while (lo < hi) {
    const uint32_t i = (lo + hi) >> 1;
    if (lw[a + i] <= W[m + d - i - 1]) lo = i + 1;
    else hi = i;
  }
  // the two fronts of each run (a front past its run's end never wins)
  const uint32_t x = a + lo, y = m + d - lo;
  const uint32_t L0 = x < cL ? lw[x] : 0xffffffffu, L1 = x + 1 < cL ? lw[x + 1] : 0xffffffffu;
  const uint32_t I0 = y < je ? W[y] : 0xffffffffu, I1 = y + 1 < je ? W[y + 1] : 0xffffffffu;
  const bool f0 = x < cL && (y >= je || L0 <= I0);  // first item a leaf
  const uint32_t L = f0 ? L1 : L0, I = f0 ? I0 : I1;
  const uint32_t xs = x + f0, ys = y + !f0;
  const bool f1 = xs < cL && (ys >= je || L <= I);  // second item a leaf
  *ia = f0 ? x : Ku + y;
  *ib = f1 ? xs : Ku + ys;
  return (f0 ? L0 : I0) + (f1 ? L : I);
}

// The two-queue Huffman merge (the two lightest fronts, a leaf first on
// equal weight) built batch by batch, giving the same tree node by node.
// S is the merged consumption order: leaves and internal nodes by weight, a
// leaf before an internal node of equal weight, internal nodes in creation
// order.  Internal node j has the items S[2j], S[2j+1] as children and sits
// at position P(j) = j + (leaves not heavier than it) of S.  Once node j0
// exists, the items of S before P(j0) are those leaves and the internal
// nodes below j0, so nodes j0+1 .. (P-2)/2, whose children all lie there,
// are built at once: node j0+1+t from the items 2t, 2t+1 of the segment
// that merges the leaves and internal nodes not yet consumed.  The next
// node takes node j0 itself and its neighbour in S (the segment's last item
// when P is odd, the item after node j0 when it is even).  Quantization-code
// histograms need about one batch per tree level.  lw: the K >= 2 leaf
// weights in order; writes W[j] (internal weights) and parent[] of every
// node but the root (node ids: leaves 0..K-1, internal K + j).  GROUP: the
// threads doing it, one warp (32) or the whole block; warp 0 of the group
// runs the searches for P.
template <int GROUP, typename PT>
__device__ void batched_merge(const uint32_t* lw, int K, uint32_t* W, PT* parent) {
  __shared__ uint32_t s_P;
  const uint32_t Ku = (uint32_t)K, r = threadIdx.x & (GROUP - 1);
  // (a, m): leaves and internal nodes consumed by nodes 0 .. j0
  uint32_t j0 = 0, a = 2, m = 0, w0 = lw[0] + lw[1];
  if (r == 0) {
    W[0] = w0;
    parent[0] = (PT)Ku;
    parent[1] = (PT)Ku;
  }
  while (j0 + 2 < Ku) {  // node Ku - 2 is the root
    uint32_t P;
    if (GROUP == 32) {
      P = j0 + warp_upper_bound(lw, a, Ku, w0);
    } else {
      if (r < 32) {
        P = j0 + warp_upper_bound(lw, a, Ku, w0);
        if (r == 0) s_P = P;
      }
      __syncthreads();
      P = s_P;
    }
    const uint32_t cL = P - j0, j1 = (P - 2) >> 1;
    for (uint32_t t = r; j0 + 1 + t <= j1; t += GROUP) {
      uint32_t ia, ib;
      const uint32_t w = seg_pair(lw, W, Ku, a, cL, m, j0, 2 * t, &ia, &ib);
      W[j0 + 1 + t] = w;
      parent[ia] = (PT)(Ku + j0 + 1 + t);
      parent[ib] = (PT)(Ku + j0 + 1 + t);
    }
    if (GROUP == 32) __syncwarp();
    else __syncthreads();
    const uint32_t jn = j1 + 1;
    uint32_t i0, i1, wn;
    if (P & 1u) {  // the segment's last item, then node j0
      const uint32_t lL = cL > a ? lw[cL - 1] : 0u, lI = j0 > m ? W[j0 - 1] : 0u;
      const bool last_leaf = j0 == m || (cL > a && lL > lI);
      i0 = last_leaf ? cL - 1 : Ku + j0 - 1;
      i1 = Ku + j0;
      wn = (last_leaf ? lL : lI) + w0;
      a = cL;
      m = j0 + 1;
    } else {  // node j0, then the next front (internal nodes j0+1 .. j1 exist)
      const uint32_t nL = cL < Ku ? lw[cL] : 0u, nI = j1 > j0 ? W[j0 + 1] : 0u;
      const bool leaf = cL < Ku && (j1 == j0 || nL <= nI);
      i0 = Ku + j0;
      i1 = leaf ? cL : Ku + j0 + 1;
      wn = w0 + (leaf ? nL : nI);
      a = cL + leaf;
      m = j0 + 1 + !leaf;
    }
    if (r == 0) {
      W[jn] = wn;
      parent[i0] = (PT)(Ku + jn);
      parent[i1] = (PT)(Ku + jn);
    }
    if (GROUP == 32) __syncwarp();
    j0 = jn;
    w0 = wn;
  }
  if (GROUP == 32) __syncwarp();
  else __syncthreads();
}

// The compacted histogram: the used symbols of each 1024-bin segment in
// symbol order, written by hist_compact_kernel for the codebook kernels.
constexpr int kHcSeg = 1024, kHcNseg = kSyms / kHcSeg, kHcThreads = 256;
struct HistList {
  uint32_t n[kHcNseg];  // used symbols of segment b
  uint2 e[kSyms];       // segment b's at [b kHcSeg, b kHcSeg + n[b]): (count, symbol)
};

// One CTA per segment: thread t reads bins 256 k + t (k = 0..3, coalesced);
// the ballot of each 32-bin run marks its used bins, runs in (k, warp) order
// are symbol order.  Also flags counts outside the alphabet and records the
// unpredictable count (code 0).
__global__ void __launch_bounds__(kHcThreads) hist_compact_kernel(const uint32_t* __restrict__ hist, uint32_t nsym,
                                                                  HistList* H, DevState* st) {
  __shared__ uint32_t s_run[4 * kHcThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t b0 = blockIdx.x * kHcSeg;
  uint32_t v[4];
  unsigned msk[4];
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = __ldcg(hist + b0 + k * kHcThreads + tid);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t sy = b0 + k * kHcThreads + tid;
    bad |= v[k] != 0 && sy >= nsym;
    msk[k] = __ballot_sync(0xffffffffu, v[k] != 0 && sy < nsym);
    if (lane == 0) s_run[k * (kHcThreads / 32) + warp] = (uint32_t)__popc(msk[k]);
  }
  __syncthreads();
  if (warp == 0) {  // exclusive prefix over the 32 runs
    const uint32_t c = s_run[lane];
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_run[lane] = x - c;
    if (lane == 31) H->n[blockIdx.x] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if ((msk[k] >> lane) & 1u) {
      const uint32_t pos = s_run[k * (kHcThreads / 32) + warp] + (uint32_t)__popc(msk[k] & ((1u << lane) - 1u));
      H->e[b0 + pos] = make_uint2(v[k], b0 + k * kHcThreads + tid);
    }
  if (bad) atomicOr(&st->flags, kFlagCorrupt);
  if (blockIdx.x == 0 && tid == 0) st->n_unpred = v[0];  // code 0 marks an unpredictable value
}

// The number K of used symbols (every thread), with s_base[b] the position
// of segment b's first used symbol.  s_base: kHcNseg + 1 shared words.
__device__ int used_count(const HistList* H, uint32_t* s_base) {
  const int lane = threadIdx.x & 31;
  static_assert(kHcNseg == 64, "two segments per lane");
  if (threadIdx.x < 32) {
    const uint32_t c0 = __ldcg(&H->n[2 * lane]), c1 = __ldcg(&H->n[2 * lane + 1]);
    uint32_t x = c0 + c1;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_base[2 * lane] = x - c0 - c1;
    s_base[2 * lane + 1] = x - c1;
    if (lane == 31) s_base[kHcNseg] = x;
  }
  __syncthreads();
  return (int)s_base[kHcNseg];
}

// emit(p, count, symbol) for the used symbol at every position p < K in
// symbol order, eight entries in flight per thread.
template <typename EmitFn>
__device__ __forceinline__ void used_entries(const HistList* H, const uint32_t* s_base, int K, EmitFn emit) {
  for (int p0 = 0; p0 < K; p0 += 8 * (int)blockDim.x) {
    uint2 e[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = p0 + u * (int)blockDim.x + (int)threadIdx.x;
      e[u] = make_uint2(0u, 0u);
      if (p < K) {
        int lo = 0, hi = kHcNseg - 1;  // the last segment starting at or before p
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_base[mid] <= (uint32_t)p) lo = mid;
          else hi = mid - 1;
        }
        e[u] = __ldcg(&H->e[lo * kHcSeg + (p - (int)s_base[lo])]);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = p0 + u * (int)blockDim.x + (int)threadIdx.x;
      if (p < K) emit(p, e[u].x, e[u].y);
    }
  }
}

struct CbGlobal {  // global scratch of the codebook kernels
  HistList hl;      // the compacted histogram
  unsigned long long keys[kSyms];  // the key arrays below: more than kSmemLeaves used symbols
  unsigned long long keys2[kSyms];
  uint32_t nf[kSyms + 16];
  uint32_t parent[2 * kSyms];
  uint16_t symord[kSyms];
};

size_t codebook_scratch_bytes() { return sizeof(CbGlobal); }

// shared memory: two key arrays, internal weights / lengths, 16-bit parents,
// used symbols in symbol order
constexpr size_t kCbOffNf = (size_t)kSmemLeaves * 16;
constexpr size_t kCbOffPar = kCbOffNf + (size_t)(kSmemLeaves + 16) * 4;
constexpr size_t kCbOffSym = kCbOffPar + (size_t)kSmemLeaves * 4;
constexpr size_t kCbSmem = kCbOffSym + (size_t)kSmemLeaves * 2;
// leaf + internal weights of up to this many leaves fit the dynamic shared
// memory when the key arrays are in global memory
constexpr int kCbSmemWeights = (int)(kCbSmem / 8);

// Depth of every leaf by walking its parents (stops past SZ3G_LMAX); returns,
// block-wide, whether some code is longer than SZ3G_LMAX.
template <typename PT>
__device__ bool leaf_depths(const PT* parent, int K, uint32_t* len) {
  const uint32_t root = (uint32_t)(2 * K - 2);
  bool deep = false;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    uint32_t v = (uint32_t)i, d = 0;
    while (v != root && d <= SZ3G_LMAX) {
      v = parent[v];
      ++d;
    }
    deep |= v != root || d > SZ3G_LMAX;
    len[i] = d;
  }
  return __syncthreads_or(deep) != 0;
}

// Code lengths of K leaves whose keys (weight << 16 | position in symbol
// order) are in `cur`, halving the weights while some code is longer than
// SZ3G_LMAX.  `other` is a second key array; leaf weights and internal
// weights go to lw_s / w_s when given (shared memory), else to the free key
// array and nf.  On return `srt` holds the leaves sorted by the (weight,
// position) of the last round and nf[i] the length of leaf srt[i].
template <typename PT>
__device__ __forceinline__ unsigned long long* code_lengths(unsigned long long* cur, unsigned long long* other,
                                                            uint32_t* nf, PT* parent, int K, uint32_t* lw_s,
                                                            uint32_t* w_s) {
  const int tid = threadIdx.x;
  unsigned long long* srt = cur;
  if (K == 1) {
    if (tid == 0) nf[0] = 1;
    __syncthreads();
    return srt;
  }
  for (int iter = 0; iter < 40; ++iter) {
    if (K <= kSmemLeaves) {  // keys in shared memory, room for the padded sort
      block_bitonic_sort<kSmemLeaves / kCbThreads>([&](int) { return cur; }, 1, K);
      srt = cur;
    } else {
      srt = block_radix_sort_w(cur, other, K);
    }
    __syncthreads();
    unsigned long long* spare = srt == cur ? other : cur;
    uint32_t* lw = lw_s ? lw_s : reinterpret_cast<uint32_t*>(spare);
    uint32_t* W = w_s ? w_s : nf;
    for (int i = tid; i < K; i += kCbThreads) lw[i] = (uint32_t)(srt[i] >> 16);
    __syncthreads();
    batched_merge<kCbThreads>(lw, K, W, parent);
    if (!leaf_depths(parent, K, nf)) break;
    for (int i = tid; i < K; i += kCbThreads) {
      const unsigned long long k = srt[i];
      const uint32_t f = (uint32_t)(k >> 16) >> 1;
      srt[i] = ((unsigned long long)(f ? f : 1u) << 16) | (k & 0xffffu);
    }
    __syncthreads();
    // the halved keys are the next round's input
    cur = srt;
    other = spare;
  }
  return srt;
}

// Alphabets up to kSpecMax symbols run their first kSpecRounds length-limit
// rounds at once inside the codebook kernel (speculative_lengths below).
constexpr int kSpecMax = 512, kSpecRounds = 4;

// Length-limit rounds of larger alphabets on separate CTAs.  Round r of the
// limit uses the weights max(1, f >> r) and does not depend on round r - 1,
// so codebook_rounds_kernel computes rounds 0 .. kCbRounds-1 at once, CTA r
// on its own scratch, and records which fit SZ3G_LMAX and their lengths; the
// codebook kernel takes the first that fits -- the round at which the
// sequential halving would have stopped -- and continues sequentially from
// round kCbRounds only when none does.
constexpr int kCbRounds = 8;
struct CbRound {
  unsigned long long keys[kSyms];
  unsigned long long keys2[kSyms];
  uint32_t nf[kSyms + 16];
  uint32_t parent[2 * kSyms];
  uint8_t lenpos[kSyms];  // code length by position in symbol order
};
struct CbRounds {
  int fits[kCbRounds];
  int pad[8];
  CbRound r[kCbRounds];
};

size_t codebook_rounds_bytes(unsigned long long max_symbols) {
  return max_symbols > (unsigned long long)kSpecMax ? sizeof(CbRounds) : 0;
}

// One round of code_lengths (no halving loop): sorts `cur` by (weight,
// position), builds the tree, and returns whether some code is longer than
// SZ3G_LMAX; *srt_out gets the sorted keys and nf[i] the length of srt[i].
template <typename PT>
__device__ bool one_round_lengths(unsigned long long* cur, unsigned long long* other, uint32_t* nf, PT* parent,
                                  int K, uint32_t* lw_s, uint32_t* w_s, unsigned long long** srt_out) {
  const int tid = threadIdx.x;
  unsigned long long* srt;
  if (K <= kSmemLeaves) {  // keys in shared memory, room for the padded sort
    block_bitonic_sort<kSmemLeaves / kCbThreads>([&](int) { return cur; }, 1, K);
    srt = cur;
  } else {
    srt = block_radix_sort_w(cur, other, K);
  }
  __syncthreads();
  unsigned long long* spare = srt == cur ? other : cur;
  uint32_t* lw = lw_s ? lw_s : reinterpret_cast<uint32_t*>(spare);
  uint32_t* W = w_s ? w_s : nf;
  for (int i = tid; i < K; i += kCbThreads) lw[i] = (uint32_t)(srt[i] >> 16);
  __syncthreads();
  batched_merge<kCbThreads>(lw, K, W, parent);
  *srt_out = srt;
  return leaf_depths(parent, K, nf);
}

// Speculative halving rounds for small alphabets.  Round i of the length
// limit uses the weights max(1, f >> i) (halving max(1, f >> 1) i times), so
// rounds 0..3 are independent: all four are sorted at once (block-wide), the
// four merges run at once on four warps (one per scheduler), and the
// first round whose codes fit SZ3G_LMAX is the answer, as if the rounds had
// run one after another.  `ka` holds the leaves in symbol order on entry.
// On success the chosen round's leaves sorted by (weight, symbol) are left
// in ka and their lengths in nf; otherwise ka holds the weights of round 4
// for the sequential rounds.  Round scratch lives in
// [region, region + 4 * kSpecRound): keys, leaf weights, internal weights
// (then lengths), parents.
constexpr int kSpecRound = kSpecMax * 8 + (kSpecMax + 4) * 4 * 2 + 2 * kSpecMax * 2;
__device__ bool speculative_lengths(unsigned long long* ka, uint32_t* nf, unsigned char* region, int K) {
  const int tid = threadIdx.x, warp = tid >> 5;
  __shared__ int s_deep[kSpecRounds];
  auto uk = [&](int i) { return reinterpret_cast<unsigned long long*>(region + i * kSpecRound); };
  auto lw = [&](int i) { return reinterpret_cast<uint32_t*>(region + i * kSpecRound + kSpecMax * 8); };
  auto nfi = [&](int i) {
    return reinterpret_cast<uint32_t*>(region + i * kSpecRound + kSpecMax * 8 + (kSpecMax + 4) * 4);
  };
  auto par = [&](int i) {
    return reinterpret_cast<uint16_t*>(region + i * kSpecRound + kSpecMax * 8 + (kSpecMax + 4) * 8);
  };
  auto key_of = [&](int i, int j) {
    const unsigned long long k = ka[j];
    const uint32_t f = (uint32_t)(k >> 16) >> i;
    return ((unsigned long long)(f ? f : 1u) << 16) | (k & 0xffffu);
  };
  if (tid < kSpecRounds) s_deep[tid] = 0;
  for (int it = tid; it < kSpecRounds * K; it += blockDim.x) {
    const int i = it / K, j = it - i * K;
    uk(i)[j] = key_of(i, j);
  }
  // 1. every round sorted by (weight, symbol) (the sort's first barrier
  //    orders the writes above)
  block_bitonic_sort<kSpecRounds * kSpecMax / kCbThreads>(uk, kSpecRounds, K);
  for (int it = tid; it < kSpecRounds * K; it += blockDim.x) {
    const int i = it / K, j = it - i * K;
    lw(i)[j] = (uint32_t)(uk(i)[j] >> 16);
  }
  __syncthreads();
  // 2. the merges at once (warps 0..3: one per scheduler)
  if (warp < kSpecRounds) batched_merge<32>(lw(warp), K, nfi(warp), par(warp));
  __syncthreads();
  // 3. depths (into nf of the round), deep rounds flagged
  const uint32_t root = (uint32_t)(2 * K - 2);
  for (int it = tid; it < kSpecRounds * K; it += blockDim.x) {
    const int i = it / K, j = it - i * K;
    uint32_t v = (uint32_t)j, d = 0;
    while (v != root && d <= SZ3G_LMAX) {
      v = par(i)[v];
      ++d;
    }
    if (v != root || d > SZ3G_LMAX) s_deep[i] = 1;
    nfi(i)[j] = d;
  }
  __syncthreads();
  int pick = -1;
  for (int i = 0; i < kSpecRounds && pick < 0; ++i)
    if (!s_deep[i]) pick = i;
  // 4. the answer (or round 4's weights) into ka / nf (K <= kSpecMax <
  //    blockDim: one leaf per thread)
  unsigned long long kk = 0;
  uint32_t ll = 0;
  if (tid < K) {
    kk = pick >= 0 ? uk(pick)[tid] : key_of(kSpecRounds, tid);
    ll = pick >= 0 ? nfi(pick)[tid] : 0u;
  }
  __syncthreads();
  if (tid < K) {
    ka[tid] = kk;
    if (pick >= 0) nf[tid] = ll;
  }
  __syncthreads();
  return pick >= 0;
}

// table[sym] = len << 24 | code for every used symbol.
__global__ void __launch_bounds__(kCbThreads) codebook_kernel(uint32_t nsym, uint32_t* table, uint8_t* len_out,
                                                              uint32_t* code_out, DevState* st, CbGlobal* g,
                                                              unsigned char* d_out, unsigned long long out_capacity,
                                                              int esz, const CbRounds* R) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_cnt[SZ3G_LMAX + 2], s_start[SZ3G_LMAX + 2], s_fc[SZ3G_LMAX + 2];
  __shared__ uint32_t s_base[kHcNseg + 1];
  const int tid = threadIdx.x;

  // 1. used symbols in symbol order, from the compacted histogram
  const int K = used_count(&g->hl, s_base);
  if (K == 0) {
    if (tid == 0) atomicOr(&st->flags, kFlagCorrupt);
    return;
  }
  const bool in_smem = K <= kSmemLeaves;
  unsigned long long* ka = in_smem ? (unsigned long long*)smem : g->keys;
  unsigned long long* kb = in_smem ? (unsigned long long*)(smem + kSmemLeaves * 8) : g->keys2;
  uint32_t* nf = in_smem ? (uint32_t*)(smem + kCbOffNf) : g->nf;
  uint16_t* symord = in_smem ? (uint16_t*)(smem + kCbOffSym) : g->symord;
  used_entries(&g->hl, s_base, K, [&](int p, uint32_t c, uint32_t sy) {
    ka[p] = ((unsigned long long)c << 16) | (uint32_t)p;  // position in symbol order
    symord[p] = (uint16_t)sy;
  });
  if (len_out || code_out)
    for (int sy = tid; sy < (int)nsym; sy += kCbThreads) {
      if (len_out) len_out[sy] = 0;
      if (code_out) code_out[sy] = 0;
    }
  __syncthreads();

  // 2. lengths (shared-memory arrays are addressed through pointers derived
  //    from the shared array itself in their own branch)
  unsigned long long* srt;
  // the first of the parallel rounds that fits, if they ran (larger alphabets)
  int pick = -1;
  if (R && K > kSpecMax)
    for (int r = 0; r < kCbRounds && pick < 0; ++r)
      if (R->fits[r]) pick = r;
  if (R && K > kSpecMax && pick < 0) {
    // none of them fits: continue the halving from round kCbRounds
    for (int i = tid; i < K; i += kCbThreads) {
      const unsigned long long k = ka[i];
      const uint32_t f = (uint32_t)(k >> 16) >> kCbRounds;
      ka[i] = ((unsigned long long)(f ? f : 1u) << 16) | (k & 0xffffu);
    }
    __syncthreads();
  }
  if (pick >= 0) {
    srt = nullptr;
  } else if (in_smem) {
    // the rounds' scratch spans the second key array and the nf / parent
    // areas, all free until the lengths are known
    static_assert(kSpecRounds * kSpecRound <= kCbOffSym - kSmemLeaves * 8, "speculative rounds fit");
    if (K > 1 && K <= kSpecMax &&
        speculative_lengths((unsigned long long*)smem, (uint32_t*)(smem + kCbOffNf), smem + kSmemLeaves * 8, K)) {
      srt = (unsigned long long*)smem;
    } else {
      srt = code_lengths((unsigned long long*)smem, (unsigned long long*)(smem + kSmemLeaves * 8),
                         (uint32_t*)(smem + kCbOffNf), (uint16_t*)(smem + kCbOffPar), K, (uint32_t*)nullptr,
                         (uint32_t*)nullptr);
    }
  } else if (K <= kCbSmemWeights) {  // leaf and internal weights in the (otherwise unused) shared memory
    srt = code_lengths(g->keys, g->keys2, g->nf, g->parent, K, (uint32_t*)smem, (uint32_t*)smem + K);
  } else {
    srt = code_lengths(g->keys, g->keys2, g->nf, g->parent, K, (uint32_t*)nullptr, (uint32_t*)nullptr);
  }
  // 3. canonical codewords: leaves ordered by (length, symbol), by a stable
  //    counting pass over the lengths in symbol order
  uint8_t* lenpos = reinterpret_cast<uint8_t*>(srt == ka ? kb : ka);  // the free key array
  if (tid <= SZ3G_LMAX + 1) s_cnt[tid] = 0;
  __syncthreads();
  for (int i0 = 0; i0 < K; i0 += kCbThreads) {
    const int i = i0 + tid;
    uint32_t L = 0;
    if (i < K) {
      if (pick >= 0) {
        L = R->r[pick].lenpos[i];
        lenpos[i] = (uint8_t)L;
      } else {
        L = nf[i];
        lenpos[(uint32_t)(srt[i] & 0xffffu)] = (uint8_t)L;
      }
    }
    warp_count(s_cnt, L, i < K);
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t start = 0, fc = 0;
    for (int L = 1; L <= SZ3G_LMAX; ++L) {
      if (L > 1) fc = (fc + s_cnt[L - 1]) << 1;
      s_fc[L] = fc;
      s_start[L] = start;
      start += s_cnt[L];
    }
    st->n_used = (uint32_t)K;
  }
  block_counting_pass<32>(
      K, [&](int i) { return (uint32_t)lenpos[i]; },
      [&](int i, uint32_t r) {
        const uint32_t L = lenpos[i], sy = symord[i], code = s_fc[L] + (r - s_start[L]);
        table[sy] = (L << 24) | code;
        if (len_out) len_out[sy] = (uint8_t)L;
        if (code_out) code_out[sy] = code;
      });
  __syncthreads();
  // 4. code-length section of the stream: (u16 symbol, u8 length) by symbol
  if (d_out) {
    const unsigned long long off = SZ3G_HEADER_BYTES + pad8(st->n_unpred * (unsigned long long)esz);
    const unsigned long long end = pad8(off + 3ull * K);
    if (end > out_capacity) {
      if (tid == 0) atomicOr(&st->flags, kFlagCapacity);
      return;
    }
    for (int i = tid; i < K; i += kCbThreads) {
      const uint32_t s = symord[i];
      unsigned char* q = d_out + off + 3ull * i;
      q[0] = (unsigned char)(s & 0xff);
      q[1] = (unsigned char)(s >> 8);
      q[2] = (unsigned char)(table[s] >> 24);
    }
    for (unsigned long long b = off + 3ull * K + tid; b < end; b += kCbThreads) d_out[b] = 0;
  }
}

__global__ void __launch_bounds__(kCbThreads) codebook_rounds_kernel(const HistList* H, CbRounds* R) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_base[kHcNseg + 1];
  const int tid = threadIdx.x, r = blockIdx.x;
  const int K = used_count(H, s_base);
  if (K <= kSpecMax) {  // small alphabets: the codebook kernel's own speculative rounds
    if (tid == 0) R->fits[r] = 0;
    return;
  }
  CbRound& g = R->r[r];
  const bool in_smem = K <= kSmemLeaves;
  unsigned long long* ka = in_smem ? (unsigned long long*)smem : g.keys;
  unsigned long long* kb = in_smem ? (unsigned long long*)(smem + kSmemLeaves * 8) : g.keys2;
  used_entries(H, s_base, K, [&](int p, uint32_t c, uint32_t) {
    const uint32_t f = c >> r;
    ka[p] = ((unsigned long long)(f ? f : 1u) << 16) | (uint32_t)p;
  });
  __syncthreads();
  unsigned long long* srt = nullptr;
  bool deep;
  uint32_t* nf;
  if (in_smem) {
    nf = (uint32_t*)(smem + kCbOffNf);
    deep = one_round_lengths(ka, kb, nf, (uint16_t*)(smem + kCbOffPar), K, (uint32_t*)nullptr, (uint32_t*)nullptr,
                             &srt);
  } else {
    nf = g.nf;
    uint32_t* lw_s = K <= kCbSmemWeights ? (uint32_t*)smem : nullptr;
    deep = one_round_lengths(ka, kb, nf, g.parent, K, lw_s, lw_s ? lw_s + K : nullptr, &srt);
  }
  if (!deep)
    for (int i = tid; i < K; i += kCbThreads) g.lenpos[(uint32_t)(srt[i] & 0xffffu)] = (uint8_t)nf[i];
  if (tid == 0) R->fits[r] = deep ? 0 : 1;
}

int launch_codebook(const uint32_t* hist, uint32_t nsym, uint32_t* table, uint8_t* len_out, uint32_t* code_out,
                    DevState* st, void* scratch, unsigned char* d_out, unsigned long long out_capacity, int esz,
                    cudaStream_t s, void* rounds) {
  auto kern = codebook_kernel;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem) != cudaSuccess)
    return SZ3G_E_CUDA;
  CbGlobal* g = (CbGlobal*)scratch;
  SZ3G_LAUNCH(kKCodebook, s, hist_compact_kernel<<<kHcNseg, kHcThreads, 0, s>>>(hist, nsym, &g->hl, st));
  if (rounds) {
    if (cudaFuncSetAttribute(codebook_rounds_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem) !=
        cudaSuccess)
      return SZ3G_E_CUDA;
    SZ3G_LAUNCH(kKCodebook, s,
                codebook_rounds_kernel<<<kCbRounds, kCbThreads, kCbSmem, s>>>(&g->hl, (CbRounds*)rounds));
  }
  SZ3G_LAUNCH(kKCodebook, s,
              kern<<<1, kCbThreads, kCbSmem, s>>>(nsym, table, len_out, code_out, st, g, d_out, out_capacity, esz,
                                                  (const CbRounds*)rounds));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// ---------------------------------------------------------------------------
// Encoder.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Decoupled look-back: exclusive prefix of chunk j's value, whole warp.  A
// wait longer than `limit` polls gives up, raises the timeout flag and
// returns the partial prefix (the caller's status then reports the timeout).
__device__ unsigned long long lookback(unsigned long long* stat, long long j, DevState* st, uint32_t limit) {
  const int lane = threadIdx.x & 31;
  unsigned long long excl = 0;
  long long base = j - 1;
  int spins = 0;
  while (base >= 0) {
    const long long idx = base - lane;
    unsigned long long v = idx >= 0 ? ld_acquire(stat + idx) : kFlagInc;
    const unsigned not_ready = __ballot_sync(0xffffffffu, (v >> 62) == 0);
    if (not_ready) {
      if ((uint32_t)++spins > limit) {
        if (lane == 0) atomicOr(&st->flags, kFlagTimeout);
        return excl;
      }
      __nanosleep(32);
      continue;
    }
    const unsigned inc = __ballot_sync(0xffffffffu, (v >> 62) == 2);
    const int stop = inc ? __ffs(inc) - 1 : 31;  // nearest inclusive predecessor
    unsigned long long part = lane <= stop ? (v & kValMask) : 0ull;
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    excl += part;
    if (inc) break;
    base -= 32;
  }
  return excl;
}

// Exclusive prefix of CTA c's value agg over the CTAs before it (warp 0 of
// the CTA, CTAs in ticket order): publishes the aggregate, looks back,
// publishes the inclusive value.
__device__ __forceinline__ unsigned long long cta_prefix(unsigned long long* stat, unsigned long long c,
                                                         unsigned long long agg, DevState* st, uint32_t limit) {
  if (threadIdx.x == 0) st_release(stat + c, (c == 0 ? kFlagInc : kFlagAgg) | agg);
  const unsigned long long ex = lookback(stat, (long long)c, st, limit);
  if (threadIdx.x == 0 && c > 0) st_release(stat + c, kFlagInc | (ex + agg));
  return ex;
}

struct EncArgs {
  const uint16_t* codes;
  const uint32_t* table;
  const void* x;                // input field (unpredictable values)
  unsigned long long n, n_chunks;
  uint32_t chunk;
  int esz;
  const uint32_t* cwords;       // words of every chunk (from count_kernel)
  const unsigned long long* wexcl;  // exclusive prefix of cwords
  const unsigned long long* zexcl;  // exclusive prefix of the zero codes per chunk
  DevState* st;
  unsigned char* d_out;         // stream mode: the output stream
  unsigned long long out_capacity;
  uint32_t* words_out;          // raw mode: payload
  uint32_t* chunk_words_out;    // raw mode: words per chunk
  uint16_t* sub_out;            // raw mode: sub-block bit lengths (nsb - 1 per chunk), or null
  uint32_t nsb;                 // 512-code sub-blocks per chunk
  unsigned long long cap_words; // raw mode
  void* unpred_out;             // raw mode: unpredictable values (or null)
  int mode;                     // kEncodeStream / kEncodeRaw
  int emit_payload;             // 0: only gather unpredictable values
  uint32_t spin_limit;          // look-back wait limit
  long long silent_chunk;       // injected failure: this chunk never publishes (-1: none)
};

constexpr int kEncWarps = 8;
constexpr int kRingWords = 200;

__device__ __forceinline__ unsigned long long map_code_to_input(const PassMap& map, unsigned long long i) {
  int lo = 0, hi = map.n - 1;
  while (lo < hi) {  // largest p with off <= i
    const int mid = (lo + hi + 1) >> 1;
    if (map.e[mid].off <= i) lo = mid;
    else hi = mid - 1;
  }
  const PassMapEntry& e = map.e[lo];
  unsigned long long j = i - e.off;
  const unsigned long long c3 = j % e.E[3];
  j /= e.E[3];
  const unsigned long long c2 = j % e.E[2];
  j /= e.E[2];
  const unsigned long long c1 = j % e.E[1];
  j /= e.E[1];
  return e.xstart + j * e.xls[0] + c1 * e.xls[1] + c2 * e.xls[2] + c3 * e.xls[3];
}

// Pass 1 of the encoder: bits (as 32-bit words) and zero codes of every chunk.
// One warp per chunk; each lane takes 16-byte pieces of eight codes, four
// pieces in flight before their table entries are looked up.
__global__ void __launch_bounds__(kEncWarps * 32) count_kernel(const uint16_t* __restrict__ codes,
                                                               const uint32_t* __restrict__ table, unsigned long long n,
                                                               unsigned long long n_chunks, uint32_t chunk,
                                                               uint32_t* cwords, uint32_t* czeros) {
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kEncWarps;
  for (unsigned long long j = (unsigned long long)blockIdx.x * kEncWarps + (threadIdx.x >> 5); j < n_chunks;
       j += nwarps) {
    const unsigned long long i0 = j * chunk;
    const uint32_t cnt = (uint32_t)min((unsigned long long)chunk, n - i0);
    const uint16_t* cp = codes + i0;
    uint32_t bits = 0, zeros = 0;
    auto piece = [&](const uint4& v) {
      const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t c0 = wv[q] & 0xffffu, c1 = wv[q] >> 16;
        bits += (__ldg(table + c0) >> 24) + (__ldg(table + c1) >> 24);
        zeros += (c0 == 0) + (c1 == 0);
      }
    };
    uint32_t t = lane * 8;
    for (; t + 3 * 256 + 8 <= cnt; t += 4 * 256) {  // four whole pieces
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(reinterpret_cast<const uint4*>(cp + t + u * 256));
#pragma unroll
      for (int u = 0; u < 4; ++u) piece(v[u]);
    }
    for (; t < cnt; t += 256) {
      if (t + 8 <= cnt) {
        piece(__ldg(reinterpret_cast<const uint4*>(cp + t)));
      } else {
        for (uint32_t u = t; u < cnt; ++u) {
          const uint32_t c = cp[u];
          bits += __ldg(table + c) >> 24;
          zeros += c == 0;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      bits += __shfl_xor_sync(0xffffffffu, bits, o);
      zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
    }
    if (lane == 0) {
      cwords[j] = (bits + 31) >> 5;
      czeros[j] = zeros;
    }
  }
}

// Pass 2: one warp per chunk writes the chunk's bits (MSB first, through a
// shared-memory word ring), its table entries, and gathers its unpredictable
// values from the input.  ONEPASS (stream mode): the warp takes its chunk by
// a ticket, counts the chunk's bits and zero codes itself and finds their
// prefixes over the earlier chunks by decoupled look-back (wstat / zstat,
// cleared with the workspace), so no count pass or scans run before it.
template <typename U, bool ONEPASS>
__global__ void __launch_bounds__(kEncWarps * 32) emit_kernel(const EncArgs a, const __grid_constant__ PassMap map,
                                                              uint32_t* ticket, unsigned long long* wstat,
                                                              unsigned long long* zstat) {
  __shared__ uint32_t ring[kEncWarps][kRingWords];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* buf = ring[w];
  for (int k = lane; k < kRingWords; k += 32) buf[k] = 0;
  __syncwarp();
  DevState* st = a.st;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kEncWarps;
  unsigned long long j = (unsigned long long)blockIdx.x * kEncWarps + w;
  for (;; j += nwarps) {
    if (ONEPASS) {
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(ticket, 1u);
      j = __shfl_sync(0xffffffffu, t, 0);
    }
    if (j >= a.n_chunks) break;
    const unsigned long long i0 = j * a.chunk;
    const uint32_t cnt = (uint32_t)min((unsigned long long)a.chunk, a.n - i0);
    const uint16_t* cp = a.codes + i0;
    unsigned long long words, wexcl, zexcl;
    if (ONEPASS) {
      uint32_t bits = 0, zeros = 0;
      for (uint32_t t = lane * 8; t < cnt; t += 256) {
        if (t + 8 <= cnt) {
          const uint4 v = *reinterpret_cast<const uint4*>(cp + t);
          const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t c0 = wv[q] & 0xffffu, c1 = wv[q] >> 16;
            bits += (a.table[c0] >> 24) + (a.table[c1] >> 24);
            zeros += (c0 == 0) + (c1 == 0);
          }
        } else {
          for (uint32_t u = t; u < cnt; ++u) {
            const uint32_t c = cp[u];
            bits += a.table[c] >> 24;
            zeros += c == 0;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        bits += __shfl_xor_sync(0xffffffffu, bits, o);
        zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
      }
      words = (bits + 31) >> 5;
      const bool publish = (long long)j != a.silent_chunk;
      if (lane == 0 && publish) {
        st_release(wstat + j, (j == 0 ? kFlagInc : kFlagAgg) | words);
        st_release(zstat + j, (j == 0 ? kFlagInc : kFlagAgg) | zeros);
      }
      wexcl = lookback(wstat, (long long)j, st, a.spin_limit);
      zexcl = lookback(zstat, (long long)j, st, a.spin_limit);
      if (lane == 0 && j > 0 && publish) {
        st_release(wstat + j, kFlagInc | (wexcl + words));
        st_release(zstat + j, kFlagInc | (zexcl + zeros));
      }
    } else {
      words = a.cwords[j];
      wexcl = a.wexcl[j];
      zexcl = a.zexcl[j];
    }
    if (lane == 0 && j == a.n_chunks - 1) st->n_words = wexcl + words;
    // destinations
    uint32_t* pay;
    uint16_t* sub = nullptr;
    U* unp;
    bool ok = true;
    if (a.mode == kEncodeStream) {
      const unsigned long long nu = st->n_unpred;
      const unsigned long long off_table = SZ3G_HEADER_BYTES + pad8(nu * a.esz);
      const unsigned long long off_chunks = off_table + pad8(3ull * st->n_used);
      const unsigned long long off_sub = off_chunks + pad8(a.n_chunks * 4);
      const unsigned long long off_payload = off_sub + pad8(a.n_chunks * (a.nsb - 1) * 2);
      unp = reinterpret_cast<U*>(a.d_out + SZ3G_HEADER_BYTES);
      pay = reinterpret_cast<uint32_t*>(a.d_out + off_payload);
      if (a.nsb > 1) sub = reinterpret_cast<uint16_t*>(a.d_out + off_sub) + j * (a.nsb - 1);
      if (off_payload + 4 * (wexcl + words) > a.out_capacity) {
        ok = false;
        if (lane == 0) atomicOr(&st->flags, kFlagCapacity);
      } else if (lane == 0) {
        *reinterpret_cast<uint32_t*>(a.d_out + off_chunks + 4 * j) = (uint32_t)words;
      }
    } else {
      unp = reinterpret_cast<U*>(a.unpred_out);
      pay = a.words_out;
      if (a.sub_out && a.nsb > 1) sub = a.sub_out + j * (a.nsb - 1);
      if (a.emit_payload) {
        if (wexcl + words > a.cap_words) {
          ok = false;
          if (lane == 0) atomicOr(&st->flags, kFlagCapacity);
        } else if (lane == 0) {
          a.chunk_words_out[j] = (uint32_t)words;
        }
      }
    }
    if (!ok) continue;
    const bool emit = a.emit_payload != 0;
    unsigned long long wpos = wexcl;  // next word to write
    uint32_t carry = 0;               // bits pending in buf[0]
    unsigned long long zpos = zexcl;
    uint32_t sbits = 0;               // bits of the current 512-code sub-block
    if (emit && sub && lane == 0)     // sub-blocks past the end of a short chunk are empty
      for (uint32_t b = (cnt + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK; b + 1 < a.nsb; ++b) sub[b] = 0;
    for (uint32_t r0 = 0; r0 < cnt; r0 += 256) {
      const uint32_t t = r0 + lane * 8;
      uint32_t c8[8];
      uint32_t nb = 0, nzl = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) c8[q] = 0xffffffffu;
      if (t + 8 <= cnt) {
        const uint4 v = *reinterpret_cast<const uint4*>(cp + t);
        c8[0] = v.x & 0xffffu; c8[1] = v.x >> 16; c8[2] = v.y & 0xffffu; c8[3] = v.y >> 16;
        c8[4] = v.z & 0xffffu; c8[5] = v.z >> 16; c8[6] = v.w & 0xffffu; c8[7] = v.w >> 16;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (t + q < cnt) c8[q] = cp[t + q];
      }
      uint32_t e8[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        e8[q] = c8[q] != 0xffffffffu ? a.table[c8[q]] : 0u;
        nb += e8[q] >> 24;
        nzl += c8[q] == 0;
      }
      uint32_t incl = nb, zincl = nzl;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        const uint32_t yz = __shfl_up_sync(0xffffffffu, zincl, o);
        if (lane >= o) {
          incl += y;
          zincl += yz;
        }
      }
      const uint32_t round_bits = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t round_zeros = __shfl_sync(0xffffffffu, zincl, 31);
      sbits += round_bits;
      if ((r0 & 256) || r0 + 256 >= cnt) {  // a sub-block ends with this round
        const uint32_t b = r0 >> 9;
        if (emit && sub && lane == 0 && b + 1 < a.nsb) sub[b] = (uint16_t)sbits;
        sbits = 0;
      }
      if (emit) {
        uint32_t o = carry + incl - nb;
        if (nb <= 64) {
          // the lane's codes concatenated in one register, then OR-ed into
          // the (at most three) ring words they cover
          unsigned long long acc = 0;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint32_t L = e8[q] >> 24;
            acc = L ? (acc << L) | (e8[q] & 0xffffffu) : acc;
          }
          if (nb) {
            const unsigned long long x = acc << (64 - nb);  // left-aligned
            const uint32_t wi = o >> 5, sh = o & 31;
            const uint32_t v0 = (uint32_t)(x >> (32 + sh)), v1 = (uint32_t)(x >> sh),
                           v2 = (uint32_t)(x << (32 - sh));
            if (v0) atomicOr(&buf[wi], v0);
            if (v1) atomicOr(&buf[wi + 1], v1);
            if (v2) atomicOr(&buf[wi + 2], v2);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint32_t L = e8[q] >> 24, val = e8[q] & 0xffffffu;
            if (L == 0) continue;
            const uint32_t wi = o >> 5, sh = o & 31;
            if (sh + L <= 32) {
              atomicOr(&buf[wi], val << (32 - sh - L));
            } else {
              atomicOr(&buf[wi], val >> (sh + L - 32));
              atomicOr(&buf[wi + 1], val << (64 - sh - L));
            }
            o += L;
          }
        }
        __syncwarp();
        const uint32_t total = carry + round_bits;
        const uint32_t full = total >> 5;
        for (uint32_t k = lane; k < full; k += 32)
          if (SZ3G_IN(wpos + k < wexcl + words, st)) pay[wpos + k] = buf[k];
        wpos += full;
        const uint32_t rest = buf[full];
        __syncwarp();
        for (uint32_t k = lane; k <= full; k += 32) buf[k] = 0;
        __syncwarp();
        carry = total & 31;
        if (lane == 0) buf[0] = carry ? rest : 0u;
        __syncwarp();
      }
      if (nzl && unp) {
        unsigned long long zr = zpos + zincl - nzl;
        bool nonfinite = false;
        for (int q = 0; q < 8; ++q) {
          if (c8[q] == 0) {
            const unsigned long long xi = map_code_to_input(map, i0 + t + q);
            const U v = reinterpret_cast<const U*>(a.x)[xi];
            if (SZ3G_IN(a.mode != kEncodeStream || zr < st->n_unpred, st)) unp[zr] = v;
            ++zr;
            // the quantizer sends every NaN / Inf to the unpredictable list
            nonfinite |= sizeof(U) == 4 ? ((v & 0x7f800000u) == 0x7f800000u)
                                        : ((v & 0x7ff0000000000000ull) == 0x7ff0000000000000ull);
          }
        }
        if (nonfinite) atomicOr(&st->flags, kFlagNonFinite);
      }
      zpos += round_zeros;
    }
    // raw mode: the number of unpredictable values is known at the last chunk
    if (a.mode == kEncodeRaw && lane == 0 && j == a.n_chunks - 1) st->n_unpred = zpos;
    if (emit) {
      if (carry && lane == 0 && SZ3G_IN(wpos < wexcl + words, st)) pay[wpos] = buf[0];
      __syncwarp();
      if (lane == 0) buf[0] = 0;
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Device-wide exclusive prefix sum of n uint32 values into uint64, one pass:
// each CTA scans a tile of kScanTile values and finds the total of the tiles
// before it by decoupled look-back.  Optionally checks that every value is
// <= limit and that the grand total equals `expect` (else: corrupt flag).
// `state` is scan_state_bytes(n) of scratch, zeroed by the launcher.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanPer = 16, kScanTile = kScanThreads * kScanPer;

size_t scan_state_bytes(unsigned long long n) { return 256 + 8 * ((n + kScanTile - 1) / kScanTile + 1); }

__global__ void __launch_bounds__(kScanThreads) scan_kernel(const uint32_t* in, unsigned long long n,
                                                            unsigned long long* out, uint32_t limit,
                                                            unsigned long long expect, int check_expect,
                                                            unsigned char* state, DevState* st, uint32_t spin_limit) {
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_excl;
  __shared__ unsigned long long s_tile;
  uint32_t* ticket = reinterpret_cast<uint32_t*>(state);
  unsigned long long* stat = reinterpret_cast<unsigned long long*>(state + 256);
  const unsigned long long ntiles = (n + kScanTile - 1) / kScanTile;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const unsigned long long t = s_tile;
  if (t >= ntiles) return;
  const unsigned long long b = t * kScanTile + (unsigned long long)threadIdx.x * kScanPer;
  uint32_t v[kScanPer];
  unsigned long long sum = 0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = b + k < n ? in[b + k] : 0u;
    if (limit && v[k] > limit) bad = true;
    sum += v[k];
  }
  unsigned long long agg;
  unsigned long long run = block_exclusive_scan(sum, s_warp, &agg);
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) st_release(stat + t, (t == 0 ? kFlagInc : kFlagAgg) | agg);
    const unsigned long long ex = lookback(stat, (long long)t, st, spin_limit);
    if (threadIdx.x == 0) {
      if (t > 0) st_release(stat + t, kFlagInc | (ex + agg));
      s_excl = ex;
      if (check_expect && t == ntiles - 1 && ex + agg != expect) atomicOr(&st->flags, kFlagCorrupt);
    }
  }
  __syncthreads();
  run += s_excl;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (b + k < n) out[b + k] = run;
    run += v[k];
  }
  if (bad) atomicOr(&st->flags, kFlagCorrupt);
}

// state_zeroed: the caller cleared `state` already (with its workspace).
int launch_scan(const uint32_t* in, unsigned long long n, unsigned long long* out, uint32_t limit,
                unsigned long long expect, int check_expect, void* state, DevState* st, cudaStream_t s,
                bool state_zeroed) {
  if (!state_zeroed && cudaMemsetAsync(state, 0, scan_state_bytes(n), s) != cudaSuccess) return SZ3G_E_CUDA;
  const unsigned long long ntiles = (n + kScanTile - 1) / kScanTile;
  SZ3G_LAUNCH(kKScan, s,
              scan_kernel<<<(unsigned)(ntiles ? ntiles : 1), kScanThreads, 0, s>>>(
                  in, n, out, limit, expect, check_expect, (unsigned char*)state, st,
                  g_debug.wait_limit ? g_debug.wait_limit : (uint32_t)kSpinLimit));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

size_t encode_scratch_bytes(unsigned long long n_chunks) {
  return 2 * ((n_chunks * 4 + 255) & ~255ull) + 2 * ((n_chunks * 8 + 255) & ~255ull) +
         2 * ((scan_state_bytes(n_chunks) + 255) & ~255ull);
}

// ---------------------------------------------------------------------------
// Stream-mode packing for fields whose chunk word offsets and zero-code
// prefixes are known (count pass, then chunk_prefix_kernel).  One warp per
// chunk, rounds of 256 codes (eight per lane): each lane concatenates the
// codewords of its codes 0-3 and of its codes 4-7 into two strings in 64-bit
// registers (a string of four codewords over 64 bits, which needs codewords
// averaging more than 16 bits, is placed as two strings of two), a warp scan
// gives each lane's bit offset, the strings are OR-ed into a shared-memory
// word ring and the round's full words leave as coalesced stores.  Zero codes (unpredictable values) are looked for once per round
// (a 16-bit minimum over the lane's codes); only rounds that hold one scan
// their positions and gather the values.
// ---------------------------------------------------------------------------
constexpr int kPackRing = 202;  // words: two guard words, one round (<= 256 x 24 bits) and the carried word

// OR a string of n (1..64) bits, right-aligned in (hi, lo), into buf so that
// it covers bits [e - n, e) (MSB first).  z zero bits follow it in its last
// word; shifted left by z the string spans the words (e-1)/32 - 2 .. (e-1)/32
// -- 32-bit funnel shifts only.
// shared-memory OR of a nonzero word, predicated (no branch)
__device__ __forceinline__ void red_or_nz(uint32_t* p, uint32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t@q red.shared.or.b32 [%0], %1;\n\t}" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(p)),
               "r"(v)
               : "memory");
}
__device__ __forceinline__ void ring_or(uint32_t* buf, uint32_t hi, uint32_t lo, uint32_t e, DevState* st) {
  const uint32_t we = (e - 1) >> 5, z = (0u - e) & 31u;
  if (!SZ3G_IN(e >= 1 && we < (uint32_t)kPackRing - 2, st)) return;
  red_or_nz(&buf[we], lo << z);
  red_or_nz(&buf[we - 1], __funnelshift_l(lo, hi, z));
  red_or_nz(&buf[we - 2], __funnelshift_l(hi, 0u, z));
}

// Packs chunk j (words payload words at word offset wexcl, its zero codes
// after zexcl earlier ones) with the calling warp; buf: the warp's ring.
template <typename U>
__device__ __forceinline__ void pack_chunk(const EncArgs& a, const PassMap& map, uint32_t* buf, int lane,
                                           unsigned long long j, uint32_t words, unsigned long long wexcl,
                                           unsigned long long zexcl, unsigned long long off_chunks,
                                           unsigned long long off_sub, unsigned long long off_payload, U* unp,
                                           unsigned long long nu) {
  DevState* st = a.st;
  const uint32_t* table = a.table;
  const unsigned long long i0 = j * a.chunk;
  const uint32_t cnt = (uint32_t)min((unsigned long long)a.chunk, a.n - i0);
  const uint16_t* cp = a.codes + i0;
  unsigned long long zpos = zexcl;
  if (lane == 0 && j == a.n_chunks - 1) st->n_words = wexcl + words;
  if (off_payload + 4 * (wexcl + words) > a.out_capacity) {
    if (lane == 0) atomicOr(&st->flags, kFlagCapacity);
    return;
  }
  if (lane == 0) *reinterpret_cast<uint32_t*>(a.d_out + off_chunks + 4 * j) = words;
  uint32_t* pay = reinterpret_cast<uint32_t*>(a.d_out + off_payload) + wexcl;
  uint16_t* sub = a.nsb > 1 ? reinterpret_cast<uint16_t*>(a.d_out + off_sub) + j * (a.nsb - 1) : nullptr;
  if (sub && lane == 0)  // sub-blocks past the end of a short chunk are empty
    for (uint32_t b = (cnt + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK; b + 1 < a.nsb; ++b) sub[b] = 0;
  uint32_t wpos = 0, carry = 0, sbits = 0;
  for (uint32_t r0 = 0; r0 < cnt; r0 += 256) {
    const uint32_t t = r0 + lane * 8;
    uint4 v = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);  // 0xffff: no code
    if (t + 8 <= cnt) {
      v = *reinterpret_cast<const uint4*>(cp + t);
    } else if (t < cnt) {
      uint32_t h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) h[q] = t + q < cnt ? cp[t + q] : 0xffffu;
      v = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
    }
    const uint32_t cw[4] = {v.x, v.y, v.z, v.w};
    // the codewords of the lane's two halves, right-aligned in (hi, lo)
    // (codewords are at most 24 bits: 32-bit funnel shifts)
    uint32_t ahi[2] = {0u, 0u}, alo[2] = {0u, 0u}, n2[2] = {0u, 0u};
    auto append = [&](int q, uint32_t e) {  // e = len << 24 | codeword
      const uint32_t L = e >> 24;
      ahi[q >> 2] = __funnelshift_l(alo[q >> 2], ahi[q >> 2], L);
      alo[q >> 2] = (alo[q >> 2] << L) | (e & 0xffffffu);
      n2[q >> 2] += L;
    };
    if (r0 + 256 <= cnt) {  // every lane has eight codes
      uint32_t e8[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) e8[q] = __ldg(table + ((q & 1) ? cw[q >> 1] >> 16 : cw[q >> 1] & 0xffffu));
#pragma unroll
      for (int q = 0; q < 8; ++q) append(q, e8[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t c = (q & 1) ? cw[q >> 1] >> 16 : cw[q >> 1] & 0xffffu;
        append(q, c != 0xffffu ? __ldg(table + c) : 0u);
      }
    }
    const uint32_t nb = n2[0] + n2[1];
    uint32_t incl = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t round_bits = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t o = carry + incl - nb;  // bit offset of the lane's strings in the ring
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t n = n2[h];
      o += n;  // the end of the half's string
      if (n <= 64) {
        if (n) ring_or(buf, ahi[h], alo[h], o, st);
      } else {  // four codewords over 64 bits: the half as two strings of two
        uint32_t op = o - n;
        for (int p = 0; p < 2; ++p) {
          uint32_t xh = 0u, xl = 0u, m = 0u;
          for (int q = 4 * h + 2 * p; q < 4 * h + 2 * p + 2; ++q) {
            const uint32_t c = (q & 1) ? cw[q >> 1] >> 16 : cw[q >> 1] & 0xffffu;
            const uint32_t e = c != 0xffffu ? __ldg(table + c) : 0u;
            xh = __funnelshift_l(xl, xh, e >> 24);
            xl = (xl << (e >> 24)) | (e & 0xffffffu);
            m += e >> 24;
          }
          op += m;
          if (m) ring_or(buf, xh, xl, op, st);
        }
      }
    }
    sbits += round_bits;
    if ((r0 & 256) || r0 + 256 >= cnt) {  // a sub-block ends with this round
      const uint32_t b = r0 >> 9;
      if (sub && lane == 0 && b + 1 < a.nsb) sub[b] = (uint16_t)sbits;
      sbits = 0;
    }
    __syncwarp();
    // the round's full words leave (and are cleared); the partial word moves
    // to the front of the ring
    const uint32_t total = carry + round_bits, full = total >> 5;
    const uint32_t rest = buf[full];
    for (uint32_t k0 = 0; k0 < full; k0 += 32) {  // warp-uniform trip count
      const uint32_t k = k0 + lane;
      if (k < full) {
        if (SZ3G_IN(wpos + k < words, st)) pay[wpos + k] = buf[k];
        buf[k] = 0;
      }
    }
    wpos += full;
    carry = total & 31;
    __syncwarp();
    if (lane == 0) {
      buf[full] = 0;
      buf[0] = carry ? rest : 0u;
    }
    __syncwarp();
    // unpredictable values of the round, in code order
    if (nu) {
      const uint32_t mn = __vminu2(__vminu2(v.x, v.y), __vminu2(v.z, v.w));
      const bool has0 = (mn & 0xffffu) == 0 || (mn >> 16) == 0;
      if (__any_sync(0xffffffffu, has0)) {
        uint32_t nz = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) nz += ((q & 1) ? cw[q >> 1] >> 16 : cw[q >> 1] & 0xffffu) == 0;
        uint32_t zincl = nz;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, zincl, s);
          if (lane >= s) zincl += y;
        }
        unsigned long long zr = zpos + zincl - nz;
        bool nonfinite = false;
        for (int q = 0; q < 8 && nz; ++q) {
          const uint32_t c = (q & 1) ? cw[q >> 1] >> 16 : cw[q >> 1] & 0xffffu;
          if (c == 0) {
            const U x = reinterpret_cast<const U*>(a.x)[map_code_to_input(map, i0 + t + q)];
            if (SZ3G_IN(zr < nu, st)) unp[zr] = x;
            ++zr;
            // the quantizer sends every NaN / Inf to the unpredictable list
            nonfinite |= sizeof(U) == 4 ? ((x & 0x7f800000u) == 0x7f800000u)
                                        : ((x & 0x7ff0000000000000ull) == 0x7ff0000000000000ull);
          }
        }
        if (nonfinite) atomicOr(&st->flags, kFlagNonFinite);
        zpos += __shfl_sync(0xffffffffu, zincl, 31);
      }
    }
  }
  if (carry && lane == 0 && SZ3G_IN(wpos < words, st)) pay[wpos] = buf[0];
  __syncwarp();
  if (lane == 0) buf[0] = 0;
  __syncwarp();
}

template <typename U>
__global__ void __launch_bounds__(kEncWarps * 32, 4) pack_kernel(const EncArgs a, const __grid_constant__ PassMap map) {
  __shared__ uint32_t ring[kEncWarps][kPackRing];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* buf = ring[w] + 2;  // buf[-2], buf[-1]: guards for strings that end in word 0 or 1
  for (int k = lane; k < kPackRing; k += 32) ring[w][k] = 0;
  __syncwarp();
  DevState* st = a.st;
  const unsigned long long nu = st->n_unpred;
  const unsigned long long off_table = SZ3G_HEADER_BYTES + pad8(nu * a.esz);
  const unsigned long long off_chunks = off_table + pad8(3ull * st->n_used);
  const unsigned long long off_sub = off_chunks + pad8(a.n_chunks * 4);
  const unsigned long long off_payload = off_sub + pad8(a.n_chunks * (a.nsb - 1) * 2);
  U* unp = reinterpret_cast<U*>(a.d_out + SZ3G_HEADER_BYTES);
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kEncWarps;
  for (unsigned long long j = (unsigned long long)blockIdx.x * kEncWarps + w; j < a.n_chunks; j += nwarps)
    pack_chunk<U>(a, map, buf, lane, j, a.cwords[j], a.wexcl[j], a.zexcl[j], off_chunks, off_sub, off_payload, unp,
                  nu);
}


// Bits (as 32-bit words) and zero codes of chunk j, counted by the calling
// warp: four 16-byte pieces of eight codes in flight per lane.
__device__ __forceinline__ void chunk_counts(const uint16_t* __restrict__ codes, const uint32_t* __restrict__ table,
                                             unsigned long long n, uint32_t chunk, unsigned long long j, int lane,
                                             uint32_t* words, uint32_t* zeros) {
  const unsigned long long i0 = j * chunk;
  const uint32_t cnt = (uint32_t)min((unsigned long long)chunk, n - i0);
  const uint16_t* cp = codes + i0;
  uint32_t bits = 0, zc = 0;
  auto piece = [&](const uint4& v) {
    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) bits += (__ldg(table + (wv[q] & 0xffffu)) >> 24) + (__ldg(table + (wv[q] >> 16)) >> 24);
    // zero codes (unpredictable values) are rare: a 16-bit minimum over the
    // eight codes finds the pieces that hold one
    const uint32_t mn = __vminu2(__vminu2(v.x, v.y), __vminu2(v.z, v.w));
    if ((mn & 0xffffu) == 0 || (mn >> 16) == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) zc += ((wv[q] & 0xffffu) == 0) + ((wv[q] >> 16) == 0);
  };
  uint32_t t = lane * 8;
  for (; t + 3 * 256 + 8 <= cnt; t += 4 * 256) {  // four whole pieces
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldg(reinterpret_cast<const uint4*>(cp + t + u * 256));
#pragma unroll
    for (int u = 0; u < 4; ++u) piece(v[u]);
  }
  for (; t < cnt; t += 256) {
    if (t + 8 <= cnt) {
      piece(__ldg(reinterpret_cast<const uint4*>(cp + t)));
    } else {
      for (uint32_t u = t; u < cnt; ++u) {
        const uint32_t c = cp[u];
        bits += __ldg(table + c) >> 24;
        zc += c == 0;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    bits += __shfl_xor_sync(0xffffffffu, bits, o);
    zc += __shfl_xor_sync(0xffffffffu, zc, o);
  }
  *words = (bits + 31) >> 5;
  *zeros = zc;
}

// ---------------------------------------------------------------------------
// Stream header (written last, once every count is known): by the encoder's
// last tile when the one-pass encoder runs, else by finalize_kernel.
// ---------------------------------------------------------------------------
struct HeaderArgs {
  unsigned char bytes[SZ3G_HEADER_BYTES];  // static fields, counts filled on device
  unsigned long long n_chunks;
  int esz;
  uint32_t nsb;  // 512-code sub-blocks per chunk
};

// The header, the padding after each section and the stream length, by
// threads tid of nthr; nw: payload words.
__device__ void write_stream_header(const HeaderArgs& h, DevState* st, unsigned char* d_out,
                                    unsigned long long out_capacity, unsigned long long nw, int tid, int nthr) {
  if (st->flags & (kFlagNonFinite | kFlagZeroRange | kFlagBadBound | kFlagCapacity | kFlagTimeout)) return;
  const unsigned long long nu = st->n_unpred;
  const uint32_t nused = st->n_used;
  const unsigned long long off_table = SZ3G_HEADER_BYTES + pad8(nu * h.esz);
  const unsigned long long off_chunks = off_table + pad8(3ull * nused);
  const unsigned long long off_sub = off_chunks + pad8(h.n_chunks * 4);
  const unsigned long long n_sub = h.n_chunks * (h.nsb - 1);
  const unsigned long long off_payload = off_sub + pad8(n_sub * 2);
  const unsigned long long end = off_payload + pad8(nw * 4);
  if (end > out_capacity) {
    if (tid == 0) atomicOr(&st->flags, kFlagCapacity);
    return;
  }
  for (int b = tid; b < SZ3G_HEADER_BYTES; b += nthr) {
    unsigned char v = h.bytes[b];
    if (b >= 56 && b < 64) v = (unsigned char)(__double_as_longlong(st->eb_abs) >> (8 * (b - 56)));
    if (b >= 64 && b < 72) v = (unsigned char)(st->ebT_bits >> (8 * (b - 64)));
    if (b >= 76 && b < 80) v = (unsigned char)(nused >> (8 * (b - 76)));
    if (b >= 88 && b < 96) v = (unsigned char)(nu >> (8 * (b - 88)));
    if (b >= 104 && b < 112) v = (unsigned char)(nw >> (8 * (b - 104)));
    d_out[b] = v;
  }
  // zero padding after the unpredictable values, the chunk table and the payload
  if (tid < 8) {
    const unsigned long long u_end = SZ3G_HEADER_BYTES + nu * h.esz;
    if (u_end + tid < off_table) d_out[u_end + tid] = 0;
    const unsigned long long c_end = off_chunks + h.n_chunks * 4;
    if (c_end + tid < off_sub) d_out[c_end + tid] = 0;
    const unsigned long long s_end = off_sub + n_sub * 2;
    if (s_end + tid < off_payload) d_out[s_end + tid] = 0;
    const unsigned long long p_end = off_payload + nw * 4;
    if (p_end + tid < end) d_out[p_end + tid] = 0;
  }
  if (tid == 0) st->out_bytes = end;
}

__global__ void finalize_kernel(const HeaderArgs h, DevState* st, unsigned char* d_out,
                                unsigned long long out_capacity) {
  write_stream_header(h, st, d_out, out_capacity, st->n_words, threadIdx.x, blockDim.x);
}

// The header's static fields and the sizes the device needs to finish it.
static HeaderArgs header_args(const Plan& pl, const sz3g_params* p) {
  HeaderArgs h;
  memset(&h, 0, sizeof(h));
  unsigned char* b = h.bytes;
  auto put = [&](int off, unsigned long long v, int n) {
    for (int i = 0; i < n; ++i) b[off + i] = (unsigned char)(v >> (8 * i));
  };
  b[0] = 'S';
  b[1] = 'Z';
  b[2] = '3';
  b[3] = 'G';
  put(4, 1, 2);
  b[6] = (unsigned char)p->dtype;
  b[7] = (unsigned char)p->ndim;
  for (int i = 0; i < 4; ++i) put(8 + 8 * i, i < (int)p->ndim ? p->dims[i] : 1, 8);
  b[40] = (unsigned char)p->eb_mode;
  b[41] = (unsigned char)p->interp;
  b[42] = p->per_level;
  b[43] = (unsigned char)pl.L;
  put(44, p->radius, 4);
  unsigned long long ebb;
  memcpy(&ebb, &p->eb, 8);
  put(48, ebb, 8);
  put(72, p->chunk_codes, 4);
  put(80, pl.N, 8);
  put(96, pl.n_chunks, 8);
  if (p->per_level) {
    for (int l = 1; l <= pl.L; ++l) {
      b[112 + l] = p->level_interp[l];
      for (int i = 0; i < 4; ++i) b[144 + 4 * l + i] = i < (int)p->ndim ? p->level_order[l][i] : 0;
    }
  }
  for (int i = 0; i < 4; ++i) b[272 + i] = i < (int)p->ndim ? p->dim_order[i] : 0;
  h.n_chunks = pl.n_chunks;
  h.esz = pl.esz;
  h.nsb = pl.nsub;
  return h;
}

// Stream-mode encoder in one pass for any number of chunks: tiles of
// kEncWarps consecutive chunks taken in ticket order; each warp counts its
// chunk, the tile's totals are published and the words and zero codes before
// the tile found by one decoupled look-back over the tiles (warp 0), then
// each warp packs its chunk (its codes read again, from the cache).  ticket,
// wstat and zstat start at zero (the compressor's workspace is cleared when
// it starts).
template <typename U>
__global__ void __launch_bounds__(kEncWarps * 32, 5) tile_pack_kernel(const EncArgs a,
                                                                       const __grid_constant__ PassMap map,
                                                                       uint32_t* ticket, unsigned long long* wstat,
                                                                       unsigned long long* zstat,
                                                                       const __grid_constant__ HeaderArgs hdr,
                                                                       int with_header) {
  __shared__ uint32_t ring[kEncWarps][kPackRing];
  __shared__ uint32_t s_words[kEncWarps], s_zeros[kEncWarps], s_tile;
  __shared__ unsigned long long s_we, s_ze;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* buf = ring[w] + 2;  // buf[-2], buf[-1]: guards for strings that end in word 0 or 1
  for (int k = lane; k < kPackRing; k += 32) ring[w][k] = 0;
  __syncwarp();
  DevState* st = a.st;
  const unsigned long long nu = st->n_unpred;
  const unsigned long long off_table = SZ3G_HEADER_BYTES + pad8(nu * a.esz);
  const unsigned long long off_chunks = off_table + pad8(3ull * st->n_used);
  const unsigned long long off_sub = off_chunks + pad8(a.n_chunks * 4);
  const unsigned long long off_payload = off_sub + pad8(a.n_chunks * (a.nsb - 1) * 2);
  U* unp = reinterpret_cast<U*>(a.d_out + SZ3G_HEADER_BYTES);
  const unsigned long long ntiles = (a.n_chunks + kEncWarps - 1) / kEncWarps;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const unsigned long long tile = s_tile;
    if (tile >= ntiles) break;
    const unsigned long long j = tile * kEncWarps + w;
    uint32_t words = 0, zeros = 0;
    if (j < a.n_chunks) chunk_counts(a.codes, a.table, a.n, a.chunk, j, lane, &words, &zeros);
    if (lane == 0) {
      s_words[w] = words;
      s_zeros[w] = zeros;
    }
    __syncthreads();
    if (w < 2) {  // warp 0: the words before the tile, warp 1: the zero codes (at once)
      const uint32_t* cnt = w == 0 ? s_words : s_zeros;
      unsigned long long* stat = w == 0 ? wstat : zstat;
      uint32_t agg = lane < kEncWarps ? cnt[lane] : 0u;
      for (int o = 16; o > 0; o >>= 1) agg += __shfl_xor_sync(0xffffffffu, agg, o);
      if (lane == 0) st_release(stat + tile, (tile == 0 ? kFlagInc : kFlagAgg) | agg);
      const unsigned long long ex = lookback(stat, (long long)tile, st, a.spin_limit);
      if (lane == 0) {
        if (tile > 0) st_release(stat + tile, kFlagInc | (ex + agg));
        if (w == 0) s_we = ex;
        else s_ze = ex;
      }
    }
    __syncthreads();
    unsigned long long wexcl = s_we, zexcl = s_ze;
    for (int q = 0; q < w; ++q) {
      wexcl += s_words[q];
      zexcl += s_zeros[q];
    }
    if (with_header && tile + 1 == ntiles) {  // every total is known once the last tile's prefix is
      unsigned long long nw = s_we;
      for (int q = 0; q < kEncWarps; ++q) nw += s_words[q];
      write_stream_header(hdr, st, a.d_out, a.out_capacity, nw, threadIdx.x, blockDim.x);
    }
    if (j < a.n_chunks)
      pack_chunk<U>(a, map, buf, lane, j, words, wexcl, zexcl, off_chunks, off_sub, off_payload, unp, nu);
    __syncthreads();  // the tile's shared counts are read before the next ticket overwrites them
  }
}

// count -> two scans -> emit (or, stream mode on at most kOnePassMaxChunks
// chunks, emit alone).  scratch: encode_scratch_bytes(n_chunks).
constexpr unsigned long long kOnePassMaxChunks = 1024;
static int encode_pipeline(EncArgs a, const PassMap* map, unsigned char* scratch, cudaStream_t s,
                           const HeaderArgs* hdr = nullptr, bool* header_written = nullptr) {
  if (header_written) *header_written = false;
  a.spin_limit = g_debug.wait_limit ? g_debug.wait_limit : (uint32_t)kSpinLimit;
  a.silent_chunk = g_debug.silent_chunk;
  const unsigned long long nch = a.n_chunks;
  const size_t a4 = (nch * 4 + 255) & ~255ull, a8 = (nch * 8 + 255) & ~255ull,
               as = (scan_state_bytes(nch) + 255) & ~255ull;
  uint32_t* cw = (uint32_t*)scratch;
  uint32_t* cz = (uint32_t*)(scratch + a4);
  unsigned long long* we = (unsigned long long*)(scratch + 2 * a4);
  unsigned long long* ze = (unsigned long long*)(scratch + 2 * a4 + a8);
  unsigned char* s1 = scratch + 2 * a4 + 2 * a8;
  unsigned char* s2 = s1 + as;
  int nb = (int)((nch + kEncWarps - 1) / kEncWarps);
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  if (a.mode == kEncodeStream && a.emit_payload && nch <= kOnePassMaxChunks) {
    // one pass: the compressor's workspace (this scratch included) was
    // cleared when it started -- cw[0] is the ticket, we / ze the look-back states.
    // Only for fields of few chunks: with thousands of chunks in flight the
    // look-back frontier (about 32 chunks per round) becomes a serial chain.
    if (a.esz == 4)
      SZ3G_LAUNCH(kKEncode, s, emit_kernel<uint32_t, true><<<nb, kEncWarps * 32, 0, s>>>(a, *map, cw, we, ze));
    else
      SZ3G_LAUNCH(kKEncode, s, emit_kernel<unsigned long long, true><<<nb, kEncWarps * 32, 0, s>>>(a, *map, cw, we, ze));
    return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
  }
  if (a.mode == kEncodeStream && a.emit_payload) {
    // counts, prefixes and packing in one pass over tiles of chunks (cw[0]
    // is the ticket, we / ze the tiles' look-back states, all cleared with
    // the compressor's workspace)
    const unsigned long long ntiles = (nch + kEncWarps - 1) / kEncWarps;
    int dev = 0, nsm = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (a.esz == 4)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tile_pack_kernel<uint32_t>, kEncWarps * 32, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tile_pack_kernel<unsigned long long>, kEncWarps * 32, 0);
    if (per < 1) per = 1;
    const unsigned ng = (unsigned)std::min<unsigned long long>(ntiles, (unsigned long long)nsm * per);
    HeaderArgs h{};
    if (hdr) h = *hdr;
    const int wh = hdr ? 1 : 0;
    if (a.esz == 4)
      SZ3G_LAUNCH(kKEncode, s, tile_pack_kernel<uint32_t><<<ng, kEncWarps * 32, 0, s>>>(a, *map, cw, we, ze, h, wh));
    else
      SZ3G_LAUNCH(kKEncode, s,
                  tile_pack_kernel<unsigned long long><<<ng, kEncWarps * 32, 0, s>>>(a, *map, cw, we, ze, h, wh));
    if (cudaGetLastError() != cudaSuccess) return SZ3G_E_CUDA;
    if (header_written) *header_written = hdr != nullptr;
    return SZ3G_OK;
  }
  SZ3G_LAUNCH(kKEncode, s, count_kernel<<<nb, kEncWarps * 32, 0, s>>>(a.codes, a.table, a.n, nch, a.chunk, cw, cz));
  if (a.mode == kEncodeStream && a.emit_payload) {
    // the prefixes (the compressor's workspace, this scratch included, was
    // cleared when it started), then the packing kernel
    int rc = launch_scan(cw, nch, we, 0, 0, 0, s1, a.st, s, true);
    if (rc) return rc;
    rc = launch_scan(cz, nch, ze, 0, 0, 0, s2, a.st, s, true);
    if (rc) return rc;
    a.cwords = cw;
    a.wexcl = we;
    a.zexcl = ze;
    if (a.esz == 4)
      SZ3G_LAUNCH(kKEncode, s, pack_kernel<uint32_t><<<nb, kEncWarps * 32, 0, s>>>(a, *map));
    else
      SZ3G_LAUNCH(kKEncode, s, pack_kernel<unsigned long long><<<nb, kEncWarps * 32, 0, s>>>(a, *map));
    return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
  }
  // stream mode: the compressor's workspace (this scratch included) was cleared when it started
  const bool zeroed = a.mode == kEncodeStream;
  int rc = launch_scan(cw, nch, we, 0, 0, 0, s1, a.st, s, zeroed);
  if (rc) return rc;
  rc = launch_scan(cz, nch, ze, 0, 0, 0, s2, a.st, s, zeroed);
  if (rc) return rc;
  a.cwords = cw;
  a.wexcl = we;
  a.zexcl = ze;
  if (a.esz == 4)
    SZ3G_LAUNCH(kKEncode, s,
                emit_kernel<uint32_t, false><<<nb, kEncWarps * 32, 0, s>>>(a, *map, nullptr, nullptr, nullptr));
  else
    SZ3G_LAUNCH(kKEncode, s,
                emit_kernel<unsigned long long, false><<<nb, kEncWarps * 32, 0, s>>>(a, *map, nullptr, nullptr,
                                                                                    nullptr));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int launch_encode(const Plan& pl, const uint16_t* codes, const uint32_t* table, const void* d_in, const PassMap* map,
                  void* scratch, DevState* st, unsigned char* d_out, unsigned long long out_capacity, int mode,
                  uint32_t* words_out, uint32_t* chunk_words_out, uint16_t* sub_out, unsigned long long cap_words,
                  cudaStream_t s, const sz3g_params* header_p, bool* header_written) {
  EncArgs a{};
  a.codes = codes;
  a.table = table;
  a.x = d_in;
  a.n = pl.N;
  a.n_chunks = pl.n_chunks;
  a.chunk = pl.chunk;
  a.esz = pl.esz;
  a.st = st;
  a.d_out = d_out;
  a.out_capacity = out_capacity;
  a.words_out = words_out;
  a.chunk_words_out = chunk_words_out;
  a.sub_out = sub_out;
  a.nsb = (pl.chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  a.cap_words = cap_words;
  a.unpred_out = nullptr;
  a.mode = mode;
  a.emit_payload = 1;
  if (header_p && mode == kEncodeStream) {
    const HeaderArgs h = header_args(pl, header_p);
    return encode_pipeline(a, map, (unsigned char*)scratch, s, &h, header_written);
  }
  if (header_written) *header_written = false;
  return encode_pipeline(a, map, (unsigned char*)scratch, s);
}

// Unpredictable values in traversal order, without encoding (stage API).
int launch_compact_unpred(const Plan& pl, const uint16_t* codes, const void* d_in, const PassMap* map, void* scratch,
                          const uint32_t* table, void* d_unpred, DevState* st, cudaStream_t s) {
  EncArgs a{};
  a.codes = codes;
  a.table = table;
  a.x = d_in;
  a.n = pl.N;
  a.n_chunks = pl.n_chunks;
  a.chunk = pl.chunk;
  a.esz = pl.esz;
  a.st = st;
  a.mode = kEncodeRaw;
  a.emit_payload = 0;
  a.nsb = (pl.chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  a.unpred_out = d_unpred;
  return encode_pipeline(a, map, (unsigned char*)scratch, s);
}

int launch_finalize(const Plan& pl, const sz3g_params* p, DevState* st, unsigned char* d_out,
                    unsigned long long out_capacity, cudaStream_t s) {
  const HeaderArgs h = header_args(pl, p);
  SZ3G_LAUNCH(kKFinalize, s, finalize_kernel<<<1, 64, 0, s>>>(h, st, d_out, out_capacity));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// ---------------------------------------------------------------------------
// Decoder.
// ---------------------------------------------------------------------------
struct DecTables {
  uint32_t lut[1 << kLutBits];   // window of kLutBits bits -> len << 16 | sym; 0 = a longer codeword
  uint32_t lim[SZ3G_LMAX + 2];   // (fc[L] + cnt[L]) << (LMAX - L): an LMAX-bit window below it
                                 // starts with a codeword of at most L bits
  uint32_t base[SZ3G_LMAX + 2];  // start[L] - fc[L] (mod 2^32): codeword c of length L is symbol
                                 // sorted[c + base[L]]
  uint32_t n_used;
  uint32_t has_zero;               // symbol 0 (the unpredictable code) has a codeword
  unsigned long long keys[kSyms];  // used symbols (length << 16 | symbol) in symbol order
  uint16_t sorted[kSyms];          // symbols by (length, symbol)
};

// Decode tables from a (symbol, length) list: either the stream's 3-byte
// records (tab != null, n_used entries) or a length per symbol (len != null).
__global__ void __launch_bounds__(kCbThreads) decode_tables_kernel(const unsigned char* tab, uint32_t n_used,
                                                                   const uint8_t* len, uint32_t nsym, DecTables* T,
                                                                   DevState* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_cnt[SZ3G_LMAX + 2];
  __shared__ int s_bad;
  __shared__ unsigned long long s_kraft;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_bad = 0;
    s_kraft = 0;
  }
  if (tid <= SZ3G_LMAX + 1) s_cnt[tid] = 0;
  __syncthreads();
  unsigned long long* keys;
  int K;
  if (tab) {
    K = (int)n_used;
    keys = K <= kSmemLeaves ? (unsigned long long*)smem : T->keys;
    for (int i = tid; i < K; i += kCbThreads) {
      const uint32_t s = tab[3 * i] | ((uint32_t)tab[3 * i + 1] << 8);
      const uint32_t L = tab[3 * i + 2];
      if (s >= nsym || L < 1 || L > SZ3G_LMAX) s_bad = 1;
      if (i > 0) {
        const uint32_t sp = tab[3 * (i - 1)] | ((uint32_t)tab[3 * (i - 1) + 1] << 8);
        if (sp >= s) s_bad = 1;
      }
      keys[i] = ((unsigned long long)(L & 31) << 16) | (s & 0xffffu);
    }
  } else {
    // compact the used symbols (symbol order), 64 per thread
    const int per = kSyms / kCbThreads;
    uint32_t mine = 0;
    for (int s = tid * per; s < tid * per + per; ++s) mine += (s < (int)nsym && len[s]) ? 1u : 0u;
    unsigned long long tot;
    unsigned long long pos = block_exclusive_scan(mine, s_warp, &tot);
    K = (int)tot;
    keys = K <= kSmemLeaves ? (unsigned long long*)smem : T->keys;
    for (int s = tid * per; s < tid * per + per && s < (int)nsym; ++s) {
      if (len[s]) {
        if (len[s] > SZ3G_LMAX) s_bad = 1;
        keys[pos++] = ((unsigned long long)(len[s] & 31) << 16) | (uint32_t)s;
      }
    }
  }
  __syncthreads();
  if (K < 1) {
    if (tid == 0) atomicOr(&st->flags, kFlagCorrupt);
    return;
  }
  // Kraft sum in units of 2^-LMAX
  for (int i0 = 0; i0 < K; i0 += kCbThreads) {
    const int i = i0 + tid;
    const uint32_t L = i < K ? (uint32_t)(keys[i] >> 16) : 0u;
    const bool ok = L >= 1 && L <= SZ3G_LMAX;
    // a warp's sum is below 32 * 2^(LMAX-1) < 2^32
    const uint32_t kr = __reduce_add_sync(0xffffffffu, ok ? 1u << (SZ3G_LMAX - L) : 0u);
    if ((tid & 31) == 0 && kr) atomicAdd(&s_kraft, (unsigned long long)kr);
    warp_count(s_cnt, L, ok);
  }
  __syncthreads();
  // a stream's table is a complete code (one symbol: one 1-bit codeword); a
  // caller's length array may be any prefix code (Kraft sum <= 1): windows
  // past its last codeword are no codeword and stop the decoder
  const unsigned long long full = 1ull << SZ3G_LMAX;
  const bool kraft_ok = tab ? (K == 1 ? s_kraft == full / 2 : s_kraft == full) : s_kraft <= full;
  if (s_bad || !kraft_ok) {
    if (tid == 0) atomicOr(&st->flags, kFlagCorrupt);
    return;
  }
  __shared__ uint32_t s_start[SZ3G_LMAX + 2], s_base[SZ3G_LMAX + 2], s_lim[SZ3G_LMAX + 2], s_cb[SZ3G_LMAX + 2];
  __shared__ uint32_t s_wc[32][SZ3G_LMAX + 2];  // per-warp counts, then offsets, of each length in a tile
  if (tid == 0) {
    uint32_t start = 0, fc = 0;
    for (int L = 1; L <= SZ3G_LMAX; ++L) {
      if (L > 1) fc = (fc + s_cnt[L - 1]) << 1;
      s_start[L] = start;
      T->base[L] = s_cb[L] = start - fc;
      T->lim[L] = s_lim[L] = (fc + s_cnt[L]) << (SZ3G_LMAX - L);
      start += s_cnt[L];
    }
    T->n_used = (uint32_t)K;
    T->has_zero = (keys[0] & 0xffffull) == 0 ? 1u : 0u;  // keys are in symbol order
  }
  if (tid <= SZ3G_LMAX + 1) s_base[tid] = 0;
  // Symbols ordered by (length, symbol): the keys are in symbol order, so a
  // stable counting sort on the length gives the order.  Tiles of one key
  // per thread: a key's rank is its length's start, plus the keys of that
  // length in earlier tiles (s_base), earlier warps of the tile and earlier
  // lanes of its warp.
  const int lane = tid & 31, warp = tid >> 5;
  for (int t0 = 0; t0 < K; t0 += kCbThreads) {
    for (int i = tid; i < 32 * (SZ3G_LMAX + 2); i += kCbThreads) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const int i = t0 + tid;
    const unsigned long long key = i < K ? keys[i] : 0ull;
    const uint32_t L = (uint32_t)(key >> 16), sym = (uint32_t)(key & 0xffffu);  // L = 0: no key
    const unsigned peers = __match_any_sync(0xffffffffu, L);
    if (lane == __ffs(peers) - 1) s_wc[warp][L] = (uint32_t)__popc(peers);
    __syncthreads();
    if (warp >= 1 && warp <= SZ3G_LMAX) {  // warp w scans the warps' counts of length w
      const uint32_t c = s_wc[lane][warp], base = s_base[warp];
      uint32_t x = c;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      s_wc[lane][warp] = base + x - c;
      __syncwarp();
      if (lane == 31) s_base[warp] = base + x;
    }
    __syncthreads();
    if (L) {
      const uint32_t r = s_start[L] + s_wc[warp][L] + (uint32_t)__popc(peers & ((1u << lane) - 1u));
      T->sorted[r] = (uint16_t)sym;
    }
    __syncthreads();
  }
  // Direct table.  The windows that start with a codeword of length L are
  // the range [lim[L-1], lim[L]) (left-justified), so a window finds its
  // length by a short walk and its symbol through the (length, symbol) order.
  for (int w = tid; w < (1 << kLutBits); w += kCbThreads) {
    const uint32_t v = (uint32_t)w << (SZ3G_LMAX - kLutBits);
    uint32_t L = 1;
    while (L <= (uint32_t)kLutBits && v >= s_lim[L]) ++L;
    uint32_t e = 0;
    if (L <= (uint32_t)kLutBits) e = (L << 16) | T->sorted[((uint32_t)w >> (kLutBits - L)) + s_cb[L]];
    T->lut[w] = e;
  }
}

struct DecArgs {
  const uint32_t* words;
  const uint32_t* chunk_words;
  const uint16_t* sub_bits;         // bit lengths of 512-code sub-blocks (nsb - 1 per chunk), or null
  unsigned long long n_chunks, n;
  unsigned long long n_words;       // payload words
  uint32_t chunk, nsb;              // nsb = 512-code sub-blocks per chunk
  uint32_t unit, upc;               // codes per decoding thread, threads per chunk
  uint32_t maxw;                    // the most words a chunk may have
  uint32_t spin_limit;              // look-back wait limit
  const DecTables* T;
  uint16_t* codes;
  uint32_t* zcnt;                   // zero codes per 512-code sub-block
  unsigned char* lb;                // look-back state (decode_state_bytes, zeroed)
  unsigned long long n_ctas;
  DevState* st;
};

// One thread decodes one unit: a 512-code sub-block when the stream carries
// sub-block lengths (its start bit is their sum), else a whole chunk.
//
// The thread's payload words pass through a ring of kDecRingW words in shared
// memory (slot q of thread t at word q * kDecThreads + t: the lanes of a warp
// never share a bank).  They arrive as 16-byte blocks copied asynchronously
// into a per-thread staging area kDecStage blocks ahead of their use.  The
// two words under the read position are kept in registers; the next
// codeword's length and symbol come from a 12-bit direct table in shared
// memory (entry: symbol << 16 | length; 0 for a longer codeword) applied to
// the 32-bit window at the read position (one funnel shift), so only the
// table read is on a code's serial path.  One ring check per eight codes
// (eight codes use at most 6 words), the word advance as a select, one byte
// permute packing two symbols, zero codes counted on the packed words, and a
// rarely taken branch for codewords longer than the table (their length by
// comparisons with the left-justified limits).
constexpr int kDecThreads = 256;
constexpr int kDecLB = 12;                        // bits of the shared-memory direct table
constexpr int kDecRingW = 16;                     // ring words per thread (a power of two)
constexpr int kDecStage = 2;                      // 16-byte blocks in flight per thread
constexpr size_t kDecOffRing = (size_t)4 << kDecLB;
constexpr size_t kDecOffStage = kDecOffRing + (size_t)kDecRingW * kDecThreads * 4;
constexpr size_t kDecodeSmem = kDecOffStage + (size_t)kDecStage * kDecThreads * 16;

__device__ __forceinline__ void dec_stage(uint4* dst, const uint4* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n\tcp.async.commit_group;" ::"r"(d), "l"(src) : "memory");
}

// A codeword longer than the direct table: its length from the left-justified
// limits, its symbol from the (length, symbol) order; symbol << 16 | length,
// or 0 when the window starts no codeword.
__device__ __forceinline__ uint32_t dec_long(uint32_t win, const uint32_t* s_lim, const uint32_t* s_base,
                                             uint32_t n_used, const uint16_t* sorted) {
  const uint32_t v = win >> (32 - SZ3G_LMAX);
  uint32_t L = kDecLB + 1;
#pragma unroll
  for (int l = kDecLB + 1; l < SZ3G_LMAX; ++l) L += v >= s_lim[l];
  const uint32_t k = (win >> (32 - L)) + s_base[L];
  if (v >= s_lim[SZ3G_LMAX] || k >= n_used) return 0u;
  return ((uint32_t)__ldg(sorted + k) << 16) | L;
}

// number of zero 16-bit halves of x
__device__ __forceinline__ uint32_t zero_halves(uint32_t x) {
  return (uint32_t)((x & 0xffffu) == 0) + (uint32_t)((x >> 16) == 0);
}

__global__ void __launch_bounds__(kDecThreads, 4) decode_kernel(const DecArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t s_lim[SZ3G_LMAX + 2], s_base[SZ3G_LMAX + 2];
  __shared__ int s_skip;
  __shared__ unsigned long long s_tk, s_ex, s_warp[32], s_cwx[kDecThreads];
  const int tid = threadIdx.x;
  unsigned long long* stat_w = reinterpret_cast<unsigned long long*>(a.lb + 256);
  if (tid == 0) s_skip = (a.st->flags & kFlagCorrupt) != 0;  // tables rejected
  uint32_t* lut = reinterpret_cast<uint32_t*>(dsm);
  // the 12-bit table from the 13-bit one (len << 16 | sym): codewords of 13
  // bits become "longer"; entries as sym << 16 | len
  for (int w = tid; w < (1 << kDecLB); w += kDecThreads) {
    const uint32_t e = a.T->lut[w << (kLutBits - kDecLB)];
    const uint32_t L = e >> 16;
    lut[w] = (L != 0 && L <= (uint32_t)kDecLB) ? ((e << 16) | L) : 0u;
  }
  if (tid <= SZ3G_LMAX + 1) {
    s_lim[tid] = a.T->lim[tid];
    s_base[tid] = a.T->base[tid];
  }
  // The CTA (one of about as many as fit on the GPU at once) takes groups of
  // kDecThreads units in ticket order until none are left: no second, partly
  // filled round of CTAs.
  for (;;) {
    __syncthreads();  // the previous group's shared state is no longer read
    if (tid == 0) s_tk = atomicAdd(reinterpret_cast<unsigned int*>(a.lb), 1u);
    __syncthreads();
    const unsigned long long c = s_tk, units = a.n_chunks * a.upc;
    if (c >= a.n_ctas) break;
    // 1. Word offsets.  The chunks whose first unit falls in this CTA are its
    //    own (one per thread at most); their exclusive prefix inside the CTA,
    //    plus the words of every chunk before them (a decoupled look-back over
    //    the CTAs before it in ticket order), gives each chunk's first word.
    //    The chunk this CTA shares with the one before starts that chunk's
    //    words before the CTA's own.  The last CTA checks the total.
    const unsigned long long jo0 = (c * kDecThreads + a.upc - 1) / a.upc;
    const unsigned long long jo1 = min(((c + 1) * kDecThreads + a.upc - 1) / a.upc, a.n_chunks);
    bool bad = false;
    uint32_t cwo = 0;
    if (jo0 + tid < jo1) {
      cwo = a.chunk_words[jo0 + tid];
      bad = cwo > a.maxw;
    }
    unsigned long long agg;
    s_cwx[tid] = block_exclusive_scan(cwo, s_warp, &agg);
    if (tid < 32) {
      const unsigned long long ex = cta_prefix(stat_w, c, agg, a.st, a.spin_limit);
      if (tid == 0) {
        s_ex = ex;
        if (c + 1 == a.n_ctas && ex + agg != a.n_words) atomicOr(&a.st->flags, kFlagCorrupt);
      }
    }
    __syncthreads();
    const unsigned long long ew = s_ex;
    // 2. The unit.  Returns true when it is corrupt.
    const unsigned long long u = c * kDecThreads + tid;
    auto decode_unit = [&]() -> bool {
      const uint32_t n_used = a.T->n_used;
      const bool count_zeros = a.T->has_zero != 0;
      uint32_t* ring = reinterpret_cast<uint32_t*>(dsm + kDecOffRing) + tid;  // word slot q at ring[q * kDecThreads]
      uint4* stg = reinterpret_cast<uint4*>(dsm + kDecOffStage) + tid;        // block slot s at stg[s * kDecThreads]
      const unsigned long long j = u / a.upc;
      const uint32_t b = (uint32_t)(u - j * a.upc);
      const uint32_t n_chunk = (uint32_t)min((unsigned long long)a.chunk, a.n - j * a.chunk);
      const uint32_t c0 = b * a.unit;
      const uint32_t nw = a.chunk_words[j];
      const uint16_t* sb = a.sub_bits ? a.sub_bits + j * (a.nsb - 1) : nullptr;
      uint32_t* zc = a.zcnt + j * a.nsb;
      auto zset = [&](uint32_t q, uint32_t v) {  // zero codes of the chunk's sub-block q
        if (SZ3G_IN(j * a.nsb + q < a.n_chunks * a.nsb, a.st)) zc[q] = v;
      };
      unsigned long long bit0 = 0;  // start bit of the unit inside the chunk
      if (sb)
        for (uint32_t q = 0; q < b; ++q) bit0 += sb[q];
      if (c0 >= n_chunk) {  // past the end of a short last chunk
        if (a.unit == SZ3G_SUBBLOCK) zset(b, 0u);
        return sb && b + 1 < a.nsb && sb[b] != 0;
      }
      const uint32_t c1 = min(c0 + a.unit, n_chunk);
      // a chunk with codes has at least one word, the unit's start bit inside
      // it, and all of its words inside the payload
      if (nw == 0 || bit0 >= 32ull * nw) return true;
      unsigned long long wj;  // the chunk's first word
      if (j >= jo0) {
        wj = ew + s_cwx[j - jo0];
      } else {
        if (ew < nw) return true;
        wj = ew - nw;
      }
      if (wj > a.n_words || nw > a.n_words - wj) return true;
      // The unit's words as a sequence of 16-byte blocks starting at the aligned
      // block that holds its first word; blocks past the payload's last one read
      // that block again (a correct code never depends on bits after its own,
      // and a decode that runs past its bits is caught by the bit count at the
      // end).
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(a.words + wj + (bit0 >> 5));
      const uint4* blk = reinterpret_cast<const uint4*>(a0 & ~(uintptr_t)15);
      const uintptr_t a_last = reinterpret_cast<uintptr_t>(a.words + a.n_words - 1) & ~(uintptr_t)15;
      const uint32_t q_last = a_last >= (a0 & ~(uintptr_t)15) ? (uint32_t)((a_last - (a0 & ~(uintptr_t)15)) >> 4) : 0u;
      constexpr uint32_t RM = kDecRingW - 1, SM_ = kDecStage - 1;
      auto stage = [&](uint32_t q) { dec_stage(stg + (q & SM_) * kDecThreads, blk + min(q, q_last)); };
      auto put = [&](uint32_t at, const uint4& v) {  // words at .. at + 3 of the sequence
        ring[((at + 0) & RM) * kDecThreads] = v.x;
        ring[((at + 1) & RM) * kDecThreads] = v.y;
        ring[((at + 2) & RM) * kDecThreads] = v.z;
        ring[((at + 3) & RM) * kDecThreads] = v.w;
      };
      stage(0);
      stage(1);
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      put(0, stg[0]);
      put(4, stg[1 * kDecThreads]);
      stage(2);
      stage(3);
      uint32_t stored = 8, next_use = 2;  // words in the ring; next staged block to take
      const uint32_t start_bit = (uint32_t)((a0 & 15) * 8) + (uint32_t)(bit0 & 31);
      // window: words wk - 2 (wa) and wk - 1 (wb); read position bp in wa
      uint32_t wk = (start_bit >> 5) + 2;
      uint32_t wa = ring[((wk - 2) & RM) * kDecThreads];
      uint32_t wb = ring[((wk - 1) & RM) * kDecThreads];
      uint32_t bp = start_bit & 31;
      uint32_t zeros = 0;
      bool fail = false;
      uint16_t* out = a.codes + j * a.chunk + c0;
      // one codeword: its entry (symbol << 16 | length), or false for a window
      // that starts no codeword
      auto one = [&](uint32_t& e) -> bool {
        const uint32_t win = __funnelshift_l(wb, wa, bp);
        e = lut[win >> (32 - kDecLB)];
        if ((e & 31u) == 0) {  // a codeword longer than the table
          e = dec_long(win, s_lim, s_base, n_used, a.T->sorted);
          if (e == 0) return false;
        }
        bp += e & 31u;
        const bool adv = bp >= 32;
        const uint32_t wn = ring[(wk & RM) * kDecThreads];
        wa = adv ? wb : wa;
        wb = adv ? wn : wb;
        wk += adv ? 1u : 0u;
        bp -= adv ? 32u : 0u;
        return true;
      };
      for (uint32_t i = c0; i < c1; i += 8, out += 8) {  // c0 is a multiple of 8
        if (i != c0 && (i & (SZ3G_SUBBLOCK - 1)) == 0) {  // whole-chunk units count per sub-block
          zset((i >> 9) - 1, zeros);
          zeros = 0;
        }
        // eight codes advance the window by at most 6 words
        while (stored < wk + 6) {
          asm volatile("cp.async.wait_group %0;" ::"n"(kDecStage - 1) : "memory");
          put(stored, stg[(next_use & SM_) * kDecThreads]);
          stored += 4;
          stage(next_use + kDecStage);  // into the slot just read
          ++next_use;
        }
        const uint32_t m = min(8u, c1 - i);
        if (m == 8) {
          uint32_t pk[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t e0 = 0, e1 = 0;
            if (!one(e0) || !one(e1)) {
              fail = true;
              break;
            }
            pk[q] = __byte_perm(e0, e1, 0x7632);  // symbol of e0 low, of e1 high
          }
          if (fail) break;
          if (count_zeros) zeros += zero_halves(pk[0]) + zero_halves(pk[1]) + zero_halves(pk[2]) + zero_halves(pk[3]);
          if (SZ3G_IN(j * a.chunk + i + 8 <= a.n, a.st))
            *reinterpret_cast<uint4*>(out) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        } else {
          for (uint32_t q = 0; q < m; ++q) {
            uint32_t e;
            if (!one(e)) {
              fail = true;
              break;
            }
            if (SZ3G_IN(j * a.chunk + i + q < a.n, a.st)) out[q] = (uint16_t)(e >> 16);
            if (count_zeros) zeros += (e >> 16) == 0;
          }
          if (fail) break;
        }
      }
      // no copy may land in shared memory after the thread has left
      asm volatile("cp.async.wait_all;" ::: "memory");
      if (fail) return true;
      zset((c1 - 1) >> 9, zeros);
      if (a.unit != SZ3G_SUBBLOCK)  // sub-blocks past the end of a short chunk
        for (uint32_t q = ((c1 - 1) >> 9) + 1; q < a.nsb; ++q) zset(q, 0u);
      // bits consumed from the chunk start; the recorded sub-block boundary
      // must be exactly where decoding ended
      const unsigned long long used = bit0 + (unsigned long long)((wk - 2) * 32u + bp - start_bit);
      if (sb && a.unit == SZ3G_SUBBLOCK && b + 1 < a.nsb && used != bit0 + sb[b]) return true;
      return used > 32ull * nw;
    };
    if (!s_skip && u < units && decode_unit()) bad = true;
    if (bad) atomicOr(&a.st->flags, kFlagCorrupt);
  }
}

size_t dec_tables_bytes() { return sizeof(DecTables); }

constexpr size_t kDecSmem = kSmemLeaves * 8;

int launch_decode_tables(const unsigned char* tab, uint32_t n_used, const uint8_t* len, uint32_t nsym, void* tables,
                         DevState* st, cudaStream_t s) {
  if (cudaFuncSetAttribute(decode_tables_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem) !=
      cudaSuccess)
    return SZ3G_E_CUDA;
  SZ3G_LAUNCH(kKDecodeTables, s, decode_tables_kernel<<<1, kCbThreads, kDecSmem, s>>>(tab, n_used, len, nsym, (DecTables*)tables, st));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// Look-back state of the decoder: a ticket and one word per CTA.
size_t decode_state_bytes(unsigned long long n_chunks, uint32_t chunk) {
  const unsigned long long nsb = (chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  return 256 + 8 * ((n_chunks * nsb + kDecThreads - 1) / kDecThreads + 1);
}

// words: payload; chunk_words: per-chunk word counts (validated here);
// sub_bits: sub-block lengths or null.  zcnt: zero codes per 512-code block.
// state: decode_state_bytes of scratch.
int launch_decode_chunks(const uint32_t* words, unsigned long long n_words, const uint32_t* chunk_words,
                         const uint16_t* sub_bits, unsigned long long n_chunks, uint32_t chunk, unsigned long long n,
                         const void* tables, uint16_t* codes, uint32_t* zcnt, void* state, DevState* st,
                         cudaStream_t s, bool state_zeroed) {
  if (!state_zeroed && cudaMemsetAsync(state, 0, decode_state_bytes(n_chunks, chunk), s) != cudaSuccess)
    return SZ3G_E_CUDA;
  DecArgs a{};
  a.words = words;
  a.chunk_words = chunk_words;
  a.sub_bits = sub_bits;
  a.n_chunks = n_chunks;
  a.n = n;
  a.n_words = n_words;
  a.chunk = chunk;
  a.nsb = (chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  a.unit = (sub_bits && a.nsb > 1) ? (uint32_t)SZ3G_SUBBLOCK : chunk;
  a.upc = (chunk + a.unit - 1) / a.unit;
  a.maxw = (uint32_t)(((unsigned long long)chunk * SZ3G_LMAX + 31) / 32);
  a.spin_limit = g_debug.wait_limit ? g_debug.wait_limit : (uint32_t)kSpinLimit;
  a.T = (const DecTables*)tables;
  a.codes = codes;
  a.zcnt = zcnt;
  a.lb = (unsigned char*)state;
  a.st = st;
  const unsigned long long threads = n_chunks * a.upc;
  a.n_ctas = threads ? (threads + kDecThreads - 1) / kDecThreads : 1;  // groups of kDecThreads units
  if (cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecodeSmem) !=
      cudaSuccess)
    return SZ3G_E_CUDA;
  int dev = 0, nsm = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, decode_kernel, kDecThreads, kDecodeSmem);
  const unsigned long long grid = min(a.n_ctas, (unsigned long long)nsm * (unsigned long long)(per > 0 ? per : 1));
  SZ3G_LAUNCH(kKDecode, s, decode_kernel<<<(unsigned)grid, kDecThreads, kDecodeSmem, s>>>(a));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// Zero-code counts per 512-code sub-block of every chunk, from a code array
// (used when codes come from the caller instead of the decoder).
__global__ void zero_count_kernel(const uint16_t* codes, unsigned long long n, uint32_t chunk, uint32_t nsb,
                                  unsigned long long n_chunks, uint32_t* zcnt) {
  const unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_chunks * nsb) return;
  const unsigned long long j = u / nsb;
  const uint32_t b = (uint32_t)(u - j * nsb);
  const unsigned long long n_chunk = min((unsigned long long)chunk, n - j * chunk);
  const unsigned long long i0 = j * chunk + (unsigned long long)b * SZ3G_SUBBLOCK;
  const unsigned long long i1 = j * chunk + min((unsigned long long)(b + 1) * SZ3G_SUBBLOCK, n_chunk);
  uint32_t z = 0;
  for (unsigned long long i = i0; i < i1; ++i) z += codes[i] == 0;
  zcnt[u] = z;
}

int launch_zero_counts(const uint16_t* codes, unsigned long long n, uint32_t chunk, unsigned long long n_chunks,
                       uint32_t* zcnt, cudaStream_t s) {
  const uint32_t nsb = (chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  const unsigned long long units = n_chunks * nsb;
  SZ3G_LAUNCH(kKZeroCount, s,
              zero_count_kernel<<<(unsigned)((units + 127) / 128), 128, 0, s>>>(codes, n, chunk, nsb, n_chunks, zcnt));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}


// table[sym] = len << 24 | code from separate arrays (stage API).
__global__ void pack_table_kernel(const uint8_t* len, const uint32_t* code, uint32_t nsym, uint32_t* table) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < (uint32_t)kSyms) table[s] = s < nsym ? (((uint32_t)len[s] << 24) | (code[s] & 0xffffffu)) : 0u;
}

int launch_pack_table(const uint8_t* len, const uint32_t* code, uint32_t nsym, uint32_t* table, cudaStream_t s) {
  SZ3G_LAUNCH(kKPackTable, s, pack_table_kernel<<<kSyms / 256, 256, 0, s>>>(len, code, nsym, table));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

}  // namespace sz3g
