// k_lz.cu -- the optional lossless stage after the Huffman coder: byte-level
// LZ77 over independent 32 KiB blocks (the dictionary coder that SZ3's
// pipelines end with; our own block format, see include/sz3g.h).
//
// Compress, one warp per block:
//   1. the block's bytes into shared memory;
//   2. match candidates of every position in parallel: 32 positions per step,
//      the lanes with equal 12-bit hashes found by __match_any_sync -- a
//      position's candidate is the nearest lower lane of its group, else the
//      table entry left by earlier steps; the group's highest lane then
//      updates the table -- and a bitmask of the positions whose candidate
//      matches in its first four bytes;
//   3. the greedy parse: the next matchable position by a ballot over the
//      bitmask words, the match extended 32 bytes per ballot, literals
//      copied by the warp;
// then the coded lengths are scanned and every payload (coded, or the raw
// block when coding does not shrink it) is gathered into place.
// Decompress, one warp per block, into shared memory: tokens read by lane 0,
// literals and matches copied by the warp (a match at distance d < 32 copies
// the d-byte period before it), every length and distance checked.
#include "internal.cuh"

namespace sz3g {

constexpr uint32_t kLzBlock = SZ3G_LZ_BLOCK;
constexpr uint32_t kLzHashBits = 12;
constexpr uint32_t kLzNone = 0xffffu;
constexpr uint32_t kLzRaw = 0x80000000u;
// shared memory of the block kernel: data (+16 pad), candidates, hash table, bitmask
constexpr size_t kLzOffCand = kLzBlock + 16;
constexpr size_t kLzOffTab = kLzOffCand + (size_t)kLzBlock * 2;
constexpr size_t kLzOffMask = kLzOffTab + ((size_t)1 << kLzHashBits) * 2;
constexpr size_t kLzSmem = kLzOffMask + (size_t)kLzBlock / 8;

__device__ __forceinline__ uint32_t lz_load4(const uint8_t* d, uint32_t i) {  // 4 bytes at any offset, little-endian
  const uint32_t* w = reinterpret_cast<const uint32_t*>(d);
  return __funnelshift_r(w[i >> 2], w[(i >> 2) + 1], 8 * (i & 3));
}

__device__ __forceinline__ uint32_t lz_hash(uint32_t v) { return (v * 2654435761u) >> (32 - kLzHashBits); }

// Writes one sequence at out[*k]: literals d[a, a + nl), then (ml > 0) a match
// of ml bytes at distance off.  Warp-wide; false when it would pass cap.
__device__ bool lz_put_seq(uint8_t* out, uint32_t* k, uint32_t cap, const uint8_t* d, uint32_t a, uint32_t nl,
                           uint32_t off, uint32_t ml) {
  const int lane = threadIdx.x & 31;
  const uint32_t xl = nl >= 15 ? (nl - 15) / 255 + 1 : 0;                       // literal-count bytes
  const uint32_t xm = (ml && ml - 4 >= 15) ? (ml - 4 - 15) / 255 + 1 : 0;       // match-length bytes
  const uint32_t need = 1 + xl + nl + (ml ? 2 + xm : 0);
  if (*k + need > cap) return false;
  uint8_t* o = out + *k;
  if (lane == 0) {
    const uint32_t tl = nl >= 15 ? 15 : nl, tm = ml == 0 ? 0 : (ml - 4 >= 15 ? 15 : ml - 4);
    o[0] = (uint8_t)(tl << 4 | tm);
    if (xl) o[xl] = (uint8_t)((nl - 15) % 255);
  }
  for (uint32_t t = lane; t + 1 < xl; t += 32) o[1 + t] = 255;
  for (uint32_t t = lane; t < nl; t += 32) o[1 + xl + t] = d[a + t];
  if (ml) {
    uint8_t* m = o + 1 + xl + nl;
    if (lane == 0) {
      m[0] = (uint8_t)(off & 0xff);
      m[1] = (uint8_t)(off >> 8);
      if (xm) m[1 + xm] = (uint8_t)((ml - 4 - 15) % 255);
    }
    for (uint32_t t = lane; t + 1 < xm; t += 32) m[2 + t] = 255;
  }
  *k += need;
  return true;
}

// One 32-thread CTA per block: coded payload to tmp + b * kLzBlock (at most
// the block's length - 1 bytes) and its size (bit 31: stored raw).
__global__ void __launch_bounds__(32) lz_block_kernel(const uint8_t* __restrict__ in, unsigned long long n,
                                                      uint8_t* __restrict__ tmp, uint32_t* __restrict__ sizes) {
  extern __shared__ __align__(16) uint8_t lsm[];
  uint8_t* d = lsm;
  uint16_t* cand = reinterpret_cast<uint16_t*>(lsm + kLzOffCand);
  uint16_t* tab = reinterpret_cast<uint16_t*>(lsm + kLzOffTab);
  uint32_t* mask = reinterpret_cast<uint32_t*>(lsm + kLzOffMask);
  const int lane = threadIdx.x;
  const unsigned long long b = blockIdx.x;
  const unsigned long long base0 = b * kLzBlock;
  const uint32_t nb = (uint32_t)min((unsigned long long)kLzBlock, n - base0);
  // 1. the block (16-byte pieces; the input is 16-byte aligned), zero padding
  const uint8_t* src = in + base0;
  const uint32_t n16 = nb / 16;
  for (uint32_t t = lane; t < n16; t += 32)
    reinterpret_cast<uint4*>(d)[t] = reinterpret_cast<const uint4*>(src)[t];
  for (uint32_t t = n16 * 16 + lane; t < nb + 16; t += 32) d[t] = t < nb ? src[t] : 0;
  for (uint32_t t = lane; t < (1u << kLzHashBits); t += 32) tab[t] = (uint16_t)kLzNone;
  const uint32_t nw = (nb + 31) / 32;
  for (uint32_t t = lane; t < nw; t += 32) mask[t] = 0;
  __syncwarp();
  // 2. candidates and the matchable bitmask
  const uint32_t npos = nb >= 4 ? nb - 3 : 0;  // positions 0..nb-4 have a hash
  for (uint32_t base = 0; base < npos; base += 32) {
    const uint32_t i = base + lane;
    const bool ok = i < npos;
    const uint32_t v = ok ? lz_load4(d, i) : 0u;
    const uint32_t h = ok ? lz_hash(v) : (0x10000u + lane);  // no lane outside the block shares a hash
    const unsigned peers = __match_any_sync(0xffffffffu, h);
    const unsigned lower = peers & ((1u << lane) - 1u);
    uint32_t c = kLzNone;
    if (ok) c = lower ? base + (31 - __clz(lower)) : tab[h];
    __syncwarp();
    if (ok && lane == 31 - __clz(peers)) tab[h] = (uint16_t)i;
    if (ok) cand[i] = (uint16_t)c;
    const bool m = ok && c != kLzNone && lz_load4(d, c) == v;
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if (lane == 0) mask[base >> 5] = bal;
    __syncwarp();
  }
  // 3. the greedy parse
  uint8_t* out = tmp + base0;
  const uint32_t cap = nb - 1;
  uint32_t pos = 0, anchor = 0, k = 0;
  bool fits = nb > 1;
  while (fits) {
    // next matchable position >= pos: lane l looks at bitmask word w0 + l
    uint32_t p = kLzNone * 65536u;  // none
    for (uint32_t w0 = pos >> 5; w0 < nw; w0 += 32) {
      const uint32_t w = w0 + lane;
      uint32_t mw = w < nw ? mask[w] : 0u;
      if (w == (pos >> 5)) mw &= ~0u << (pos & 31);
      const unsigned any = __ballot_sync(0xffffffffu, mw != 0);
      if (any) {
        const int fl = __ffs(any) - 1;
        const uint32_t mf = __shfl_sync(0xffffffffu, mw, fl);
        p = (w0 + fl) * 32 + (__ffs(mf) - 1);
        break;
      }
    }
    if (p >= npos) break;
    const uint32_t c = cand[p];
    uint32_t len = 4;
    for (;;) {  // extend while the next byte equals (the source may overlap p)
      const uint32_t q = p + len + lane;
      const bool eq = q < nb && d[c + len + lane] == d[q];
      const unsigned miss = __ballot_sync(0xffffffffu, !eq);
      if (miss) {
        len += __ffs(miss) - 1;
        break;
      }
      len += 32;
    }
    fits = lz_put_seq(out, &k, cap, d, anchor, p - anchor, p - c, len);
    __syncwarp();
    pos = anchor = p + len;
  }
  if (fits) fits = lz_put_seq(out, &k, cap, d, anchor, nb - anchor, 0, 0);
  if (lane == 0) sizes[b] = fits ? k : (nb | kLzRaw);
}

// Payload lengths rounded up to 4 bytes (and, decompressing, checked against
// the block lengths).
__global__ void lz_lens_kernel(const uint32_t* sizes, unsigned long long nblk, unsigned long long n, uint32_t* lens,
                               DevState* st) {
  const unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  const uint32_t s = sizes[b];
  const uint32_t len = s & ~kLzRaw;
  const uint32_t nb = (uint32_t)min((unsigned long long)kLzBlock, n - b * kLzBlock);
  if ((s & kLzRaw) ? len != nb : (len == 0 || len >= nb)) atomicOr(&st->flags, kFlagCorrupt);
  lens[b] = (len + 3) & ~3u;
}

// The stream: header, size table, payloads at data0 + off[b] (padded).  One CTA per block.
__global__ void lz_gather_kernel(const uint8_t* __restrict__ in, unsigned long long n, const uint8_t* __restrict__ tmp,
                                 const uint32_t* __restrict__ sizes, const unsigned long long* __restrict__ off,
                                 unsigned long long nblk, unsigned long long data0, uint8_t* __restrict__ out,
                                 DevState* st) {
  const unsigned long long b = blockIdx.x;
  if (b == 0) {
    for (unsigned long long t = threadIdx.x; t < data0; t += blockDim.x) {
      uint8_t v = 0;
      if (t < 4) v = (uint8_t)("SZLZ"[t]);
      else if (t < 8) v = (uint8_t)(kLzBlock >> (8 * (t - 4)));
      else if (t < 16) v = (uint8_t)(n >> (8 * (t - 8)));
      else if (t < 20) v = (uint8_t)(nblk >> (8 * (t - 16)));
      else if (t >= SZ3G_LZ_HEADER && t < SZ3G_LZ_HEADER + 4 * nblk)
        v = (uint8_t)(sizes[(t - SZ3G_LZ_HEADER) / 4] >> (8 * ((t - SZ3G_LZ_HEADER) % 4)));
      out[t] = v;
    }
    if (threadIdx.x == 0) st->out_bytes = data0 + off[nblk - 1] + (((sizes[nblk - 1] & ~kLzRaw) + 3) & ~3u);
  }
  const uint32_t s = sizes[b];
  const uint32_t len = s & ~kLzRaw, len4 = (len + 3) & ~3u;
  const uint8_t* src = (s & kLzRaw) ? in + b * kLzBlock : tmp + b * kLzBlock;
  uint8_t* dst = out + data0 + off[b];
  // 4-byte words while the source has them (the input's last block may end mid-word)
  const uint32_t nw = len / 4;
  for (uint32_t t = threadIdx.x; t < nw; t += blockDim.x)
    reinterpret_cast<uint32_t*>(dst)[t] = reinterpret_cast<const uint32_t*>(src)[t];
  for (uint32_t t = nw * 4 + threadIdx.x; t < len4; t += blockDim.x) dst[t] = t < len ? src[t] : 0;
}

// One 32-thread CTA per block, decoded into shared memory, then copied out.
__global__ void __launch_bounds__(32) lz_decode_kernel(const uint8_t* __restrict__ stream, unsigned long long bytes,
                                                       const uint32_t* __restrict__ sizes,
                                                       const unsigned long long* __restrict__ off,
                                                       unsigned long long data0, unsigned long long n,
                                                       uint8_t* __restrict__ out, DevState* st) {
  extern __shared__ __align__(16) uint8_t lsm[];
  const int lane = threadIdx.x;
  const unsigned long long b = blockIdx.x;
  if (st->flags & kFlagCorrupt) return;
  const uint32_t nb = (uint32_t)min((unsigned long long)kLzBlock, n - b * kLzBlock);
  const uint32_t s = sizes[b];
  const uint32_t len = s & ~kLzRaw;
  const unsigned long long at = data0 + off[b];
  uint8_t* dst = out + b * kLzBlock;
  if (at + len > bytes) {
    if (lane == 0) atomicOr(&st->flags, kFlagCorrupt);
    return;
  }
  const uint8_t* p = stream + at;
  if (s & kLzRaw) {  // (length checked equal to the block's by the lengths kernel)
    for (uint32_t t = lane; t < len; t += 32) dst[t] = p[t];
    return;
  }
  uint8_t* o8 = lsm;
  uint32_t q = 0, o = 0;
  bool bad = false;
  for (;;) {
    // token and literal count (lane 0), broadcast
    uint32_t nl = 0, ml = 0, qq = q;
    int fail = 0;
    if (lane == 0) {
      if (qq >= len) {
        fail = 1;
      } else {
        const uint32_t t = p[qq++];
        nl = t >> 4;
        ml = t & 15;
        if (nl == 15)
          for (;;) {
            if (qq >= len) {
              fail = 1;
              break;
            }
            const uint32_t x = p[qq++];
            nl += x;
            if (x != 255) break;
          }
      }
    }
    fail = __shfl_sync(0xffffffffu, fail, 0);
    nl = __shfl_sync(0xffffffffu, nl, 0);
    ml = __shfl_sync(0xffffffffu, ml, 0);
    qq = __shfl_sync(0xffffffffu, qq, 0);
    if (fail || qq + nl > len || o + nl > nb) {
      bad = true;
      break;
    }
    for (uint32_t t = lane; t < nl; t += 32) o8[o + t] = p[qq + t];
    q = qq + nl;
    o += nl;
    __syncwarp();
    if (q == len) {  // the last sequence: literals only
      bad = ml != 0;
      break;
    }
    // distance and match length (lane 0), broadcast
    uint32_t dist = 0;
    qq = q;
    if (lane == 0) {
      if (qq + 2 > len) {
        fail = 1;
      } else {
        dist = (uint32_t)p[qq] | ((uint32_t)p[qq + 1] << 8);
        qq += 2;
        ml += 4;
        if (ml == 19)
          for (;;) {
            if (qq >= len) {
              fail = 1;
              break;
            }
            const uint32_t x = p[qq++];
            ml += x;
            if (x != 255) break;
          }
      }
    }
    fail = __shfl_sync(0xffffffffu, fail, 0);
    dist = __shfl_sync(0xffffffffu, dist, 0);
    ml = __shfl_sync(0xffffffffu, ml, 0);
    qq = __shfl_sync(0xffffffffu, qq, 0);
    if (fail || dist == 0 || dist > o || ml > nb - o) {
      bad = true;
      break;
    }
    if (dist >= 32) {  // each 32-byte step reads only bytes written before it
      for (uint32_t t0 = 0; t0 < ml; t0 += 32) {
        const uint32_t t = t0 + lane;
        if (t < ml) o8[o + t] = o8[o + t - dist];
        __syncwarp();
      }
    } else {  // the dist-byte period before the match, repeated
      for (uint32_t t = lane; t < ml; t += 32) o8[o + t] = o8[o - dist + t % dist];
    }
    __syncwarp();
    q = qq;
    o += ml;
  }
  if (!bad && o != nb) bad = true;
  if (bad) {
    if (lane == 0) atomicOr(&st->flags, kFlagCorrupt);
    return;
  }
  for (uint32_t t = lane; t < nb; t += 32) dst[t] = o8[t];
}

size_t lz_workspace_bytes(unsigned long long n) {
  const unsigned long long nblk = (n + kLzBlock - 1) / kLzBlock;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return up(sizeof(DevState)) + up(scan_state_bytes(nblk)) + up(nblk * (size_t)kLzBlock) + up(nblk * 4) * 2 +
         up(nblk * 8);
}

namespace {
struct LzWs {
  DevState* st;
  unsigned char* scan;
  uint8_t* tmp;
  uint32_t *sizes, *lens;
  unsigned long long* off;
};
LzWs lz_layout(unsigned char* ws, unsigned long long nblk) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  LzWs w;
  size_t k = 0;
  w.st = (DevState*)(ws + k);
  k += up(sizeof(DevState));
  w.scan = ws + k;  // cleared with the status block
  k += up(scan_state_bytes(nblk));
  w.tmp = ws + k;
  k += up(nblk * (size_t)kLzBlock);
  w.sizes = (uint32_t*)(ws + k);
  k += up(nblk * 4);
  w.lens = (uint32_t*)(ws + k);
  k += up(nblk * 4);
  w.off = (unsigned long long*)(ws + k);
  return w;
}
}  // namespace

int launch_lz_compress(const void* d_in, unsigned long long n, void* d_out, unsigned char* ws, cudaStream_t s,
                       DevState** st_out) {
  const unsigned long long nblk = (n + kLzBlock - 1) / kLzBlock;
  const unsigned long long data0 = (SZ3G_LZ_HEADER + 4 * nblk + 7) & ~7ull;
  LzWs w = lz_layout(ws, nblk);
  *st_out = w.st;
  if (cudaMemsetAsync(ws, 0, (size_t)(w.tmp - ws), s) != cudaSuccess) return SZ3G_E_CUDA;
  if (nblk == 0) {  // the header alone
    if (cudaMemsetAsync(d_out, 0, data0, s) != cudaSuccess) return SZ3G_E_CUDA;
    if (cudaMemcpyAsync(d_out, "SZLZ", 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return SZ3G_E_CUDA;
    const uint32_t bs = kLzBlock;
    if (cudaMemcpyAsync((uint8_t*)d_out + 4, &bs, 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return SZ3G_E_CUDA;
    const unsigned long long hb = data0;
    if (cudaMemcpyAsync(&w.st->out_bytes, &hb, 8, cudaMemcpyHostToDevice, s) != cudaSuccess) return SZ3G_E_CUDA;
    return SZ3G_OK;
  }
  if (cudaFuncSetAttribute(lz_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLzSmem) !=
      cudaSuccess)
    return SZ3G_E_CUDA;
  SZ3G_LAUNCH(kKLossless, s,
              lz_block_kernel<<<(unsigned)nblk, 32, kLzSmem, s>>>((const uint8_t*)d_in, n, w.tmp, w.sizes));
  SZ3G_LAUNCH(kKLossless, s, lz_lens_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(w.sizes, nblk, n, w.lens,
                                                                                           w.st));
  const int rc = launch_scan(w.lens, nblk, w.off, 0, 0, 0, w.scan, w.st, s, true);
  if (rc) return rc;
  SZ3G_LAUNCH(kKLossless, s,
              lz_gather_kernel<<<(unsigned)nblk, 256, 0, s>>>((const uint8_t*)d_in, n, w.tmp, w.sizes, w.off, nblk,
                                                              data0, (uint8_t*)d_out, w.st));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int launch_lz_decompress(const void* d_stream, unsigned long long bytes, unsigned long long n, void* d_out,
                         unsigned char* ws, cudaStream_t s, DevState** st_out) {
  const unsigned long long nblk = (n + kLzBlock - 1) / kLzBlock;
  const unsigned long long data0 = (SZ3G_LZ_HEADER + 4 * nblk + 7) & ~7ull;
  LzWs w = lz_layout(ws, nblk);
  *st_out = w.st;
  if (cudaMemsetAsync(ws, 0, (size_t)(w.tmp - ws), s) != cudaSuccess) return SZ3G_E_CUDA;
  if (nblk == 0) return SZ3G_OK;
  const uint32_t* sizes = (const uint32_t*)((const uint8_t*)d_stream + SZ3G_LZ_HEADER);
  SZ3G_LAUNCH(kKLossless, s,
              lz_lens_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(sizes, nblk, n, w.lens, w.st));
  const int rc = launch_scan(w.lens, nblk, w.off, 0, 0, 0, w.scan, w.st, s, true);
  if (rc) return rc;
  if (cudaFuncSetAttribute(lz_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLzBlock) !=
      cudaSuccess)
    return SZ3G_E_CUDA;
  SZ3G_LAUNCH(kKLossless, s,
              lz_decode_kernel<<<(unsigned)nblk, 32, kLzBlock, s>>>((const uint8_t*)d_stream, bytes, sizes, w.off,
                                                                     data0, n, (uint8_t*)d_out, w.st));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

}  // namespace sz3g
