// SZ3-Pastri modules on the quantize / encode path.
//
// Unpred-aware quantizer (Sec. 4.2): values of T aligned to the exponent e =
// floor(log2(eb)) of the bound, q = trunc(v / 2^e) (|v - q 2^e| < 2^e <= eb),
// stored as a sign plane and B magnitude planes, most significant first
// (stream layout in include/sz3g.h).  Two kernels: a scan for B and the
// finiteness / width checks, then the planes, a tile of 1024 values (32 plane
// words) per CTA iteration -- a warp turns its 32 magnitudes into the 32
// plane words of their bits with one 32 x 32 bit-matrix transpose across the
// lanes (five exchange rounds), the words of a tile meet in shared memory and
// every plane row of the tile leaves as one coalesced 128-byte store.  The
// decoder stages a tile's plane words in shared memory and runs the same
// transpose backwards (it is its own inverse).
//
// Fixed Huffman (Sec. 3.2 Encoder, the predefined tree of SZ-Pastri): the
// lengths and canonical codewords of the predefined code over the 2r
// quantization codes, each thread placing its symbols by the closed forms of
// the distance classes (no histogram, no tree, nothing stored).
#include <cmath>

#include "internal.cuh"

namespace sz3g {

namespace {

constexpr int kBpThreads = 256;
constexpr int kBpTile = 1024;  // values per tile: 32 words of each plane
constexpr uint32_t kBpMaxB = 62;

struct BpState {
  uint32_t flags;
  uint32_t B;
  unsigned long long out_bytes;
};

// v / 2^e rounded toward zero, as its magnitude and sign; false when it is
// 2^62 or wider.  In T: scaling by a power of two is exact unless the result
// leaves T's range, and then it is either too wide (overflow) or below 1
// (underflow, truncated to 0) either way -- so float data never needs FP64.
__device__ __forceinline__ bool bp_align(float v, int e, unsigned long long* mag, bool* neg) {
  const float w = scalbnf(v, -e);
  if (!(fabsf(w) < 0x1p62f)) return false;
  const float t = truncf(w);
  *mag = (unsigned long long)fabsf(t);
  *neg = t < 0.0f;
  return true;
}
__device__ __forceinline__ bool bp_align(double v, int e, unsigned long long* mag, bool* neg) {
  const double w = scalbn(v, -e);
  if (!(fabs(w) < 0x1p62)) return false;
  const double t = trunc(w);
  *mag = (unsigned long long)fabs(t);
  *neg = t < 0.0;
  return true;
}

// 32 x 32 bit-matrix transpose across a warp: bit j of lane i's input is
// bit i of lane j's output.  Five rounds; in round s a lane swaps, with the
// lane s away, the bit columns whose index differs from its own in bit s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int sft = 16 >> r;
    const uint32_t m = masks[r];
    const uint32_t t = __shfl_xor_sync(0xffffffffu, x, sft);
    x = (lane & sft) ? ((x & ~m) | ((t & ~m) >> sft)) : ((x & m) | ((t & m) << sft));
  }
  return x;
}

constexpr int kBpRow = 33;  // shared-memory words per plane row of a tile (padded: no bank conflicts)

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_scan_kernel(const T* __restrict__ v, unsigned long long n, int e,
                                                            BpState* st) {
  uint32_t width = 0;
  bool bad = false, wide = false;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  auto take = [&](T x) {
    if (!isfinite(x)) {
      bad = true;
      return;
    }
    unsigned long long mag;
    bool neg;
    if (!bp_align(x, e, &mag, &neg)) {
      wide = true;
      return;
    }
    const uint32_t bl = mag ? 64u - (uint32_t)__clzll((long long)mag) : 0u;
    width = bl > width ? bl : width;
  };
  unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {  // four loads in flight
    const T x0 = __ldcs(v + i), x1 = __ldcs(v + i + stride), x2 = __ldcs(v + i + 2 * stride),
            x3 = __ldcs(v + i + 3 * stride);
    take(x0), take(x1), take(x2), take(x3);
  }
  for (; i < n; i += stride) take(__ldcs(v + i));
  width = __reduce_max_sync(0xffffffffu, width);
  const bool any_bad = __any_sync(0xffffffffu, bad), any_wide = __any_sync(0xffffffffu, wide);
  if ((threadIdx.x & 31) == 0) {
    if (width) atomicMax(&st->B, width);
    if (any_bad) atomicOr(&st->flags, kFlagNonFinite);
    if (any_wide) atomicOr(&st->flags, kFlagBadBound);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_encode_kernel(const T* __restrict__ v, unsigned long long n, int e,
                                                              uint32_t dtype, unsigned long long W,
                                                              unsigned long long cap, uint8_t* out, BpState* st) {
  __shared__ uint32_t sm[(kBpMaxB + 1) * kBpRow];
  if (st->flags) return;
  const uint32_t B = st->B;
  const unsigned long long total = SZ3G_BP_HEADER + 4ull * W * (1ull + B);
  if (total > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&st->flags, kFlagCapacity);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t* h = reinterpret_cast<uint32_t*>(out);
    h[0] = 0x50425a53u;  // "SZBP"
    h[1] = dtype;
    h[2] = (uint32_t)n, h[3] = (uint32_t)(n >> 32);
    h[4] = (uint32_t)e;
    h[5] = B;
    h[6] = (uint32_t)W, h[7] = (uint32_t)(W >> 32);
    st->out_bytes = total;
  }
  uint32_t* planes = reinterpret_cast<uint32_t*>(out + SZ3G_BP_HEADER);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long ntiles = (n + kBpTile - 1) / kBpTile;
  for (unsigned long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
#pragma unroll 1
    for (int k = 0; k < kBpTile / 32 / (kBpThreads / 32); ++k) {
      const int g = warp + (kBpThreads / 32) * k;
      const unsigned long long i = t * kBpTile + (unsigned long long)g * 32 + lane;
      unsigned long long mag = 0;
      bool neg = false;
      if (i < n) bp_align(v[i], e, &mag, &neg);  // in range: the scan found no wider value
      const uint32_t sw = __ballot_sync(0xffffffffu, neg);
      if (lane == 0) sm[g] = sw;
      // lane b receives the plane word of bit b (plane B - b)
      const uint32_t lo = warp_transpose32((uint32_t)mag, lane);
      if ((uint32_t)lane < B) sm[(B - lane) * kBpRow + g] = lo;
      if (B > 32) {
        const uint32_t hi = warp_transpose32((uint32_t)(mag >> 32), lane);
        if ((uint32_t)lane + 32 < B) sm[(B - 32 - lane) * kBpRow + g] = hi;
      }
    }
    __syncthreads();
    const unsigned long long w0 = t * 32;
    for (uint32_t idx = threadIdx.x; idx < (B + 1) * 32; idx += kBpThreads) {
      const uint32_t p = idx >> 5, g = idx & 31;
      if (w0 + g < W) planes[(unsigned long long)p * W + w0 + g] = sm[p * kBpRow + g];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_decode_kernel(const uint32_t* __restrict__ planes,
                                                              unsigned long long n, unsigned long long W, uint32_t B,
                                                              int e, T* __restrict__ out) {
  __shared__ uint32_t sm[(kBpMaxB + 1) * kBpRow];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long ntiles = (n + kBpTile - 1) / kBpTile;
  for (unsigned long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const unsigned long long w0 = t * 32;
    for (uint32_t idx = threadIdx.x; idx < (B + 1) * 32; idx += kBpThreads) {
      const uint32_t p = idx >> 5, g = idx & 31;
      sm[p * kBpRow + g] = w0 + g < W ? planes[(unsigned long long)p * W + w0 + g] : 0u;
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < kBpTile / 32 / (kBpThreads / 32); ++k) {
      const int g = warp + (kBpThreads / 32) * k;
      const unsigned long long i = t * kBpTile + (unsigned long long)g * 32 + lane;
      // lane b holds the plane word of bit b; the transpose gives lane i its bits
      const uint32_t wlo = (uint32_t)lane < B ? sm[(B - lane) * kBpRow + g] : 0u;
      unsigned long long mag = warp_transpose32(wlo, lane);
      if (B > 32) {
        const uint32_t whi = (uint32_t)lane + 32 < B ? sm[(B - 32 - lane) * kBpRow + g] : 0u;
        mag |= (unsigned long long)warp_transpose32(whi, lane) << 32;
      }
      T r;
      if (sizeof(T) == 4 && B <= 24) {  // |q| < 2^24: exact in float, one rounding at most (underflow)
        r = (T)scalbnf((float)mag, e);
      } else {
        r = (T)scalbn((double)mag, e);
      }
      if ((sm[g] >> lane) & 1u) r = -r;  // the sign plane is row 0
      if (i < n) out[i] = r;
    }
    __syncthreads();
  }
}

__global__ void fixed_table_kernel(uint32_t r, uint8_t* __restrict__ len, uint32_t* __restrict__ code) {
  __shared__ uint32_t first[SZ3G_LMAX + 1];
  if (threadIdx.x == 0) {
    uint32_t cnt[SZ3G_LMAX + 1];
    for (int l = 0; l <= SZ3G_LMAX; ++l) cnt[l] = 0;
    cnt[1] = 1;             // code r
    cnt[SZ3G_LMAX] += 1;    // code 0
    for (uint32_t c = 1; c <= 16; ++c) {
      const uint32_t kmin = 1u << (c - 1), kmax = min((1u << c) - 1u, r - 1u);
      if (kmax < kmin) break;
      cnt[c >= 11 ? SZ3G_LMAX : 2 * c + 2] += 2 * (kmax - kmin + 1);
    }
    uint32_t f = 0;
    first[0] = 0;
    for (int l = 1; l <= SZ3G_LMAX; ++l) {
      f = (f + cnt[l - 1]) << 1;
      first[l] = f;
    }
  }
  __syncthreads();
  const uint32_t nlow = r > 1024u ? r - 1024u : 0u;  // codes 1 .. r - 1024: distance >= 1024
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < 2 * r; s += gridDim.x * blockDim.x) {
    uint32_t l, rank;
    const uint32_t k = s > r ? s - r : r - s;
    if (s == 0) {
      l = SZ3G_LMAX, rank = 0;
    } else if (k == 0) {
      l = 1, rank = 0;
    } else {
      const uint32_t c = 32u - (uint32_t)__clz((int)k);
      if (c <= 10) {
        const uint32_t kmin = 1u << (c - 1), kmax = min((1u << c) - 1u, r - 1u);
        l = 2 * c + 2;
        rank = s < r ? s - (r - kmax) : (kmax - kmin + 1) + (s - (r + kmin));
      } else {
        l = SZ3G_LMAX;
        rank = s < r ? s : 1 + nlow + (s - (r + 1024u));
      }
    }
    len[s] = (uint8_t)l;
    code[s] = first[l] + rank;
  }
}

int bp_grid(unsigned long long n, int per_sm) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned long long tiles = (n + kBpTile - 1) / kBpTile;
  const unsigned long long cap = (unsigned long long)nsm * per_sm;
  return (int)(tiles < cap ? (tiles ? tiles : 1) : cap);
}

}  // namespace

int bitplane_exponent(double eb, int* e) {
  if (!(eb > 0) || !std::isfinite(eb)) return SZ3G_E_INVAL;
  int ex = 0;
  (void)std::frexp(eb, &ex);  // eb = m 2^ex, m in [0.5, 1)
  *e = ex - 1;
  return SZ3G_OK;
}

size_t bp_state_bytes() { return 256; }

int launch_bitplane_encode(uint32_t dtype, const void* d_values, unsigned long long n, int e, void* d_out,
                           unsigned long long cap, void* d_state, cudaStream_t s) {
  BpState* st = (BpState*)d_state;
  if (cudaMemsetAsync(st, 0, sizeof(BpState), s) != cudaSuccess) return SZ3G_E_CUDA;
  const unsigned long long W = (n + 31) / 32;
  const int g1 = bp_grid(n, 8), g2 = bp_grid(n, 8);
  if (dtype == SZ3G_F32) {
    if (n)
      SZ3G_LAUNCH(kKBitplane, s, bp_scan_kernel<float><<<g1, kBpThreads, 0, s>>>((const float*)d_values, n, e, st));
    SZ3G_LAUNCH(kKBitplane, s,
                bp_encode_kernel<float><<<g2, kBpThreads, 0, s>>>((const float*)d_values, n, e, dtype, W, cap,
                                                                   (uint8_t*)d_out, st));
  } else {
    if (n)
      SZ3G_LAUNCH(kKBitplane, s, bp_scan_kernel<double><<<g1, kBpThreads, 0, s>>>((const double*)d_values, n, e, st));
    SZ3G_LAUNCH(kKBitplane, s,
                bp_encode_kernel<double><<<g2, kBpThreads, 0, s>>>((const double*)d_values, n, e, dtype, W, cap,
                                                                    (uint8_t*)d_out, st));
  }
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int read_bitplane_state(const void* d_state, uint32_t* flags, unsigned long long* out_bytes, cudaStream_t s) {
  BpState h;
  if (cudaMemcpyAsync(&h, d_state, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SZ3G_E_CUDA;
  *flags = h.flags;
  *out_bytes = h.out_bytes;
  return SZ3G_OK;
}

int launch_bitplane_decode(uint32_t dtype, const void* d_stream, unsigned long long n, unsigned long long W,
                           uint32_t B, int e, void* d_out, cudaStream_t s) {
  if (!n) return SZ3G_OK;
  const uint32_t* planes = (const uint32_t*)((const uint8_t*)d_stream + SZ3G_BP_HEADER);
  const int g = bp_grid(n, 8);
  if (dtype == SZ3G_F32)
    SZ3G_LAUNCH(kKBitplane, s, bp_decode_kernel<float><<<g, kBpThreads, 0, s>>>(planes, n, W, B, e, (float*)d_out));
  else
    SZ3G_LAUNCH(kKBitplane, s, bp_decode_kernel<double><<<g, kBpThreads, 0, s>>>(planes, n, W, B, e, (double*)d_out));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int launch_huffman_fixed(uint32_t radius, uint8_t* d_len, uint32_t* d_code, cudaStream_t s) {
  SZ3G_LAUNCH(kKFixedTable, s, fixed_table_kernel<<<1, 1024, 0, s>>>(radius, d_len, d_code));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

}  // namespace sz3g
