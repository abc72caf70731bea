// SZ3-Pastri modules on the quantize / encode path.
//
// Unpred-aware quantizer (Sec. 4.2): values of T aligned to the exponent e =
// floor(log2(eb)) of the bound, q = trunc(v / 2^e) (|v - q 2^e| < 2^e <= eb),
// stored as a sign plane and B magnitude planes, most significant first
// (stream layout in include/sz3g.h).  Two kernels: a scan for B and the
// finiteness / width checks, then the planes, a tile of 1024 values (32 plane
// words) per CTA iteration -- each warp turns 32 values into one word of a
// plane with a ballot, the words of a tile meet in shared memory and every
// plane row of the tile leaves as one coalesced 128-byte store.  The decoder
// stages a tile's plane words in shared memory and rebuilds each value from
// its bit of every plane word (a broadcast read per plane).
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

// v / 2^e rounded toward zero (in double; exact while it fits 62 bits)
template <typename T>
__device__ __forceinline__ double bp_aligned(T v, int e) {
  return trunc(scalbn((double)v, -e));
}

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_scan_kernel(const T* __restrict__ v, unsigned long long n, int e,
                                                            BpState* st) {
  uint32_t width = 0;
  bool bad = false, wide = false;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double x = (double)v[i];
    if (!isfinite(x)) {
      bad = true;
      continue;
    }
    const double w = scalbn(x, -e);
    if (!(fabs(w) < 0x1p62)) {
      wide = true;
      continue;
    }
    const unsigned long long mag = (unsigned long long)fabs(trunc(w));
    const uint32_t bl = mag ? 64u - (uint32_t)__clzll((long long)mag) : 0u;
    width = bl > width ? bl : width;
  }
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
  __shared__ uint32_t sm[(kBpMaxB + 1) * 32];
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
      const double q = i < n ? bp_aligned(v[i], e) : 0.0;
      const unsigned long long mag = (unsigned long long)fabs(q);
      const uint32_t sw = __ballot_sync(0xffffffffu, q < 0.0);
      if (lane == 0) sm[g] = sw;
      for (uint32_t b = 0; b < B; ++b) {
        const uint32_t wd = __ballot_sync(0xffffffffu, (mag >> b) & 1ull);
        const uint32_t p = 1 + (B - 1 - b);
        if (lane == (int)(p & 31)) sm[p * 32 + g] = wd;
      }
    }
    __syncthreads();
    const unsigned long long w0 = t * 32;
    for (uint32_t idx = threadIdx.x; idx < (B + 1) * 32; idx += kBpThreads) {
      const uint32_t p = idx >> 5, g = idx & 31;
      if (w0 + g < W) planes[(unsigned long long)p * W + w0 + g] = sm[idx];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kBpThreads) bp_decode_kernel(const uint32_t* __restrict__ planes,
                                                              unsigned long long n, unsigned long long W, uint32_t B,
                                                              int e, T* __restrict__ out) {
  __shared__ uint32_t sm[(kBpMaxB + 1) * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long ntiles = (n + kBpTile - 1) / kBpTile;
  for (unsigned long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const unsigned long long w0 = t * 32;
    for (uint32_t idx = threadIdx.x; idx < (B + 1) * 32; idx += kBpThreads) {
      const uint32_t p = idx >> 5, g = idx & 31;
      sm[idx] = w0 + g < W ? planes[(unsigned long long)p * W + w0 + g] : 0u;
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < kBpTile / 32 / (kBpThreads / 32); ++k) {
      const int g = warp + (kBpThreads / 32) * k;
      const unsigned long long i = t * kBpTile + (unsigned long long)g * 32 + lane;
      unsigned long long mag = 0;
      for (uint32_t b = 0; b < B; ++b) {
        const uint32_t p = 1 + (B - 1 - b);
        mag |= (unsigned long long)((sm[p * 32 + g] >> lane) & 1u) << b;
      }
      double r = scalbn((double)mag, e);
      if ((sm[g] >> lane) & 1u) r = -r;
      if (i < n) out[i] = (T)r;
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
    if (n) SZ3G_LAUNCH(kKBitplane, s, bp_scan_kernel<float><<<g1, kBpThreads, 0, s>>>((const float*)d_values, n, e, st));
    SZ3G_LAUNCH(kKBitplane, s,
                bp_encode_kernel<float><<<g2, kBpThreads, 0, s>>>((const float*)d_values, n, e, dtype, W, cap,
                                                                   (uint8_t*)d_out, st));
  } else {
    if (n) SZ3G_LAUNCH(kKBitplane, s, bp_scan_kernel<double><<<g1, kBpThreads, 0, s>>>((const double*)d_values, n, e, st));
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
