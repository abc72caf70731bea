// static_ws.cu -- the chunked Huffman decoder with its scratch in a fixed
// device array, for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc (or any allocating routine) from the
// code that decodes: a host whose device memory is owned entirely by another
// allocator (a framework pool that has reserved all of it), or a
// latency-sensitive path where an allocation may block on the device or fail
// part-way through a run.  sz3g_huffman_decode_static serves them: it takes
// the same arguments as sz3g_huffman_decode, but its scratch lives in the
// file-scope array below, so the call allocates nothing.
//
// The array is part of the library image: every GPU that loads the library
// holds kStaticScratchBytes of it until the process exits.  All calls share
// it, so two calls whose GPU work overlaps (on different streams, or from
// different host threads) race on it; run them one after another.
#include <mutex>

#include "internal.cuh"

namespace sz3g {

size_t dec_tables_bytes();
size_t decode_state_bytes(unsigned long long n_chunks, uint32_t chunk);
int launch_decode_tables(const unsigned char* tab, uint32_t n_used, const uint8_t* len, uint32_t nsym, void* tables,
                         DevState* st, cudaStream_t s);
int launch_decode_chunks(const uint32_t* words, unsigned long long n_words, const uint32_t* chunk_words,
                         const uint16_t* sub_bits, unsigned long long n_chunks, uint32_t chunk, unsigned long long n,
                         const void* tables, uint16_t* codes, uint32_t* zcnt, void* state, DevState* st,
                         cudaStream_t s, bool state_zeroed = false);

constexpr size_t kStaticScratchBytes = 4u << 20;  // 4 MiB

// The scratch.  In host code this name is only a host-side handle, not a
// device address: the address a kernel may use comes from
// cudaGetSymbolAddress, taken once per device below.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up on the first
// call on each device, with that device current).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return SZ3G_E_INVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SZ3G_E_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SZ3G_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

}  // namespace sz3g

using namespace sz3g;

extern "C" int sz3g_huffman_decode_static(const uint32_t* d_words, uint64_t n_words, const uint32_t* d_chunk_words,
                                          const uint16_t* d_sub_bits, uint32_t chunk, const uint8_t* d_len,
                                          uint32_t nsym, uint16_t* d_codes, uint64_t n, void* stream) {
  if (!d_words || !d_chunk_words || !d_len || !d_codes || n < 1 || nsym < 1 || nsym > (uint32_t)kSyms || chunk < 8 ||
      chunk > 65536 || chunk % 8 || ((uintptr_t)d_codes % 16) != 0)
    return SZ3G_E_INVAL;
  const unsigned long long nch = (n + chunk - 1) / chunk;
  // no stream with more chunks than 4-byte counts fit in the array can fit;
  // refusing it here also keeps the size sums below from wrapping
  if (nch > kStaticScratchBytes / 4) return SZ3G_E_CAPACITY;
  const unsigned long long nsb = (chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  // layout inside the fixed array; a stream too long for it is refused
  const size_t o_st = 0;
  const size_t o_tab = o_st + up256(sizeof(DevState));
  const size_t o_zc = o_tab + up256(dec_tables_bytes());
  const size_t o_scan = o_zc + up256(nch * nsb * 4);
  const size_t need = o_scan + up256(decode_state_bytes(nch, chunk));
  if (need > kStaticScratchBytes) return SZ3G_E_CAPACITY;
  void* base = nullptr;
  const int rc0 = scratch_address(&base);
  if (rc0 != SZ3G_OK) return rc0;
  unsigned char* ws = (unsigned char*)base;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = (DevState*)(ws + o_st);
  // the status block starts at zero on every call (earlier calls left theirs)
  if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_CUDA;
  }
  int rc = launch_decode_tables(nullptr, 0, d_len, nsym, ws + o_tab, st, s);
  if (rc == SZ3G_OK)
    rc = launch_decode_chunks(d_words, n_words, d_chunk_words, d_sub_bits, nch, chunk, n, ws + o_tab, d_codes,
                              (uint32_t*)(ws + o_zc), ws + o_scan, st, s);
  if (rc != SZ3G_OK) {
    // work already queued may still use the array: let it finish before the
    // caller can start another call
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return rc;
  }
  DevState h;
  if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_CUDA;
  }
  // the same flag-to-status mapping as sz3g_huffman_decode
  return stream_status(h.flags);
}
