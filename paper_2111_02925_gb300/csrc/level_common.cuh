// level_common.cuh -- shared by the level kernels: their arguments,
// asynchronous copies into shared memory (element cp.async, tensor and bulk
// copies completing on an mbarrier) and the lookup of an unpredictable
// value's position.
#pragma once

#include <cuda.h>

#include "internal.cuh"

namespace sz3g {

constexpr int kHistWin = 2048;  // shared-memory histogram window around the radius

template <typename T>
struct LevelArgs {
  const T* x;          // compress: input of the level (the field, or its decimated copy)
  unsigned long long xs[3];  // compress: element strides in x of one G_k step along axes 0..2
  const T* Rc;         // R_{k+1}
  T* Rout;             // R_k, or the field on decompress at k = 0
  uint16_t* codes;
  uint32_t* hist;
  DevState* st;
  const T* unpred;     // decompress
  unsigned long long n_unpred;
  const unsigned long long* zunit;  // zeros before each 512-code sub-block
  int radius;
  T ebT;               // decompress (compress reads the device state)
  int codes_padded;    // decompress: at least 256 readable bytes follow the codes
#ifdef SZ3G_CHECK
  unsigned long long n_codes;  // codes in the array (index checks)
  unsigned long long n_out;    // elements of Rout (index checks)
#endif
};

// Asynchronous 4- or 8-byte global -> shared copy.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- tensor copies (TMA) ----------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          (uint32_t)__cvta_generic_to_shared(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"((uint32_t)__cvta_generic_to_shared(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
constexpr int kWaitLimit = 1 << 22;  // bounded wait on a tensor copy

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of
// 16), completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes), "r"((uint32_t)__cvta_generic_to_shared(bar))
               : "memory");
}

// Position of the unpredictable value of code i among all zero codes: the
// zeros before its 512-code sub-block plus those before it inside it.
__device__ __forceinline__ unsigned long long rank_of_zero(const uint16_t* codes, unsigned long long i, uint32_t chunk,
                                                           uint32_t nsub, const unsigned long long* zunit) {
  const unsigned long long c = i / chunk;
  const unsigned long long r = i - c * chunk;
  const unsigned long long b = r >> 9;
  unsigned long long rank = zunit[c * nsub + b];
  for (unsigned long long q = c * chunk + (b << 9); q < i; ++q) rank += codes[q] == 0;
  return rank;
}

}  // namespace sz3g
