// k_interp.cu -- error bound, and the level-by-level interpolation passes
// (predict + quantize on compress, predict + recover on decompress).
//
// Generic form: one launch per pass of the schedule, one thread per point of
// the pass, reading the compact recon grid R_k of the level.  Coordinates are
// padded to 4 axes, so this form handles every rank 1..4.
#include <cstdio>
#include <type_traits>

#include "internal.cuh"

namespace sz3g {

// ---------------------------------------------------------------------------
// Error bound (REL: eb * (max - min), the range-normalised bound of the
// paper's throughput experiment, Sec. 6.2).
// ---------------------------------------------------------------------------
constexpr int kRangeThreads = 512;
constexpr int kRangeBlocks = 152 * 4;

template <typename T>
__device__ __forceinline__ bool finite_val(T v) {
  return isfinite(v);
}

__device__ __forceinline__ bool is_normal_f(float v) {
  uint32_t e = (__float_as_uint(v) >> 23) & 0xffu;
  return e != 0 && e != 0xffu;
}
__device__ __forceinline__ bool is_normal_d(double v) {
  unsigned long long e = ((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffull;
  return e != 0 && e != 0x7ffull;
}

// eb_T = the absolute bound rounded toward zero into T; ebr = fl_T(1 / eb_T).
__device__ bool bound_into(float*, double e, DevState* st) {
  float t = (float)e;  // round to nearest
  if ((double)t > e) t = __uint_as_float(__float_as_uint(t) - 1u);  // next toward 0 (t > 0)
  if (!is_normal_f(t)) return false;
  float r = 1.0f / t;
  if (!is_normal_f(r)) return false;
  st->ebT_bits = __float_as_uint(t);
  st->ebr_bits = __float_as_uint(r);
  return true;
}
__device__ bool bound_into(double*, double e, DevState* st) {
  double t = e;
  if (!is_normal_d(t)) return false;
  double r = 1.0 / t;
  if (!is_normal_d(r)) return false;
  st->ebT_bits = (unsigned long long)__double_as_longlong(t);
  st->ebr_bits = (unsigned long long)__double_as_longlong(r);
  return true;
}

// The bound from the (REL) value range or the absolute eb.
template <typename T>
__device__ void set_bound(int eb_mode, double eb, T mn, T mx, DevState* st) {
  double e = eb;
  if (eb_mode == SZ3G_EB_REL) {
    if (st->flags & kFlagNonFinite) return;
    const double range = (double)mx - (double)mn;
    if (range == 0.0) {
      atomicOr(&st->flags, kFlagZeroRange);
      return;
    }
    e = eb * range;
  }
  if (!(e > 0.0) || !isfinite(e) || !bound_into((T*)nullptr, e, st)) {
    atomicOr(&st->flags, kFlagBadBound);
    return;
  }
  st->eb_abs = e;
}

template <typename T>
__device__ __forceinline__ void block_minmax(T& mn, T& mx, T* smn, T* smx) {
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    smn[w] = mn;
    smx[w] = mx;
  }
  __syncthreads();
  if (w == 0) {
    mn = lane < kRangeThreads / 32 ? smn[lane] : smn[0];
    mx = lane < kRangeThreads / 32 ? smx[lane] : smx[0];
    for (int o = 16; o > 0; o >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
  }
}

// Where the range pass also writes the decimated copies X_k = x[::2^k, ::2^k,
// ::2^k], k = 1 .. kmax (rows of the padded 3-D view, each a whole number of
// 16-byte vectors): the inputs of the coarser levels, written from the rows
// it reads anyway.
constexpr int kRangePyr = 16;  // most levels written by the range pass
template <typename T>
struct RangeRows {
  T* X1;                      // null: flat pass, no copy
  unsigned long long a1, a2;  // extents of axes 1 and 2 (rows: a0 x a1, row length a2)
  unsigned long long rows;    // a0 * a1
  unsigned long long p0, p1;  // X_1 strides (elements) along axes 0 and 1
  int kmax;                   // X_2 .. X_kmax too (kmax <= 1: X_1 only)
  unsigned long long off[kRangePyr + 1], q0[kRangePyr + 1], q1[kRangePyr + 1];  // X_k: offset from X_1, strides
};

// Min / max / finiteness of the field with 16-byte loads (the field is 16-byte
// aligned), four in flight per thread; each block writes its partial result
// and the last block to finish reduces them and sets the bound.  With
// rows.X1 the field is walked row by row (a warp per row), and the rows with
// even coordinates on axes 0 and 1 also write their even elements to X_1.
template <typename T>
__global__ void __launch_bounds__(kRangeThreads) range_partial_kernel(const T* __restrict__ x,
                                                                       unsigned long long n, T* part,
                                                                       DevState* st, int eb_mode, double eb,
                                                                       const RangeRows<T> rows) {
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int kPer = 16 / sizeof(T);
  T mn = x[0], mx = x[0];
  bool bad = false;
  auto take = [&](T v) {
    bad |= !finite_val(v);
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  };
  auto take_v = [&](const V& v) {
    if constexpr (sizeof(T) == 4) {
      take(v.x); take(v.y); take(v.z); take(v.w);
    } else {
      take(v.x); take(v.y);
    }
  };
  const V* xv = reinterpret_cast<const V*>(x);
  if (rows.X1) {
    const unsigned long long vpr = rows.a2 / kPer;  // vectors per row
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (unsigned long long r = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         r < rows.rows; r += nw) {
      const unsigned long long i = r / rows.a1, j = r - i * rows.a1;
      const V* rp = xv + r * vpr;
      T* dp = ((i | j) & 1) ? nullptr : rows.X1 + (i >> 1) * rows.p0 + (j >> 1) * rows.p1;
      for (unsigned long long v0 = lane; v0 < vpr; v0 += 128) {
        V q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (v0 + 32 * u < vpr) q[u] = __ldcs(rp + v0 + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned long long v = v0 + 32 * u;
          if (v >= vpr) continue;
          take_v(q[u]);
          if (dp) {
            if constexpr (sizeof(T) == 4) {
              *reinterpret_cast<float2*>(dp + 2 * v) = make_float2(q[u].x, q[u].z);
            } else {
              dp[v] = q[u].x;
            }
            // X_k, k >= 2: element c = e >> k of rows with i, j multiples of
            // 2^k, for the vector's first element e = kPer v a multiple of 2^k
            for (int k = 2; k <= rows.kmax; ++k) {
              const unsigned long long mk = (1ull << k) - 1;
              const int sv = k - (sizeof(T) == 4 ? 2 : 1);  // e multiple of 2^k <=> v multiple of 2^sv
              if (((i | j) & mk) != 0 || (v & ((1ull << sv) - 1)) != 0) break;
              rows.X1[rows.off[k] + (i >> k) * rows.q0[k] + (j >> k) * rows.q1[k] + (v >> sv)] = q[u].x;
            }
          }
        }
      }
    }
  } else {
    const unsigned long long nv = n / kPer;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < nv; i += 4 * stride) {
      const V v0 = __ldcs(xv + i), v1 = __ldcs(xv + i + stride), v2 = __ldcs(xv + i + 2 * stride),
              v3 = __ldcs(xv + i + 3 * stride);
      take_v(v0); take_v(v1); take_v(v2); take_v(v3);
    }
    for (; i < nv; i += stride) take_v(__ldcs(xv + i));
    for (unsigned long long t = nv * kPer + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += stride)
      take(x[t]);
  }
  __shared__ T smn[kRangeThreads / 32], smx[kRangeThreads / 32];
  __shared__ bool s_last;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->flags, kFlagNonFinite);
  block_minmax(mn, mx, smn, smx);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = mn;
    part[2 * blockIdx.x + 1] = mx;
    __threadfence();
    s_last = atomicAdd(&st->range_ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // last block: reduce the partial results
  __threadfence();
  mn = __ldcg(part);
  mx = __ldcg(part + 1);
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    mn = fmin(mn, __ldcg(part + 2 * k));
    mx = fmax(mx, __ldcg(part + 2 * k + 1));
  }
  __syncthreads();
  block_minmax(mn, mx, smn, smx);
  if (threadIdx.x == 0) set_bound<T>(eb_mode, eb, mn, mx, st);
}

// Absolute bound only (no range needed).
template <typename T>
__global__ void eb_kernel(int eb_mode, double eb, DevState* st) {
  if (threadIdx.x == 0) set_bound<T>(eb_mode, eb, T(0), T(0), st);
}

size_t range_scratch_bytes(const Plan&) { return (size_t)kRangeBlocks * 2 * 8; }

int launch_range_eb(const Plan& pl, const void* d_in, DevState* st, void* scratch, size_t scratch_bytes,
                    int eb_mode, double eb, cudaStream_t s, void* X1, bool* wrote_pyr) {
  if (scratch_bytes < range_scratch_bytes(pl)) return SZ3G_E_CAPACITY;
  if (wrote_pyr) *wrote_pyr = false;
  int nparts = 1;
  if (eb_mode == SZ3G_EB_REL) {
    const int per = 16 / pl.esz;
    unsigned long long want = (pl.N / per + kRangeThreads * 4 - 1) / (kRangeThreads * 4);
    nparts = (int)(want < kRangeBlocks ? (want ? want : 1) : kRangeBlocks);
    // the decimated copies the levels read (X_1 .. X_{kc-1}, kc the coarse
    // group's grid) come with the pass when rows are whole vectors
    const int kmax = coarse_grid(pl) - 1;
    const bool rows_ok = X1 && pl.n[0] == 1 && pl.L >= 1 && pl.n[3] % (unsigned long long)per == 0 &&
                         kmax <= kRangePyr;
    auto fill = [&](auto& r, auto* base) {
      r.X1 = base;
      r.a1 = pl.n[2];
      r.a2 = pl.n[3];
      r.rows = pl.n[1] * pl.n[2];
      r.p1 = xk_pitch(pl, 1);
      r.p0 = r.p1 * pl.gm[1][2];
      r.kmax = kmax;
      for (int k = 2; k <= kmax; ++k) {
        r.off[k] = xpyr_offset(pl, k) / pl.esz;
        r.q1[k] = xk_pitch(pl, k);
        r.q0[k] = r.q1[k] * pl.gm[k][2];
      }
    };
    if (pl.dtype == SZ3G_F32) {
      RangeRows<float> r{};
      if (rows_ok) fill(r, (float*)X1);
      SZ3G_LAUNCH(kKRange, s,
                  range_partial_kernel<float><<<nparts, kRangeThreads, 0, s>>>((const float*)d_in, pl.N,
                                                                                (float*)scratch, st, eb_mode, eb, r));
    } else {
      RangeRows<double> r{};
      if (rows_ok) fill(r, (double*)X1);
      SZ3G_LAUNCH(kKRange, s,
                  range_partial_kernel<double><<<nparts, kRangeThreads, 0, s>>>((const double*)d_in, pl.N,
                                                                                 (double*)scratch, st, eb_mode, eb, r));
    }
    if (wrote_pyr) *wrote_pyr = rows_ok;
  } else if (pl.dtype == SZ3G_F32) {
    SZ3G_LAUNCH(kKEb, s, eb_kernel<float><<<1, 32, 0, s>>>(eb_mode, eb, st));
  } else {
    SZ3G_LAUNCH(kKEb, s, eb_kernel<double><<<1, 32, 0, s>>>(eb_mode, eb, st));
  }
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// ---------------------------------------------------------------------------
// Helpers shared by the pass kernels.
// ---------------------------------------------------------------------------
constexpr uint32_t kFatal = kFlagNonFinite | kFlagZeroRange | kFlagBadBound;
constexpr uint32_t kNoCode = 0xffffffffu;

// Warp-aggregated histogram update: lanes holding the same code add once.
__device__ __forceinline__ void warp_hist_add(uint32_t* hist, uint32_t code) {
  const unsigned peers = __match_any_sync(0xffffffffu, code);
  const int lane = threadIdx.x & 31;
  if (code != kNoCode && lane == __ffs(peers) - 1) atomicAdd(&hist[code], (uint32_t)__popc(peers));
}

// Rank of the unpredictable value at code index i: zeros before it.
// zunit[c*nsub + b]: zeros before 512-code sub-block b of chunk c.
__device__ __forceinline__ unsigned long long unpred_rank(const uint16_t* codes, unsigned long long i,
                                                          uint32_t chunk, uint32_t nsub,
                                                          const unsigned long long* zunit) {
  const unsigned long long c = i / chunk;
  const unsigned long long r = i - c * chunk;
  const unsigned long long b = r >> 9;
  unsigned long long rank = zunit[c * nsub + b];
  for (unsigned long long k = c * chunk + (b << 9); k < i; ++k) rank += codes[k] == 0;
  return rank;
}

// ---------------------------------------------------------------------------
// Anchor (point 0, prediction 0) and the lift from G_{k+1} to G_k.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void anchor_quantize_kernel(const T* x, uint16_t* codes, T* Rtop, uint32_t* hist, DevState* st,
                                       int radius) {
  if (threadIdx.x != 0 || (st->flags & kFatal)) return;
  const T ebT = bits_to<T>(st->ebT_bits), ebr = bits_to<T>(st->ebr_bits);
  T v = x[0], r;
  if (!isfinite(v)) atomicOr(&st->flags, kFlagNonFinite);
  uint32_t c = quantize_point<T>(v, T(0), ebT, ebr, radius, r);
  codes[0] = (uint16_t)c;
  Rtop[0] = r;
  atomicAdd(&hist[c], 1u);
  if (c == 0) atomicAdd(&st->n_unpred, 1ull);
}

template <typename T>
__global__ void anchor_recover_kernel(const uint16_t* codes, const T* unpred, unsigned long long n_unpred, T* Rtop,
                                      DevState* st, int radius, T ebT) {
  if (threadIdx.x != 0) return;
  uint32_t c = codes[0];
  if (c >= 2u * (uint32_t)radius) {
    atomicOr(&st->flags, kFlagCorrupt);
    Rtop[0] = T(0);
  } else if (c == 0) {
    if (n_unpred == 0) {
      atomicOr(&st->flags, kFlagCorrupt);
      Rtop[0] = T(0);
    } else {
      Rtop[0] = unpred[0];
    }
  } else {
    Rtop[0] = recover_point<T>(T(0), c, radius, ebT);
  }
}

// R_k[2c] = R_{k+1}[c] for every point c of G_{k+1}.
template <typename T>
__global__ void lift_kernel(const T* __restrict__ Rc, T* __restrict__ Rf, unsigned long long nc, uint32_t c1,
                            uint32_t c2, uint32_t c3, unsigned long long fs0, unsigned long long fs1,
                            unsigned long long fs2) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += stride) {
    unsigned long long t = i;
    const unsigned long long g3 = t % c3;
    t /= c3;
    const unsigned long long g2 = t % c2;
    t /= c2;
    const unsigned long long g1 = t % c1;
    t /= c1;
    const unsigned long long g0 = t;
    Rf[2 * (g0 * fs0 + g1 * fs1 + g2 * fs2 + g3)] = Rc[i];
  }
}

// ---------------------------------------------------------------------------
// One pass, generic form.
// ---------------------------------------------------------------------------
struct PassGeom {
  unsigned long long gi, xi;
  uint32_t i, n;
  unsigned long long st;
};

__device__ __forceinline__ PassGeom pass_point(const PassDesc& pd, unsigned long long j) {
  PassGeom g;
  unsigned long long t = j;
  unsigned long long c[4];
  c[3] = t % pd.E[3];
  t /= pd.E[3];
  c[2] = t % pd.E[2];
  t /= pd.E[2];
  c[1] = t % pd.E[1];
  t /= pd.E[1];
  c[0] = t;
  g.gi = 0;
  g.xi = 0;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const unsigned long long q = pd.start[d] + pd.step[d] * c[d];
    g.gi += q * pd.gstride[d];
    g.xi += q * pd.xstride[d];
    if (d == pd.axis) g.i = (uint32_t)q;
  }
  g.n = pd.m[pd.axis];
  g.st = pd.gstride[pd.axis];
  return g;
}

template <typename T>
__device__ __forceinline__ T pass_predict(const T* R, const PassGeom& g, int interp) {
  const bool has_b = g.i + 1 < g.n, has_c = g.i >= 3, has_d = g.i + 3 < g.n;
  const T a = R[g.gi - g.st];
  const T b = has_b ? R[g.gi + g.st] : T(0);
  const T c = has_c ? R[g.gi - 3 * g.st] : T(0);
  const T d = has_d ? R[g.gi + 3 * g.st] : T(0);
  return interp_predict<T>(a, b, c, d, has_b, has_c, has_d, interp);
}

template <typename T>
__global__ void __launch_bounds__(256) pass_quantize_kernel(const PassDesc pd, const T* __restrict__ x, T* R,
                                                            uint16_t* __restrict__ codes, uint32_t* hist,
                                                            DevState* st, int radius) {
  if (st->flags & kFatal) return;
  const T ebT = bits_to<T>(st->ebT_bits), ebr = bits_to<T>(st->ebr_bits);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  bool bad = false;
  unsigned int nz = 0;
  for (unsigned long long jb = (unsigned long long)blockIdx.x * blockDim.x; jb < pd.count; jb += stride) {
    const unsigned long long j = jb + threadIdx.x;
    uint32_t code = kNoCode;
    if (j < pd.count) {
      const PassGeom g = pass_point(pd, j);
      const T pred = pass_predict<T>(R, g, pd.interp);
      const T v = x[g.xi];
      bad |= !isfinite(v);
      T r;
      code = quantize_point<T>(v, pred, ebT, ebr, radius, r);
      codes[pd.off + j] = (uint16_t)code;
      R[g.gi] = r;
      nz += code == 0;
    }
    warp_hist_add(hist, code);
  }
  if (bad) atomicOr(&st->flags, kFlagNonFinite);
  if (nz) atomicAdd(&st->n_unpred, (unsigned long long)nz);
}

template <typename T>
__global__ void __launch_bounds__(256) pass_recover_kernel(const PassDesc pd, const uint16_t* __restrict__ codes,
                                                           const T* __restrict__ unpred,
                                                           unsigned long long n_unpred,
                                                           const unsigned long long* zunit,
                                                           uint32_t chunk, uint32_t nsub, T* R, DevState* st,
                                                           int radius, T ebT) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < pd.count; j += stride) {
    const PassGeom g = pass_point(pd, j);
    const uint32_t c = codes[pd.off + j];
    T v;
    if (c == 0) {
      const unsigned long long rk = unpred_rank(codes, pd.off + j, chunk, nsub, zunit);
      if (rk < n_unpred) {
        v = unpred[rk];
      } else {
        atomicOr(&st->flags, kFlagCorrupt);
        v = T(0);
      }
    } else if (c >= 2u * (uint32_t)radius) {
      atomicOr(&st->flags, kFlagCorrupt);
      v = T(0);
    } else {
      const T pred = pass_predict<T>(R, g, pd.interp);
      v = recover_point<T>(pred, c, radius, ebT);
    }
    R[g.gi] = v;
  }
}

static unsigned grid_for(unsigned long long n, int threads) {
  unsigned long long b = (n + threads - 1) / threads;
  const unsigned long long cap = 152ull * 16;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
static void lift(const Plan& pl, int k, const T* Rc, T* Rf, cudaStream_t s) {
  // G_{k+1} -> even points of G_k
  const unsigned long long* mc = pl.gm[k + 1];
  const unsigned long long* mf = pl.gm[k];
  const unsigned long long fs2 = mf[3], fs1 = fs2 * mf[2], fs0 = fs1 * mf[1];
  const unsigned long long nc = pl.gsize[k + 1];
  SZ3G_LAUNCH(kKLift, s, lift_kernel<T><<<grid_for(nc, 256), 256, 0, s>>>(Rc, Rf, nc, (uint32_t)mc[1], (uint32_t)mc[2], (uint32_t)mc[3], fs0,
                                                   fs1, fs2));
}

template <typename T>
static int quantize_levels_t(const Plan& pl, const T* x, uint16_t* codes, void* const* R, uint32_t* hist,
                             DevState* st, cudaStream_t s) {
  SZ3G_LAUNCH(kKAnchor, s, anchor_quantize_kernel<T><<<1, 32, 0, s>>>(x, codes, (T*)R[pl.L], hist, st, (int)pl.radius));
  int pi = 0;
  for (int l = pl.L; l >= 1; --l) {
    const int k = l - 1;
    lift<T>(pl, k, (const T*)R[k + 1], (T*)R[k], s);
    for (; pi < pl.n_pass && pl.pass[pi].grid == k; ++pi) {
      const PassDesc& pd = pl.pass[pi];
      SZ3G_LAUNCH(kKPassQuantize, s, pass_quantize_kernel<T><<<grid_for(pd.count, 256), 256, 0, s>>>(pd, x, (T*)R[k], codes, hist, st,
                                                                      (int)pl.radius));
    }
  }
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int launch_quantize_levels(const Plan& pl, const void* d_in, uint16_t* codes, void* const* R, uint32_t* hist,
                           DevState* st, void* X1, bool pyr_ready, cudaStream_t s, LevelQueue* lq, int field) {
  if (level_path_ok(pl)) return launch_quantize_fused(pl, d_in, codes, R, hist, st, X1, pyr_ready, s, lq, field);
  if (pl.dtype == SZ3G_F32) return quantize_levels_t<float>(pl, (const float*)d_in, codes, R, hist, st, s);
  return quantize_levels_t<double>(pl, (const double*)d_in, codes, R, hist, st, s);
}

template <typename T>
static int recover_levels_t(const Plan& pl, const uint16_t* codes, const T* unpred, unsigned long long n_unpred,
                            const unsigned long long* zunit, void* const* R, T* out,
                            DevState* st, T ebT, cudaStream_t s) {
  T* top = pl.L == 0 ? out : (T*)R[pl.L];
  SZ3G_LAUNCH(kKAnchor, s, anchor_recover_kernel<T><<<1, 32, 0, s>>>(codes, unpred, n_unpred, top, st, (int)pl.radius, ebT));
  int pi = 0;
  for (int l = pl.L; l >= 1; --l) {
    const int k = l - 1;
    T* Rf = k == 0 ? out : (T*)R[k];
    lift<T>(pl, k, (const T*)R[k + 1], Rf, s);
    for (; pi < pl.n_pass && pl.pass[pi].grid == k; ++pi) {
      const PassDesc& pd = pl.pass[pi];
      SZ3G_LAUNCH(kKPassRecover, s, pass_recover_kernel<T><<<grid_for(pd.count, 256), 256, 0, s>>>(pd, codes, unpred, n_unpred, zunit,
                                                                     pl.chunk, pl.nsub, Rf, st, (int)pl.radius,
                                                                     ebT));
    }
  }
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int launch_recover_levels(const Plan& pl, const uint16_t* codes, const void* unpred, unsigned long long n_unpred,
                          const unsigned long long* zunit, void* const* R, void* d_out,
                          DevState* st, unsigned long long ebT_bits, bool codes_padded, cudaStream_t s,
                          LevelQueue* lq, int field) {
  if (level_path_ok(pl))
    return launch_recover_fused(pl, codes, unpred, n_unpred, zunit, R, d_out, st, ebT_bits, codes_padded, s, lq,
                                field);
  if (pl.dtype == SZ3G_F32) {
    float e;
    uint32_t b = (uint32_t)ebT_bits;
    memcpy(&e, &b, 4);
    return recover_levels_t<float>(pl, codes, (const float*)unpred, n_unpred, zunit, R, (float*)d_out, st, e,
                                   s);
  }
  double e;
  memcpy(&e, &ebT_bits, 8);
  return recover_levels_t<double>(pl, codes, (const double*)unpred, n_unpred, zunit, R, (double*)d_out, st, e,
                                  s);
}

}  // namespace sz3g
