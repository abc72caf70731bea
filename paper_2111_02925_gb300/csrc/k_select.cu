// k_select.cu -- per-level choice of interpolation and axis order.
//
// For level l (stride s = 2^(l-1), grid G_{l-1}) and each of 8 candidates
// c = 2 o + interp (o an axis order of kOrders), every point of the level
// inside the sample blocks (or every point, with no blocks) is predicted from
// the ORIGINAL values along its pass axis -- the last axis of the order on
// which its coordinate in G_{l-1} is odd -- and quantized; the candidate's
// cost is the Shannon bits of the codes plus 8 sizeof(T) bits per
// unpredictable value.  The sampling selector takes, per level, the
// candidate of least cost (ties: the lower index); the learned selector feeds
// 16 features of the level, computed from the same sample blocks, to a small
// network (k_mlp.cu).  This estimate reads the composite / best-fit predictor
// of the paper (Sec. 3.1) and the per-level tuning of SZ3-Interp (Sec. 6.2).
//
// Sample block b of level l covers, per axis d, span_d = min(16, m_d) grid
// points starting at splitmix64(seed ^ l << 48 ^ b << 8 ^ d) mod
// (m_d - span_d + 1), SplitMix64 being the published output function; a
// point in several blocks counts once (for its first block).
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace sz3g {

constexpr int kSelCand = 8, kSelFeat = 16, kSelMaxBlocks = 1024, kSelThreads = 256;

struct SelLevel {
  int ndim;                     // rank (1..3), axes padded in front to 3
  int m[3];                     // extents of G_{l-1}
  unsigned long long st[3];     // element strides of one G_{l-1} step
  unsigned long long n[3];      // field extents
  unsigned long long s;         // stride 2^(l-1)
  int nblk;                     // 0: the whole grid as one block
  int lo[kSelMaxBlocks][3];     // (device copy) block starts
  int span[3];                  // block extents (all blocks alike)
};

// Axis k of order o (in the field's own axis numbering), orders packed one
// hex digit per axis: 3-D (0,1,2), (1,2,0), (2,0,1), (2,1,0); 2-D (0,1),
// (1,0), (0,1), (1,0); 1-D (0).
__host__ __device__ inline int sel_axis(int ndim, int o, int k) {
  if (ndim == 3) {
    const unsigned t = o == 0 ? 0x012u : (o == 1 ? 0x120u : (o == 2 ? 0x201u : 0x210u));
    return (int)((t >> (4 * (2 - k))) & 0xfu);
  }
  if (ndim == 2) {
    const unsigned t = (o & 1) ? 0x10u : 0x01u;
    return (int)((t >> (4 * (1 - k))) & 0xfu);
  }
  return 0;
}

static unsigned long long splitmix64(unsigned long long key) {
  unsigned long long z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Host: geometry and sample blocks of level l.
static void sel_level(const Plan& pl, int l, int nblocks, unsigned long long seed, SelLevel* g) {
  std::memset(g, 0, sizeof(*g));
  const int nd = pl.ndim, off = 4 - nd;
  g->ndim = nd;
  g->s = 1ull << (l - 1);
  for (int d = 0; d < nd; ++d) {
    g->n[d] = pl.n[off + d];
    g->m[d] = (int)((g->n[d] + g->s - 1) / g->s);
    g->st[d] = pl.fstride[off + d] * g->s;
    g->span[d] = g->m[d] < 16 ? g->m[d] : 16;
  }
  g->nblk = nblocks > kSelMaxBlocks ? kSelMaxBlocks : nblocks;
  if (g->nblk == 0)
    for (int d = 0; d < nd; ++d) g->span[d] = g->m[d];
  for (int b = 0; b < g->nblk; ++b)
    for (int d = 0; d < nd; ++d) {
      const unsigned long long key = seed ^ ((unsigned long long)l << 48) ^ ((unsigned long long)b << 8) ^ (unsigned long long)d;
      g->lo[b][d] = (int)(splitmix64(key) % (unsigned long long)(g->m[d] - g->span[d] + 1));
    }
}

// Grid point of item u (block, then row-major inside the block); false when
// it is past the items or already inside an earlier block.
__device__ __forceinline__ bool sel_point(const SelLevel& g, unsigned long long u, int* gc) {
  unsigned long long per = 1;
  for (int d = 0; d < g.ndim; ++d) per *= (unsigned long long)g.span[d];
  const unsigned long long nb = g.nblk ? (unsigned long long)g.nblk : 1ull;
  if (u >= per * nb) return false;
  const int b = (int)(u / per);
  unsigned long long r = u - (unsigned long long)b * per;
  for (int d = g.ndim - 1; d >= 0; --d) {
    gc[d] = (g.nblk ? g.lo[b][d] : 0) + (int)(r % (unsigned long long)g.span[d]);
    r /= (unsigned long long)g.span[d];
  }
  for (int e = 0; e < b; ++e) {
    bool in = true;
    for (int d = 0; d < g.ndim && in; ++d) in = gc[d] >= g.lo[e][d] && gc[d] < g.lo[e][d] + g.span[d];
    if (in) return false;
  }
  return true;
}

// Prediction from x along axis a (coordinate i = gc[a] s in the field).
template <typename T>
__device__ __forceinline__ T sel_pred(const SelLevel& g, const T* p, int a, int ga, int interp) {
  const unsigned long long st = g.st[a];
  const unsigned long long i = (unsigned long long)ga * g.s, n = g.n[a], s = g.s;
  const bool hb = i + s < n, hc = i >= 3 * s, hd = i + 3 * s < n;
  const T va = p[-(long long)st];
  const T vb = hb ? p[st] : T(0);
  const T vc = hc ? p[-3 * (long long)st] : T(0);
  const T vd = hd ? p[3 * st] : T(0);
  return interp_predict<T>(va, vb, vc, vd, hb, hc, hd, interp);
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads) sel_hist_kernel(const SelLevel* __restrict__ gl, const T* __restrict__ x,
                                                                const DevState* st, uint32_t radius,
                                                                uint32_t* hist /* [8][2r] */) {
  const SelLevel& g = *gl;
  const T ebT = bits_to<T>(st->ebT_bits), ebr = bits_to<T>(st->ebr_bits);
  int gc[3] = {0, 0, 0};
  const unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!sel_point(g, u, gc)) return;
  bool odd = false;
  unsigned long long idx = 0;
  for (int d = 0; d < g.ndim; ++d) {
    odd |= (gc[d] & 1) != 0;
    idx += (unsigned long long)gc[d] * g.st[d];
  }
  if (!odd) return;  // a point of a coarser level
  const T* p = x + idx;
  const T xv = *p;
  for (int c = 0; c < kSelCand; ++c) {
    int a = -1;
    for (int k = g.ndim - 1; k >= 0 && a < 0; --k) {
      const int ax = sel_axis(g.ndim, c / 2, k);
      if (gc[ax] & 1) a = ax;
    }
    T r;
    const uint32_t code = quantize_point<T>(xv, sel_pred<T>(g, p, a, gc[a], c % 2), ebT, ebr, (int)radius, r);
    atomicAdd(&hist[(size_t)c * 2 * radius + code], 1u);
  }
}

// Costs of every (level, candidate): one CTA each.
__global__ void __launch_bounds__(kSelThreads) sel_cost_kernel(const uint32_t* hist, uint32_t radius, int esz,
                                                               double* cost) {
  const uint32_t* h = hist + (size_t)blockIdx.x * 2 * radius;
  double n = 0.0, acc = 0.0;
  for (uint32_t i = threadIdx.x; i < 2 * radius; i += blockDim.x) {
    const double v = (double)h[i];
    n += v;
    if (h[i]) acc += v * log2(v);
  }
  __shared__ double sn[kSelThreads], sa[kSelThreads];
  sn[threadIdx.x] = n;
  sa[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kSelThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sa[threadIdx.x] += sa[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double N = sn[0];
    cost[blockIdx.x] = N == 0.0 ? 0.0 : N * log2(N) - sa[0] + 8.0 * (double)esz * (double)h[0];
  }
}

// Feature accumulators of one level (see sel_features_kernel).
struct SelAcc {
  double se[3][2], sr[3][2];
  unsigned long long ce[3], cr[3], n_flat, n_all, n_lvl, n_big[2];
};

template <typename T>
__global__ void __launch_bounds__(kSelThreads) sel_acc_kernel(const SelLevel* __restrict__ gl, const T* __restrict__ x,
                                                               const DevState* st, SelAcc* acc) {
  const SelLevel& g = *gl;
  const double eb = (double)bits_to<T>(st->ebT_bits);
  double se[3][2] = {{0, 0}, {0, 0}, {0, 0}}, sr[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  unsigned long long ce[3] = {0, 0, 0}, cr[3] = {0, 0, 0}, n_flat = 0, n_all = 0, n_lvl = 0, n_big[2] = {0, 0};
  int gc[3] = {0, 0, 0};
  const unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (sel_point(g, u, gc)) {
    unsigned long long idx = 0;
    bool odd = false;
    for (int d = 0; d < g.ndim; ++d) {
      idx += (unsigned long long)gc[d] * g.st[d];
      odd |= (gc[d] & 1) != 0;
    }
    const T* p = x + idx;
    const double v = (double)*p;
    bool flat_ok = true;
    double dmax = 0.0;
    for (int d = 0; d < g.ndim; ++d) {
      const unsigned long long s1 = g.st[d];
      if ((gc[d] & 1) && gc[d] + 1 < g.m[d]) {
        const double a0 = (double)p[-(long long)s1], b0 = (double)p[s1];
        const double lin = fabs(v - (a0 + b0) * 0.5);
        double cub = lin;
        if (gc[d] >= 3 && gc[d] + 3 < g.m[d]) {
          const double c0 = (double)p[-3 * (long long)s1], d0 = (double)p[3 * s1];
          cub = fabs(v - (9.0 * (a0 + b0) - (c0 + d0)) * 0.0625);
        }
        se[d][0] += lin;
        se[d][1] += cub;
        ++ce[d];
      }
      if (gc[d] + 2 < g.m[d]) {
        const double d1 = (double)p[s1] - v, d2 = (double)p[2 * s1] - v;
        sr[d][0] += d1 * d1;
        sr[d][1] += d2 * d2;
        ++cr[d];
      }
      if (gc[d] + 1 < g.m[d]) {
        const double dd = fabs((double)p[s1] - v);
        if (dd > dmax) dmax = dd;
      } else {
        flat_ok = false;
      }
    }
    if (flat_ok) {
      ++n_all;
      if (dmax <= eb) ++n_flat;
    }
    if (odd) {
      int a = -1;
      for (int k = g.ndim - 1; k >= 0 && a < 0; --k)
        if (gc[k] & 1) a = k;  // axis order (0, 1, 2)
      ++n_lvl;
      for (int it = 0; it < 2; ++it)
        if (fabs(v - (double)sel_pred<T>(g, p, a, gc[a], it)) > 64.0 * eb) ++n_big[it];
    }
  }
  // block reduction, then one atomic per accumulator and CTA
  __shared__ double sd[kSelThreads / 32][12];
  __shared__ unsigned long long su[kSelThreads / 32][11];
  double dv[12] = {se[0][0], se[0][1], se[1][0], se[1][1], se[2][0], se[2][1],
                   sr[0][0], sr[0][1], sr[1][0], sr[1][1], sr[2][0], sr[2][1]};
  unsigned long long uv[11] = {ce[0], ce[1], ce[2], cr[0], cr[1], cr[2], n_flat, n_all, n_lvl, n_big[0], n_big[1]};
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 12; ++k)
    for (int o = 16; o > 0; o >>= 1) dv[k] += __shfl_xor_sync(0xffffffffu, dv[k], o);
  for (int k = 0; k < 11; ++k)
    for (int o = 16; o > 0; o >>= 1) uv[k] += __shfl_xor_sync(0xffffffffu, uv[k], o);
  if (lane == 0) {
    for (int k = 0; k < 12; ++k) sd[w][k] = dv[k];
    for (int k = 0; k < 11; ++k) su[w][k] = uv[k];
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    double t = 0.0;
    for (int q = 0; q < kSelThreads / 32; ++q) t += sd[q][threadIdx.x];
    if (t != 0.0) atomicAdd(&(&acc->se[0][0])[threadIdx.x], t);
  } else if (threadIdx.x >= 32 && threadIdx.x < 43) {
    unsigned long long t = 0;
    for (int q = 0; q < kSelThreads / 32; ++q) t += su[q][threadIdx.x - 32];
    if (t) atomicAdd(&(&acc->ce[0])[threadIdx.x - 32], t);
  }
}

// The 16 features of every level from its accumulators.
__global__ void sel_features_kernel(const SelAcc* acc, const SelLevel* gls, int L, const DevState* st, int esz,
                                    double range, double* feat, float* feat_f) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;  // level index l - 1
  if (li >= L) return;
  const SelAcc& A = acc[li];
  const SelLevel& g = gls[li];
  const double eb = esz == 4 ? (double)__uint_as_float((uint32_t)st->ebT_bits) : __longlong_as_double((long long)st->ebT_bits);
  const double tiny = eb * eb * 1e-6;
  double f[kSelFeat];
  for (int d = 0; d < 3; ++d) {
    f[3 * d + 0] = A.ce[d] ? log2(1.0 + A.se[d][0] / (double)A.ce[d] / eb) : 0.0;
    f[3 * d + 1] = A.ce[d] ? log2(1.0 + A.se[d][1] / (double)A.ce[d] / eb) : 0.0;
    f[3 * d + 2] = A.cr[d] ? log2((A.sr[d][1] / (double)A.cr[d] + tiny) / (A.sr[d][0] / (double)A.cr[d] + tiny)) : 0.0;
  }
  f[9] = (double)(li + 1) / (double)L;
  f[10] = (double)li;
  f[11] = range > 0.0 ? log10(eb / range) : 0.0;
  f[12] = A.n_all ? (double)A.n_flat / (double)A.n_all : 0.0;
  f[13] = A.n_lvl ? (double)A.n_big[0] / (double)A.n_lvl : 0.0;
  f[14] = A.n_lvl ? (double)A.n_big[1] / (double)A.n_lvl : 0.0;
  f[15] = log2((double)g.m[g.ndim - 1] / (double)g.m[0]);
  for (int k = 0; k < kSelFeat; ++k) {
    if (feat) feat[li * kSelFeat + k] = f[k];
    if (feat_f) feat_f[li * kSelFeat + k] = (float)f[k];
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

size_t range_scratch_bytes(const Plan& pl);

struct SelScratch {
  DevState st;
  double range[2];
};

size_t select_scratch_bytes(const Plan& pl) {
  const size_t L = (size_t)pl.L;
  return 512 + range_scratch_bytes(pl) + L * sizeof(SelLevel) + L * kSelCand * 2 * pl.radius * 4 + L * sizeof(SelAcc) +
         L * kSelCand * 8 + L * kSelFeat * 8 + 4096;
}

// Bound (and, for the features, the value range) of the field, then the
// costs (h_cost: L x 8) and / or the features (d_feat_f: L x 16 floats on the
// device; h_feat: L x 16 doubles) of every level.
int launch_select(const Plan& pl, const sz3g_params* p, const void* d_x, int nblocks, unsigned long long seed,
                  unsigned char* ws, double* h_cost, double* h_feat, float* d_feat_f, cudaStream_t s) {
  const int L = pl.L;
  if (pl.ndim > 3 || L < 1) return SZ3G_E_INVAL;
  size_t off = 0;
  auto take = [&](size_t b) {
    unsigned char* q = ws + off;
    off += (b + 255) & ~(size_t)255;
    return q;
  };
  DevState* st = (DevState*)take(sizeof(DevState));
  DevState* st2 = (DevState*)take(sizeof(DevState));
  void* rsc = take(range_scratch_bytes(pl));
  SelLevel* gl = (SelLevel*)take((size_t)L * sizeof(SelLevel));
  uint32_t* hist = (uint32_t*)take((size_t)L * kSelCand * 2 * pl.radius * 4);
  SelAcc* acc = (SelAcc*)take((size_t)L * sizeof(SelAcc));
  double* cost = (double*)take((size_t)L * kSelCand * 8);
  double* feat = (double*)take((size_t)L * kSelFeat * 8);
  // one pass over the field: its value range (the REL bound of eb = 1 is
  // exactly max - min), then the bound rounded into T as the compressor does
  if (cudaMemsetAsync(st2, 0, sizeof(DevState), s) != cudaSuccess) return SZ3G_E_CUDA;
  int rc = launch_range_eb(pl, d_x, st2, rsc, range_scratch_bytes(pl), SZ3G_EB_REL, 1.0, s);
  if (rc) return rc;
  double range = 0.0;
  {
    DevState hs;
    if (cudaMemcpyAsync(&hs, st2, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SZ3G_E_CUDA;
    if (hs.flags & kFlagNonFinite) return SZ3G_E_NONFINITE;
    if (hs.flags & kFlagZeroRange) {
      if (p->eb_mode == SZ3G_EB_REL) return SZ3G_E_ZERO_RANGE_REL;
    } else {
      range = hs.eb_abs;
    }
    DevState b;
    std::memset(&b, 0, sizeof(b));
    const double e = p->eb_mode == SZ3G_EB_REL ? p->eb * range : p->eb;
    if (!(e > 0.0) || !std::isfinite(e)) return SZ3G_E_INVAL;
    if (pl.esz == 4) {
      float t = (float)e;
      if ((double)t > e) t = std::nextafter(t, 0.0f);
      if (!std::isnormal(t) || !std::isnormal(1.0f / t)) return SZ3G_E_INVAL;
      const float r = 1.0f / t;
      uint32_t tb, rb;
      std::memcpy(&tb, &t, 4);
      std::memcpy(&rb, &r, 4);
      b.ebT_bits = tb;
      b.ebr_bits = rb;
    } else {
      const double t = e, r = 1.0 / t;
      if (!std::isnormal(t) || !std::isnormal(r)) return SZ3G_E_INVAL;
      std::memcpy(&b.ebT_bits, &t, 8);
      std::memcpy(&b.ebr_bits, &r, 8);
    }
    b.eb_abs = e;
    if (cudaMemcpyAsync(st, &b, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SZ3G_E_CUDA;
  }
  std::vector<SelLevel> hg(L);
  for (int l = 1; l <= L; ++l) sel_level(pl, l, nblocks, seed, &hg[l - 1]);
  if (cudaMemcpyAsync(gl, hg.data(), (size_t)L * sizeof(SelLevel), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SZ3G_E_CUDA;
  if (h_cost) {
    if (cudaMemsetAsync(hist, 0, (size_t)L * kSelCand * 2 * pl.radius * 4, s) != cudaSuccess) return SZ3G_E_CUDA;
    for (int l = 1; l <= L; ++l) {
      const SelLevel& g = hg[l - 1];
      unsigned long long items = g.nblk ? (unsigned long long)g.nblk : 1ull;
      for (int d = 0; d < g.ndim; ++d) items *= (unsigned long long)g.span[d];
      const unsigned blocks = (unsigned)((items + kSelThreads - 1) / kSelThreads);
      if (pl.dtype == SZ3G_F32)
        SZ3G_LAUNCH(kKSelect, s,
                    sel_hist_kernel<float><<<blocks, kSelThreads, 0, s>>>(gl + (l - 1), (const float*)d_x, st,
                                                                          pl.radius,
                                                                          hist + (size_t)(l - 1) * kSelCand * 2 * pl.radius));
      else
        SZ3G_LAUNCH(kKSelect, s,
                    sel_hist_kernel<double><<<blocks, kSelThreads, 0, s>>>(gl + (l - 1), (const double*)d_x, st,
                                                                           pl.radius,
                                                                           hist + (size_t)(l - 1) * kSelCand * 2 * pl.radius));
    }
    SZ3G_LAUNCH(kKSelect, s, sel_cost_kernel<<<L * kSelCand, kSelThreads, 0, s>>>(hist, pl.radius, pl.esz, cost));
    if (cudaMemcpyAsync(h_cost, cost, (size_t)L * kSelCand * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SZ3G_E_CUDA;
  }
  if (h_feat || d_feat_f) {
    if (cudaMemsetAsync(acc, 0, (size_t)L * sizeof(SelAcc), s) != cudaSuccess) return SZ3G_E_CUDA;
    for (int l = 1; l <= L; ++l) {
      const SelLevel& g = hg[l - 1];
      unsigned long long items = g.nblk ? (unsigned long long)g.nblk : 1ull;
      for (int d = 0; d < g.ndim; ++d) items *= (unsigned long long)g.span[d];
      const unsigned blocks = (unsigned)((items + kSelThreads - 1) / kSelThreads);
      if (pl.dtype == SZ3G_F32)
        SZ3G_LAUNCH(kKSelect, s,
                    sel_acc_kernel<float><<<blocks, kSelThreads, 0, s>>>(gl + (l - 1), (const float*)d_x, st,
                                                                         acc + (l - 1)));
      else
        SZ3G_LAUNCH(kKSelect, s,
                    sel_acc_kernel<double><<<blocks, kSelThreads, 0, s>>>(gl + (l - 1), (const double*)d_x, st,
                                                                          acc + (l - 1)));
    }
    SZ3G_LAUNCH(kKSelect, s,
                sel_features_kernel<<<1, 32, 0, s>>>(acc, gl, L, st, pl.esz, range, feat, d_feat_f));
    if (h_feat && cudaMemcpyAsync(h_feat, feat, (size_t)L * kSelFeat * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SZ3G_E_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return SZ3G_E_CUDA;
  DevState hs;
  if (cudaMemcpy(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) return SZ3G_E_CUDA;
  if (hs.flags & kFlagNonFinite) return SZ3G_E_NONFINITE;
  if (hs.flags & kFlagZeroRange) return SZ3G_E_ZERO_RANGE_REL;
  if (hs.flags) return SZ3G_E_INVAL;
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

}  // namespace sz3g

namespace sz3g {
int launch_mlp_forward(const float* w, const float* feat, const uint8_t* mask, uint32_t B, float* logits,
                       cudaStream_t s);

// Candidates a rank can use: 2-D lists its two orders twice, 1-D has one.
static bool sel_valid(int ndim, int c) { return ndim == 3 || (ndim == 2 && c < 4) || (ndim == 1 && c < 2); }

namespace {
struct SelWs {
  void* p = nullptr;
  ~SelWs() {
    if (p) cudaFree(p);
  }
};

int sel_prepare(const sz3g_params* p, const void* d_x, Plan* pl, SelWs* ws, size_t extra) {
  if (!p || !d_x || ((uintptr_t)d_x % 16) != 0) return SZ3G_E_INVAL;
  int rc = make_plan(p, pl);
  if (rc) return rc;
  if (pl->ndim > 3 || pl->L < 1) return SZ3G_E_INVAL;
  if (cudaMalloc(&ws->p, select_scratch_bytes(*pl) + extra) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_NOMEM;
  }
  return SZ3G_OK;
}
}  // namespace
}  // namespace sz3g

using namespace sz3g;

extern "C" {

int sz3g_select_costs(const sz3g_params* p, const void* d_x, uint32_t nblocks, uint64_t seed, double* h_cost,
                      void* stream) {
  Plan pl;
  SelWs ws;
  if (!h_cost) return SZ3G_E_INVAL;
  int rc = sel_prepare(p, d_x, &pl, &ws, 0);
  if (rc) return rc;
  return launch_select(pl, p, d_x, (int)nblocks, seed, (unsigned char*)ws.p, h_cost, nullptr, nullptr,
                       (cudaStream_t)stream);
}

int sz3g_select_features(const sz3g_params* p, const void* d_x, uint32_t nblocks, uint64_t seed, double* h_feat,
                         void* stream) {
  Plan pl;
  SelWs ws;
  if (!h_feat) return SZ3G_E_INVAL;
  int rc = sel_prepare(p, d_x, &pl, &ws, 0);
  if (rc) return rc;
  return launch_select(pl, p, d_x, (int)nblocks, seed, (unsigned char*)ws.p, nullptr, h_feat, nullptr,
                       (cudaStream_t)stream);
}

int sz3g_select_sampled(const sz3g_params* p, const void* d_x, uint32_t nblocks, uint64_t seed, uint8_t* h_choice,
                        void* stream) {
  Plan pl;
  SelWs ws;
  if (!h_choice) return SZ3G_E_INVAL;
  int rc = sel_prepare(p, d_x, &pl, &ws, 0);
  if (rc) return rc;
  std::vector<double> cost((size_t)pl.L * kSelCand);
  rc = launch_select(pl, p, d_x, (int)nblocks, seed, (unsigned char*)ws.p, cost.data(), nullptr, nullptr,
                     (cudaStream_t)stream);
  if (rc) return rc;
  h_choice[0] = 0;
  for (int l = 1; l <= pl.L; ++l) {
    int best = 0;
    for (int c = 1; c < kSelCand; ++c)
      if (sel_valid(pl.ndim, c) && cost[(size_t)(l - 1) * kSelCand + c] < cost[(size_t)(l - 1) * kSelCand + best]) best = c;
    h_choice[l] = (uint8_t)best;
  }
  return SZ3G_OK;
}

int sz3g_select_learned(const sz3g_params* p, const void* d_x, const float* d_w, uint32_t nblocks, uint64_t seed,
                        uint8_t* h_choice, void* stream) {
  Plan pl;
  SelWs ws;
  if (!h_choice || !d_w) return SZ3G_E_INVAL;
  const size_t extra = 32 * (kSelFeat * 4 + kSelCand + kSelCand * 4) + 1024;
  int rc = sel_prepare(p, d_x, &pl, &ws, extra);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = (unsigned char*)ws.p + ((select_scratch_bytes(pl) + 255) & ~(size_t)255);
  float* feat = (float*)base;
  uint8_t* mask = base + 32 * kSelFeat * 4;
  float* logits = (float*)(base + 32 * kSelFeat * 4 + 256);
  rc = launch_select(pl, p, d_x, (int)nblocks, seed, (unsigned char*)ws.p, nullptr, nullptr, feat, s);
  if (rc) return rc;
  uint8_t hm[32 * kSelCand];
  for (int l = 0; l < pl.L; ++l)
    for (int c = 0; c < kSelCand; ++c) hm[l * kSelCand + c] = sel_valid(pl.ndim, c) ? 1 : 0;
  if (cudaMemcpyAsync(mask, hm, (size_t)pl.L * kSelCand, cudaMemcpyHostToDevice, s) != cudaSuccess) return SZ3G_E_CUDA;
  rc = launch_mlp_forward(d_w, feat, mask, (uint32_t)pl.L, logits, s);
  if (rc) return rc;
  std::vector<float> lg((size_t)pl.L * kSelCand);
  if (cudaMemcpyAsync(lg.data(), logits, lg.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SZ3G_E_CUDA;
  h_choice[0] = 0;
  for (int l = 1; l <= pl.L; ++l) {
    int best = 0;
    for (int c = 1; c < kSelCand; ++c)
      if (sel_valid(pl.ndim, c) && lg[(size_t)(l - 1) * kSelCand + c] > lg[(size_t)(l - 1) * kSelCand + best]) best = c;
    h_choice[l] = (uint8_t)best;
  }
  return SZ3G_OK;
}

}  // extern "C"
