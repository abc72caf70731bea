// k_fine.cu -- register-blocked level kernel for grids refined in axis order
// (0, 1, 2) (3-D) or (1, 2) (2-D: axis 0 is a unit axis).
//
// One launch per grid G_k.  The level's passes (Sec. 6.2, multilevel
// interpolation: refine axis 0, then 1, then 2 at the finest stride of G_k)
// split the points of G_k by the parity of their coordinates: pass 0 takes
// (odd i, even j, even k), pass 1 (any i, odd j, even k), pass 2 (any i, any j,
// odd k).  Passes 0 and 1 read and write only even-k points, so a tile keeps
// the even-k points of its rows in a separate shared-memory plane E (the
// coarse points R_{k+1} copied in, then the pass-0 and pass-1 results); pass 2
// then reads, for a run of four odd points along k, the seven even values
// around them with two 16-byte loads.
//
// Tile: T0 x T1 x 64 points (i, j, k); 4 x 16 x 64 in 3-D, 1 x 64 x 64 in 2-D.
// Staged per tile on one mbarrier per buffer (kStages buffers):
//   x box   (compress) input rows i in [A0, A0+T0), j in [A1-2, A1+T1+3),
//           k in [A2-4, A2+68)                      -- tensor copy
//   C box   R_{k+1} points (i/2, j/2, k/2) around the tile    -- tensor copy
//   codes   (recover) every row of codes the tile's passes read -- one
//           tensor copy per pass when each pass's codes form 16-byte
//           aligned rows (the pass's lattice as a 3-D array of 2-byte codes),
//           else one bulk copy per row (or 16-byte cp.async pieces)
// With two stages the next tile's copies are issued before the current tile
// is computed; with one (the configuration in use) they are issued when the
// tile starts and other CTAs of the SM cover the wait.
// Halo points (pass-0/1 points just outside the tile that pass 1/2 read) are
// evaluated redundantly and never written; points outside the grid are
// skipped.  Tiles on a face of the grid take the one-sided predictors through
// per-row (passes 0, 1) and per-point (pass 2) boundary flags.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <functional>
#include <type_traits>

#include "internal.cuh"
#include "level_common.cuh"

namespace sz3g {

// Threads per CTA, CTAs per SM and staging depth (1: the copies of a tile are
// issued when the tile starts; 2: the next tile's copies are issued while the
// current tile is computed).  Measured on 512^3: many small single-stage CTAs
// (other CTAs of the SM compute while one waits for its copies) beat fewer,
// double-buffered ones -- compress 0.62 vs 0.73 ms, recover 0.48 vs 0.53 ms.
// Recover stages the tile's code rows with 16-byte cp.async pieces spread
// over the threads (true) or one bulk copy per row (false).
constexpr bool kCodeCpAsync = false;
// Code rows by one bulk copy per row, each row's thread announcing its own
// bytes with an arrival on the tile's mbarrier (which then expects one
// arrival per staged row): no byte count through shared memory and no extra
// barrier (true); or the two forms above (false).
constexpr bool kCodeRowArrive = true;
// Pass 2 moves the four codes of a run as one 8-, two 4- or four 2-byte
// accesses by the alignment of the run's first code (true), or one 2-byte
// access per code (false).
constexpr bool kPackCodes = true;
// Histogram update without a branch: every code adds to the shared window
// (codes outside it to a spare slot that is never flushed) and, when outside,
// also to the global histogram (true); or window-or-global by a branch (false).
constexpr bool kHistSpare = true;

// Recover runs levels of many tiles with 128 threads per CTA (more CTAs per
// SM cover the staging waits) and levels of at most kWideTiles tiles per SM,
// where a tile's own latency is the time, with 256 (WIDE).
template <bool COMP, bool WIDE = false>
struct FineThreads {
  static constexpr int kN = (COMP || WIDE) ? 256 : 128, kMinBlocks = (COMP || WIDE) ? 4 : 8, kStages = 1;
};
constexpr int kWideTiles = 4;

template <int T0>
struct FineShape {
  static constexpr bool kHas0 = T0 > 1;                   // axis 0 refined
  static constexpr int kT0 = T0, kT1 = T0 > 1 ? 16 : 64, kW = 64;
  static constexpr int kXJ = kT1 + 5;                     // x box / E rows: j = A1 - 2 + j21
  static constexpr int kXK = kW + 8;                      // x box columns: k = A2 - 4 + c
  static constexpr int kEK = kXK / 2;                     // even-k values per row: k = A2 - 4 + 2 ke
  static constexpr int kPairs = kEK / 2;                  // tasks of two even-k points per row
  static constexpr int kCI = T0 > 1 ? 5 : 1;              // coarse box: i/2 = A0/2 - 1 + ci (3-D)
  static constexpr int kCJ = kT1 / 2 + 3;                 //             j/2 = A1/2 - 1 + cj
  static constexpr int kCK = 40;                          //             k/2 = A2/2 - 4 + ck
  static constexpr int kEvenI = T0 > 1 ? 2 : 1;           // tile rows along i that are even
  static constexpr int kCopyTasks = kEvenI * kCJ * kPairs;
  static constexpr int kP0Tasks = T0 > 1 ? 2 * kCJ * kPairs : 0;
  static constexpr int kP1Tasks = kT0 * (kT1 / 2) * kPairs;
  static constexpr int kP2Tasks = kT0 * kT1 * (kW / 8);   // runs of four odd points
  // code rows (recover): pass 2 rows of 32 codes, pass 1 / pass 0 rows of 36
  static constexpr int kR2 = kT0 * kT1, kR1 = kT0 * (kT1 / 2), kR0 = T0 > 1 ? 2 * kCJ : 0;
  static constexpr int kL2 = 40, kL01 = 48;               // u16 slots per staged row (80 / 96 bytes)
  static constexpr int kCodeSlots = kR2 * kL2 + (kR1 + kR0) * kL01;
};

// Shared-memory layout: tensor-copy destinations on 128-byte boundaries,
// buffers padded so that the second buffer stays aligned.
template <typename T, bool COMP, int T0>
struct FineLayout {
  using S = FineShape<T0>;
  static constexpr int kSt = FineThreads<COMP>::kStages;
  static constexpr size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }
  static constexpr int kXB = COMP ? (int)(up(S::kT0 * S::kXJ * S::kXK * sizeof(T), 128) / sizeof(T)) : 0;
  static constexpr int kCB = (int)(up(S::kCI * S::kCJ * S::kCK * sizeof(T), 128) / sizeof(T));
  static constexpr int kKB = COMP ? 0 : (int)up(S::kCodeSlots, 64);
  static constexpr size_t kOffX = 0;
  static constexpr size_t kOffC = kOffX + kSt * (size_t)kXB * sizeof(T);
  static constexpr size_t kOffE = kOffC + kSt * (size_t)kCB * sizeof(T);
  static constexpr size_t kOffK = up(kOffE + (size_t)S::kT0 * S::kXJ * S::kEK * sizeof(T), 128);
  static constexpr size_t kOffH = kOffK + kSt * (size_t)kKB * 2;
  static constexpr size_t kOffBar = up(kOffH + (COMP ? (kHistWin + 1) * 4 : 0), 16);
  static constexpr size_t kBytes = kOffBar + 16;
};

struct FineDesc {
  int m0, m1, m2;              // extents of G_k (m0 = 1 in 2-D)
  int nt1, nt2;                // tiles along j, k
  uint32_t tile0, ntiles;       // tiles [tile0, ntiles) of this launch
  uint32_t off[3];             // first code of passes 0, 1, 2 (pass 0 unused in 2-D)
  uint32_t E1[3], E2[3];       // lattice extents of each pass along j and k
  uint32_t rs0, rs1;           // output row strides (elements) along i, j; contiguous along k
  uint32_t chunk, nsub;
  int write_out;
  uint32_t tensor_bytes;       // bytes of the x and coarse boxes of one tile
  int code_tma;                // recover: code rows by one tensor copy per pass
  int code_al;                 // bit p: pass p's code pairs (p < 2) or runs of four (p = 2) are
                               // 4- or 8-byte aligned, in global and in the staged rows
};

// ---- vector helpers -----------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* v) {  // 4 consecutive, 16-byte aligned
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else {
    const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
  }
}
template <typename T>
__device__ __forceinline__ void ld2(const T* p, T* v) {  // 2 consecutive, 2 * sizeof(T)-aligned
  if constexpr (sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x, v[1] = q.y;
  } else {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x, v[1] = q.y;
  }
}
template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
  if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
  else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
template <typename T>
__device__ __forceinline__ void st4(T* p, T a, T b, T c, T d) {  // 16-byte aligned
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
  }
}

// Four consecutive codes as one 8-, two 4- or four 2-byte accesses, by the
// alignment of the first.
__device__ __forceinline__ void put_codes4(uint16_t* p, const uint32_t* c) {
  const uint32_t lo = c[0] | (c[1] << 16), hi = c[2] | (c[3] << 16);
  const uintptr_t ad = reinterpret_cast<uintptr_t>(p);
  if ((ad & 7) == 0) {
    *reinterpret_cast<uint2*>(p) = make_uint2(lo, hi);
  } else if ((ad & 3) == 0) {
    reinterpret_cast<uint32_t*>(p)[0] = lo;
    reinterpret_cast<uint32_t*>(p)[1] = hi;
  } else {
    p[0] = (uint16_t)c[0], p[1] = (uint16_t)c[1], p[2] = (uint16_t)c[2], p[3] = (uint16_t)c[3];
  }
}
__device__ __forceinline__ void get_codes4(const uint16_t* p, uint32_t* c) {
  const uintptr_t ad = reinterpret_cast<uintptr_t>(p);
  if ((ad & 7) == 0) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    c[0] = v.x & 0xffffu, c[1] = v.x >> 16, c[2] = v.y & 0xffffu, c[3] = v.y >> 16;
  } else if ((ad & 3) == 0) {
    const uint32_t v0 = reinterpret_cast<const uint32_t*>(p)[0], v1 = reinterpret_cast<const uint32_t*>(p)[1];
    c[0] = v0 & 0xffffu, c[1] = v0 >> 16, c[2] = v1 & 0xffffu, c[3] = v1 >> 16;
  } else {
    c[0] = p[0], c[1] = p[1], c[2] = p[2], c[3] = p[3];
  }
}

// Task t of a sweep over nrows rows of kPairs = 18 pairs: the first 16 pairs
// of every row, then the last two of every row, so that the 16 lanes of a
// half-warp take 16 pairs of one row (8-byte shared accesses without bank
// conflicts) instead of straddling two rows.
__device__ __forceinline__ void pair_task(int t, int nrows, int& row, int& pr) {
  const int n16 = nrows * 16;
  if (t < n16) {
    row = t >> 4;
    pr = t & 15;
  } else {
    const int u = t - n16;
    row = u >> 1;
    pr = 16 + (u & 1);
  }
}

// Per-thread results of the tile passes, flushed once per CTA.
struct FineAcc {
  bool bad;  // recover: a code outside [0, 2r) or an unpredictable value past the list
};

// Quantize (compress) or recover (decompress) one point whose prediction is
// p; returns its reconstruction.  `code_in` is the stored code (recover).
template <typename T, bool COMP>
__device__ __forceinline__ T fine_point(const LevelArgs<T>& a, const FineDesc& d, uint32_t* hwin, int hlo, T x, T p,
                                        T ebT, T ebr, bool own, uint32_t ci, uint32_t code_in, FineAcc& acc,
                                        uint32_t* code_out = nullptr) {
  if (COMP) {
    T r;
    const uint32_t code = quantize_point<T>(x, p, ebT, ebr, a.radius, r);
    if (own) {
      // (unpredictable values -- also every non-finite input -- are counted by
      // histogram bin 0 and checked for finiteness where the encoder gathers
      // them)
      if (code_out) *code_out = code;
      else if (SZ3G_IN(ci < a.n_codes, a.st)) a.codes[ci] = (uint16_t)code;
      const uint32_t bn = code - (uint32_t)hlo;
      if (kHistSpare) {
        const bool far = bn >= (uint32_t)kHistWin;
        atomicAdd(&hwin[far ? (uint32_t)kHistWin : bn], 1u);
        if (far) atomicAdd(&a.hist[code], 1u);
      } else {
        if (bn < (uint32_t)kHistWin) atomicAdd(&hwin[bn], 1u);
        else atomicAdd(&a.hist[code], 1u);
      }
    }
    return r;
  } else {
    if (code_in == 0) {
      const unsigned long long rk = rank_of_zero(a.codes, ci, d.chunk, d.nsub, a.zunit);
      if (rk < a.n_unpred) return a.unpred[rk];
      acc.bad = true;
      return T(0);
    }
    if (code_in >= 2u * (uint32_t)a.radius) {
      acc.bad = true;
      return T(0);
    }
    return recover_point<T>(p, code_in, a.radius, ebT);
  }
}

// N points of one task with every point inside the grid: compress quantizes
// them and counts the owned ones (codes away from the shared window reach the
// global histogram on a path taken once per task); recover reconstructs them,
// sending codes 0 (unpredictable) and codes past the alphabet through
// fine_point on a path taken once per task.  cq receives the codes (compress).
template <typename T, bool COMP, int N>
__device__ __forceinline__ void fine_points(const LevelArgs<T>& a, const FineDesc& d, uint32_t* hwin, int hlo,
                                            const T* x, const T* p, T ebT, T ebr, const bool* own, uint32_t ci0,
                                            const uint32_t* kin, FineAcc& acc, T* r, uint32_t* cq) {
  if (COMP) {
    bool anyfar = false;
#pragma unroll
    for (int u = 0; u < N; ++u) cq[u] = quantize_point<T>(x[u], p[u], ebT, ebr, a.radius, r[u]);
#pragma unroll
    for (int u = 0; u < N; ++u) {
      const uint32_t bn = cq[u] - (uint32_t)hlo;
      const bool far = bn >= (uint32_t)kHistWin;
      if (own[u]) atomicAdd(&hwin[far ? (uint32_t)kHistWin : bn], 1u);
      anyfar |= far && own[u];
    }
    if (anyfar)
      for (int u = 0; u < N; ++u)
        if (own[u] && cq[u] - (uint32_t)hlo >= (uint32_t)kHistWin) atomicAdd(&a.hist[cq[u]], 1u);
  } else {
    const uint32_t lim = 2u * (uint32_t)a.radius - 1u;
    bool rare = false;
#pragma unroll
    for (int u = 0; u < N; ++u) rare |= (kin[u] - 1u) >= lim;
    if (!rare) {
#pragma unroll
      for (int u = 0; u < N; ++u) r[u] = recover_point<T>(p[u], kin[u], a.radius, ebT);
    } else {
      for (int u = 0; u < N; ++u)
        r[u] = fine_point<T, false>(a, d, hwin, hlo, T(0), p[u], ebT, ebr, true, ci0 + u, kin[u], acc);
    }
  }
}

// First code of a staged row and where its aligned 16-byte copy starts
// (codes before the array start, only at rows whose leading points lie
// outside the grid, are never read).
__device__ __forceinline__ void code_row(long long c0, long long* a16, int* o) {
  long long al = c0 >= 0 ? (c0 & ~7ll) : 0;
  *a16 = al;
  *o = (int)(c0 - al);
}

template <typename T, bool COMP, int INTERP, int T0, bool WIDE>
__global__ void __launch_bounds__(FineThreads<COMP, WIDE>::kN, FineThreads<COMP, WIDE>::kMinBlocks)
    fine_kernel(const FineDesc d, const LevelArgs<T> a, const __grid_constant__ CUtensorMap tmx,
                const __grid_constant__ CUtensorMap tmc, const __grid_constant__ CUtensorMap tmk0,
                const __grid_constant__ CUtensorMap tmk1, const __grid_constant__ CUtensorMap tmk2) {
  using S = FineShape<T0>;
  using L = FineLayout<T, COMP, T0>;
  constexpr int kFineThreads = FineThreads<COMP, WIDE>::kN;
  constexpr int XB = L::kXB, CB = L::kCB, KB = L::kKB;  // elements per buffer
  extern __shared__ __align__(128) unsigned char sm[];
  T* Xs = reinterpret_cast<T*>(sm + L::kOffX);              // [2][XB] (compress)
  T* Cs = reinterpret_cast<T*>(sm + L::kOffC);              // [2][CB]
  T* E = reinterpret_cast<T*>(sm + L::kOffE);               // even-k plane
  uint16_t* Ks = reinterpret_cast<uint16_t*>(sm + L::kOffK);  // [2][KB] (recover)
  uint32_t* hwin = reinterpret_cast<uint32_t*>(sm + L::kOffH);  // [kHistWin] (compress)
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::kOffBar);  // [2]
  __shared__ int s_bad, s_timeout;
  __shared__ uint32_t s_bytes[2];
  const int tid = threadIdx.x;
  DevState* st = a.st;
  // two values into the even-k plane at element offset off
  auto est2 = [&](int off, T v0, T v1) {
    if (SZ3G_IN(off >= 0 && off + 2 <= S::kT0 * S::kXJ * S::kEK, st)) st2(E + off, v0, v1);
  };
  if (COMP && (st->flags & (kFlagNonFinite | kFlagZeroRange | kFlagBadBound))) return;
  if (!COMP && (st->flags & kFlagCorrupt)) return;
  const T ebT = COMP ? bits_to<T>(st->ebT_bits) : a.ebT;
  const T ebr = COMP ? bits_to<T>(st->ebr_bits) : T(0);
  const int hlo = a.radius - kHistWin / 2;
  const int m0 = d.m0, m1 = d.m1, m2 = d.m2;
  if (COMP)
    for (int i = tid; i <= kHistWin; i += kFineThreads) hwin[i] = 0;
  if (tid == 0) {
    s_bad = 0;
    s_timeout = 0;
    s_bytes[0] = s_bytes[1] = 0;
    // recover with per-row arrivals: one arrival per staged code row
    const uint32_t arrivals =
        (!COMP && kCodeRowArrive && !d.code_tma) ? (uint32_t)(S::kR2 + S::kR1 + S::kR0) : 1u;
    mbar_init(&bar[0], arrivals);
    mbar_init(&bar[1], arrivals);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  FineAcc acc{false};

  auto tile_origin = [&](uint32_t tile, int& A0, int& A1, int& A2) {
    const uint32_t t2 = tile % (uint32_t)d.nt2, r = tile / (uint32_t)d.nt2;
    const uint32_t t1 = r % (uint32_t)d.nt1, t0 = r / (uint32_t)d.nt1;
    A0 = (int)t0 * S::kT0;
    A1 = (int)t1 * S::kT1;
    A2 = (int)t2 * S::kW;
  };
  // code rows of a tile: first code of each staged row
  auto row_c0 = [&](int A0, int A1, int A2, int r, int& which, int& slot, bool& valid) -> long long {
    if (r < S::kR2) {  // pass 2 row (i, j) of the tile
      const int i = A0 + r / S::kT1, j = A1 + r % S::kT1;
      which = 2;
      slot = r * S::kL2;
      valid = i < m0 && j < m1;
      return (long long)d.off[2] + ((long long)i * d.E1[2] + j) * d.E2[2] + A2 / 2;
    }
    r -= S::kR2;
    if (r < S::kR1) {  // pass 1 row (i, odd j)
      const int i = A0 + r / (S::kT1 / 2), j = A1 + 2 * (r % (S::kT1 / 2)) + 1;
      which = 1;
      slot = S::kR2 * S::kL2 + r * S::kL01;
      valid = i < m0 && j < m1;
      return (long long)d.off[1] + ((long long)i * d.E1[1] + (j - 1) / 2) * d.E2[1] + (A2 / 2 - 2);
    }
    r -= S::kR1;  // pass 0 row (odd i, even j)
    const int i = A0 + 2 * (r / S::kCJ) + 1, j = A1 - 2 + 2 * (r % S::kCJ);
    which = 0;
    slot = S::kR2 * S::kL2 + (S::kR1 + r) * S::kL01;
    valid = i < m0 && j >= 0 && j < m1;
    return (long long)d.off[0] + ((long long)(i - 1) / 2 * d.E1[0] + j / 2) * d.E2[0] + (A2 / 2 - 2);
  };
  // issue the copies of `tile` into buffer b (compress: tensor copies and the
  // arrival; recover: also the code rows, whose bytes are summed in
  // s_bytes[b] and announced by finish_issue after a barrier)
  auto issue = [&](uint32_t tile, int b) {
    int A0, A1, A2;
    tile_origin(tile, A0, A1, A2);
    if (!COMP && d.code_tma) {
      // the code rows of each pass as one box of the pass's code lattice, laid
      // out as the per-row copies place them: pass-2 rows of 40 codes from
      // k/2 = A2/2, pass-1 and pass-0 rows of 48 from A2/2 - 8 (rows and
      // codes outside the lattice read as 0 and are never used)
      if (tid == 0) {
        uint16_t* Kb = Ks + b * KB;
        fence_proxy_async_smem();
        mbar_expect_tx(&bar[b], d.tensor_bytes + (uint32_t)S::kCodeSlots * 2u);
        tma_load_3d(Cs + b * CB, &tmc, A2 / 2 - 4, A1 / 2 - 1, S::kHas0 ? A0 / 2 - 1 : 0, &bar[b]);
        tma_load_3d(Kb, &tmk2, A2 / 2, A1, A0, &bar[b]);
        tma_load_3d(Kb + S::kR2 * S::kL2, &tmk1, A2 / 2 - 8, A1 / 2, A0, &bar[b]);
        if (S::kHas0) tma_load_3d(Kb + S::kR2 * S::kL2 + S::kR1 * S::kL01, &tmk0, A2 / 2 - 8, A1 / 2 - 1, A0 / 2, &bar[b]);
      }
      return;
    }
    if (!COMP && kCodeRowArrive) {
      // row r by thread r: its arrival announces its bytes (thread 0 also the
      // coarse box's), then its copy
      if (tid < S::kR2 + S::kR1 + S::kR0) {
        int which, slot;
        bool valid;
        const long long c0 = row_c0(A0, A1, A2, tid, which, slot, valid);
        long long al = 0;
        int o = 0;
        if (valid) code_row(c0, &al, &o);
        const uint32_t want = which == 2 ? S::kL2 * 2 : S::kL01 * 2;
        // the row's copy stays inside the codes and the padding after them
        const bool inb = !valid || SZ3G_IN((unsigned long long)al + want / 2 <=
                                               a.n_codes + (a.codes_padded ? 128ull : 0ull), st);
        const uint32_t bytes = valid && inb ? want : 0u;
        fence_proxy_async_smem();
        mbar_expect_tx(&bar[b], bytes + (tid == 0 ? d.tensor_bytes : 0u));
        if (tid == 0)
          tma_load_3d(Cs + b * CB, &tmc, A2 / 2 - 4, A1 / 2 - 1, S::kHas0 ? A0 / 2 - 1 : 0, &bar[b]);
        if (bytes) bulk_load(Ks + b * KB + slot, a.codes + al, bytes, &bar[b]);
      }
      return;
    }
    if (tid == 0) {
      fence_proxy_async_smem();
      if (COMP || kCodeCpAsync) {
        mbar_expect_tx(&bar[b], d.tensor_bytes);
      }
      if (COMP) {
        tma_load_3d(Xs + b * XB, &tmx, A2 - 4, A1 - 2, A0, &bar[b]);
      }
      tma_load_3d(Cs + b * CB, &tmc, A2 / 2 - 4, A1 / 2 - 1, S::kHas0 ? A0 / 2 - 1 : 0, &bar[b]);
    }
    if (!COMP && kCodeCpAsync) {
      // every 16-byte piece of every staged row, spread over the threads
      constexpr int kItems = S::kR2 * (S::kL2 / 8) + (S::kR1 + S::kR0) * (S::kL01 / 8);
      for (int it = tid; it < kItems; it += kFineThreads) {
        int r, q;
        if (it < S::kR2 * (S::kL2 / 8)) {
          r = it / (S::kL2 / 8);
          q = it % (S::kL2 / 8);
        } else {
          const int u = it - S::kR2 * (S::kL2 / 8);
          r = S::kR2 + u / (S::kL01 / 8);
          q = u % (S::kL01 / 8);
        }
        int which, slot;
        bool valid;
        const long long c0 = row_c0(A0, A1, A2, r, which, slot, valid);
        if (valid) {
          long long al;
          int o;
          code_row(c0, &al, &o);
          const uint32_t d16 = (uint32_t)__cvta_generic_to_shared(Ks + b * KB + slot + 8 * q);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d16), "l"(a.codes + al + 8 * q) : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else if (!COMP && tid < S::kR2 + S::kR1 + S::kR0) {
      int which, slot;
      bool valid;
      const long long c0 = row_c0(A0, A1, A2, tid, which, slot, valid);
      if (valid) {
        long long al;
        int o;
        code_row(c0, &al, &o);
        const uint32_t bytes = which == 2 ? S::kL2 * 2 : S::kL01 * 2;
        fence_proxy_async_smem();
        bulk_load(Ks + b * KB + slot, a.codes + al, bytes, &bar[b]);
        atomicAdd(&s_bytes[b], bytes);
      }
    }
  };
  auto finish_issue = [&](int b) {  // after a barrier that follows issue(b)
    if (!COMP && tid == 0 && !kCodeCpAsync && !kCodeRowArrive) {
      mbar_expect_tx(&bar[b], d.tensor_bytes + s_bytes[b]);
      s_bytes[b] = 0;
    }
  };

  constexpr int ST = FineThreads<COMP>::kStages;
  uint32_t phase[2] = {0u, 0u};
  uint32_t tile = d.tile0 + blockIdx.x;
  if (ST == 2) {
    if (tile < d.ntiles) issue(tile, 0);
    __syncthreads();
    if (tile < d.ntiles) finish_issue(0);
  }
  int b = 0;
  for (; tile < d.ntiles; tile += gridDim.x, b ^= (ST == 2 ? 1 : 0)) {
    const uint32_t next = tile + gridDim.x;
    const bool has_next = ST == 2 && next < d.ntiles;
    if (ST == 1) {  // the buffer is free: the previous tile ended with a barrier
      issue(tile, 0);
      if (!COMP && !kCodeCpAsync && !kCodeRowArrive) {
        __syncthreads();
        finish_issue(0);
      }
    }
    if (has_next) issue(next, b ^ 1);
    // wait for this tile's copies
    {
      int spins = 0;
      bool done = true;
      while (!mbar_try_wait(&bar[b], phase[b])) {
        if (++spins > kWaitLimit) {
          s_timeout = 1;
          done = false;
          break;
        }
      }
      if (done) phase[b] ^= 1u;
      if (!COMP && kCodeCpAsync) {
        if (ST == 2 && has_next) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
    }
    __syncthreads();
    if (s_timeout) {
      if (has_next) finish_issue(b ^ 1);  // so that the copies in flight can be waited for
      break;
    }
    if (has_next) finish_issue(b ^ 1);
    int A0, A1, A2;
    tile_origin(tile, A0, A1, A2);
    const T* X = Xs + b * XB;
    const T* C = Cs + b * CB;
    const uint16_t* K = Ks + b * KB;
    // tiles away from every face: all points in the grid, every neighbour of
    // every pass present (compile-time predictor, no per-point checks)
    const bool edgek = !(A2 >= 4 && A2 + S::kW + 4 <= m2);
    const bool in0 = !S::kHas0 || (A0 >= 4 && A0 + S::kT0 + 4 <= m0);
    const bool in1 = A1 >= 4 && A1 + S::kT1 + 4 <= m1;
    auto passes = [&](auto interior_tag) {
      constexpr bool IN = decltype(interior_tag)::value;
      // ---- coarse points into E, and pass 0 (odd i, even j) ----------------
      // pass-0 tasks start on a warp boundary (kCopyPad), so that their
      // half-warps take whole rows as well
      constexpr int kCopyPad = (S::kCopyTasks + 31) & ~31;
      for (int t = tid; t < kCopyPad + S::kP0Tasks; t += kFineThreads) {
        if (t < S::kCopyTasks) {
          static_assert(S::kPairs == 18, "pair_task takes rows of 18 pairs");
          int pr, row;
          pair_task(t, S::kCopyTasks / S::kPairs, row, pr);
          const int e = row / S::kCJ, cj = row % S::kCJ;
          T v[2];
          ld2(C + ((e + (S::kHas0 ? 1 : 0)) * S::kCJ + cj) * S::kCK + 2 * pr + 2, v);
          est2(((2 * e) * S::kXJ + 2 * cj) * S::kEK + 2 * pr, v[0], v[1]);
          continue;
        }
        if (t < kCopyPad) continue;
        if constexpr (S::kHas0) {
          const int u = t - kCopyPad;
          int pr, row;
          pair_task(u, S::kP0Tasks / S::kPairs, row, pr);
          const int eo = row / S::kCJ, cj = row % S::kCJ;
          const int i = A0 + 2 * eo + 1, j = A1 - 2 + 2 * cj;
          if (!IN && (i >= m0 || j < 0 || j >= m1)) continue;
          const int ke = 2 * pr, k = A2 - 4 + 2 * ke;
          const bool hb = IN || i + 1 < m0, hc = IN || i >= 3, hd = IN || i + 3 < m0;
          T va[2], vb[2], vc[2], vd[2];
          const T* Cr = C + cj * S::kCK + ke + 2;
          ld2(Cr + (eo + 1) * S::kCJ * S::kCK, va);
          ld2(Cr + (eo + 2) * S::kCJ * S::kCK, vb);
          ld2(Cr + (eo + 0) * S::kCJ * S::kCK, vc);
          ld2(Cr + (eo + 3) * S::kCJ * S::kCK, vd);
          T xv[4] = {T(0), T(0), T(0), T(0)};
          if (COMP) ld4(X + ((2 * eo + 1) * S::kXJ + 2 * cj) * S::kXK + 2 * ke, xv);
          const int c0 = (int)d.off[0] + ((i - 1) / 2 * (int)d.E1[0] + j / 2) * (int)d.E2[0] + (A2 / 2 - 2);
          const bool ownj = j >= A1 && j < A1 + S::kT1;
          const uint16_t* kr = nullptr;
          if (!COMP) {
            long long al;
            int o;
            code_row(c0, &al, &o);
            kr = K + S::kR2 * S::kL2 + (S::kR1 + row) * S::kL01 + o + ke;
          }
          T r[2];
          if (IN) {
            const T p2[2] = {interp_predict<T>(va[0], vb[0], vc[0], vd[0], true, true, true, INTERP),
                             interp_predict<T>(va[1], vb[1], vc[1], vd[1], true, true, true, INTERP)};
            const bool own2[2] = {ownj && ke >= 2 && ke < 2 + S::kW / 2, ownj && ke + 1 >= 2 && ke + 1 < 2 + S::kW / 2};
            const T x2[2] = {xv[0], xv[2]};
            uint32_t k2[2] = {0u, 0u}, q2[2];
            if (!COMP) {
              if (d.code_al & 1) {
                const uint32_t v = *reinterpret_cast<const uint32_t*>(kr);
                k2[0] = v & 0xffffu, k2[1] = v >> 16;
              } else {
                k2[0] = kr[0], k2[1] = kr[1];
              }
            }
            fine_points<T, COMP, 2>(a, d, hwin, hlo, x2, p2, ebT, ebr, own2, (uint32_t)(c0 + ke), k2, acc, r, q2);
            if (COMP) {
              // (ke is even: both points of the pair are owned or neither)
              if ((d.code_al & 1) && own2[0]) {
                if (SZ3G_IN((unsigned long long)(long long)(c0 + ke) + 2 <= a.n_codes, st))
                  *reinterpret_cast<uint32_t*>(a.codes + c0 + ke) = q2[0] | (q2[1] << 16);
              } else {
                if (own2[0] && SZ3G_IN((unsigned long long)(long long)(c0 + ke) < a.n_codes, st))
                  a.codes[c0 + ke] = (uint16_t)q2[0];
                if (own2[1] && SZ3G_IN((unsigned long long)(long long)(c0 + ke + 1) < a.n_codes, st))
                  a.codes[c0 + ke + 1] = (uint16_t)q2[1];
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int kq = k + 2 * q;
              r[q] = T(0);
              if (kq < 0 || kq >= m2) continue;
              const T p = interp_predict<T>(va[q], vb[q], vc[q], vd[q], hb, hc, hd, INTERP);
              const bool own = ownj && ke + q >= 2 && ke + q < 2 + S::kW / 2;
              r[q] = fine_point<T, COMP>(a, d, hwin, hlo, xv[2 * q], p, ebT, ebr, own, (uint32_t)(c0 + ke + q),
                                         COMP ? 0u : (uint32_t)kr[q], acc);
            }
          }
          est2(((2 * eo + 1) * S::kXJ + 2 * cj) * S::kEK + ke, r[0], r[1]);
        }
      }
      __syncthreads();

      // ---- pass 1 (any i, odd j) --------------------------------------------
      for (int t = tid; t < S::kP1Tasks; t += kFineThreads) {
        int pr, row;
        pair_task(t, S::kP1Tasks / S::kPairs, row, pr);
        const int i4 = row / (S::kT1 / 2), jo = row % (S::kT1 / 2);
        const int i = A0 + i4, j = A1 + 2 * jo + 1;
        if (!IN && (i >= m0 || j >= m1)) continue;
        const int ke = 2 * pr, k = A2 - 4 + 2 * ke;
        const int j21 = 2 * jo + 3;
        const bool hb = IN || j + 1 < m1, hc = IN || j >= 3, hd = IN || j + 3 < m1;
        const T* Er = E + (i4 * S::kXJ + j21) * S::kEK + ke;
        T va[2], vb[2], vc[2], vd[2];
        ld2(Er - S::kEK, va);
        ld2(Er + S::kEK, vb);
        ld2(Er - 3 * S::kEK, vc);
        ld2(Er + 3 * S::kEK, vd);
        T xv[4] = {T(0), T(0), T(0), T(0)};
        if (COMP) ld4(X + (i4 * S::kXJ + j21) * S::kXK + 2 * ke, xv);
        const int c0 = (int)d.off[1] + (i * (int)d.E1[1] + (j - 1) / 2) * (int)d.E2[1] + (A2 / 2 - 2);
        const uint16_t* kr = nullptr;
        if (!COMP) {
          long long al;
          int o;
          code_row(c0, &al, &o);
          kr = K + S::kR2 * S::kL2 + row * S::kL01 + o + ke;
        }
        T r[2];
        if (IN) {
          const T p2[2] = {interp_predict<T>(va[0], vb[0], vc[0], vd[0], true, true, true, INTERP),
                           interp_predict<T>(va[1], vb[1], vc[1], vd[1], true, true, true, INTERP)};
          const bool own2[2] = {ke >= 2 && ke < 2 + S::kW / 2, ke + 1 >= 2 && ke + 1 < 2 + S::kW / 2};
          const T x2[2] = {xv[0], xv[2]};
          uint32_t k2[2] = {0u, 0u}, q2[2];
          if (!COMP) {
            if (d.code_al & 2) {
              const uint32_t v = *reinterpret_cast<const uint32_t*>(kr);
              k2[0] = v & 0xffffu, k2[1] = v >> 16;
            } else {
              k2[0] = kr[0], k2[1] = kr[1];
            }
          }
          fine_points<T, COMP, 2>(a, d, hwin, hlo, x2, p2, ebT, ebr, own2, (uint32_t)(c0 + ke), k2, acc, r, q2);
          if (COMP) {
            if ((d.code_al & 2) && own2[0]) {
              if (SZ3G_IN((unsigned long long)(long long)(c0 + ke) + 2 <= a.n_codes, st))
                *reinterpret_cast<uint32_t*>(a.codes + c0 + ke) = q2[0] | (q2[1] << 16);
            } else {
              if (own2[0] && SZ3G_IN((unsigned long long)(long long)(c0 + ke) < a.n_codes, st))
                a.codes[c0 + ke] = (uint16_t)q2[0];
              if (own2[1] && SZ3G_IN((unsigned long long)(long long)(c0 + ke + 1) < a.n_codes, st))
                a.codes[c0 + ke + 1] = (uint16_t)q2[1];
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int kq = k + 2 * q;
            r[q] = T(0);
            if (kq < 0 || kq >= m2) continue;
            const T p = interp_predict<T>(va[q], vb[q], vc[q], vd[q], hb, hc, hd, INTERP);
            const bool own = ke + q >= 2 && ke + q < 2 + S::kW / 2;
            r[q] = fine_point<T, COMP>(a, d, hwin, hlo, xv[2 * q], p, ebT, ebr, own, (uint32_t)(c0 + ke + q),
                                       COMP ? 0u : (uint32_t)kr[q], acc);
          }
        }
        est2((i4 * S::kXJ + j21) * S::kEK + ke, r[0], r[1]);
      }
      __syncthreads();

      // ---- pass 2 (any i, any j, odd k): runs of four ------------------------
      for (int t = tid; t < S::kP2Tasks; t += kFineThreads) {
        const int q4 = t & 7, row = t >> 3;
        const int i4 = row / S::kT1, j16 = row % S::kT1;
        const int i = A0 + i4, j = A1 + j16;
        if (!IN && (i >= m0 || j >= m1)) continue;
        const int j21 = j16 + 2;
        const T* Er = E + (i4 * S::kXJ + j21) * S::kEK + 4 * q4;
        T e[8];
        ld4(Er, e);
        ld4(Er + 4, e + 4);
        T xo[4] = {T(0), T(0), T(0), T(0)};
        if (COMP) {
          // the run's eight x values as two 16-byte loads; the upper four
          // lanes of each group of eight load the second half first, so that
          // the eight lanes of one load touch distinct banks
          const bool sw = (q4 & 4) != 0;
          T xa[4], xb[4];
          const T* xr = X + (i4 * S::kXJ + j21) * S::kXK + 8 * q4 + 4;
          ld4(xr + (sw ? 4 : 0), xa);
          ld4(xr + (sw ? 0 : 4), xb);
          xo[0] = sw ? xb[1] : xa[1];
          xo[1] = sw ? xb[3] : xa[3];
          xo[2] = sw ? xa[1] : xb[1];
          xo[3] = sw ? xa[3] : xb[3];
        }
        const int c0 = (int)d.off[2] + (i * (int)d.E1[2] + j) * (int)d.E2[2] + A2 / 2;
        const uint32_t ci = (uint32_t)(c0 + 4 * q4);
        const uint16_t* kr = nullptr;
        if (!COMP) {
          long long al;
          int o;
          code_row(c0, &al, &o);
          kr = K + row * S::kL2 + o + 4 * q4;
        }
        const int k0 = A2 + 8 * q4;  // first (even) k of the run's eight points
        T r[4];
        if (IN || !edgek) {
          uint32_t kin[4] = {0u, 0u, 0u, 0u}, cq[4] = {0u, 0u, 0u, 0u};
          if (!COMP) {
            if (kPackCodes) {
              if (d.code_al & 4) {
                const uint2 v = *reinterpret_cast<const uint2*>(kr);
                kin[0] = v.x & 0xffffu, kin[1] = v.x >> 16, kin[2] = v.y & 0xffffu, kin[3] = v.y >> 16;
              } else {
                get_codes4(kr, kin);
              }
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) kin[u] = kr[u];
            }
          }
          T p4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            p4[u] = interp_predict<T>(e[u + 2], e[u + 3], e[u + 1], e[u + 4], true, true, true, INTERP);
          const bool own4[4] = {true, true, true, true};
          fine_points<T, COMP, 4>(a, d, hwin, hlo, xo, p4, ebT, ebr, own4, ci, kin, acc, r, cq);
          if (COMP && SZ3G_IN((unsigned long long)ci + 4 <= a.n_codes, st)) {
            if (d.code_al & 4)
              *reinterpret_cast<uint2*>(a.codes + ci) = make_uint2(cq[0] | (cq[1] << 16), cq[2] | (cq[3] << 16));
            else
              put_codes4(a.codes + ci, cq);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int kk = k0 + 2 * u + 1;
            r[u] = T(0);
            if (kk >= m2) continue;
            const bool hb = kk + 1 < m2, hc = kk >= 3, hd = kk + 3 < m2;
            const T p = interp_predict<T>(e[u + 2], hb ? e[u + 3] : T(0), hc ? e[u + 1] : T(0),
                                          hd ? e[u + 4] : T(0), hb, hc, hd, INTERP);
            r[u] = fine_point<T, COMP>(a, d, hwin, hlo, xo[u], p, ebT, ebr, true, ci + u,
                                       COMP ? 0u : (uint32_t)kr[u], acc);
          }
        }
        if (d.write_out) {
          const unsigned long long od =
              (unsigned long long)i * d.rs0 + (unsigned long long)j * d.rs1 + (unsigned long long)k0;
          T* dst = a.Rout + od;
          if (IN || k0 + 8 <= m2) {
            if (SZ3G_IN(od + 8 <= a.n_out, st)) {
              st4(dst, e[2], r[0], e[3], r[1]);
              st4(dst + 4, e[4], r[2], e[5], r[3]);
            }
          } else {
            const T v8[8] = {e[2], r[0], e[3], r[1], e[4], r[2], e[5], r[3]};
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8)
              if (k0 + s8 < m2 && SZ3G_IN(od + s8 < a.n_out, st)) dst[s8] = v8[s8];
          }
        }
      }
      __syncthreads();
    };
    if (in0 && in1 && !edgek) passes(std::true_type{});
    else passes(std::false_type{});
  }

  // ---- flush the per-CTA counters
  if (acc.bad) s_bad = 1;
  __syncthreads();
  if (s_timeout) {
    // give copies still in flight a last bounded chance to land
    for (int q = 0; q < 2; ++q) {
      int spins = 0;
      while (!mbar_try_wait(&bar[q], phase[q]) && ++spins < kWaitLimit) {
      }
    }
    if (tid == 0) atomicOr(&st->flags, kFlagTimeout);
  }
  if (COMP) {
    for (int i = tid; i < kHistWin; i += kFineThreads)
      if (hwin[i]) atomicAdd(&a.hist[hlo + i], hwin[i]);
  } else if (tid == 0 && s_bad) {
    atomicOr(&st->flags, kFlagCorrupt);
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// 3-D tensor map over rows of m2 elements (row stride s1, plane stride s0
// elements) with a box of b0 x b1 x b2 elements (T: float, double or the
// 2-byte codes).
template <typename T>
static bool fine_map(CUtensorMap* map, const T* base, int m0, int m1, int m2, unsigned long long s0,
                     unsigned long long s1, int b0, int b1, int b2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)m2, (cuuint64_t)m1, (cuuint64_t)m0};
  const cuuint64_t strides[2] = {(cuuint64_t)s1 * sizeof(T), (cuuint64_t)s0 * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)b2, (cuuint32_t)b1, (cuuint32_t)b0};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 2   ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                : sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return enc(map, dt, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Whether the register-blocked kernel takes level k (the passes of G_k in
// plan order): 3-D grids refined in axis order (0, 1, 2) or 2-D grids in
// (1, 2), with 16-byte aligned rows for the tensor copies.
bool fine_eligible(const Plan& pl, int k, bool comp, const void* x, const unsigned long long* xs, const void* Rc,
                   const void* Rout, bool to_field) {
  if (pl.ndim < 2 || pl.n[0] != 1) return false;
  int ax[4], P = 0;
  for (int i = 0; i < pl.n_pass; ++i)
    if (pl.pass[i].grid == k) {
      if (P == 4) return false;
      ax[P++] = pl.pass[i].axis;
    }
  const unsigned long long* m = pl.gm[k];
  const bool three = m[1] > 1;
  if (three ? !(P == 3 && ax[0] == 1 && ax[1] == 2 && ax[2] == 3) : !(P == 2 && ax[0] == 2 && ax[1] == 3))
    return false;
  const size_t esz = (size_t)pl.esz;
  const unsigned long long* mc = pl.gm[k + 1];
  auto rows16 = [&](unsigned long long e2) { return (e2 * esz) % 16 == 0; };
  if (!rows16(mc[3]) || ((uintptr_t)Rc % 16) != 0) return false;
  // compress reads x by tensor copies: contiguous rows, 16-byte strides
  if (comp && (xs[2] != 1 || !rows16(xs[1]) || !rows16(xs[0]) || ((uintptr_t)x % 16) != 0)) return false;
  if (Rout && (!rows16(to_field ? pl.n[3] : m[3]) || ((uintptr_t)Rout % 16) != 0)) return false;
  return m[2] >= 2 && m[3] >= 2 && pl.gsize[k] <= 0xffffffffull;
}

// Tiles of the plane groups [g0, g1) along axis 0 (T0 planes of G_k each).
template <typename T, bool COMP, int T0>
static int launch_fine_t(const Plan& pl, int k, const LevelArgs<T>& a, bool to_field, cudaStream_t s,
                         uint32_t g0 = 0, uint32_t g1 = 0xffffffffu) {
  using S = FineShape<T0>;
  FineDesc d;
  memset(&d, 0, sizeof(d));
  const unsigned long long* m = pl.gm[k];
  d.m0 = (int)m[1];
  d.m1 = (int)m[2];
  d.m2 = (int)m[3];
  d.nt1 = (d.m1 + S::kT1 - 1) / S::kT1;
  d.nt2 = (d.m2 + S::kW - 1) / S::kW;
  const int nt0 = (d.m0 + S::kT0 - 1) / S::kT0;
  if (g1 > (uint32_t)nt0) g1 = (uint32_t)nt0;
  if (g0 >= g1) return SZ3G_OK;
  d.tile0 = g0 * (uint32_t)d.nt1 * (uint32_t)d.nt2;
  d.ntiles = g1 * (uint32_t)d.nt1 * (uint32_t)d.nt2;
  int p = S::kHas0 ? 0 : 1;
  int interp = SZ3G_LINEAR;
  uint32_t E0[3] = {0u, 0u, 0u};  // lattice extent of each pass along axis 0
  for (int i = 0; i < pl.n_pass; ++i) {
    const PassDesc& pd = pl.pass[i];
    if (pd.grid != k) continue;
    d.off[p] = (uint32_t)pd.off;
    E0[p] = pd.E[1];
    d.E1[p] = pd.E[2];
    d.E2[p] = pd.E[3];
    interp = pd.interp;
    ++p;
  }
  d.write_out = a.Rout != nullptr;
  if (to_field) {
    d.rs1 = (uint32_t)pl.fstride[2];
    d.rs0 = (uint32_t)pl.fstride[1];
  } else {
    d.rs1 = (uint32_t)m[3];
    d.rs0 = (uint32_t)(m[3] * m[2]);
  }
  d.chunk = pl.chunk;
  d.nsub = pl.nsub;
  const unsigned long long* mc = pl.gm[k + 1];
  CUtensorMap tmx, tmc;
  memset(&tmx, 0, sizeof(tmx));
  memset(&tmc, 0, sizeof(tmc));
  bool ok = fine_map<T>(&tmc, a.Rc, (int)mc[1], (int)mc[2], (int)mc[3], mc[3] * mc[2], mc[3], S::kCI, S::kCJ, S::kCK);
  d.tensor_bytes = (uint32_t)(S::kCI * S::kCJ * S::kCK * sizeof(T));
  if (COMP) {
    ok = ok && fine_map<T>(&tmx, a.x, d.m0, d.m1, d.m2, a.xs[0], a.xs[1], S::kT0, S::kXJ, S::kXK);
    d.tensor_bytes += (uint32_t)(S::kT0 * S::kXJ * S::kXK * sizeof(T));
  }
  // pairs of codes (passes 0, 1: the pair starts at an even lattice index)
  // and runs of four (pass 2: at a multiple of four) start on 4- and 8-byte
  // boundaries when the pass's first code and row length allow it
  if ((uintptr_t)a.codes % 8 == 0) {
    for (int q = S::kHas0 ? 0 : 1; q < 2; ++q)
      if (d.off[q] % 2 == 0 && d.E2[q] % 2 == 0) d.code_al |= 1 << q;
    if (d.off[2] % 4 == 0 && d.E2[2] % 4 == 0) d.code_al |= 4;
  }
  CUtensorMap tmk[3];
  memset(tmk, 0, sizeof(tmk));
  if (!COMP) {
    // code rows by tensor copies when every pass's codes start on a 16-byte
    // boundary and its rows are a multiple of 16 bytes long
    bool tma = ((uintptr_t)a.codes % 16) == 0;
    for (int q = S::kHas0 ? 0 : 1; q < 3; ++q) tma = tma && d.E2[q] % 8 == 0 && d.off[q] % 8 == 0;
    if (tma) {
      for (int q = S::kHas0 ? 0 : 1; q < 3 && ok; ++q) {
        const int rows = q == 2 ? S::kT1 : (q == 1 ? S::kT1 / 2 : S::kCJ);
        const int planes = q == 0 ? 2 : S::kT0;
        ok = fine_map<uint16_t>(&tmk[q], a.codes + d.off[q], (int)E0[q], (int)d.E1[q], (int)d.E2[q],
                                (unsigned long long)d.E1[q] * d.E2[q], d.E2[q], planes, rows,
                                q == 2 ? S::kL2 : S::kL01);
      }
      d.code_tma = 1;
    }
  }
  if (!ok) return SZ3G_E_CUDA;
  const size_t smem = FineLayout<T, COMP, T0>::kBytes;
  int dev = 0, nsm = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool wide = !COMP && d.ntiles - d.tile0 <= (uint32_t)(kWideTiles * nsm);
  decltype(&fine_kernel<T, COMP, SZ3G_CUBIC, T0, false>) kern;
  if constexpr (COMP)
    kern = interp == SZ3G_CUBIC ? fine_kernel<T, COMP, SZ3G_CUBIC, T0, false> : fine_kernel<T, COMP, SZ3G_LINEAR, T0, false>;
  else if (wide)
    kern = interp == SZ3G_CUBIC ? fine_kernel<T, COMP, SZ3G_CUBIC, T0, true> : fine_kernel<T, COMP, SZ3G_LINEAR, T0, true>;
  else
    kern = interp == SZ3G_CUBIC ? fine_kernel<T, COMP, SZ3G_CUBIC, T0, false> : fine_kernel<T, COMP, SZ3G_LINEAR, T0, false>;
  const int nthr = wide ? FineThreads<COMP, true>::kN : FineThreads<COMP, false>::kN;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SZ3G_E_CUDA;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, nthr, smem);
  if (per < 1) per = 1;
  unsigned long long grid = (unsigned long long)nsm * per;
  if (g_level_cta_cap > 0 && grid > (unsigned long long)g_level_cta_cap) grid = (unsigned long long)g_level_cta_cap;
  if (grid > d.ntiles - d.tile0) grid = d.ntiles - d.tile0;
  SZ3G_LAUNCH(COMP ? kKLevelQuantize : kKLevelRecover, s,
              kern<<<(unsigned)grid, nthr, smem, s>>>(d, a, tmx, tmc, tmk[0], tmk[1], tmk[2]));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

template <typename T, bool COMP>
int launch_fine(const Plan& pl, int k, const LevelArgs<T>& a, bool to_field, cudaStream_t s) {
  return pl.gm[k][1] > 1 ? launch_fine_t<T, COMP, 4>(pl, k, a, to_field, s)
                         : launch_fine_t<T, COMP, 1>(pl, k, a, to_field, s);
}

// The finest level of a decompress (3-D, to the field) in `slabs` launches of
// consecutive plane groups; after each, `done(first_plane, planes)` is called
// on the host with the field planes that launch completed.
template <typename T>
int launch_fine_slabs(const Plan& pl, const LevelArgs<T>& a, cudaStream_t s, int slabs,
                      const std::function<int(unsigned long long, unsigned long long)>& done) {
  constexpr int T0 = 4;
  const unsigned long long m0 = pl.gm[0][1];
  const uint32_t ng = (uint32_t)((m0 + T0 - 1) / T0);
  const uint32_t per = (ng + (uint32_t)slabs - 1) / (uint32_t)slabs;
  for (uint32_t g0 = 0; g0 < ng; g0 += per) {
    const uint32_t g1 = g0 + per < ng ? g0 + per : ng;
    const int rc = launch_fine_t<T, false, T0>(pl, 0, a, true, s, g0, g1);
    if (rc != SZ3G_OK) return rc;
    const unsigned long long p0 = (unsigned long long)g0 * T0, p1 = (unsigned long long)g1 * T0 < m0 ? g1 * T0 : m0;
    const int rd = done(p0, p1 - p0);
    if (rd != SZ3G_OK) return rd;
  }
  return SZ3G_OK;
}
template int launch_fine_slabs<float>(const Plan&, const LevelArgs<float>&, cudaStream_t, int,
                                      const std::function<int(unsigned long long, unsigned long long)>&);
template int launch_fine_slabs<double>(const Plan&, const LevelArgs<double>&, cudaStream_t, int,
                                       const std::function<int(unsigned long long, unsigned long long)>&);

template int launch_fine<float, true>(const Plan&, int, const LevelArgs<float>&, bool, cudaStream_t);
template int launch_fine<float, false>(const Plan&, int, const LevelArgs<float>&, bool, cudaStream_t);
template int launch_fine<double, true>(const Plan&, int, const LevelArgs<double>&, bool, cudaStream_t);
template int launch_fine<double, false>(const Plan&, int, const LevelArgs<double>&, bool, cudaStream_t);

}  // namespace sz3g
