// k_sweep.cu -- plane-pair sweep kernel for grids refined in axis order
// (0, 1, 2) (3-D) or (1, 2) (2-D: axis 0 is a unit axis).
//
// One launch per grid G_k.  The level's passes (Sec. 6.2, multilevel
// interpolation at the finest stride of G_k: refine axis 0, then 1, then 2)
// split the points of G_k by coordinate parity: pass 0 takes (odd i, even j,
// even k), pass 1 (any i, odd j, even k), pass 2 (any i, any j, odd k).
//
// A CTA owns the two planes i = 2p, 2p + 1 of G_k, a run of row pairs
// (j = 2b, 2b + 1 for b in [b0, b1)) and a segment of KW points along k, and
// sweeps the row pairs in order.  It keeps, per plane, the even-k values of
// the even rows in a ring E (eight rows) and of the odd row in E1 (two
// buffers).  Step b, with one barrier:
//   B  row c = b + 3 of E: the coarse row R_{k+1}[p][c] (plane 2p) and the
//      pass-0 row of plane 2p + 1, predicted along i from the coarse rows of
//      planes p - 1 .. p + 2;
//   C  pass 1 at j = 2b + 1 for both planes, along j from E rows b - 1 .. b + 2
//      (written by earlier steps), into E1[b & 1];
//   -- barrier --
//   D  pass 2 on the four rows (2p | 2p + 1) x (2b | 2b + 1), along k from
//      the even values of the row; the rows leave as (even, odd) runs.
// B and C share a barrier interval because C reads only rows finished one
// step earlier; the next step's B and C write a ring row and an E1 buffer
// that D does not read.  Every point is predicted once (the ring slides
// instead of re-reading a halo), except the even columns next to the k
// segment (passes 0 and 1 evaluate them, never written, so that pass 2 has
// its neighbours) and the four rows evaluated before a run to fill the ring.
//
// Work is spread in runs of four consecutive columns: a thread of B or C
// takes four even columns of one row, a thread of D four odd points (and the
// four even points between them) of one row, so shared-memory reads, code
// reads and the field's stores are vector accesses.
//
// Inputs arrive by asynchronous copies, two steps ahead, into one of three
// slots per CTA, each on its own mbarrier: the four coarse rows (one tensor
// copy), the input rows (compress: tensor copies) or the code rows of the
// step (recover: one bulk copy per row, 16-byte aligned).  Boundary rules
// along i and j are uniform per CTA and step; along k they are per point,
// with a compile-time interior form for segments away from both ends.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "internal.cuh"
#include "level_common.cuh"

namespace sz3g {

constexpr int kSwThreads = 128;
constexpr int kSwKW = 256;  // points of a k segment (kSwThreads odd points x 2)
constexpr int kSwJS = 16;   // row pairs of a run
constexpr int kSwSlots = 4;  // copy slots; copies run kSwSlots - 1 steps ahead
constexpr int kSwRing = 8;  // even rows kept per plane

template <typename T>
struct SwShape {
  static constexpr int kHE = 4;                        // extra even columns on each side (runs of four)
  static constexpr int kCW = kSwKW / 2 + 2 * kHE;      // even columns of an E row (a multiple of 4)
  static constexpr int kQuads = kCW / 4;               // runs of four even columns in an E row
  static constexpr int kXW = kSwKW + 4 * kHE;          // input points of a row segment (compress)
  static constexpr int kXH = kXW / 2;                  // one tensor copy of a row: half of it (<= 256 elements)
  // u16 slots of a staged code row: the row, up to 7 codes of alignment in
  // front and a run of four read past its end
  static constexpr int kCodeRow = ((kCW + 7 + 7) / 8) * 8 + 8;
  static_assert(kCW % 4 == 0 && kXH % 8 == 0, "runs of four even columns, runs of eight input points");
};

// Shared-memory layout (bytes), tensor-copy destinations on 128-byte boundaries.
template <typename T, bool COMP>
struct SwLayout {
  using S = SwShape<T>;
  static constexpr size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }
  static constexpr size_t kCoarse = up((size_t)4 * S::kCW * sizeof(T), 128);   // 4 coarse rows
  // input rows (compress): [half][plane][row][kXH] for rows 2b, 2b + 1 of both
  // planes (the second plane unused in 2-D), then the two halves of row
  // (2p + 1, 2c), each copy on a 128-byte boundary
  static constexpr size_t kXB0 = up((size_t)S::kXH * sizeof(T), 128);
  static constexpr size_t kXA = up((size_t)4 * S::kXW * sizeof(T), 128);
  static constexpr size_t kXrows = COMP ? kXA + 2 * kXB0 : 0;
  static constexpr size_t kCodes = COMP ? 0 : up((size_t)7 * S::kCodeRow * 2, 128);    // 7 code rows
  static constexpr size_t kSlot = kCoarse + kXrows + kCodes;
  static constexpr size_t kOffSlots = 0;
  static constexpr size_t kOffE = kOffSlots + kSwSlots * kSlot;                           // [2][kSwRing][kCW]
  static constexpr size_t kOffE1 = kOffE + up((size_t)2 * kSwRing * S::kCW * sizeof(T), 16);  // [2 bufs][2][kCW]
  static constexpr size_t kOffH = kOffE1 + up((size_t)4 * S::kCW * sizeof(T), 16);
  static constexpr size_t kOffBar = up(kOffH + (COMP ? (kHistWin + 1) * 4 : 0), 16);
  static constexpr size_t kBytes = kOffBar + 8 * kSwSlots;
};

struct SweepDesc {
  int m0, m1, m2;           // extents of G_k (m0 = 1 in 2-D)
  int mc0, mc1, mc2;        // extents of G_{k+1}
  int cpl, xpl;             // planes of the coarse box (4 in 3-D, 1 in 2-D) and of the input box (2 / 1)
  uint32_t nks, njs;        // k segments, runs of row pairs
  uint32_t item0, nitems;   // items [item0, nitems) of this launch (plane pair major)
  uint32_t off[3];          // first code of passes 0, 1, 2 (a field's code indices fit in 32 bits)
  uint32_t E1[3], E2[3];    // lattice extents of each pass along j and k
  uint32_t rs0, rs1;        // output element strides along i, j (contiguous along k)
  uint32_t chunk, nsub;
  int write_out;
};

// four consecutive values (16-byte aligned in shared memory)
template <typename T>
__device__ __forceinline__ void sw_ld4(const T* p, T* v) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else {
    const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
  }
}
template <typename T>
__device__ __forceinline__ void sw_st4(T* p, T a, T b, T c, T d) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
  }
}
// four consecutive u16 codes at any 2-byte alignment, as one 8-, two 4- or
// four 2-byte accesses
__device__ __forceinline__ void sw_codes_in(const uint16_t* p, uint32_t* c) {
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
__device__ __forceinline__ void sw_codes_out(uint16_t* p, const uint32_t* c) {
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

template <typename T, bool COMP, int INTERP>
__global__ void __launch_bounds__(kSwThreads, sizeof(T) == 4 ? 8 : 6)
    sweep_kernel(const SweepDesc d, const LevelArgs<T> a, const __grid_constant__ CUtensorMap tmc,
                 const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmx1) {
  using S = SwShape<T>;
  using L = SwLayout<T, COMP>;
  constexpr int CW = S::kCW, HE = S::kHE, XW = S::kXW, XH = S::kXH, CR = S::kCodeRow, NQ = S::kQuads;
  extern __shared__ __align__(128) unsigned char sm[];
  T* E = reinterpret_cast<T*>(sm + L::kOffE);    // E[(plane * kSwRing + (c & 7)) * CW + e]
  T* E1 = reinterpret_cast<T*>(sm + L::kOffE1);  // E1[((b & 1) * 2 + plane) * CW + e]
  uint32_t* hwin = reinterpret_cast<uint32_t*>(sm + L::kOffH);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::kOffBar);
  __shared__ int s_bad, s_timeout;
  const int tid = threadIdx.x;
  DevState* st = a.st;
  if (COMP && (st->flags & (kFlagNonFinite | kFlagZeroRange | kFlagBadBound))) return;
  if (!COMP && (st->flags & kFlagCorrupt)) return;
  const uint32_t item = d.item0 + blockIdx.x;
  if (item >= d.nitems) return;
  const T ebT = COMP ? bits_to<T>(st->ebT_bits) : a.ebT;
  const T ebr = COMP ? bits_to<T>(st->ebr_bits) : T(0);
  const int radius = a.radius;
  const uint32_t r2m1 = 2u * (uint32_t)radius - 1u;
  const int hlo = radius - kHistWin / 2;
  const int m0 = d.m0, m1 = d.m1, m2 = d.m2, mc1 = d.mc1, mc2 = d.mc2;
  // item -> (plane pair, run, k segment)
  const uint32_t ks = item % d.nks, r0 = item / d.nks;
  const uint32_t js = r0 % d.njs, pp = r0 / d.njs;
  const int ie = 2 * (int)pp, io = ie + 1;
  const bool has_io = io < m0;
  const int K0 = (int)ks * kSwKW;
  const int kc0 = K0 / 2 - HE;  // even column of E index 0
  const int b0 = (int)js * kSwJS, b1 = min(b0 + kSwJS, mc1);
  const int zb = d.cpl == 4 ? 1 : 0;  // box plane of coarse plane pp
  // code indices (every code index of a field fits in 32 bits): the pass-0
  // row (pp, c) starts at base0 + c E20, the pass-1 row (ie + q, b) at
  // base1 + q pl1 + b E21, the pass-2 row (ie + q, j) at base2 + q pl2 + j E22
  const uint32_t E20 = d.E2[0], E21 = d.E2[1], E22 = d.E2[2];
  const uint32_t pl1 = d.E1[1] * E21, pl2 = d.E1[2] * E22;
  const uint32_t base0 = d.off[0] + pp * d.E1[0] * E20;
  const uint32_t base1 = d.off[1] + (uint32_t)ie * pl1;
  const uint32_t base2 = d.off[2] + (uint32_t)ie * pl2;
  const int lo01 = max(kc0, 0), lo2 = K0 / 2;  // first staged lattice column of pass-0/1 and pass-2 rows

  // ---- per-thread roles, fixed for the whole sweep
  // B / C: a run of four even columns (B: the new E row; C: one plane's odd row)
  const int role = tid < NQ ? 0 : (tid < 3 * NQ ? 1 : 2);
  const int cq = (role == 1 && tid - NQ >= NQ) ? 1 : 0;
  const int qd = role == 0 ? tid : (role == 1 ? tid - NQ - cq * NQ : 0);
  const int qe = 4 * qd, col0 = kc0 + qe;
  const bool q_in = col0 >= 0 && col0 < mc2 && (role == 0 ? has_io : (cq == 0 || has_io));
  const int q_nv = min(4, mc2 - col0);  // points of the run inside the grid
  const bool q_own = col0 >= K0 / 2 && col0 < K0 / 2 + kSwKW / 2;
  const bool hb0 = io + 1 < m0, hc0 = io >= 3, hd0 = io + 3 < m0;  // pass 0 (along i), uniform
  // D: four odd points and the four even points before them, of one row
  const int dw = tid >> 5, rr = tid & 31, dq = dw & 1, tj = dw >> 1;
  const int kk = K0 / 2 + 4 * rr, de = HE + 4 * rr;
  const bool d_in = ie + dq < m0 && 2 * kk < m2;
  const int d_nv = min(4, max(0, (m2 - 2 * kk) >> 1));  // odd points inside the grid
  const bool d_full = 2 * kk + 8 <= m2;
  const bool d_edge = !((K0 >= 4 && K0 + kSwKW + 4 <= m2) || (kk >= 1 && 2 * kk + 10 < m2));
  // input offsets inside a slot's input rows (compress)
  const int xoffB = [&] {
    const int u = 2 * qe, h = u >= XH ? 1 : 0;
    return (int)((L::kXA + h * L::kXB0) / sizeof(T)) + (u - h * XH);
  }();
  const int xoffC = [&] {
    const int u = 2 * qe, h = u >= XH ? 1 : 0;
    return (h * 2 + cq) * 2 * XH + XH + (u - h * XH);
  }();
  const int xoffD = [&] {
    const int u = 8 * rr + 2 * HE, h = u >= XH ? 1 : 0;
    return (h * 2 + dq) * 2 * XH + tj * XH + (u - h * XH);
  }();

  if (COMP)
    for (int i = tid; i <= kHistWin; i += kSwThreads) hwin[i] = 0;
  if (tid == 0) {
    s_bad = 0;
    s_timeout = 0;
    for (int q = 0; q < kSwSlots; ++q) mbar_init(&bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool bad = false;

  // code row r of iteration v (recover): 0 the pass-0 row (pp, c = v + 3),
  // 1-2 the pass-1 rows (ie | io, b = v), 3-6 the pass-2 rows (ie, 2b),
  // (io, 2b), (ie, 2b + 1), (io, 2b + 1); false when the row is not staged
  auto code_row = [&](int v, int r, uint32_t* row0, int* lo, int* hi) -> bool {
    const int c = v + 3, b = v;
    if (r == 0) {
      if (!has_io || c < 0 || c >= mc1) return false;
      *row0 = base0 + (uint32_t)c * E20;
      *lo = lo01, *hi = min(kc0 + CW, (int)E20);
    } else if (r <= 2) {
      if (b < b0 || 2 * b + 1 >= m1 || (r == 2 && !has_io)) return false;
      *row0 = base1 + (r == 2 ? pl1 : 0u) + (uint32_t)b * E21;
      *lo = lo01, *hi = min(kc0 + CW, (int)E21);
    } else {
      const int q = (r - 3) & 1, j = 2 * b + ((r - 3) >> 1);
      if (b < b0 || j >= m1 || (q && !has_io)) return false;
      *row0 = base2 + (q ? pl2 : 0u) + (uint32_t)j * E22;
      *lo = lo2, *hi = min(K0 / 2 + kSwKW / 2, (int)E22);
    }
    return *lo < *hi;
  };

  // The copies of iteration n (v = b0 - 4 + n) into slot n % kSwSlots,
  // issued by the 32 lanes of one warp: lane 0 the coarse box; compress:
  // lanes 1-2 the halves of the step's input box, lanes 3-4 those of row
  // (io, 2c); recover: lanes 1-7 the code rows 0-6.  Lane 0 announces the
  // total bytes on the slot's mbarrier before any copy is issued.
  auto issue = [&](int n) {
    const int lane = tid & 31;
    const int v = b0 - 4 + n, c = v + 3;
    unsigned char* slot = sm + L::kOffSlots + (size_t)(n % kSwSlots) * L::kSlot;
    uint64_t* br = &bar[n % kSwSlots];
    const bool rowB = c >= 0 && c < mc1;
    const bool stepCD = v >= b0;
    uint32_t bytes = 0, al = 0;
    if (lane == 0) {
      if (rowB) bytes = d.cpl * CW * sizeof(T);
    } else if (COMP) {
      if (lane <= 2 && stepCD) bytes = d.xpl * XW * sizeof(T);
      else if (lane >= 3 && lane <= 4 && rowB && has_io) bytes = XH * sizeof(T);
    } else if (lane <= 7) {
      uint32_t row0;
      int lo, hi;
      if (code_row(v, lane - 1, &row0, &lo, &hi)) {
        al = (row0 + (uint32_t)lo) & ~7u;
        bytes = ((row0 + (uint32_t)hi - al + 7u) & ~7u) * 2u;
      }
    }
    uint32_t total = bytes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(br, total);
    }
    __syncwarp();
    if (bytes == 0) return;
    fence_proxy_async_smem();
    if (lane == 0) {
      tma_load_3d(slot, &tmc, kc0, c, (int)pp - zb, br);
    } else if (COMP) {
      unsigned char* xb = slot + L::kCoarse;
      // planes ie, io x rows 2b, 2b + 1 in two halves along k, and the two
      // halves of row (io, 2c) (rows and planes past the grid read the fill value)
      if (lane == 1) tma_load_3d(xb, &tmx, K0 - 2 * HE, 2 * v, ie, br);
      else if (lane == 2) tma_load_3d(xb + (size_t)4 * XH * sizeof(T), &tmx, K0 - 2 * HE + XH, 2 * v, ie, br);
      else if (lane == 3) tma_load_3d(xb + L::kXA, &tmx1, K0 - 2 * HE, 2 * c, io, br);
      else tma_load_3d(xb + L::kXA + L::kXB0, &tmx1, K0 - 2 * HE + XH, 2 * c, io, br);
    } else {
      uint16_t* cs = reinterpret_cast<uint16_t*>(slot + L::kCoarse);
      bulk_load(cs + (lane - 1) * CR, a.codes + al, bytes, br);
    }
  };

  // Recover a run of four points from their predictions and codes; nv: the
  // points inside the grid.  Codes 0 (unpredictable) and codes past the
  // alphabet take the per-point path, once per run.
  auto rec4 = [&](const T* p4, const uint32_t* k4, uint32_t ci0, int nv, T* r4) {
    bool rare = nv < 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) rare |= (k4[t] - 1u) >= r2m1;
    if (!rare) {
#pragma unroll
      for (int t = 0; t < 4; ++t) r4[t] = recover_point<T>(p4[t], k4[t], radius, ebT);
      return;
    }
    for (int t = 0; t < nv; ++t) {
      const uint32_t code = k4[t];
      if (code - 1u < r2m1) {
        r4[t] = recover_point<T>(p4[t], code, radius, ebT);
      } else {
        r4[t] = T(0);
        if (code == 0) {
          const unsigned long long rk = rank_of_zero(a.codes, ci0 + t, d.chunk, d.nsub, a.zunit);
          if (rk < a.n_unpred) r4[t] = a.unpred[rk];
          else bad = true;
        } else {
          bad = true;
        }
      }
    }
  };
  // Quantize a run of four points; own: count the first nv of them in the
  // histogram.  Codes outside the shared window also go to the global
  // histogram, checked once per run.
  auto quant4 = [&](const T* x4, const T* p4, bool own, int nv, uint32_t* q4, T* r4) {
#pragma unroll
    for (int t = 0; t < 4; ++t) q4[t] = quantize_point<T>(x4[t], p4[t], ebT, ebr, radius, r4[t]);
    if (!own) return;
    if (nv == 4) {
      bool anyfar = false;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint32_t bn = q4[t] - (uint32_t)hlo;
        const bool far = bn >= (uint32_t)kHistWin;
        atomicAdd(&hwin[far ? (uint32_t)kHistWin : bn], 1u);
        anyfar |= far;
      }
      if (anyfar)
        for (int t = 0; t < 4; ++t)
          if (q4[t] - (uint32_t)hlo >= (uint32_t)kHistWin) atomicAdd(&a.hist[q4[t]], 1u);
    } else {
      for (int t = 0; t < nv; ++t) {
        const uint32_t bn = q4[t] - (uint32_t)hlo;
        if (bn < (uint32_t)kHistWin) atomicAdd(&hwin[bn], 1u);
        else atomicAdd(&a.hist[q4[t]], 1u);
      }
    }
  };
  // the first nv of four codes to global memory
  auto put_codes = [&](uint16_t* co, const uint32_t* q4, int nv) {
    if (nv == 4) {
      sw_codes_out(co, q4);
    } else {
      for (int t = 0; t < nv; ++t) co[t] = (uint16_t)q4[t];
    }
  };

  const int n_iter = b1 - b0 + 4;
  if (tid < 32)
    for (int q = 0; q < kSwSlots - 1 && q < n_iter; ++q) issue(q);
  uint32_t phase = 0;  // bit q: parity of slot q
  for (int n = 0; n < n_iter; ++n) {
    const int v = b0 - 4 + n, c = v + 3, b = v;
    const int sl = n % kSwSlots;
    const unsigned char* slot = sm + L::kOffSlots + (size_t)sl * L::kSlot;
    const T* Cb = reinterpret_cast<const T*>(slot);  // [box plane][CW]
    const T* xs = reinterpret_cast<const T*>(slot + L::kCoarse);
    const uint16_t* cs = reinterpret_cast<const uint16_t*>(slot + L::kCoarse);
    const bool stepCD = v >= b0;
    const int j1 = 2 * b + 1;
    {
      int spins = 0;
      while (!mbar_try_wait(&bar[sl], (phase >> sl) & 1u)) {
        if (++spins > kWaitLimit) {
          s_timeout = 1;
          break;
        }
      }
      phase ^= 1u << sl;
    }
    if (role == 0) {
      // ---- B: E row c ---------------------------------------------------------
      if (c >= 0 && c < mc1) {
        T cz[4];
        sw_ld4(Cb + zb * CW + qe, cz);
        sw_st4(E + (c & 7) * CW + qe, cz[0], cz[1], cz[2], cz[3]);
        if (q_in) {
          T ca[4], cb[4], cc[4], cd[4], p4[4], r4[4];
          sw_ld4(Cb + 1 * CW + qe, ca);
          sw_ld4(Cb + 2 * CW + qe, cb);
          sw_ld4(Cb + 0 * CW + qe, cc);
          sw_ld4(Cb + 3 * CW + qe, cd);
#pragma unroll
          for (int t = 0; t < 4; ++t) p4[t] = interp_predict<T>(ca[t], cb[t], cc[t], cd[t], hb0, hc0, hd0, INTERP);
          const uint32_t row0 = base0 + (uint32_t)c * E20;
          if (COMP) {  // input points 2 col0 .. 2 col0 + 6 of row (io, 2c)
            T xa[4], xb[4], x4[4];
            sw_ld4(xs + xoffB, xa);
            sw_ld4(xs + xoffB + 4, xb);
            x4[0] = xa[0], x4[1] = xa[2], x4[2] = xb[0], x4[3] = xb[2];
            uint32_t q4[4];
            const bool own = q_own && c >= b0 && c < b1;
            quant4(x4, p4, own, q_nv, q4, r4);
            if (own) put_codes(a.codes + row0 + col0, q4, q_nv);
          } else {
            uint32_t k4[4];
            sw_codes_in(cs + ((row0 + (uint32_t)lo01) & 7u) + (col0 - lo01), k4);
            rec4(p4, k4, row0 + (uint32_t)col0, q_nv, r4);
          }
          sw_st4(E + (kSwRing + (c & 7)) * CW + qe, r4[0], r4[1], r4[2], r4[3]);
        }
      }
    } else if (role == 1 && stepCD && j1 < m1 && q_in) {
      // ---- C: pass 1 at j = 2b + 1 ----------------------------------------------
      const bool hb = j1 + 1 < m1, hc = j1 >= 3, hd = j1 + 3 < m1;
      const T* Eq = E + cq * kSwRing * CW + qe;
      T ea[4], eb[4], ec[4], ed[4], p4[4], r4[4];
      sw_ld4(Eq + (b & 7) * CW, ea);
      sw_ld4(Eq + ((b + 1) & 7) * CW, eb);
      sw_ld4(Eq + ((b + 7) & 7) * CW, ec);
      sw_ld4(Eq + ((b + 2) & 7) * CW, ed);
#pragma unroll
      for (int t = 0; t < 4; ++t) p4[t] = interp_predict<T>(ea[t], eb[t], ec[t], ed[t], hb, hc, hd, INTERP);
      const uint32_t row0 = base1 + (cq ? pl1 : 0u) + (uint32_t)b * E21;
      if (COMP) {  // input points 2 col0 .. of row (ie + cq, 2b + 1)
        T xa[4], xb[4], x4[4];
        sw_ld4(xs + xoffC, xa);
        sw_ld4(xs + xoffC + 4, xb);
        x4[0] = xa[0], x4[1] = xa[2], x4[2] = xb[0], x4[3] = xb[2];
        uint32_t q4[4];
        quant4(x4, p4, q_own, q_nv, q4, r4);
        if (q_own) put_codes(a.codes + row0 + col0, q4, q_nv);
      } else {
        uint32_t k4[4];
        sw_codes_in(cs + (1 + cq) * CR + ((row0 + (uint32_t)lo01) & 7u) + (col0 - lo01), k4);
        rec4(p4, k4, row0 + (uint32_t)col0, q_nv, r4);
      }
      sw_st4(E1 + ((b & 1) * 2 + cq) * CW + qe, r4[0], r4[1], r4[2], r4[3]);
    }
    __syncthreads();
    if (s_timeout) break;
    if (tid >= 3 * 32 && n + kSwSlots - 1 < n_iter) issue(n + kSwSlots - 1);  // the warp with the least B / C work
    if (!stepCD) continue;  // filling the ring
    // ---- D: pass 2 on rows (ie | io) x (2b | 2b + 1) ------------------------------
    const int j = 2 * b + tj;
    if (d_in && j < m1) {
      const T* Er = tj ? E1 + ((b & 1) * 2 + dq) * CW : E + (dq * kSwRing + (b & 7)) * CW;
      T ev[12];  // even columns kk - 4 .. kk + 7
      sw_ld4(Er + de - 4, ev);
      sw_ld4(Er + de, ev + 4);
      sw_ld4(Er + de + 4, ev + 8);
      // the interior formula; runs within three points of either end redo it
      // with the boundary rules
      T p4[4], o4[4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        p4[t] = interp_predict<T>(ev[4 + t], ev[5 + t], ev[3 + t], ev[6 + t], true, true, true, INTERP);
      if (d_edge) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int k = 2 * (kk + t) + 1;
          p4[t] = interp_predict<T>(ev[4 + t], ev[5 + t], ev[3 + t], ev[6 + t], k + 1 < m2, k >= 3, k + 3 < m2,
                                    INTERP);
        }
      }
      const uint32_t row0 = base2 + (dq ? pl2 : 0u) + (uint32_t)j * E22;
      if (COMP) {  // input points 2 kk .. 2 kk + 7 of row (i, j): the odd ones
        T xa[4], xb[4], x4[4];
        sw_ld4(xs + xoffD, xa);
        sw_ld4(xs + xoffD + 4, xb);
        x4[0] = xa[1], x4[1] = xa[3], x4[2] = xb[1], x4[3] = xb[3];
        uint32_t q4[4];
        quant4(x4, p4, true, d_nv, q4, o4);
        put_codes(a.codes + row0 + kk, q4, d_nv);
      } else {
        uint32_t k4[4];
        sw_codes_in(cs + (3 + dw) * CR + ((row0 + (uint32_t)lo2) & 7u) + 4 * rr, k4);
        rec4(p4, k4, row0 + (uint32_t)kk, d_nv, o4);
      }
      if (d.write_out) {
        T* dst = a.Rout + ((uint32_t)(ie + dq) * d.rs0 + (uint32_t)j * d.rs1 + 2u * (uint32_t)kk);
        if (d_full) {
          sw_st4(dst, ev[4], o4[0], ev[5], o4[1]);
          sw_st4(dst + 4, ev[6], o4[2], ev[7], o4[3]);
        } else {
          const T v8[8] = {ev[4], o4[0], ev[5], o4[1], ev[6], o4[2], ev[7], o4[3]};
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (2 * kk + t < m2) dst[t] = v8[t];
        }
      }
    }
  }

  // ---- flush the per-CTA counters
  if (bad) s_bad = 1;
  __syncthreads();
  if (s_timeout) {
    // give copies still in flight a last bounded chance to land
    for (int q = 0; q < kSwSlots; ++q) {
      int spins = 0;
      while (!mbar_try_wait(&bar[q], (phase >> q) & 1u) && ++spins < kWaitLimit) {
      }
    }
    if (tid == 0) atomicOr(&st->flags, kFlagTimeout);
  }
  if (COMP) {
    for (int i = tid; i < kHistWin; i += kSwThreads)
      if (hwin[i]) atomicAdd(&a.hist[hlo + i], hwin[i]);
  } else if (tid == 0 && s_bad) {
    atomicOr(&st->flags, kFlagCorrupt);
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

template <typename T>
static bool sweep_map(CUtensorMap* map, const T* base, int m0, int m1, int m2, unsigned long long s0,
                      unsigned long long s1, int b0, int b1, int b2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)m2, (cuuint64_t)m1, (cuuint64_t)m0};
  const cuuint64_t strides[2] = {(cuuint64_t)s1 * sizeof(T), (cuuint64_t)s0 * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)b2, (cuuint32_t)b1, (cuuint32_t)b0};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return enc(map, dt, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, bool COMP>
int launch_sweep(const Plan& pl, int k, const LevelArgs<T>& a, bool to_field, cudaStream_t s) {
  using S = SwShape<T>;
  SweepDesc d;
  memset(&d, 0, sizeof(d));
  const unsigned long long* m = pl.gm[k];
  const unsigned long long* mc = pl.gm[k + 1];
  d.m0 = (int)m[1];
  d.m1 = (int)m[2];
  d.m2 = (int)m[3];
  d.mc0 = (int)mc[1];
  d.mc1 = (int)mc[2];
  d.mc2 = (int)mc[3];
  d.nks = (uint32_t)((d.m2 + kSwKW - 1) / kSwKW);
  d.njs = (uint32_t)((d.mc1 + kSwJS - 1) / kSwJS);
  const unsigned long long items = (unsigned long long)d.mc0 * d.njs * d.nks;
  if (items == 0 || items > 0x7fffffffull) return SZ3G_E_INVAL;
  d.item0 = 0;
  d.nitems = (uint32_t)items;
  int p = m[1] > 1 ? 0 : 1;
  int interp = SZ3G_LINEAR;
  for (int i = 0; i < pl.n_pass; ++i) {
    const PassDesc& pd = pl.pass[i];
    if (pd.grid != k) continue;
    d.off[p] = (uint32_t)pd.off;
    d.E1[p] = (uint32_t)pd.E[2];
    d.E2[p] = (uint32_t)pd.E[3];
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
  d.cpl = d.m0 > 1 ? 4 : 1;
  d.xpl = d.m0 > 1 ? 2 : 1;
  CUtensorMap tmc, tmx, tmx1;
  memset(&tmc, 0, sizeof(tmc));
  memset(&tmx, 0, sizeof(tmx));
  memset(&tmx1, 0, sizeof(tmx1));
  bool ok = sweep_map<T>(&tmc, a.Rc, d.mc0, d.mc1, d.mc2, mc[3] * mc[2], mc[3], d.cpl, 1, S::kCW);
  if (COMP) {
    ok = ok && sweep_map<T>(&tmx, a.x, d.m0, d.m1, d.m2, a.xs[0], a.xs[1], d.xpl, 2, S::kXH);
    ok = ok && sweep_map<T>(&tmx1, a.x, d.m0, d.m1, d.m2, a.xs[0], a.xs[1], 1, 1, S::kXH);
  }
  if (!ok) return SZ3G_E_CUDA;
  const size_t smem = SwLayout<T, COMP>::kBytes;
  auto kern = interp == SZ3G_CUBIC ? sweep_kernel<T, COMP, SZ3G_CUBIC> : sweep_kernel<T, COMP, SZ3G_LINEAR>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SZ3G_E_CUDA;
  SZ3G_LAUNCH(COMP ? kKLevelQuantize : kKLevelRecover, s,
              kern<<<(unsigned)items, kSwThreads, smem, s>>>(d, a, tmc, tmx, tmx1));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

template int launch_sweep<float, true>(const Plan&, int, const LevelArgs<float>&, bool, cudaStream_t);
template int launch_sweep<float, false>(const Plan&, int, const LevelArgs<float>&, bool, cudaStream_t);
template int launch_sweep<double, true>(const Plan&, int, const LevelArgs<double>&, bool, cudaStream_t);
template int launch_sweep<double, false>(const Plan&, int, const LevelArgs<double>&, bool, cudaStream_t);

}  // namespace sz3g
