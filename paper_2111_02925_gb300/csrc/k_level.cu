// k_level.cu -- fused level kernels for fields of rank <= 3 (coordinates
// padded to 3 axes).
//
// level_kernel: one launch per grid G_k that is larger than the coarse group.
// A persistent CTA walks the tiles of G_k; for each tile it stages in shared
// memory a box V holding the input values (compress) and the coarse
// reconstruction R_{k+1} (all-even points), runs every pass of the level on the
// box (the tile plus the halo points whose reconstruction later passes read),
// writes the codes of the tile's own points in traversal order, and writes the
// tile of R_k that the next finer level reads.  Decompress is the same walk
// with codes read instead of computed.
//
// Halos: the last pass reads neighbours at +-1 and +-3 along its axis; those
// points belong to earlier passes, so a pass p is evaluated on the tile
// extended by 2 (low) / 3 (high) along the axes of the passes after p, and the
// first pass reads coarse points up to 3 away along its own axis, so the box
// spans the tile plus that halo on every refined axis.  It is staged with
// cp.async copies (all in flight at once), only at the points some pass reads.
// Halo points are evaluated redundantly with the same arithmetic and never
// written.
//
// coarse_kernel: one CTA evaluates every level whose grid has at most
// kCoarseMax points, in traversal order, on a shared-memory copy of the
// coarsest such grid G_kc (strided in place), then writes R_kc.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <functional>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "internal.cuh"
#include "level_common.cuh"

namespace sz3g {

constexpr int kLevelThreads = 256;

struct LevelDesc {
  int k, P, interp, write_out;
  int ax[3];      // axis of pass p
  int pos[3];     // order position of axis d, -1 for a unit axis
  int m[3];       // extents of G_k
  int B[3];       // tile extents
  int nt[3];      // tiles per axis
  int vext[3], vlo[3];  // box extent and low halo per axis
  uint32_t ntiles;
  uint32_t off[3];      // first code of each pass
  uint32_t E[3][3];     // pass lattice extents
  uint32_t xs[3];       // input stride of one G_k step
  uint32_t rs[3];       // strides of the output grid (R_k or the field)
  uint32_t rcs[3];      // strides of R_{k+1} (rcs[2] == 1)
  uint32_t chunk, nsub;
  // tensor-copy staging
  int xb0_tile;         // input box spans only the tile along axis 0
  int cw[3];            // coarse box extents (compact), cw[2] a multiple of 16 bytes
  int calign;           // coarse box start alignment along axis 2 (elements)
  int fast012;          // the specialised 4 x 16 x 56 interior tile applies
  uint32_t smem_c, smem_h, smem_bar;  // byte offsets of the coarse box, histogram, barrier
};


__device__ __forceinline__ int floor_to(int v, int a) {  // a power of two
  return v & ~(a - 1);
}

constexpr int kUnroll = 4;  // rows a warp works on at once

struct TileGeo {
  int A0, A1, A2, E0, E1, E2, lo0, lo1, lo2;
};

// One pass of a level on the staged box V.  Warps take the rows of the pass
// region (tile on the axes refined so far, tile + halo on later ones); lanes
// run along axis 2.  INTERIOR: every neighbour at +-1 and +-3 exists, so the
// prediction needs no boundary cases.
template <typename T, bool COMP, int INTERP, bool INTERIOR>
__device__ __forceinline__ void level_pass(const LevelDesc& d, const LevelArgs<T>& a, T* V, uint32_t* hwin,
                                           const TileGeo& g, int p, T ebT, T ebr, int hlo, unsigned int& my_nz,
                                           bool& my_bad) {
  constexpr int kWarps = kLevelThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ve2 = d.vext[2], vs0 = d.vext[1] * d.vext[2];
  const int pos0 = d.pos[0], pos1 = d.pos[1], pos2 = d.pos[2];
  const int radius = a.radius;
  const int ax = d.ax[p];
  int s0[3], sp[3], cnt[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int pq = q == 0 ? pos0 : (q == 1 ? pos1 : pos2);
    const int Aq = q == 0 ? g.A0 : (q == 1 ? g.A1 : g.A2);
    const int Eq = q == 0 ? g.E0 : (q == 1 ? g.E1 : g.E2);
    const bool ext = pq > p;  // axis refined by a later pass: halo of 2 below, 3 above
    const int rlo = ext ? max(Aq - 2, 0) : Aq;
    const int rhi = ext ? min(Aq + d.B[q] + 3, d.m[q]) : Eq;
    int st0 = rlo, stp = 1;
    if (q == ax) {
      st0 = rlo | 1;
      stp = 2;
    } else if (ext || pq < 0) {
      st0 = (rlo + 1) & ~1;
      stp = 2;
    }
    s0[q] = st0;
    sp[q] = stp;
    cnt[q] = rhi > st0 ? (rhi - st0 + stp - 1) / stp : 0;
  }
  const int vst = ax == 2 ? 1 : (ax == 1 ? ve2 : vs0);
  const int n_ax = d.m[ax];
  // lattice coordinate per axis: c >> 1 on the pass axis and on later /
  // unit axes, c on axes refined earlier in this level
  const int sh0 = (pos0 >= 0 && pos0 < p) ? 0 : 1, sh1 = (pos1 >= 0 && pos1 < p) ? 0 : 1,
            sh2 = (pos2 >= 0 && pos2 < p) ? 0 : 1;
  const uint32_t PE1 = d.E[p][1], PE2 = d.E[p][2];
  const uint32_t poff = d.off[p];
  const int rows = cnt[0] * cnt[1];
  const int c2first = s0[2], c2step = sp[2], n2 = cnt[2];
  int j0 = cnt[1] ? warp / cnt[1] : 0, j1 = cnt[1] ? warp - j0 * cnt[1] : 0;
  for (int r0 = warp; r0 < rows; r0 += kWarps * kUnroll) {
    int vrow[kUnroll];
    uint32_t crow[kUnroll];
    bool orow[kUnroll], rok[kUnroll];
    int irow[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {  // rows r0 + u * kWarps
      const int c0 = s0[0] + sp[0] * j0, c1 = s0[1] + sp[1] * j1;
      rok[u] = r0 + u * kWarps < rows;
      vrow[u] = (c0 - g.lo0) * vs0 + (c1 - g.lo1) * ve2 - g.lo2;
      crow[u] = poff + (((uint32_t)c0 >> sh0) * PE1 + ((uint32_t)c1 >> sh1)) * PE2;
      orow[u] = c0 >= g.A0 && c0 < g.E0 && c1 >= g.A1 && c1 < g.E1;
      irow[u] = ax == 0 ? c0 : c1;
      j1 += kWarps;
      while (j1 >= cnt[1] && cnt[1] > 0) {
        j1 -= cnt[1];
        ++j0;
      }
    }
    for (int j2b = 0; j2b < n2; j2b += 32) {
      const int j2 = j2b + lane;
      const int c2 = c2first + c2step * j2;
      const bool own2 = c2 >= g.A2 && c2 < g.E2;
      T pred[kUnroll], xv[kUnroll];
      // phase 1: loads and predictions
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        pred[u] = T(0);
        xv[u] = T(0);
        if (rok[u] && j2 < n2) {
          const int v = vrow[u] + c2;
          if (INTERIOR) {
            const T va = V[v - vst], vb = V[v + vst], vc = V[v - 3 * vst], vd = V[v + 3 * vst];
            pred[u] = interp_predict<T>(va, vb, vc, vd, true, true, true, INTERP);
          } else {
            const int i = ax == 2 ? c2 : irow[u];
            const bool hb = i + 1 < n_ax, hc = i >= 3, hd = i + 3 < n_ax;
            const T va = V[v - vst];
            const T vb = hb ? V[v + vst] : T(0);
            const T vc = hc ? V[v - 3 * vst] : T(0);
            const T vd = hd ? V[v + 3 * vst] : T(0);
            pred[u] = interp_predict<T>(va, vb, vc, vd, hb, hc, hd, INTERP);
          }
          if (COMP) xv[u] = V[v];
        }
      }
      // phase 2: quantize / recover, stores
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (!(rok[u] && j2 < n2)) continue;
        const int v = vrow[u] + c2;
        const uint32_t ci = crow[u] + ((uint32_t)c2 >> sh2);
        if (COMP) {
          T rr;
          const uint32_t code = quantize_point<T>(xv[u], pred[u], ebT, ebr, radius, rr);
          V[v] = rr;
          if (orow[u] && own2) {
            a.codes[ci] = (uint16_t)code;
            if (code == 0) {  // unpredictable: also where a non-finite input ends up
              ++my_nz;
              my_bad |= !isfinite(xv[u]);
            }
            const int b = (int)code - hlo;
            if (b >= 0 && b < kHistWin) atomicAdd(&hwin[b], 1u);
            else atomicAdd(&a.hist[code], 1u);
          }
        } else {
          const uint32_t code = a.codes[ci];
          T rr;
          if (code == 0) {
            const unsigned long long rk = rank_of_zero(a.codes, ci, d.chunk, d.nsub, a.zunit);
            if (rk < a.n_unpred) {
              rr = a.unpred[rk];
            } else {
              rr = T(0);
              my_bad = true;
            }
          } else if (code >= 2u * (uint32_t)radius) {
            rr = T(0);
            my_bad = true;
          } else {
            rr = recover_point<T>(pred[u], code, radius, ebT);
          }
          V[v] = rr;
        }
      }
    }
  }
}

// Region of one pass inside the box for a tile away from every grid face, in
// box coordinates (the same for all such tiles): first, step and count per
// axis; the shift that maps a coordinate to its lattice coordinate; the
// ownership window; the box stride along the pass axis.
struct PassRegion {
  int f[3], s[3], n[3];
  int sh[3];
  int olo[3], ohi[3];  // owned box coordinates [olo, ohi)
  int vst;
  uint32_t E1, E2, off;
};

__device__ void make_regions(const LevelDesc& d, PassRegion* R) {
  for (int p = 0; p < d.P; ++p) {
    PassRegion& g = R[p];
    const int ax = d.ax[p];
    for (int q = 0; q < 3; ++q) {
      const int pq = d.pos[q];
      const bool ext = pq > p;
      const int rlo = ext ? -2 : 0, rhi = ext ? d.B[q] + 3 : d.B[q];  // relative to the tile start (even)
      int st0 = rlo, stp = 1;
      if (q == ax) {
        st0 = rlo | 1;
        stp = 2;
      } else if (ext || pq < 0) {
        st0 = (rlo + 1) & ~1;
        stp = 2;
      }
      g.f[q] = st0 + d.vlo[q];
      g.s[q] = stp;
      g.n[q] = rhi > st0 ? (rhi - st0 + stp - 1) / stp : 0;
      g.sh[q] = (pq >= 0 && pq < p) ? 0 : 1;
      g.olo[q] = d.vlo[q];
      g.ohi[q] = d.vlo[q] + d.B[q];
    }
    g.vst = ax == 2 ? 1 : (ax == 1 ? d.vext[2] : d.vext[1] * d.vext[2]);
    g.E1 = d.E[p][1];
    g.E2 = d.E[p][2];
    g.off = d.off[p];
  }
}

// One pass on a tile away from every grid face: every neighbour at +-1 and
// +-3 exists.  Each warp takes a contiguous run of rows of the region, each
// lane a fixed column; two rows are loaded before either is stored.
template <typename T, bool COMP, int INTERP>
__device__ __forceinline__ void level_pass_interior(const LevelDesc& d, const LevelArgs<T>& a, T* V, uint32_t* hwin,
                                                    const PassRegion& g, int A0, int A1, int A2, T ebT, T ebr,
                                                    int hlo, unsigned int& my_nz, bool& my_bad) {
  constexpr int kWarps = kLevelThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ve2 = d.vext[2], vs0 = d.vext[1] * ve2;
  const int radius = a.radius;
  const int vst = g.vst;
  const uint32_t tilebase =
      g.off + (((uint32_t)A0 >> g.sh[0]) * g.E1 + ((uint32_t)A1 >> g.sh[1])) * g.E2 + ((uint32_t)A2 >> g.sh[2]);
  const int rows = g.n[0] * g.n[1];
  const int rb = (rows * warp) / kWarps, re = (rows * (warp + 1)) / kWarps;
  if (rb >= re) return;
  for (int seg = 0; seg < g.n[2]; seg += 32) {
    const int j2 = seg + lane;
    const bool col = j2 < g.n[2];
    const int b2 = g.f[2] + g.s[2] * j2;
    const int rel2 = b2 - d.vlo[2];
    const uint32_t cl2 = (uint32_t)(rel2 >> g.sh[2]);
    const bool own2 = b2 >= g.olo[2] && b2 < g.ohi[2];
    int j0 = rb / g.n[1], j1 = rb - j0 * g.n[1];
    for (int r = rb; r < re; r += 2) {
      const bool two = r + 1 < re;
      int v[2];
      uint32_t ci[2];
      bool own[2];
      T pred[2], xv[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int b0 = g.f[0] + g.s[0] * j0, b1 = g.f[1] + g.s[1] * j1;
        const int rel0 = b0 - d.vlo[0], rel1 = b1 - d.vlo[1];
        v[u] = b0 * vs0 + b1 * ve2 + b2;
        ci[u] = tilebase + ((uint32_t)(rel0 >> g.sh[0]) * g.E1 + (uint32_t)(rel1 >> g.sh[1])) * g.E2 + cl2;
        own[u] = own2 && b0 >= g.olo[0] && b0 < g.ohi[0] && b1 >= g.olo[1] && b1 < g.ohi[1];
        if (++j1 == g.n[1]) {
          j1 = 0;
          ++j0;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        pred[u] = T(0);
        xv[u] = T(0);
        if (col && (u == 0 || two)) {
          const T* w = V + v[u];
          pred[u] = interp_predict<T>(w[-vst], w[vst], w[-3 * vst], w[3 * vst], true, true, true, INTERP);
          if (COMP) xv[u] = w[0];
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!col || !(u == 0 || two)) continue;
        if (COMP) {
          T rr;
          const uint32_t code = quantize_point<T>(xv[u], pred[u], ebT, ebr, radius, rr);
          V[v[u]] = rr;
          if (own[u]) {
            a.codes[ci[u]] = (uint16_t)code;
            if (code == 0) {  // unpredictable: also where a non-finite input ends up
              ++my_nz;
              my_bad |= !isfinite(xv[u]);
            }
            const int bn = (int)code - hlo;
            if (bn >= 0 && bn < kHistWin) atomicAdd(&hwin[bn], 1u);
            else atomicAdd(&a.hist[code], 1u);
          }
        } else {
          const uint32_t code = a.codes[ci[u]];
          T rr;
          if (code == 0) {
            const unsigned long long rk = rank_of_zero(a.codes, ci[u], d.chunk, d.nsub, a.zunit);
            if (rk < a.n_unpred) {
              rr = a.unpred[rk];
            } else {
              rr = T(0);
              my_bad = true;
            }
          } else if (code >= 2u * (uint32_t)radius) {
            rr = T(0);
            my_bad = true;
          } else {
            rr = recover_point<T>(pred[u], code, radius, ebT);
          }
          V[v[u]] = rr;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Specialised interior tile for 3-D grids refined in axis order (0, 1, 2) with
// 4 x 16 x 56 tiles: the box (9 x 21 x 64, low halos 2, 2, 4), the pass
// regions, strides and lattice shifts are compile-time constants, so each
// point costs its loads, the predictor, the quantizer and its stores.
// ---------------------------------------------------------------------------
constexpr int kT0 = 4, kT1 = 16, kT2 = 56;                 // tile
constexpr int kX0 = kT0 + 5, kX1 = kT1 + 5, kX2 = kT2 + 8;  // box
constexpr int kXS1 = kX2, kXS0 = kX1 * kX2;                 // box strides
constexpr int kH0 = 2, kH1 = 2, kH2 = 4;                    // low halos

template <typename T, bool COMP, int INTERP, int PASS, bool EDGE2>
__device__ __forceinline__ void pass012(const LevelDesc& d, const LevelArgs<T>& a, T* V, uint32_t* hwin, int A0,
                                        int A1, int A2, int E2, T ebT, T ebr, int hlo, unsigned int& my_nz,
                                        bool& my_bad) {
  // region of the pass in box coordinates: first, step, count per axis
  constexpr int F0 = PASS == 0 ? kH0 + 1 : kH0, S0 = PASS == 0 ? 2 : 1, N0 = PASS == 0 ? kT0 / 2 : kT0;
  constexpr int F1 = PASS == 0 ? 0 : (PASS == 1 ? kH1 + 1 : kH1), S1 = PASS == 2 ? 1 : 2;
  constexpr int N1 = PASS == 0 ? (kT1 + 6) / 2 : (PASS == 1 ? kT1 / 2 : kT1);
  constexpr int F2 = PASS == 2 ? kH2 + 1 : kH2 - 2, S2 = 2, N2 = PASS == 2 ? kT2 / 2 : (kT2 + 6) / 2;
  constexpr int VST = PASS == 0 ? kXS0 : (PASS == 1 ? kXS1 : 1);
  constexpr int SH0 = PASS == 0 ? 1 : 0, SH1 = PASS == 2 ? 0 : 1;  // lattice shifts (axis 2: 1)
  constexpr int ROWS = N0 * N1;
  constexpr int kWarps = kLevelThreads / 32;
  constexpr int KMAX = (ROWS + kWarps - 1) / kWarps;
  static_assert(N2 <= 32, "one lane per column");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int radius = a.radius;
  const uint32_t E1 = d.E[PASS][1], E2L = d.E[PASS][2];
  const uint32_t tilebase =
      d.off[PASS] + (((uint32_t)A0 >> SH0) * E1 + ((uint32_t)A1 >> SH1)) * E2L + ((uint32_t)A2 >> 1);
  const int b2 = F2 + S2 * lane;
  const int c2 = A2 - kH2 + b2;  // grid coordinate of the column
  const uint32_t cl2 = (uint32_t)((b2 - kH2) >> 1);
  const bool own2 = b2 >= kH2 && c2 < E2;
  // EDGE2: the tile touches a face along axis 2: columns past the grid drop
  // out, and the axis-2 pass needs its boundary cases
  const int m2 = d.m[2];
  bool col = lane < N2;
  if (EDGE2) col = col && c2 >= 0 && (PASS == 2 ? c2 < E2 : c2 < m2);
  const bool hb = !EDGE2 || PASS != 2 || c2 + 1 < m2, hc = !EDGE2 || PASS != 2 || c2 >= 3,
             hd = !EDGE2 || PASS != 2 || c2 + 3 < m2;
  if (!col) return;
#pragma unroll
  for (int k = 0; k < KMAX; k += 2) {
    int v[2];
    uint32_t ci[2];
    bool own[2], ok[2];
    T pred[2], xv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = warp + kWarps * (k + u);
      ok[u] = k + u < KMAX && r < ROWS;
      const int j0 = r / N1, j1 = r - (r / N1) * N1;
      const int b0 = F0 + S0 * j0, b1 = F1 + S1 * j1;
      v[u] = b0 * kXS0 + b1 * kXS1 + b2;
      ci[u] = tilebase + ((uint32_t)((b0 - kH0) >> SH0) * E1 + (uint32_t)((b1 - kH1) >> SH1)) * E2L + cl2;
      own[u] = own2 && b0 >= kH0 && b0 < kH0 + kT0 && b1 >= kH1 && b1 < kH1 + kT1;
      pred[u] = T(0);
      xv[u] = T(0);
      if (ok[u]) {
        const T* w = V + v[u];
        if (EDGE2 && PASS == 2) {
          const T vb = hb ? w[VST] : T(0), vc = hc ? w[-3 * VST] : T(0), vd = hd ? w[3 * VST] : T(0);
          pred[u] = interp_predict<T>(w[-VST], vb, vc, vd, hb, hc, hd, INTERP);
        } else {
          pred[u] = interp_predict<T>(w[-VST], w[VST], w[-3 * VST], w[3 * VST], true, true, true, INTERP);
        }
        if (COMP) xv[u] = w[0];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!ok[u]) continue;
      if (COMP) {
        T rr;
        const uint32_t code = quantize_point<T>(xv[u], pred[u], ebT, ebr, radius, rr);
        V[v[u]] = rr;
        if (own[u]) {
          a.codes[ci[u]] = (uint16_t)code;
          if (code == 0) {
            ++my_nz;
            my_bad |= !isfinite(xv[u]);
          }
          const int bn = (int)code - hlo;
          if (bn >= 0 && bn < kHistWin) atomicAdd(&hwin[bn], 1u);
          else atomicAdd(&a.hist[code], 1u);
        }
      } else {
        const uint32_t code = a.codes[ci[u]];
        T rr;
        if (code == 0) {
          const unsigned long long rk = rank_of_zero(a.codes, ci[u], d.chunk, d.nsub, a.zunit);
          if (rk < a.n_unpred) {
            rr = a.unpred[rk];
          } else {
            rr = T(0);
            my_bad = true;
          }
        } else if (code >= 2u * (uint32_t)radius) {
          rr = T(0);
          my_bad = true;
        } else {
          rr = recover_point<T>(pred[u], code, radius, ebT);
        }
        V[v[u]] = rr;
      }
    }
  }
}

// Coarse values of a specialised interior tile from the coarse box C to the
// all-even positions of V (every one lies inside the grid).
template <typename T>
__device__ __forceinline__ void scatter012(const LevelDesc& d, T* V, const T* C, int coff2) {
  constexpr int NI0 = (kX0 + 1) / 2, NI1 = (kX1 + 1) / 2, NI2 = kX2 / 2;  // 5, 11, 32
  constexpr int TOT = NI0 * NI1 * NI2;
  const int cw2 = d.cw[2], cst0 = d.cw[1] * d.cw[2];
#pragma unroll
  for (int k = 0; k < (TOT + kLevelThreads - 1) / kLevelThreads; ++k) {
    const int e = threadIdx.x + kLevelThreads * k;
    if (e < TOT) {
      const int i2 = e % NI2, i1 = (e / NI2) % NI1, i0 = e / (NI2 * NI1);
      V[2 * i0 * kXS0 + 2 * i1 * kXS1 + 2 * i2] = C[i0 * cst0 + i1 * cw2 + i2 + coff2];
    }
  }
}

// The owned 4 x 16 x (E2 - A2) tile of V to the output grid.
template <typename T>
__device__ __forceinline__ void write012(const LevelDesc& d, const LevelArgs<T>& a, const T* V, int A0, int A1,
                                         int A2, int E2) {
  constexpr int kWarps = kLevelThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w2 = E2 - A2;
#pragma unroll
  for (int k = 0; k < kT0 * kT1 / kWarps; ++k) {
    const int r = warp + kWarps * k;
    const int q0 = r / kT1, q1 = r % kT1;
    T* dst = a.Rout + ((uint32_t)(A0 + q0) * d.rs[0] + (uint32_t)(A1 + q1) * d.rs[1] + (uint32_t)A2);
    const T* src = V + (q0 + kH0) * kXS0 + (q1 + kH1) * kXS1 + kH2;
#pragma unroll
    for (int q2 = lane; q2 < kT2; q2 += 32)
      if (q2 < w2) dst[q2] = src[q2];
  }
}

// Work on a box region is distributed as (row, 32-wide segment) items over the
// warps of the CTA: lanes run along axis 2, the contiguous axis.  A pass
// handles kUnroll items per warp at a time: all their loads are issued before
// any result is stored (the points a pass writes are never its own inputs).

// Per-CTA state of the level kernels across the tiles a CTA processes.
template <typename T>
struct LevelCtx {
  T* V;
  T* C;
  uint32_t* hwin;
  uint64_t* bar;
  PassRegion* reg;
  int* s_timeout;
  uint32_t phase;
  unsigned int my_nz;
  bool my_bad;
  T ebT, ebr;
  int hlo;
};

// One tile of a grid level: stage its box, run the level's passes, write the
// output tile.  Returns false when a bounded wait gave up.
template <typename T, bool COMP, bool TMA, int INTERP>
__device__ __forceinline__ bool level_tile(const LevelDesc& d, const LevelArgs<T>& a, const CUtensorMap* tmx,
                                           const CUtensorMap* tmc, uint32_t tile, LevelCtx<T>& c) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kLevelThreads / 32;
  T* V = c.V;
  T* C = c.C;
  uint32_t* hwin = c.hwin;
  uint64_t* bar = c.bar;
  const T ebT = c.ebT, ebr = c.ebr;
  const int hlo = c.hlo;
  const int ve1 = d.vext[1], ve2 = d.vext[2];
  const int vs0 = ve1 * ve2;
  const int m0 = d.m[0], m1 = d.m[1], m2 = d.m[2];
  const int pos0 = d.pos[0], pos1 = d.pos[1], pos2 = d.pos[2];
  (void)tid;
  (void)C;
  (void)bar;
  const int t2 = (int)(tile % (uint32_t)d.nt[2]);
  const int t1 = (int)((tile / (uint32_t)d.nt[2]) % (uint32_t)d.nt[1]);
  const int t0 = (int)(tile / ((uint32_t)d.nt[2] * (uint32_t)d.nt[1]));
  const int A0 = t0 * d.B[0], A1 = t1 * d.B[1], A2 = t2 * d.B[2];
  const int E0 = min(A0 + d.B[0], m0), E1 = min(A1 + d.B[1], m1), E2 = min(A2 + d.B[2], m2);
  const int lo0 = A0 - d.vlo[0], lo1 = A1 - d.vlo[1], lo2 = A2 - d.vlo[2];

  if (TMA) {
    // ---- stage with two tensor copies: the input box (compress) and the
    //      coarse box of R_{k+1}; then spread the coarse values over V
    const int cs0 = lo0 >> 1, cs1 = lo1 >> 1, cs2 = floor_to(lo2 >> 1, d.calign);
    if (tid == 0) {
      fence_proxy_async_smem();  // earlier generic writes to V / C precede the copies
      const uint32_t cbytes = (uint32_t)(d.cw[0] * d.cw[1] * d.cw[2] * (int)sizeof(T));
      const int xb0 = d.xb0_tile ? d.B[0] : d.vext[0];
      const uint32_t xbytes = COMP ? (uint32_t)(xb0 * vs0 * (int)sizeof(T)) : 0u;
      mbar_expect_tx(bar, cbytes + xbytes);
      if (COMP) tma_load_3d(V + (d.xb0_tile ? d.vlo[0] * vs0 : 0), tmx, lo2, lo1, d.xb0_tile ? A0 : lo0, bar);
      tma_load_3d(C, tmc, cs2, cs1, cs0, bar);
    }
    int spins = 0;
    while (!mbar_try_wait(bar, c.phase)) {
      if (++spins > kWaitLimit) {
        *c.s_timeout = 1;
        break;
      }
    }
    c.phase ^= 1u;
    __syncthreads();
    if (*c.s_timeout) return false;
    const bool fast = d.fast012 && (A0 >= 6 && A0 + kT0 + 6 <= m0) && (A1 >= 6 && A1 + kT1 + 6 <= m1);
    if (fast) {
      scatter012<T>(d, V, C, (lo2 >> 1) - cs2);
      __syncthreads();
    } else {
    // coarse values to the all-even positions of V
    const int i0a = (max(lo0, 0) + 1) >> 1, i0b = min(lo0 + d.vext[0] - 1, m0 - 1) >> 1;
    const int i1a = (max(lo1, 0) + 1) >> 1, i1b = min(lo1 + ve1 - 1, m1 - 1) >> 1;
    const int i2a = (max(lo2, 0) + 1) >> 1, i2b = min(lo2 + ve2 - 1, m2 - 1) >> 1;
    const int n2 = i2b - i2a + 1, n1 = i1b - i1a + 1, n0 = i0b - i0a + 1;
    const int cst1 = d.cw[2], cst0 = d.cw[1] * d.cw[2];
    if (n0 > 0 && n1 > 0 && n2 > 0) {
      const int nseg = (n2 + 31) >> 5;
      const int items = n0 * n1 * nseg;
      for (int it = warp; it < items; it += kWarps) {
        const int r = it / nseg, seg = it - r * nseg;
        const int q0 = r / n1, q1 = r - q0 * n1;
        const int q2 = seg * 32 + lane;
        if (q2 >= n2) continue;
        const int i0 = i0a + q0, i1 = i1a + q1, i2 = i2a + q2;
        V[(2 * i0 - lo0) * vs0 + (2 * i1 - lo1) * ve2 + (2 * i2 - lo2)] =
            C[(i0 - cs0) * cst0 + (i1 - cs1) * cst1 + (i2 - cs2)];
      }
    }
    __syncthreads();
    }
  } else {
    // ---- stage with element copies, only the points some pass reads
    const int nseg = (ve2 + 31) >> 5;
    const int items = d.vext[0] * ve1 * nseg;
    for (int it = warp; it < items; it += kWarps) {
      const int r = it / nseg, seg = it - r * nseg;
      const int b0 = r / ve1, b1 = r - b0 * ve1;
      const int c0 = lo0 + b0, c1 = lo1 + b1;
      if (c0 < 0 || c1 < 0 || c0 >= m0 || c1 >= m1) continue;
      const int b2 = seg * 32 + lane;
      const int c2 = lo2 + b2;
      if (b2 >= ve2 || c2 < 0 || c2 >= m2) continue;
      T* vp = V + r * ve2 + b2;
      const bool odd01 = ((c0 | c1) & 1) != 0;
      if (!odd01 && !(c2 & 1)) {
        cp_async_elem(vp, a.Rc + ((uint32_t)(c0 >> 1) * d.rcs[0] + (uint32_t)(c1 >> 1) * d.rcs[1] +
                                  (uint32_t)(c2 >> 1)));
      } else if (COMP) {
        // evaluated by pass p = the latest axis (in order) with an odd
        // coordinate, on the tile range of the axes up to p
        int p = -1;
        if ((c0 & 1) && pos0 > p) p = pos0;
        if ((c1 & 1) && pos1 > p) p = pos1;
        if ((c2 & 1) && pos2 > p) p = pos2;
        bool need = true;
        if (pos0 >= 0 && pos0 <= p && (c0 < A0 || c0 >= E0)) need = false;
        if (pos1 >= 0 && pos1 <= p && (c1 < A1 || c1 >= E1)) need = false;
        if (pos2 >= 0 && pos2 <= p && (c2 < A2 || c2 >= E2)) need = false;
        if (need) cp_async_elem(vp, a.x + ((uint32_t)c0 * d.xs[0] + (uint32_t)c1 * d.xs[1] + (uint32_t)c2 * d.xs[2]));
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }

  // ---- the passes of the level (tiles away from every grid face take the
  //      branch-free interior form)
  const bool interior = (pos0 < 0 || (A0 >= 6 && A0 + d.B[0] + 6 <= m0)) &&
                        (pos1 < 0 || (A1 >= 6 && A1 + d.B[1] + 6 <= m1)) &&
                        (pos2 < 0 || (A2 >= 6 && A2 + d.B[2] + 6 <= m2));
  // the specialised tile: interior along axes 0 and 1; a face along axis 2
  // only changes the columns and the axis-2 pass
  const bool fast = d.fast012 && (A0 >= 6 && A0 + kT0 + 6 <= m0) && (A1 >= 6 && A1 + kT1 + 6 <= m1);
  const bool edge2 = !(A2 >= 6 && A2 + kT2 + 6 <= m2);
  if (fast && !edge2) {
    pass012<T, COMP, INTERP, 0, false>(d, a, V, hwin, A0, A1, A2, E2, ebT, ebr, hlo, c.my_nz, c.my_bad);
    __syncthreads();
    pass012<T, COMP, INTERP, 1, false>(d, a, V, hwin, A0, A1, A2, E2, ebT, ebr, hlo, c.my_nz, c.my_bad);
    __syncthreads();
    pass012<T, COMP, INTERP, 2, false>(d, a, V, hwin, A0, A1, A2, E2, ebT, ebr, hlo, c.my_nz, c.my_bad);
    __syncthreads();
  } else if (fast) {
    pass012<T, COMP, INTERP, 0, true>(d, a, V, hwin, A0, A1, A2, E2, ebT, ebr, hlo, c.my_nz, c.my_bad);
    __syncthreads();
    pass012<T, COMP, INTERP, 1, true>(d, a, V, hwin, A0, A1, A2, E2, ebT, ebr, hlo, c.my_nz, c.my_bad);
    __syncthreads();
    pass012<T, COMP, INTERP, 2, true>(d, a, V, hwin, A0, A1, A2, E2, ebT, ebr, hlo, c.my_nz, c.my_bad);
    __syncthreads();
  } else {
    for (int p = 0; p < d.P; ++p) {
      const TileGeo g{A0, A1, A2, E0, E1, E2, lo0, lo1, lo2};
      if (interior)
        level_pass_interior<T, COMP, INTERP>(d, a, V, hwin, c.reg[p], A0, A1, A2, ebT, ebr, hlo, c.my_nz, c.my_bad);
      else
        level_pass<T, COMP, INTERP, false>(d, a, V, hwin, g, p, ebT, ebr, hlo, c.my_nz, c.my_bad);
      __syncthreads();
    }
  }

  // ---- write the tile of the output grid
  if (d.write_out && fast) {
    write012<T>(d, a, V, A0, A1, A2, E2);
  } else if (d.write_out) {
    const int w1 = E1 - A1, w2 = E2 - A2;
    const int rows = (E0 - A0) * w1;
    int q0 = warp / w1, q1 = warp - (warp / w1) * w1;
    for (int r = warp; r < rows; r += kWarps) {
      const int c0 = A0 + q0, c1 = A1 + q1;
      T* dst = a.Rout + ((uint32_t)c0 * d.rs[0] + (uint32_t)c1 * d.rs[1] + (uint32_t)A2 * d.rs[2]);
      const T* src = V + ((c0 - lo0) * vs0 + (c1 - lo1) * ve2 + (A2 - lo2));
      for (int q2 = lane; q2 < w2; q2 += 32) dst[(uint32_t)q2 * d.rs[2]] = src[q2];
      q1 += kWarps;
      while (q1 >= w1) {
        q1 -= w1;
        ++q0;
      }
    }
  }
  __syncthreads();
  return true;
}

template <typename T, bool COMP, bool TMA, int INTERP>
__global__ void __launch_bounds__(kLevelThreads, 3) level_kernel(const LevelDesc d, const LevelArgs<T> a,
                                                              const __grid_constant__ CUtensorMap tmx,
                                                              const __grid_constant__ CUtensorMap tmc) {
  extern __shared__ __align__(128) unsigned char sm[];
  T* V = reinterpret_cast<T*>(sm);
  T* C = reinterpret_cast<T*>(sm + d.smem_c);
  uint32_t* hwin = reinterpret_cast<uint32_t*>(sm + d.smem_h);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + d.smem_bar);
  __shared__ unsigned long long s_nz;
  __shared__ int s_bad, s_timeout;
  const int tid = threadIdx.x;
  DevState* st = a.st;
  if (COMP && (st->flags & (kFlagNonFinite | kFlagZeroRange | kFlagBadBound))) return;
  if (!COMP && (st->flags & kFlagCorrupt)) return;
  const T ebT = COMP ? bits_to<T>(st->ebT_bits) : a.ebT;
  const T ebr = COMP ? bits_to<T>(st->ebr_bits) : T(0);
  const int radius = a.radius;
  const int hlo = radius - kHistWin / 2;
  if (COMP)
    for (int i = tid; i < kHistWin; i += kLevelThreads) hwin[i] = 0;
  if (tid == 0) {
    s_nz = 0;
    s_bad = 0;
    s_timeout = 0;
    if (TMA) {
      mbar_init(bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __shared__ PassRegion s_reg[3];
  if (tid == 0) make_regions(d, s_reg);
  __syncthreads();

  LevelCtx<T> c{V, C, hwin, bar, s_reg, &s_timeout, 0u, 0u, false, ebT, ebr, hlo};
  for (uint32_t tile = blockIdx.x; tile < d.ntiles; tile += gridDim.x)
    if (!level_tile<T, COMP, TMA, INTERP>(d, a, &tmx, &tmc, tile, c)) break;
  const uint32_t phase = c.phase;
  const unsigned int my_nz = c.my_nz;
  const bool my_bad = c.my_bad;

  // ---- flush the per-CTA counters
  if (my_nz) atomicAdd(&s_nz, (unsigned long long)my_nz);
  if (my_bad) s_bad = 1;
  __syncthreads();
  if (TMA && s_timeout) {
    // give an outstanding copy a last bounded chance to land before exiting
    int spins = 0;
    while (!mbar_try_wait(bar, phase ^ 1u) && ++spins < kWaitLimit) {
    }
    if (tid == 0) atomicOr(&st->flags, kFlagTimeout);
  }
  if (COMP) {
    for (int i = tid; i < kHistWin; i += kLevelThreads)
      if (hwin[i]) atomicAdd(&a.hist[hlo + i], hwin[i]);
    if (tid == 0) {
      if (s_nz) atomicAdd(&st->n_unpred, s_nz);
      if (s_bad) atomicOr(&st->flags, kFlagNonFinite);
    }
  } else if (tid == 0 && s_bad) {
    atomicOr(&st->flags, kFlagCorrupt);
  }
}

// ---------------------------------------------------------------------------
// Coarse group: every level whose grid is small, one CTA.
// ---------------------------------------------------------------------------
constexpr int kCoarseThreads = 1024;
constexpr unsigned long long kCoarseMax = 4096;  // points of the largest coarse-group grid
constexpr int kCoarseMaxPasses = 96;

// Division of a 32-bit n by an invariant d >= 1 by one multiply-high, after
// Granlund and Montgomery ("Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n) and
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for every n < 2^32.
struct DivU32 {
  uint32_t m, s1, s2;
};
static DivU32 divu32(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  const unsigned long long m = (((1ull << l) - d) << 32) / d + 1;
  return DivU32{(uint32_t)m, l < 1 ? l : 1u, l > 1 ? l - 1 : 0u};
}
__device__ __forceinline__ uint32_t div_by(uint32_t n, const DivU32& v) {
  const uint32_t t = __umulhi(v.m, n);
  return (t + ((n - t) >> v.s1)) >> v.s2;
}

struct CoarsePass {
  unsigned long long off;
  uint32_t count;
  uint32_t E[3];
  DivU32 dE2, dE1;      // division by E[2] and by E[1]
  uint32_t start[3], step[3];
  uint32_t m_ax;        // extent of the pass axis in G_grid
  int ax, interp, scale_log;  // scale_log = grid - kc
  unsigned long long xs[3];   // input strides of one G_grid step
};

struct CoarseDesc {
  int n_pass, kc;
  uint32_t mk[3];              // extents of G_kc
  uint32_t gs[3];              // strides of G_kc (compact)
  unsigned long long rs[3];    // strides of the output grid (R_kc or the field)
  unsigned long long xk[3];    // compress: input strides of one G_kc step
  CoarsePass pass[kCoarseMaxPasses];
  uint32_t chunk, nsub;
};

// Shared memory of the coarse kernel: the reconstruction of G_kc, then
// (recover) the group's codes in traversal order.
__host__ __device__ constexpr size_t coarse_off_codes(size_t npts, size_t esz) {
  return (npts * esz + 15) & ~(size_t)15;
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(kCoarseThreads) coarse_kernel(const __grid_constant__ CoarseDesc d,
                                                                const LevelArgs<T> a) {
  extern __shared__ __align__(128) unsigned char sm[];
  T* R = reinterpret_cast<T*>(sm);
  const uint32_t npts = d.mk[0] * d.mk[1] * d.mk[2];
  uint16_t* Kc = reinterpret_cast<uint16_t*>(sm + coarse_off_codes(npts, sizeof(T)));  // recover
  T* Xs = reinterpret_cast<T*>(sm + coarse_off_codes(npts, sizeof(T)));  // compress: input at every point of G_kc
  const int tid = threadIdx.x;
  DevState* st = a.st;
  if (COMP && (st->flags & (kFlagNonFinite | kFlagZeroRange | kFlagBadBound))) return;
  if (!COMP && (st->flags & kFlagCorrupt)) return;
  const T ebT = COMP ? bits_to<T>(st->ebT_bits) : a.ebT;
  const T ebr = COMP ? bits_to<T>(st->ebr_bits) : T(0);
  const int radius = a.radius;
  __shared__ unsigned int s_nz;
  __shared__ int s_bad;
  // the pass descriptors, copied once (indexed reads of the parameter space
  // would wait for the constant cache on every pass)
  __shared__ CoarsePass s_pass[kCoarseMaxPasses];
  static_assert(sizeof(CoarsePass) % 4 == 0, "pass descriptors copy as words");
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(d.pass);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_pass);
    const int nw = d.n_pass * (int)(sizeof(CoarsePass) / 4);
    for (int i = tid; i < nw; i += kCoarseThreads) dst[i] = src[i];
  }
  // recover: the group's codes (the first npts codes of the traversal) in one
  // round of coalesced loads, so that no pass waits for global memory
  if (!COMP) {
    for (uint32_t i = tid; i < npts; i += kCoarseThreads) Kc[i] = a.codes[i];
    __syncthreads();
  } else {
    // compress: the input at every point of G_kc (at most 4 per thread), all
    // loads in flight at once, indexed like the reconstruction
    static_assert(kCoarseMax <= 4 * kCoarseThreads, "four points per thread");
    T xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t v = tid + u * kCoarseThreads;
      if (v < npts) {
        const uint32_t c2 = v % d.mk[2], c1 = (v / d.mk[2]) % d.mk[1], c0 = v / (d.mk[2] * d.mk[1]);
        xv[u] = a.x[c0 * d.xk[0] + c1 * d.xk[1] + c2 * d.xk[2]];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (tid + u * kCoarseThreads < npts) Xs[tid + u * kCoarseThreads] = xv[u];
    __syncthreads();
  }
  if (tid == 0) {
    s_nz = 0;
    s_bad = 0;
    // anchor: point 0, prediction 0
    T r;
    if (COMP) {
      const T xv = Xs[0];
      const uint32_t code = quantize_point<T>(xv, T(0), ebT, ebr, radius, r);
      a.codes[0] = (uint16_t)code;
      atomicAdd(&a.hist[code], 1u);
      if (code == 0) s_nz = 1;
      if (!isfinite(xv)) s_bad = 1;
    } else {
      const uint32_t code = Kc[0];
      if (code == 0) {
        if (a.n_unpred) {
          r = a.unpred[0];
        } else {
          r = T(0);
          s_bad = 1;
        }
      } else if (code >= 2u * (uint32_t)radius) {
        r = T(0);
        s_bad = 1;
      } else {
        r = recover_point<T>(T(0), code, radius, ebT);
      }
    }
    R[0] = r;
  }
  __syncthreads();
  for (int q = 0; q < d.n_pass; ++q) {
    const CoarsePass& P = s_pass[q];
    const uint32_t sc = 1u << P.scale_log;
    const uint32_t vst = sc * d.gs[P.ax];
    for (uint32_t j = tid; j < P.count; j += kCoarseThreads) {
      const uint32_t q1 = div_by(j, P.dE2), j0 = div_by(q1, P.dE1);
      const uint32_t j2 = j - q1 * P.E[2], j1 = q1 - j0 * P.E[1];
      const uint32_t g0 = P.start[0] + P.step[0] * j0, g1 = P.start[1] + P.step[1] * j1,
                     g2 = P.start[2] + P.step[2] * j2;
      const uint32_t v = sc * (g0 * d.gs[0] + g1 * d.gs[1] + g2 * d.gs[2]);
      const uint32_t i = P.ax == 0 ? g0 : (P.ax == 1 ? g1 : g2);
      const bool hb = i + 1 < P.m_ax, hc = i >= 3, hd = i + 3 < P.m_ax;
      const T va = R[v - vst];
      const T vb = hb ? R[v + vst] : T(0);
      const T vc = hc ? R[v - 3 * vst] : T(0);
      const T vd = hd ? R[v + 3 * vst] : T(0);
      const T pred = interp_predict<T>(va, vb, vc, vd, hb, hc, hd, P.interp);
      const unsigned long long ci = P.off + j;
      T r;
      if (COMP) {
        const T xv = Xs[v];
        const uint32_t code = quantize_point<T>(xv, pred, ebT, ebr, radius, r);
        if (SZ3G_IN(ci < a.n_codes && ci < npts, st)) a.codes[ci] = (uint16_t)code;
        atomicAdd(&a.hist[code], 1u);
        if (code == 0) atomicAdd(&s_nz, 1u);
        if (!isfinite(xv)) s_bad = 1;
      } else {
        const uint32_t code = SZ3G_IN(ci < npts, st) ? Kc[ci] : 0u;
        if (code == 0) {
          const unsigned long long rk = rank_of_zero(a.codes, ci, d.chunk, d.nsub, a.zunit);
          if (rk < a.n_unpred) {
            r = a.unpred[rk];
          } else {
            r = T(0);
            s_bad = 1;
          }
        } else if (code >= 2u * (uint32_t)radius) {
          r = T(0);
          s_bad = 1;
        } else {
          r = recover_point<T>(pred, code, radius, ebT);
        }
      }
      if (SZ3G_IN(v < npts && v >= vst && (!hb || v + vst < npts) && (!hc || v >= 3 * vst) &&
                      (!hd || v + 3 * vst < npts), st))
        R[v] = r;
    }
    // a pass of at most 32 points followed by another runs on warp 0 alone:
    // a warp barrier suffices between them (the condition is the same for
    // every thread)
    if (P.count <= 32 && q + 1 < d.n_pass && s_pass[q + 1].count <= 32) __syncwarp();
    else __syncthreads();
  }
  // write G_kc
  const uint32_t tot = a.Rout ? d.mk[0] * d.mk[1] * d.mk[2] : 0u;
  for (uint32_t f = tid; f < tot; f += kCoarseThreads) {
    const uint32_t c2 = f % d.mk[2], c1 = (f / d.mk[2]) % d.mk[1], c0 = f / (d.mk[2] * d.mk[1]);
    const unsigned long long od =
        (unsigned long long)c0 * d.rs[0] + (unsigned long long)c1 * d.rs[1] + (unsigned long long)c2 * d.rs[2];
    if (SZ3G_IN(od < a.n_out, st)) a.Rout[od] = R[c0 * d.gs[0] + c1 * d.gs[1] + c2 * d.gs[2]];
  }
  if (tid == 0) {
    if (COMP) {
      if (s_nz) atomicAdd(&st->n_unpred, (unsigned long long)s_nz);
      if (s_bad) atomicOr(&st->flags, kFlagNonFinite);
    } else if (s_bad) {
      atomicOr(&st->flags, kFlagCorrupt);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

int g_level_cta_cap = 0;

bool level_path_ok(const Plan& pl) { return pl.n[0] == 1; }  // rank <= 3

// k_fine.cu
bool fine_eligible(const Plan& pl, int k, bool comp, const void* x, const unsigned long long* xs, const void* Rc,
                   const void* Rout, bool to_field);
template <typename T, bool COMP>
int launch_fine(const Plan& pl, int k, const LevelArgs<T>& a, bool to_field, cudaStream_t s);
template <typename T>
int launch_fine_slabs(const Plan& pl, const LevelArgs<T>& a, cudaStream_t s, int slabs,
                      const std::function<int(unsigned long long, unsigned long long)>& done);

int coarse_grid(const Plan& pl) {
  int kc = pl.L;
  while (kc > 0 && pl.gsize[kc - 1] <= kCoarseMax) --kc;
  return kc;
}

thread_local const SlabSink* g_slab_sink = nullptr;

bool recover_writes_out_once(const Plan& pl, const void* d_out) {
  alignas(16) static const unsigned char kAlignedRc[16] = {};
  return level_path_ok(pl) && coarse_grid(pl) > 0 && pl.gm[0][1] > 1 &&
         fine_eligible(pl, 0, false, nullptr, nullptr, kAlignedRc, d_out, true);
}

static void tile_shape(const Plan& pl, int k, const int* pos, int* B) {
  const unsigned long long* m = pl.gm[k];  // padded 4 axes; 3-D axes are 1..3
  uint32_t want[3];
  const int rank3 = (m[1] > 1) + (m[2] > 1) + (m[3] > 1);
  // even extents (a tile starts on an even coordinate); along axis 2 the
  // evaluated rows hold B/2 or B/2 + 3 points, close to a 32-lane multiple
  if (rank3 <= 1) {
    want[0] = want[1] = 1;
    want[2] = 2048;
  } else if (m[1] == 1) {
    want[0] = 1;
    want[1] = 32;
    want[2] = 120;
  } else {
    want[0] = 4;
    want[1] = 16;
    want[2] = 56;
  }
  for (int q = 0; q < 3; ++q) {
    const unsigned long long e = m[q + 1];
    B[q] = e <= want[q] ? (int)e : (int)want[q];
    (void)pos;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 3-D tensor map over a dense row-major grid (extents m0, m1, m2; axis 2
// contiguous) with a box of b0 x b1 x b2 elements.
template <typename T>
static bool encode_map(CUtensorMap* map, const T* base, int m0, int m1, int m2, int b0, int b1, int b2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)m2, (cuuint64_t)m1, (cuuint64_t)m0};
  const cuuint64_t strides[2] = {(cuuint64_t)m2 * sizeof(T), (cuuint64_t)m1 * m2 * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)b2, (cuuint32_t)b1, (cuuint32_t)b0};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  return enc(map, dt, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t up128(size_t x) { return (x + 127) & ~(size_t)127; }

// Descriptor, shared-memory bytes and (when tensor copies are allowed and
// possible) tensor maps of one grid level on the generic kernel.  d->P == 0:
// the grid has no passes.
template <typename T, bool COMP>
static int level_desc(const Plan& pl, int k, const LevelArgs<T>& a, bool allow_tma, LevelDesc* dp, size_t* smem,
                      CUtensorMap* tmxp, CUtensorMap* tmcp, bool* tma_out) {
  LevelDesc& d = *dp;
  memset(&d, 0, sizeof(d));
  d.k = k;
  d.write_out = a.Rout != nullptr;
  for (int q = 0; q < 3; ++q) {
    d.m[q] = (int)pl.gm[k][q + 1];
    d.pos[q] = -1;
  }
  int P = 0;
  for (int i = 0; i < pl.n_pass; ++i) {
    const PassDesc& pd = pl.pass[i];
    if (pd.grid != k) continue;
    d.ax[P] = pd.axis - 1;
    d.pos[pd.axis - 1] = P;
    d.off[P] = (uint32_t)pd.off;
    for (int q = 0; q < 3; ++q) d.E[P][q] = pd.E[q + 1];
    d.interp = pd.interp;
    ++P;
  }
  d.P = P;
  if (P == 0) return SZ3G_OK;  // d.P == 0: nothing to launch
  tile_shape(pl, k, d.pos, d.B);
  const unsigned long long* mc = pl.gm[k + 1];
  const int mc0 = (int)mc[1], mc1 = (int)mc[2], mc2 = (int)mc[3];
  const int esz = (int)sizeof(T), al = 16 / esz;
  // tensor copies: the coarse grid rows (and, on compress, the input rows of a
  // finest-level grid) must be 16-byte multiples, the box start along axis 2
  // a 16-byte boundary (tile starts are multiples of `al`)
  bool tma = allow_tma && (size_t)mc2 * esz % 16 == 0 && (size_t)mc1 * mc2 * esz % 16 == 0 && d.B[2] % al == 0 &&
             ((uintptr_t)a.Rc % 16) == 0 && tensor_map_encoder() != nullptr;
  if (COMP)
    tma = tma && k == 0 && (size_t)d.m[2] * esz % 16 == 0 && (size_t)d.m[1] * d.m[2] * esz % 16 == 0 &&
          ((uintptr_t)a.x % 16) == 0;
  // a tensor-copy box has at most 256 elements per dimension
  for (int q = 0; q < 3; ++q) tma = tma && d.B[q] + 8 <= 256;
  d.ntiles = 1;
  for (int q = 0; q < 3; ++q) {
    d.nt[q] = (d.m[q] + d.B[q] - 1) / d.B[q];
    d.ntiles *= (uint32_t)d.nt[q];
    const bool refined = d.pos[q] >= 0;
    if (q == 2 && refined) {
      d.vlo[q] = 4;  // box start on a 16-byte boundary (tensor copies)
      d.vext[q] = d.B[q] + 8;
    } else {
      d.vlo[q] = refined ? 2 : 0;
      d.vext[q] = d.B[q] + (refined ? 5 : 0);
    }
    d.xs[q] = (uint32_t)a.xs[q];
  }
  d.rcs[2] = 1;
  d.rcs[1] = (uint32_t)mc2;
  d.rcs[0] = (uint32_t)mc2 * (uint32_t)mc1;
  if (k == 0 && !COMP) {
    for (int q = 0; q < 3; ++q) d.rs[q] = (uint32_t)pl.fstride[q + 1];
  } else {
    d.rs[2] = 1;
    d.rs[1] = (uint32_t)pl.gm[k][3];
    d.rs[0] = (uint32_t)(pl.gm[k][3] * pl.gm[k][2]);
  }
  d.chunk = pl.chunk;
  d.nsub = pl.nsub;
  d.fast012 = d.P == 3 && d.pos[0] == 0 && d.pos[1] == 1 && d.pos[2] == 2 && d.B[0] == kT0 && d.B[1] == kT1 &&
              d.B[2] == kT2 && d.vext[0] == kX0 && d.vext[1] == kX1 && d.vext[2] == kX2 && d.vlo[0] == kH0 &&
              d.vlo[1] == kH1 && d.vlo[2] == kH2 && d.rs[2] == 1;
  const size_t vbytes = (size_t)d.vext[0] * d.vext[1] * d.vext[2] * esz;
  CUtensorMap& tmx = *tmxp;
  CUtensorMap& tmc = *tmcp;
  memset(&tmx, 0, sizeof(tmx));
  memset(&tmc, 0, sizeof(tmc));
  size_t cbytes = 0;
  if (tma) {
    d.calign = al;
    for (int q = 0; q < 2; ++q) d.cw[q] = ((d.vext[q] - 1) >> 1) + 1;
    d.cw[2] = (((d.vext[2] - 1) >> 1) + 1 + al - 1 + al - 1) / al * al;
    cbytes = (size_t)d.cw[0] * d.cw[1] * d.cw[2] * esz;
    const size_t plane = (size_t)d.vext[1] * d.vext[2] * esz;
    d.xb0_tile = d.pos[0] == 0 && (plane * d.vlo[0]) % 128 == 0;
    const int xb0 = d.xb0_tile ? d.B[0] : d.vext[0];
    bool okm = encode_map<T>(&tmc, a.Rc, mc0, mc1, mc2, d.cw[0], d.cw[1], d.cw[2]);
    if (COMP) okm = okm && encode_map<T>(&tmx, a.x, d.m[0], d.m[1], d.m[2], xb0, d.vext[1], d.vext[2]);
    if (!okm) return SZ3G_E_CUDA;
  }
  d.smem_c = (uint32_t)up128(vbytes);
  d.smem_h = (uint32_t)up128(d.smem_c + cbytes);
  d.smem_bar = (uint32_t)(d.smem_h + (COMP ? kHistWin * 4 : 0));
  *smem = d.smem_bar + 16;
  *tma_out = tma;
  return SZ3G_OK;
}

template <typename T, bool COMP>
static int run_level(const Plan& pl, int k, const LevelArgs<T>& a, cudaStream_t s) {
  if ((COMP || a.codes_padded) && fine_eligible(pl, k, COMP, a.x, a.xs, a.Rc, a.Rout, !COMP && k == 0))
    return launch_fine<T, COMP>(pl, k, a, !COMP && k == 0, s);
  LevelDesc d;
  size_t smem = 0;
  CUtensorMap tmx, tmc;
  bool tma = false;
  const int rc = level_desc<T, COMP>(pl, k, a, true, &d, &smem, &tmx, &tmc, &tma);
  if (rc != SZ3G_OK || d.P == 0) return rc;
  auto kern = tma ? (d.interp == SZ3G_CUBIC ? level_kernel<T, COMP, true, SZ3G_CUBIC>
                                            : level_kernel<T, COMP, true, SZ3G_LINEAR>)
                  : (d.interp == SZ3G_CUBIC ? level_kernel<T, COMP, false, SZ3G_CUBIC>
                                            : level_kernel<T, COMP, false, SZ3G_LINEAR>);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SZ3G_E_CUDA;
  int dev = 0, nsm = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kLevelThreads, smem);
  if (per < 1) per = 1;
  unsigned long long grid = (unsigned long long)nsm * per;
  if (g_level_cta_cap > 0 && grid > (unsigned long long)g_level_cta_cap) grid = (unsigned long long)g_level_cta_cap;
  if (grid > d.ntiles) grid = d.ntiles;
  SZ3G_LAUNCH(COMP ? kKLevelQuantize : kKLevelRecover, s,
              kern<<<(unsigned)grid, kLevelThreads, smem, s>>>(d, a, tmx, tmc));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// ---------------------------------------------------------------------------
// Cross-field work queue (batches).  The levels below the coarse group of
// every field of a batch are collected instead of launched, and one
// persistent kernel per direction and type walks their tiles: a CTA takes the
// next chunk of tiles by a ticket, loads its level's descriptor and arguments into
// shared memory when the level changes (flushing the previous level's
// histogram window and counters to its field), waits until its field's next
// coarser level has counted all its tiles done, runs the tile and counts it
// done.  The queue lists every field's levels coarse to fine (k descending),
// so a tile waits only on tiles taken before it; a CTA takes a tile only
// once it runs, so every awaited tile is held by a running CTA.  counters:
// [0] the ticket, [1 + i] chunks of level i done, [1 + nlev] set when a wait
// gave up (every later wait then gives up at once).  Counts are of chunks.
// ---------------------------------------------------------------------------
template <typename T>
struct QLevel {
  LevelDesc d;
  LevelArgs<T> a;
  int dep;          // index of the level whose reconstruction this one reads (-1: none in the queue)
  uint32_t first;   // queue index of the level's first chunk
  uint32_t chunks;  // chunks of up to kQueueChunk consecutive tiles
  uint32_t extra;   // injected failure (tests): chunks awaited beyond the dependency's own (else 0)
};

constexpr uint32_t kQueueChunk = 8;  // tiles per ticket (one level's, consecutive)

constexpr int kQueueSpinLimit = 1 << 24;  // x ~100 ns: the bound on one dependency wait

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T, bool COMP>
__global__ void __launch_bounds__(kLevelThreads, 3) level_queue_kernel(const QLevel<T>* __restrict__ q, int nlev,
                                                                    uint32_t total, uint32_t* counters,
                                                                    uint32_t spin_limit) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ LevelDesc s_d;
  __shared__ LevelArgs<T> s_a;
  __shared__ PassRegion s_reg[3];
  __shared__ unsigned long long s_nz;
  __shared__ int s_bad, s_timeout, s_skip, s_late, s_lev;
  __shared__ uint32_t s_item;
  const int tid = threadIdx.x;
  int cur = -1;
  LevelCtx<T> c{};
  c.reg = s_reg;
  c.s_timeout = &s_timeout;
  if (tid == 0) {
    s_nz = 0;
    s_bad = 0;
    s_timeout = 0;
  }
  // the per-CTA counters and histogram window of the current level to its field
  auto flush = [&]() {
    if (c.my_nz) atomicAdd(&s_nz, (unsigned long long)c.my_nz);
    if (c.my_bad) s_bad = 1;
    __syncthreads();
    DevState* st = s_a.st;
    if (COMP) {
      for (int i = tid; i < kHistWin; i += kLevelThreads)
        if (c.hwin[i]) atomicAdd(&s_a.hist[c.hlo + i], c.hwin[i]);
      if (tid == 0) {
        if (s_nz) atomicAdd(&st->n_unpred, s_nz);
        if (s_bad) atomicOr(&st->flags, kFlagNonFinite);
      }
    } else if (tid == 0 && s_bad) {
      atomicOr(&st->flags, kFlagCorrupt);
    }
    __syncthreads();
    if (tid == 0) {
      s_nz = 0;
      s_bad = 0;
    }
    c.my_nz = 0;
    c.my_bad = false;
  };
  for (;;) {
    if (tid == 0) {
      const uint32_t it = atomicAdd(&counters[0], 1u);
      int li = -1;
      if (it < total) {  // the last level whose first tile is not after it
        int lo = 0, hi = nlev - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (q[mid].first <= it) lo = mid;
          else hi = mid - 1;
        }
        li = lo;
      }
      s_item = it;
      s_lev = li;
    }
    __syncthreads();
    const uint32_t it = s_item;
    const int li = s_lev;
    if (it >= total) break;
    if (li != cur) {
      if (cur >= 0) flush();
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&q[li].d);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_d);
      for (int i = tid; i < (int)(sizeof(LevelDesc) / 4); i += kLevelThreads) dst[i] = src[i];
      const uint32_t* sa = reinterpret_cast<const uint32_t*>(&q[li].a);
      uint32_t* da = reinterpret_cast<uint32_t*>(&s_a);
      for (int i = tid; i < (int)(sizeof(LevelArgs<T>) / 4); i += kLevelThreads) da[i] = sa[i];
      __syncthreads();
      if (tid == 0) {
        make_regions(s_d, s_reg);
        const uint32_t f = s_a.st->flags;
        s_skip = COMP ? (f & (kFlagNonFinite | kFlagZeroRange | kFlagBadBound)) != 0 : (f & kFlagCorrupt) != 0;
      }
      c.V = reinterpret_cast<T*>(sm);
      c.C = reinterpret_cast<T*>(sm + s_d.smem_c);
      c.hwin = reinterpret_cast<uint32_t*>(sm + s_d.smem_h);
      c.bar = nullptr;
      c.ebT = COMP ? bits_to<T>(s_a.st->ebT_bits) : s_a.ebT;
      c.ebr = COMP ? bits_to<T>(s_a.st->ebr_bits) : T(0);
      c.hlo = s_a.radius - kHistWin / 2;
      if (COMP)
        for (int i = tid; i < kHistWin; i += kLevelThreads) c.hwin[i] = 0;
      __syncthreads();
      cur = li;
    }
    // the next coarser level of the field must be complete
    if (tid == 0) {
      s_late = 0;
      const int dep = q[li].dep;
      if (dep >= 0) {
        const uint32_t need = q[dep].chunks + q[li].extra;
        volatile uint32_t* abort_flag = counters + 1 + nlev;  // set by the first wait that gave up
        uint32_t spins = 0;
        while (ld_acquire_u32(&counters[1 + dep]) < need) {
          if (++spins > spin_limit || *abort_flag) {
            s_late = 1;
            atomicOr(&s_a.st->flags, kFlagTimeout);
            atomicExch(counters + 1 + nlev, 1u);
            break;
          }
          __nanosleep(100);
        }
        __threadfence();
      }
    }
    __syncthreads();
    if (!s_skip && !s_late) {
      const uint32_t t0 = (it - q[li].first) * kQueueChunk, t1 = min(t0 + kQueueChunk, s_d.ntiles);
      for (uint32_t tile = t0; tile < t1; ++tile) {
        if (s_d.interp == SZ3G_CUBIC)
          level_tile<T, COMP, false, SZ3G_CUBIC>(s_d, s_a, nullptr, nullptr, tile, c);
        else
          level_tile<T, COMP, false, SZ3G_LINEAR>(s_d, s_a, nullptr, nullptr, tile, c);
      }
    }
    // every thread's writes of the tile, then the tile counted done
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(&counters[1 + li], 1u);
  }
  if (cur >= 0) flush();
}

template <typename T>
struct QItem {
  const Plan* pl;
  int k, field;
  LevelArgs<T> a;
};

struct LevelQueue {
  bool comp = false;
  std::vector<QItem<float>> f32;
  std::vector<QItem<double>> f64;
  std::vector<unsigned char> h32, h64;  // QLevel arrays built at launch time
  int n32 = 0, n64 = 0;
  void* dev = nullptr;                  // counters of both types, then the QLevel arrays
  size_t cap = 0, off32 = 0, off64 = 0, cnt64 = 0;
};

LevelQueue* level_queue_new(bool comp) {
  LevelQueue* q = new LevelQueue;
  q->comp = comp;
  return q;
}

void level_queue_free(LevelQueue* q) {
  if (!q) return;
  if (q->dev) cudaFree(q->dev);
  delete q;
}

int level_queue_reserve(LevelQueue* q, size_t max_levels) {
  const size_t cnt = (max_levels + 2) * 4 * 2 + 512;
  const size_t need = cnt + (max_levels + 1) * (sizeof(QLevel<double>) + 256);
  if (q->dev && q->cap >= need) return SZ3G_OK;
  if (q->dev) cudaFree(q->dev);
  q->dev = nullptr;
  if (cudaMalloc(&q->dev, need) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_NOMEM;
  }
  q->cap = need;
  q->cnt64 = ((max_levels + 2) * 4 + 255) & ~(size_t)255;
  q->off32 = (2 * q->cnt64 + 255) & ~(size_t)255;
  q->off64 = q->off32;  // set once the f32 array size is known
  return SZ3G_OK;
}

int level_queue_count(const LevelQueue* q) { return (int)(q->f32.size() + q->f64.size()); }

template <typename T>
static std::vector<QItem<T>>& queue_items(LevelQueue* q);
template <>
std::vector<QItem<float>>& queue_items<float>(LevelQueue* q) { return q->f32; }
template <>
std::vector<QItem<double>>& queue_items<double>(LevelQueue* q) { return q->f64; }

template <typename T>
static void queue_add(LevelQueue* q, const Plan& pl, int k, int field, const LevelArgs<T>& a) {
  queue_items<T>(q).push_back(QItem<T>{&pl, k, field, a});
}

// Descriptors of one type's levels in queue order (into `host`), then the
// counters cleared and the kernel launched on s.
template <typename T, bool COMP>
static int queue_launch_t(LevelQueue* q, std::vector<unsigned char>& host, size_t dev_off, uint32_t* counters,
                          size_t counter_bytes, cudaStream_t s) {
  const std::vector<QItem<T>>& items = queue_items<T>(q);
  host.clear();
  if (items.empty()) return SZ3G_OK;
  std::vector<int> order(items.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (items[x].k != items[y].k) return items[x].k > items[y].k;
    return items[x].field < items[y].field;
  });
  std::vector<QLevel<T>> lv;
  lv.reserve(items.size());
  std::unordered_map<int, int> last;  // field -> its latest queued (so nearest coarser) level
  size_t smem = 0;
  uint32_t total = 0;
  bool stalled = false;
  for (int i : order) {
    const QItem<T>& it = items[i];
    QLevel<T> e;
    memset(&e, 0, sizeof(e));
    CUtensorMap tmx, tmc;
    bool tma = false;
    size_t sm = 0;
    const int rc = level_desc<T, COMP>(*it.pl, it.k, it.a, false, &e.d, &sm, &tmx, &tmc, &tma);
    if (rc != SZ3G_OK) return rc;
    if (e.d.P == 0) continue;
    e.a = it.a;
    const auto f = last.find(it.field);
    e.dep = f == last.end() ? -1 : f->second;
    e.first = total;
    e.chunks = (e.d.ntiles + kQueueChunk - 1) / kQueueChunk;
    // injected stall: the first level at or after the given index that waits on another
    e.extra = 0;
    if (!stalled && g_debug.queue_stall >= 0 && (long long)lv.size() >= g_debug.queue_stall && e.dep >= 0) {
      e.extra = 1;
      stalled = true;
    }
    total += e.chunks;
    smem = std::max(smem, sm);
    last[it.field] = (int)lv.size();
    lv.push_back(e);
  }
  if ((lv.size() + 2) * 4 > counter_bytes || dev_off + lv.size() * sizeof(QLevel<T>) > q->cap) return SZ3G_E_INVAL;
  host.resize(lv.size() * sizeof(QLevel<T>));
  if (!lv.empty()) memcpy(host.data(), lv.data(), host.size());
  if (total == 0) return SZ3G_OK;
  auto kern = level_queue_kernel<T, COMP>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return SZ3G_E_CUDA;
  int dev = 0, nsm = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kLevelThreads, smem);
  if (per < 1) per = 1;
  unsigned long long grid = (unsigned long long)nsm * per;
  if (grid > total) grid = total;
  if (cudaMemsetAsync(counters, 0, (lv.size() + 2) * 4, s) != cudaSuccess) return SZ3G_E_CUDA;
  SZ3G_LAUNCH(COMP ? kKLevelQuantize : kKLevelRecover, s,
              kern<<<(unsigned)grid, kLevelThreads, smem, s>>>(
                  reinterpret_cast<const QLevel<T>*>((unsigned char*)q->dev + dev_off), (int)lv.size(), total,
                  counters, g_debug.wait_limit ? g_debug.wait_limit : (uint32_t)kQueueSpinLimit));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int level_queue_launch(LevelQueue* q, cudaStream_t s) {
  if (!q->dev || (size_t)level_queue_count(q) + 2 > q->cnt64 / 4) return SZ3G_E_INVAL;
  uint32_t* c32 = (uint32_t*)q->dev;
  uint32_t* c64 = (uint32_t*)((unsigned char*)q->dev + q->cnt64);
  int rc = q->comp ? queue_launch_t<float, true>(q, q->h32, q->off32, c32, q->cnt64, s)
                   : queue_launch_t<float, false>(q, q->h32, q->off32, c32, q->cnt64, s);
  if (rc != SZ3G_OK) return rc;
  q->off64 = (q->off32 + q->h32.size() + 255) & ~(size_t)255;
  rc = q->comp ? queue_launch_t<double, true>(q, q->h64, q->off64, c64, q->cnt64, s)
               : queue_launch_t<double, false>(q, q->h64, q->off64, c64, q->cnt64, s);
  return rc;
}

int level_queue_upload(LevelQueue* q) {
  if (!q->h32.empty() && cudaMemcpy((unsigned char*)q->dev + q->off32, q->h32.data(), q->h32.size(),
                                    cudaMemcpyHostToDevice) != cudaSuccess)
    return SZ3G_E_CUDA;
  if (!q->h64.empty() && cudaMemcpy((unsigned char*)q->dev + q->off64, q->h64.data(), q->h64.size(),
                                    cudaMemcpyHostToDevice) != cudaSuccess)
    return SZ3G_E_CUDA;
  return SZ3G_OK;
}

template <typename T, bool COMP>
static int run_coarse(const Plan& pl, int kc, const LevelArgs<T>& a, cudaStream_t s) {
  CoarseDesc d;
  memset(&d, 0, sizeof(d));
  d.kc = kc;
  for (int q = 0; q < 3; ++q) d.mk[q] = (uint32_t)pl.gm[kc][q + 1];
  d.gs[2] = 1;
  d.gs[1] = d.mk[2];
  d.gs[0] = d.mk[2] * d.mk[1];
  if (kc == 0 && !COMP) {
    for (int q = 0; q < 3; ++q) d.rs[q] = pl.fstride[q + 1];
  } else {
    for (int q = 0; q < 3; ++q) d.rs[q] = d.gs[q];
  }
  int n = 0;
  for (int i = 0; i < pl.n_pass; ++i) {
    const PassDesc& pd = pl.pass[i];
    if (pd.grid < kc) continue;
    if (n >= kCoarseMaxPasses) return SZ3G_E_INVAL;
    CoarsePass& c = d.pass[n++];
    c.off = pd.off;
    c.count = (uint32_t)pd.count;
    for (int q = 0; q < 3; ++q) {
      c.E[q] = pd.E[q + 1];
      c.start[q] = pd.start[q + 1];
      c.step[q] = pd.step[q + 1];
      c.xs[q] = pd.xstride[q + 1];
    }
    if (c.E[1] == 0 || c.E[2] == 0) return SZ3G_E_INVAL;
    c.dE2 = divu32(c.E[2]);
    c.dE1 = divu32(c.E[1]);
    if (pd.grid == kc)
      for (int q = 0; q < 3; ++q) d.xk[q] = pd.xstride[q + 1];
    c.ax = pd.axis - 1;
    c.m_ax = pd.m[pd.axis];
    c.interp = pd.interp;
    c.scale_log = pd.grid - kc;
    // the group's codes are the first codes of the traversal: recover
    // stages them by code index
    if (c.off + c.count > pl.gsize[kc]) return SZ3G_E_INVAL;
  }
  if (pl.gsize[kc] > kCoarseMax) return SZ3G_E_INVAL;  // one CTA holds the group (four points per thread)
  d.n_pass = n;
  d.chunk = pl.chunk;
  d.nsub = pl.nsub;
  const size_t smem = coarse_off_codes((size_t)pl.gsize[kc], sizeof(T)) + (size_t)pl.gsize[kc] * (COMP ? sizeof(T) : 2);
  if (cudaFuncSetAttribute(coarse_kernel<T, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return SZ3G_E_CUDA;
  SZ3G_LAUNCH(COMP ? kKCoarseQuantize : kKCoarseRecover, s,
              coarse_kernel<T, COMP><<<1, kCoarseThreads, smem, s>>>(d, a));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

// X_k[i][j][c] = src[2i][2j][2c] (src = the field for k = 1, else X_{k-1}):
// the decimated pyramid that the levels on G_1 and coarser read contiguously
// (and by tensor copies) instead of the field at stride 2^k.  One warp per
// output row; rows of X_k pitched to 16 bytes.
template <typename T>
__global__ void decimate_kernel(const T* __restrict__ src, unsigned long long s0, unsigned long long s1,
                                T* __restrict__ dst, int m0, int m1, int m2, unsigned long long p0,
                                unsigned long long p1) {
  const unsigned long long row = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= (unsigned long long)m0 * m1) return;
  const int lane = threadIdx.x & 31;
  const unsigned long long i = row / (unsigned)m1, j = row % (unsigned)m1;
  const T* sp = src + 2 * i * s0 + 2 * j * s1;
  T* dp = dst + i * p0 + j * p1;
  for (int c = lane; c < m2; c += 32) dp[c] = __ldcs(sp + 2 * c);
}

// X_2 .. X_kmax from X_1 in one pass: one warp per row of X_2; a point of X_2
// whose coordinates are multiples of 2^(k-2) is also the point of X_k.
struct PyrDesc {
  int kmax;
  int m[32][3];                    // extents of G_k
  unsigned long long off[32];      // element offset of X_k
  unsigned long long p0[32], p1[32];
};

template <typename T>
__global__ void pyramid_kernel(T* __restrict__ X, const __grid_constant__ PyrDesc d) {
  const unsigned long long row = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= (unsigned long long)d.m[2][0] * d.m[2][1]) return;
  const int lane = threadIdx.x & 31;
  const unsigned long long i = row / (unsigned)d.m[2][1], j = row % (unsigned)d.m[2][1];
  const T* src = X + d.off[1] + 2 * i * d.p0[1] + 2 * j * d.p1[1];
  for (int c = lane; c < d.m[2][2]; c += 32) {
    const T v = src[2 * c];
    X[d.off[2] + i * d.p0[2] + j * d.p1[2] + c] = v;
    for (int k = 3; k <= d.kmax; ++k) {
      const int sh = k - 2;
      if (((i | j | (unsigned long long)c) & ((1ull << sh) - 1)) != 0) break;
      X[d.off[k] + (i >> sh) * d.p0[k] + (j >> sh) * d.p1[k] + (c >> sh)] = v;
    }
  }
}

// X_1 .. X_kmax into the pyramid, unless the range pass wrote them.
static int launch_decimate(const Plan& pl, const void* x, unsigned char* X, int kmax, bool pyr_ready, cudaStream_t s) {
  if (pyr_ready) return SZ3G_OK;  // the range pass wrote X_1 .. X_kmax
  {
    const unsigned long long* m = pl.gm[1];
    const unsigned long long p1 = xk_pitch(pl, 1), p0 = p1 * m[2];
    const unsigned blocks = (unsigned)((m[1] * m[2] + 7) / 8);
    if (pl.dtype == SZ3G_F32)
      SZ3G_LAUNCH(kKDecimate, s,
                  decimate_kernel<float><<<blocks, 256, 0, s>>>((const float*)x, pl.fstride[1], pl.fstride[2],
                                                                (float*)X, (int)m[1], (int)m[2], (int)m[3], p0, p1));
    else
      SZ3G_LAUNCH(kKDecimate, s,
                  decimate_kernel<double><<<blocks, 256, 0, s>>>((const double*)x, pl.fstride[1], pl.fstride[2],
                                                                 (double*)X, (int)m[1], (int)m[2], (int)m[3], p0, p1));
    if (cudaGetLastError() != cudaSuccess) return SZ3G_E_CUDA;
  }
  if (kmax < 2) return SZ3G_OK;
  PyrDesc d;
  memset(&d, 0, sizeof(d));
  d.kmax = kmax;
  for (int k = 1; k <= kmax && k < 32; ++k) {
    for (int q = 0; q < 3; ++q) d.m[k][q] = (int)pl.gm[k][q + 1];
    d.off[k] = xpyr_offset(pl, k) / pl.esz;
    d.p1[k] = xk_pitch(pl, k);
    d.p0[k] = d.p1[k] * pl.gm[k][2];
  }
  const unsigned blocks = (unsigned)(((unsigned long long)d.m[2][0] * d.m[2][1] + 7) / 8);
  if (pl.dtype == SZ3G_F32)
    SZ3G_LAUNCH(kKDecimate, s, pyramid_kernel<float><<<blocks, 256, 0, s>>>((float*)X, d));
  else
    SZ3G_LAUNCH(kKDecimate, s, pyramid_kernel<double><<<blocks, 256, 0, s>>>((double*)X, d));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

template <typename T>
static int quantize_fused(const Plan& pl, const T* x, uint16_t* codes, void* const* R, uint32_t* hist, DevState* st,
                          void* X, bool pyr_ready, cudaStream_t s, LevelQueue* lq, int field) {
  const int kc = coarse_grid(pl);
  LevelArgs<T> a{};
  a.x = x;
  for (int q = 0; q < 3; ++q) a.xs[q] = pl.fstride[q + 1];
  a.codes = codes;
#ifdef SZ3G_CHECK
  a.n_codes = pl.N;
#endif
  a.hist = hist;
  a.st = st;
  a.radius = (int)pl.radius;
  a.Rout = kc == 0 ? nullptr : (T*)R[kc];  // the finest grid's reconstruction is not kept
#ifdef SZ3G_CHECK
  a.n_out = kc == 0 ? 0 : pl.gsize[kc];
#endif
  int rc = run_coarse<T, true>(pl, kc, a, s);
  if (rc) return rc;
  // levels on G_1 and coarser read the decimated pyramid
  const bool dec = X && kc >= 2;
  if (dec) {
    rc = launch_decimate(pl, x, (unsigned char*)X, kc - 1, pyr_ready, s);
    if (rc) return rc;
  }
  for (int k = kc - 1; k >= 0; --k) {
    a.Rc = (const T*)R[k + 1];
    a.Rout = k == 0 ? nullptr : (T*)R[k];
#ifdef SZ3G_CHECK
    a.n_out = k == 0 ? 0 : pl.gsize[k];
#endif
    if (dec && k >= 1) {
      a.x = (const T*)((unsigned char*)X + xpyr_offset(pl, k));
      a.xs[1] = xk_pitch(pl, k);
      a.xs[0] = a.xs[1] * pl.gm[k][2];
      a.xs[2] = 1;
    } else {
      a.x = x;
      for (int q = 0; q < 3; ++q) a.xs[q] = pl.fstride[q + 1] << k;
    }
    if (lq) {
      queue_add<T>(lq, pl, k, field, a);
      continue;
    }
    rc = run_level<T, true>(pl, k, a, s);
    if (rc) return rc;
  }
  return SZ3G_OK;
}

// The finest level in slabs of planes, each slab copied to the host on the
// sink's stream as soon as its launch is done; the copies join back into s.
template <typename T>
static int recover_finest_to_host(const Plan& pl, const LevelArgs<T>& a, cudaStream_t s, const SlabSink& sink) {
  const unsigned long long plane = pl.fstride[1] * pl.esz;
  auto done = [&](unsigned long long p0, unsigned long long np) -> int {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return SZ3G_E_CUDA;
    const bool ok = cudaEventRecord(ev, s) == cudaSuccess && cudaStreamWaitEvent(sink.copy, ev, 0) == cudaSuccess &&
                    cudaMemcpyAsync((unsigned char*)sink.h_out + p0 * plane, (const unsigned char*)a.Rout + p0 * plane,
                                    np * plane, cudaMemcpyDeviceToHost, sink.copy) == cudaSuccess;
    cudaEventDestroy(ev);
    return ok ? SZ3G_OK : SZ3G_E_CUDA;
  };
  int rc = launch_fine_slabs<T>(pl, a, s, sink.slabs, done);
  cudaEvent_t join;
  if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) return SZ3G_E_CUDA;
  const bool ok = cudaEventRecord(join, sink.copy) == cudaSuccess && cudaStreamWaitEvent(s, join, 0) == cudaSuccess;
  cudaEventDestroy(join);
  if (rc == SZ3G_OK && !ok) rc = SZ3G_E_CUDA;
  return rc;
}

template <typename T>
static int recover_fused(const Plan& pl, const uint16_t* codes, const T* unpred, unsigned long long n_unpred,
                         const unsigned long long* zunit, void* const* R, T* out, DevState* st,
                         T ebT, bool codes_padded, cudaStream_t s, LevelQueue* lq, int field) {
  const int kc = coarse_grid(pl);
  LevelArgs<T> a{};
  a.codes = const_cast<uint16_t*>(codes);
#ifdef SZ3G_CHECK
  a.n_codes = pl.N;
#endif
  a.st = st;
  a.radius = (int)pl.radius;
  a.unpred = unpred;
  a.n_unpred = n_unpred;
  a.zunit = zunit;
  a.ebT = ebT;
  a.codes_padded = codes_padded;
  a.Rout = kc == 0 ? out : (T*)R[kc];
#ifdef SZ3G_CHECK
  a.n_out = kc == 0 ? pl.N : pl.gsize[kc];
#endif
  int rc = run_coarse<T, false>(pl, kc, a, s);
  if (rc) return rc;
  for (int k = kc - 1; k >= 0; --k) {
    a.Rc = (const T*)R[k + 1];
    a.Rout = k == 0 ? out : (T*)R[k];
#ifdef SZ3G_CHECK
    a.n_out = k == 0 ? pl.N : pl.gsize[k];
#endif
    if (lq) {
      queue_add<T>(lq, pl, k, field, a);
      continue;
    }
    if (k == 0 && g_slab_sink && a.codes_padded && recover_writes_out_once(pl, out)) {
      rc = recover_finest_to_host(pl, a, s, *g_slab_sink);
      if (rc) return rc;
      continue;
    }
    rc = run_level<T, false>(pl, k, a, s);
    if (rc) return rc;
  }
  return SZ3G_OK;
}

int launch_quantize_fused(const Plan& pl, const void* d_in, uint16_t* codes, void* const* R, uint32_t* hist,
                          DevState* st, void* X, bool pyr_ready, cudaStream_t s, LevelQueue* lq, int field) {
  if (pl.dtype == SZ3G_F32)
    return quantize_fused<float>(pl, (const float*)d_in, codes, R, hist, st, X, pyr_ready, s, lq, field);
  return quantize_fused<double>(pl, (const double*)d_in, codes, R, hist, st, X, pyr_ready, s, lq, field);
}

int launch_recover_fused(const Plan& pl, const uint16_t* codes, const void* unpred, unsigned long long n_unpred,
                         const unsigned long long* zunit, void* const* R, void* d_out,
                         DevState* st, unsigned long long ebT_bits, bool codes_padded, cudaStream_t s,
                         LevelQueue* lq, int field) {
  if (pl.dtype == SZ3G_F32) {
    float e;
    uint32_t b = (uint32_t)ebT_bits;
    memcpy(&e, &b, 4);
    return recover_fused<float>(pl, codes, (const float*)unpred, n_unpred, zunit, R, (float*)d_out, st, e,
                                codes_padded, s, lq, field);
  }
  double e;
  memcpy(&e, &ebT_bits, 8);
  return recover_fused<double>(pl, codes, (const double*)unpred, n_unpred, zunit, R, (double*)d_out, st, e,
                               codes_padded, s, lq, field);
}

}  // namespace sz3g
