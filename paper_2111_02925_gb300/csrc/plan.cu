// plan.cu -- parameter validation and the host-side schedule of one field.
//
// The schedule follows the multilevel interpolation of SZ3-Interp (SZ3 paper
// Sec. 6.2) as read for this library: after the anchor (point 0), level l =
// L..1 refines the grid of stride 2^(l-1); within a level the axes are refined
// one after another in `order`, and each refinement (a "pass") predicts the
// points whose coordinate on the pass axis is an odd multiple of the stride.
//
// Points of stride-2^k form the compact grid G_k (extents ceil(n / 2^k)); level
// l = k + 1 is then the finest level of G_k, and its passes are the
// sub-lattices of G_k with an odd coordinate on the pass axis, any coordinate
// on axes refined earlier in the level and an even one on the others.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace sz3g {

static bool is_perm(const uint8_t* o, uint32_t nd) {
  uint32_t seen = 0;
  for (uint32_t k = 0; k < nd; ++k) {
    if (o[k] >= nd || (seen >> o[k]) & 1u) return false;
    seen |= 1u << o[k];
  }
  return true;
}

int make_plan(const sz3g_params* p, Plan* pl) {
  if (!p || !pl) return SZ3G_E_INVAL;
  std::memset(pl, 0, sizeof(*pl));
  if (p->dtype != SZ3G_F32 && p->dtype != SZ3G_F64) return SZ3G_E_INVAL;
  if (p->ndim < 1 || p->ndim > 4) return SZ3G_E_INVAL;
  if (p->eb_mode != SZ3G_EB_ABS && p->eb_mode != SZ3G_EB_REL) return SZ3G_E_INVAL;
  if (!(p->eb > 0.0) || !std::isfinite(p->eb)) return SZ3G_E_INVAL;
  if (p->radius < 2 || p->radius > 32768) return SZ3G_E_INVAL;
  if (p->chunk_codes < 8 || p->chunk_codes > 65536 || p->chunk_codes % 8) return SZ3G_E_INVAL;
  if (p->per_level > 1) return SZ3G_E_INVAL;
  const uint32_t nd = p->ndim;
  const int off = 4 - (int)nd;  // leading unit axes
  unsigned long long N = 1, maxn = 1;
  for (uint32_t d = 0; d < nd; ++d) {
    unsigned long long e = p->dims[d];
    if (e < 1 || e > (1ull << 31)) return SZ3G_E_INVAL;
    if (N > (1ull << 31) / e) return SZ3G_E_INVAL;
    N *= e;
    if (e > maxn) maxn = e;
  }
  int L = 0;
  while ((1ull << L) < maxn) ++L;
  if (p->per_level) {
    for (int l = 1; l <= L; ++l)
      if (p->level_interp[l] > SZ3G_CUBIC || !is_perm(p->level_order[l], nd)) return SZ3G_E_INVAL;
  } else {
    if (p->interp > SZ3G_CUBIC || !is_perm(p->dim_order, nd)) return SZ3G_E_INVAL;
  }
  pl->dtype = (int)p->dtype;
  pl->esz = p->dtype == SZ3G_F32 ? 4 : 8;
  pl->ndim = (int)nd;
  pl->L = L;
  pl->radius = p->radius;
  pl->chunk = p->chunk_codes;
  pl->N = N;
  for (int d = 0; d < 4; ++d) pl->n[d] = d < off ? 1 : p->dims[d - off];
  pl->fstride[3] = 1;
  for (int d = 2; d >= 0; --d) pl->fstride[d] = pl->fstride[d + 1] * pl->n[d + 1];
  for (int k = 0; k <= L; ++k) {
    unsigned long long sz = 1;
    for (int d = 0; d < 4; ++d) {
      unsigned long long s = 1ull << k;
      pl->gm[k][d] = (pl->n[d] + s - 1) >> k;
      sz *= pl->gm[k][d];
    }
    pl->gsize[k] = sz;
  }
  // Passes in traversal order.
  unsigned long long pos = 1;  // code 0 is the anchor
  int np = 0;
  for (int l = L; l >= 1; --l) {
    const int k = l - 1;
    const uint8_t* ord = p->per_level ? p->level_order[l] : p->dim_order;
    const int interp = p->per_level ? p->level_interp[l] : (int)p->interp;
    const unsigned long long* m = pl->gm[k];
    unsigned long long gstride[4];
    gstride[3] = 1;
    for (int d = 2; d >= 0; --d) gstride[d] = gstride[d + 1] * m[d + 1];
    for (uint32_t kk = 0; kk < nd; ++kk) {
      const int a = ord[kk] + off;
      PassDesc& pd = pl->pass[np];
      std::memset(&pd, 0, sizeof(pd));
      unsigned long long cnt = 1;
      for (int d = 0; d < 4; ++d) {
        bool earlier = false;
        for (uint32_t j = 0; j < kk; ++j)
          if (ord[j] + off == d) earlier = true;
        if (d == a) {
          pd.start[d] = 1;
          pd.step[d] = 2;
          pd.E[d] = (uint32_t)(m[d] / 2);
        } else if (earlier) {
          pd.start[d] = 0;
          pd.step[d] = 1;
          pd.E[d] = (uint32_t)m[d];
        } else {
          pd.start[d] = 0;
          pd.step[d] = 2;
          pd.E[d] = (uint32_t)((m[d] + 1) / 2);
        }
        cnt *= pd.E[d];
        pd.m[d] = (uint32_t)m[d];
        pd.gstride[d] = gstride[d];
        pd.xstride[d] = pl->fstride[d] << k;
      }
      if (cnt == 0) continue;  // a unit axis has nothing to refine
      pd.off = pos;
      pd.count = cnt;
      pd.axis = a;
      pd.interp = interp;
      pd.grid = k;
      pos += cnt;
      ++np;
    }
  }
  if (pos != N) return SZ3G_E_INVAL;  // cannot happen for a valid shape
  pl->n_pass = np;
  pl->n_chunks = (N + pl->chunk - 1) / pl->chunk;
  pl->nsub = (pl->chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  return SZ3G_OK;
}

void make_pass_map(const Plan& pl, PassMap* map) {
  std::memset(map, 0, sizeof(*map));
  map->e[0].off = 0;
  for (int d = 0; d < 4; ++d) map->e[0].E[d] = 1;
  for (int i = 0; i < pl.n_pass; ++i) {
    const PassDesc& pd = pl.pass[i];
    PassMapEntry& e = map->e[i + 1];
    e.off = pd.off;
    e.xstart = 0;
    for (int d = 0; d < 4; ++d) {
      e.E[d] = pd.E[d];
      e.xstart += (unsigned long long)pd.start[d] * pd.xstride[d];
      e.xls[d] = (unsigned long long)pd.step[d] * pd.xstride[d];
    }
  }
  map->n = pl.n_pass + 1;
}

}  // namespace sz3g
