/* szlz.c -- serial reference of the optional lossless stage after the
 * Huffman coder (TEST INFRASTRUCTURE; see sz3o.h for the stream layout).
 *
 * SZ3 follows its entropy coder with a general-purpose dictionary coder
 * (the paper's pipelines end in a lossless compressor).  This is a byte-level
 * LZ77 of our own definition, chosen so that the GPU can find every
 * position's match candidate in parallel:
 *   - independent blocks of SZLZ_BLOCK bytes;
 *   - h(i) = (little-endian u32 of bytes i..i+3) * 2654435761 mod 2^32 >> 20;
 *   - cand(i) = the last j < i of the block with h(j) = h(i), over ALL
 *     positions 0..n_b-4 (not only those the parse visits); none if no such j;
 *   - matchable(i): cand(i) exists and bytes cand(i)..+3 equal bytes i..i+3;
 *   - greedy parse: from `pos`, take the first matchable p >= pos, extend the
 *     match while the next byte equals (it may overlap p), emit the literals
 *     since the last match and the match, continue after it; the bytes after
 *     the last match are the final literals;
 *   - a block whose coded form is not shorter than the block is stored raw.
 */
#include <stdint.h>
#include <string.h>

#include "sz3o.h"

#define SZLZ_HASH_BITS 12
#define SZLZ_NONE 0xffffffffu

static uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static uint32_t lz_hash(const uint8_t* p) { return (uint32_t)(rd32(p) * 2654435761u) >> (32 - SZLZ_HASH_BITS); }

static uint64_t up4(uint64_t x) { return (x + 3) & ~(uint64_t)3; }

uint64_t sz3o_lz_bound(uint64_t n) {
  const uint64_t nb = (n + SZLZ_BLOCK - 1) / SZLZ_BLOCK;
  return SZLZ_HEADER + 4 * nb + 8 + n + 4 * nb;
}

/* a length field continued by 255-bytes: writes v (>= 15 already taken out) */
static uint64_t put_ext(uint8_t* o, uint64_t k, uint64_t cap, uint64_t v, int* over) {
  while (v >= 255) {
    if (k >= cap) {
      *over = 1;
      return k;
    }
    o[k++] = 255;
    v -= 255;
  }
  if (k >= cap) {
    *over = 1;
    return k;
  }
  o[k++] = (uint8_t)v;
  return k;
}

/* one sequence: literals lit[0..nl), then (if ml) a match of ml bytes at
 * distance off; returns the new output length, *over set past cap */
static uint64_t put_seq(uint8_t* o, uint64_t k, uint64_t cap, const uint8_t* lit, uint64_t nl, uint32_t off,
                        uint64_t ml, int* over) {
  if (k >= cap) {
    *over = 1;
    return k;
  }
  const uint32_t tl = nl >= 15 ? 15 : (uint32_t)nl;
  const uint32_t tm = ml == 0 ? 0 : (ml - 4 >= 15 ? 15 : (uint32_t)(ml - 4));
  o[k++] = (uint8_t)(tl << 4 | tm);
  if (nl >= 15) k = put_ext(o, k, cap, nl - 15, over);
  if (*over || k + nl > cap) {
    *over = 1;
    return k;
  }
  memcpy(o + k, lit, nl);
  k += nl;
  if (ml == 0) return k;
  if (k + 2 > cap) {
    *over = 1;
    return k;
  }
  o[k++] = (uint8_t)(off & 0xff);
  o[k++] = (uint8_t)(off >> 8);
  if (ml - 4 >= 15) k = put_ext(o, k, cap, ml - 4 - 15, over);
  return k;
}

/* coded form of one block into o (at most cap = nb - 1 bytes); returns its
 * length, or 0 when it would not be shorter than the block */
static uint64_t lz_block(const uint8_t* in, uint64_t nb, uint8_t* o, uint64_t cap) {
  static uint32_t last[1u << SZLZ_HASH_BITS];
  static uint32_t cand[SZLZ_BLOCK];
  for (uint32_t h = 0; h < (1u << SZLZ_HASH_BITS); ++h) last[h] = SZLZ_NONE;
  for (uint64_t i = 0; i < nb; ++i) cand[i] = SZLZ_NONE;
  for (uint64_t i = 0; i + 4 <= nb; ++i) {
    const uint32_t h = lz_hash(in + i);
    cand[i] = last[h];
    last[h] = (uint32_t)i;
  }
  uint64_t pos = 0, anchor = 0, k = 0;
  int over = 0;
  for (;;) {
    uint64_t p = pos;
    while (p + 4 <= nb && !(cand[p] != SZLZ_NONE && rd32(in + cand[p]) == rd32(in + p))) ++p;
    if (p + 4 > nb) break;
    const uint64_t c = cand[p];
    uint64_t len = 4;
    while (p + len < nb && in[c + len] == in[p + len]) ++len;
    k = put_seq(o, k, cap, in + anchor, p - anchor, (uint32_t)(p - c), len, &over);
    if (over) return 0;
    pos = anchor = p + len;
  }
  k = put_seq(o, k, cap, in + anchor, nb - anchor, 0, 0, &over);
  return over ? 0 : k;
}

int sz3o_lz_compress(const void* in_, uint64_t n, void* out_, uint64_t cap, uint64_t* out_bytes) {
  const uint8_t* in = (const uint8_t*)in_;
  uint8_t* out = (uint8_t*)out_;
  const uint64_t nblk = (n + SZLZ_BLOCK - 1) / SZLZ_BLOCK;
  const uint64_t data0 = (SZLZ_HEADER + 4 * nblk + 7) & ~(uint64_t)7;
  if (!out || !out_bytes || (n && !in) || nblk > 0xffffffffull || cap < data0) return SZ3O_E_CAPACITY;
  memset(out, 0, data0);
  memcpy(out, "SZLZ", 4);
  const uint32_t bs = SZLZ_BLOCK;
  memcpy(out + 4, &bs, 4);
  memcpy(out + 8, &n, 8);
  const uint32_t nb32 = (uint32_t)nblk;
  memcpy(out + 16, &nb32, 4);
  static uint8_t tmp[SZLZ_BLOCK];
  uint64_t k = data0;
  for (uint64_t b = 0; b < nblk; ++b) {
    const uint64_t nb = (b + 1) * SZLZ_BLOCK <= n ? SZLZ_BLOCK : n - b * SZLZ_BLOCK;
    const uint8_t* src = in + b * SZLZ_BLOCK;
    const uint64_t cb = nb > 1 ? lz_block(src, nb, tmp, nb - 1) : 0;
    uint32_t size;
    const uint8_t* pay;
    if (cb) {
      size = (uint32_t)cb;
      pay = tmp;
    } else {
      size = (uint32_t)nb | 0x80000000u;
      pay = src;
    }
    const uint64_t len = size & 0x7fffffffu;
    if (k + up4(len) > cap) return SZ3O_E_CAPACITY;
    memcpy(out + SZLZ_HEADER + 4 * b, &size, 4);
    memcpy(out + k, pay, len);
    memset(out + k + len, 0, up4(len) - len);
    k += up4(len);
  }
  *out_bytes = k;
  return SZ3O_OK;
}

/* a length continued by 255-bytes: adds them to *v; 0 when the payload ends */
static int get_ext(const uint8_t* p, uint64_t end, uint64_t* k, uint64_t* v) {
  for (;;) {
    if (*k >= end) return 0;
    const uint8_t b = p[(*k)++];
    *v += b;
    if (b != 255) return 1;
  }
}

int sz3o_lz_decompress(const void* in_, uint64_t bytes, void* out_, uint64_t cap, uint64_t* out_n) {
  const uint8_t* in = (const uint8_t*)in_;
  uint8_t* out = (uint8_t*)out_;
  if (!in || bytes < SZLZ_HEADER || memcmp(in, "SZLZ", 4) != 0) return SZ3O_E_CORRUPT;
  uint32_t bs, nblk32;
  uint64_t n;
  memcpy(&bs, in + 4, 4);
  memcpy(&n, in + 8, 8);
  memcpy(&nblk32, in + 16, 4);
  const uint64_t nblk = nblk32;
  if (bs != SZLZ_BLOCK || nblk != (n + SZLZ_BLOCK - 1) / SZLZ_BLOCK) return SZ3O_E_CORRUPT;
  const uint64_t data0 = (SZLZ_HEADER + 4 * nblk + 7) & ~(uint64_t)7;
  if (data0 > bytes) return SZ3O_E_CORRUPT;
  if (n > cap || (n && !out)) return SZ3O_E_CAPACITY;
  uint64_t k = data0;
  for (uint64_t b = 0; b < nblk; ++b) {
    uint32_t size;
    memcpy(&size, in + SZLZ_HEADER + 4 * b, 4);
    const uint64_t nb = (b + 1) * SZLZ_BLOCK <= n ? SZLZ_BLOCK : n - b * SZLZ_BLOCK;
    const uint64_t len = size & 0x7fffffffu;
    if (k + len > bytes) return SZ3O_E_CORRUPT;
    uint8_t* dst = out + b * SZLZ_BLOCK;
    const uint8_t* p = in + k;
    if (size & 0x80000000u) {
      if (len != nb) return SZ3O_E_CORRUPT;
      memcpy(dst, p, nb);
    } else {
      uint64_t q = 0, o = 0;
      for (;;) {
        if (q >= len) return SZ3O_E_CORRUPT;
        const uint8_t t = p[q++];
        uint64_t nl = t >> 4, ml = t & 15;
        if (nl == 15 && !get_ext(p, len, &q, &nl)) return SZ3O_E_CORRUPT;
        if (q + nl > len || o + nl > nb) return SZ3O_E_CORRUPT;
        memcpy(dst + o, p + q, nl);
        q += nl;
        o += nl;
        if (q == len) {  /* the last sequence: literals only */
          if (ml != 0) return SZ3O_E_CORRUPT;
          break;
        }
        if (q + 2 > len) return SZ3O_E_CORRUPT;
        const uint64_t off = (uint64_t)p[q] | ((uint64_t)p[q + 1] << 8);
        q += 2;
        ml += 4;
        if (ml == 19 && !get_ext(p, len, &q, &ml)) return SZ3O_E_CORRUPT;
        if (off == 0 || off > o || o + ml > nb) return SZ3O_E_CORRUPT;
        for (uint64_t i = 0; i < ml; ++i) dst[o + i] = dst[o + i - off];  /* may overlap */
        o += ml;
      }
      if (o != nb) return SZ3O_E_CORRUPT;
    }
    k += up4(len);
  }
  if (out_n) *out_n = n;
  return SZ3O_OK;
}
