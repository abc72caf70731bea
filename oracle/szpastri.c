/* szpastri.c -- serial reference of the two SZ3-Pastri modules on the
 * quantize / encode path (TEST INFRASTRUCTURE; declarations and stream
 * layout in sz3o.h).
 *
 * Unpred-aware quantizer (Sec. 4.2): values are aligned to the exponent of
 * the error bound and stored as integers, bitplane by bitplane from the most
 * significant one, so that the high planes are long runs of zeros for a
 * later lossless stage.  Our reading of the alignment step:
 *   e    = floor(log2(eb))            (2^e <= eb < 2^(e+1))
 *   q_i  = trunc(v_i / 2^e)           (|v_i - q_i 2^e| < 2^e <= eb)
 *   B    = bit length of max |q_i|    (0 when every q_i is 0)
 * and the value it decodes to is q_i 2^e, exactly representable in T.
 *
 * Fixed Huffman encoder (Sec. 3.2 Encoder, the predefined tree of
 * SZ-Pastri): a prefix code over the quantization codes [0, 2r) that is
 * fixed in advance instead of built from the histogram and stored.  Our
 * predefined code: code r (zero error) 1 bit; codes at distance k >= 1 from
 * r, in the distance class c = bit length of k, 2c + 2 bits (a two-sided
 * Elias-gamma shape); classes c >= 11 and code 0 (unpredictable) 24 bits,
 * the stream's longest codeword.  Codewords are canonical over these
 * lengths (sz3o_canonical_codes).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "sz3o.h"

int sz3o_bitplane_exponent(double eb, int32_t* e) {
  int ex = 0;
  if (!e || !(eb > 0) || !isfinite(eb)) return SZ3O_E_INVAL;
  (void)frexp(eb, &ex); /* eb = m 2^ex, m in [0.5, 1) */
  *e = (int32_t)(ex - 1);
  return SZ3O_OK;
}

uint64_t sz3o_bitplane_bound(uint64_t n) { return SZBP_HEADER + 4ull * ((n + 31) / 32) * 64ull; }

static double value_at(uint32_t dtype, const void* v, uint64_t i) {
  return dtype == 0 ? (double)((const float*)v)[i] : ((const double*)v)[i];
}

static void put_u32(uint8_t* p, uint32_t x) { memcpy(p, &x, 4); }
static void put_u64(uint8_t* p, uint64_t x) { memcpy(p, &x, 8); }

int sz3o_bitplane_encode(uint32_t dtype, const void* v, uint64_t n, double eb, void* out_, uint64_t cap,
                         uint64_t* out_bytes) {
  uint8_t* out = (uint8_t*)out_;
  int32_t e;
  uint64_t i, maxmag = 0, W = (n + 31) / 32, total;
  uint32_t B = 0, b;
  if (dtype > 1 || !out_bytes || (n && !v) || sz3o_bitplane_exponent(eb, &e) != SZ3O_OK) return SZ3O_E_INVAL;
  /* pass 1: every value aligned, the widest magnitude; a non-finite value
   * anywhere is reported before an aligned integer past 62 bits */
  {
    int bad = 0, wide = 0;
    for (i = 0; i < n; ++i) {
      const double x = value_at(dtype, v, i);
      double w;
      if (!isfinite(x)) {
        bad = 1;
        continue;
      }
      w = ldexp(x, -e);
      if (!(fabs(w) < 0x1p62)) {
        wide = 1;
        continue;
      }
      {
        const uint64_t mag = (uint64_t)fabs(trunc(w));
        if (mag > maxmag) maxmag = mag;
      }
    }
    if (bad) return SZ3O_E_NONFINITE;
    if (wide) return SZ3O_E_INVAL;
  }
  while (B < 64 && (maxmag >> B)) ++B;
  total = SZBP_HEADER + 4ull * W * (1ull + B);
  if (!out || cap < total) return SZ3O_E_CAPACITY;
  memset(out, 0, total);
  memcpy(out, "SZBP", 4);
  put_u32(out + 4, dtype);
  put_u64(out + 8, n);
  put_u32(out + 16, (uint32_t)e);
  put_u32(out + 20, B);
  put_u64(out + 24, W);
  /* pass 2: the sign plane, then the magnitude planes from bit B-1 down */
  for (i = 0; i < n; ++i) {
    const double t = trunc(ldexp(value_at(dtype, v, i), -e));
    const uint64_t mag = (uint64_t)fabs(t);
    uint8_t* planes = out + SZBP_HEADER;
    const uint64_t w = i / 32;
    const uint32_t bit = 1u << (i % 32);
    uint32_t word;
    if (t < 0) {
      memcpy(&word, planes + 4 * w, 4);
      word |= bit;
      memcpy(planes + 4 * w, &word, 4);
    }
    for (b = 0; b < B; ++b) {
      const uint64_t p = 1 + (uint64_t)(B - 1 - b); /* plane index: MSB first after the signs */
      if (!((mag >> b) & 1)) continue;
      memcpy(&word, planes + 4 * (p * W + w), 4);
      word |= bit;
      memcpy(planes + 4 * (p * W + w), &word, 4);
    }
  }
  *out_bytes = total;
  return SZ3O_OK;
}

int sz3o_bitplane_decode(const void* in_, uint64_t bytes, void* out, uint64_t cap, uint64_t* n_out) {
  const uint8_t* in = (const uint8_t*)in_;
  uint32_t dtype, B, eu, b;
  uint64_t n, W, i;
  int32_t e;
  if (!in || bytes < SZBP_HEADER || memcmp(in, "SZBP", 4) != 0) return SZ3O_E_CORRUPT;
  memcpy(&dtype, in + 4, 4);
  memcpy(&n, in + 8, 8);
  memcpy(&eu, in + 16, 4);
  memcpy(&B, in + 20, 4);
  memcpy(&W, in + 24, 8);
  e = (int32_t)eu;
  if (dtype > 1 || B > 62 || W != (n + 31) / 32 || n > (1ull << 40)) return SZ3O_E_CORRUPT;
  if (bytes < SZBP_HEADER + 4ull * W * (1ull + B)) return SZ3O_E_CORRUPT;
  if (n * (dtype == 0 ? 4u : 8u) > cap || (n && !out)) return SZ3O_E_CAPACITY;
  for (i = 0; i < n; ++i) {
    const uint8_t* planes = in + SZBP_HEADER;
    const uint64_t w = i / 32;
    const uint32_t sh = (uint32_t)(i % 32);
    uint32_t word;
    uint64_t mag = 0;
    double r;
    for (b = 0; b < B; ++b) {
      const uint64_t p = 1 + (uint64_t)(B - 1 - b);
      memcpy(&word, planes + 4 * (p * W + w), 4);
      mag |= (uint64_t)((word >> sh) & 1) << b;
    }
    memcpy(&word, planes + 4 * w, 4);
    r = ldexp((double)mag, e);
    if ((word >> sh) & 1) r = -r;
    if (dtype == 0) ((float*)out)[i] = (float)r;
    else ((double*)out)[i] = r;
  }
  if (n_out) *n_out = n;
  return SZ3O_OK;
}

int sz3o_huffman_fixed_lengths(uint32_t radius, uint8_t* len) {
  uint32_t s;
  if (!len || radius < 2 || radius > 32768) return SZ3O_E_INVAL;
  len[0] = SZ3O_LMAX;
  for (s = 1; s < 2 * radius; ++s) {
    const uint32_t k = s > radius ? s - radius : radius - s;
    uint32_t c = 0;
    while ((k >> c) != 0) ++c; /* bit length of k */
    len[s] = (uint8_t)(k == 0 ? 1 : (c >= 11 ? SZ3O_LMAX : 2 * c + 2));
  }
  return SZ3O_OK;
}
