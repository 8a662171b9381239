// Host AFL encoder (Section 3.2) and the hlr_afl_encode entry point.
//
// One unit of n values is stored as follows. m_min is the smallest nonzero magnitude; every
// magnitude is scaled by 1/m_min and shifted by +1 (the remark of Section 3.2), giving v >= 2
// for nonzero values and v = 1 for zeros. v is rounded half-up to m = ceil(-log2 u) mantissa
// bits on its FP64 bit pattern (a carry runs into the exponent); the stored exponent field is
// the unbiased exponent of v (>= 0) in e bits, e the smallest width that holds the largest
// field. The code of value j is sign | field | mantissa (sign on top), w = 1 + e + m bits,
// placed at stream bits [j w, (j+1) w), LSB-first, zero-padded to 16 bytes.
// Compiled with -ffp-contract=off: every FP64 operation is a separately rounded IEEE op.
#include <cmath>
#include <cstring>

#include "hlr_internal.h"

namespace hlr {

int mantissa_bits(double u) {
  int E = 0;
  std::frexp(u, &E);  // u = f 2^E with f in [1/2, 1) -> ceil(-log2 u) = 1 - E
  int m = 1 - E;
  if (m < 0) m = 0;
  if (m > 52) m = 52;
  return m;
}

static inline uint64_t dbits(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
}

static inline uint64_t round_bits(double v, int m) {
  uint64_t b = dbits(v);
  if (m < 52) {
    b += uint64_t(1) << (51 - m);
    b &= ~((uint64_t(1) << (52 - m)) - 1);
  }
  return b;
}

static inline int bit_length(uint64_t x) {
  int l = 0;
  while (x) {
    ++l;
    x >>= 1;
  }
  return l;
}

bool afl_params(const double *a, int64_t n, double u, AflParams *p) {
  p->m = mantissa_bits(u);
  double m_min = INFINITY;
  for (int64_t j = 0; j < n; ++j) {
    double x = a[j];
    if (!std::isfinite(x)) return false;
    double ax = std::fabs(x);
    if (ax != 0.0 && ax < m_min) m_min = ax;
  }
  if (!(m_min < INFINITY)) {  // all zero
    p->m_min = 0.0;
    p->e = 0;
    p->w = 1 + p->m;
    return true;
  }
  int64_t fmax = 0;
  for (int64_t j = 0; j < n; ++j) {
    double v = std::fabs(a[j]) / m_min + 1.0;
    int64_t field = int64_t(round_bits(v, p->m) >> 52) - 1023;
    if (field > fmax) fmax = field;
  }
  p->m_min = m_min;
  p->e = bit_length(uint64_t(fmax));
  p->w = 1 + p->e + p->m;
  return true;
}

void afl_pack(const double *a, int64_t n, const AflParams &p, uint8_t *out) {
  const int e = p.e, m = p.m, w = p.w;
  uint64_t *words = reinterpret_cast<uint64_t *>(out);  // out is 16-byte aligned
  const uint64_t mmask = (uint64_t(1) << 52) - 1;
  for (int64_t j = 0; j < n; ++j) {
    uint64_t code = 0;
    if (p.m_min != 0.0) {
      double v = std::fabs(a[j]) / p.m_min + 1.0;
      uint64_t b = round_bits(v, m);
      uint64_t field = (b >> 52) - 1023;
      uint64_t mant = (b & mmask) >> (52 - m);
      uint64_t sign = a[j] < 0.0 ? 1 : 0;
      code = (sign << (e + m)) | (field << m) | mant;
    }
    uint64_t bit = uint64_t(j) * uint64_t(w);
    uint64_t wi = bit >> 6;
    unsigned off = unsigned(bit & 63);
    words[wi] |= code << off;
    if (off + unsigned(w) > 64) words[wi + 1] |= code >> (64 - off);
  }
}

}  // namespace hlr

extern "C" int hlr_afl_encode(const double *a, int64_t n, double u, double *m_min, int32_t *e,
                              int32_t *m, uint8_t *out, size_t cap, size_t *nbytes) {
  using namespace hlr;
  if (n < 0 || (n > 0 && !a) || !m_min || !e || !m || !nbytes)
    return set_error(HLR_ERR_INVALID, "hlr_afl_encode: null argument or negative n");
  if (!(u > 0.0) || !std::isfinite(u))
    return set_error(HLR_ERR_INVALID, "hlr_afl_encode: precision must be positive and finite");
  AflParams p;
  if (!afl_params(a, n, u, &p)) return set_error(HLR_ERR_INVALID, "hlr_afl_encode: non-finite input");
  size_t need = padded16(afl_bytes(n, p.w));
  *m_min = p.m_min;
  *e = p.e;
  *m = p.m;
  *nbytes = need;
  if (cap < need) return set_error(HLR_ERR_OOM, "hlr_afl_encode: output buffer too small");
  if (need == 0) return HLR_OK;
  // pack into an aligned scratch buffer so that 64-bit word access is valid
  std::vector<uint64_t> tmp(need / 8 + 1, 0);
  afl_pack(a, n, p, reinterpret_cast<uint8_t *>(tmp.data()));
  std::memcpy(out, tmp.data(), need);
  return HLR_OK;
}
