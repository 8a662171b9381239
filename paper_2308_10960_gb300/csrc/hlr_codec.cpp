// Host AFL encoder (Section 3.2), its byte-aligned variants (AFLP, BFL, DFL) and the
// hlr_afl_encode / hlr_encode entry points.
//
// One unit of n values is stored as follows. m_min is the smallest nonzero magnitude; every
// magnitude is scaled by 1/m_min and shifted by +1 (the remark of Section 3.2), giving v >= 2
// for nonzero values and v = 1 for zeros. v is rounded half-up to m = ceil(-log2 u) mantissa
// bits on its FP64 bit pattern (a carry runs into the exponent); the stored exponent field is
// the unbiased exponent of v (>= 0) in e bits, e the smallest width that holds the largest
// field. The code of value j is sign | field | mantissa (sign on top), w = 1 + e + m bits,
// placed at stream bits [j w, (j+1) w), LSB-first, zero-padded to 16 bytes.
// AFLP raises m to the smallest m' for which 1 + e + m' is a multiple of 8. BFL stores the top
// 1 + 8 + m' bits of the FP32 pattern of the value (cast to nearest, then rounded half up to
// m' in {7, 15, 23}); DFL the top 1 + 11 + m' bits of the FP64 pattern rounded half up to
// m' in {4, 12, ..., 52}.
// MP (Section 3.3) stores each unit as IEEE FP16, FP32 or FP64 bit patterns (round to nearest
// even), the cheapest of the three whose unit roundoff 2^-11, 2^-24, 2^-53 is <= u.
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

static bool afl_params_m(const double *a, int64_t n, int m, AflParams *p);

bool afl_params(const double *a, int64_t n, double u, AflParams *p) { return afl_params_m(a, n, mantissa_bits(u), p); }

static bool afl_params_m(const double *a, int64_t n, int m, AflParams *p) {
  p->kind = VF_AFL;
  p->m = m;
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

static inline uint32_t fbits(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  return b;
}

// x rounded to nearest even into an IEEE binary16 pattern; false if it overflows. The
// quantum of the result is 2^(max(E, -14) - 10) for x = f 2^E, f in [1, 2) (2^-24 for the
// subnormal range): x / quantum rounded to an integer q is the significand with the implicit
// bit, and (E + 15) << 10 plus q - 1024 the pattern (a carry of q to 2048 moves into the
// exponent; below 2^-14 the pattern is q itself).
static bool half_bits(double x, uint16_t *out) {
  if (!std::isfinite(x)) return false;
  const double ax = std::fabs(x);
  int E = 0;
  std::frexp(ax, &E);
  const int ue = ax == 0.0 ? -25 : E - 1;
  const int qe = (ue < -14 ? -14 : ue) - 10;
  const double q = std::nearbyint(std::ldexp(ax, -qe));  // exact scaling, ties to even
  uint64_t code;
  if (ue < -14) {
    code = uint64_t(q);
  } else {
    code = (uint64_t(ue + 15) << 10) + uint64_t(q) - 1024;
    if (code >= 0x7C00) return false;
  }
  if (x < 0.0 || (x == 0.0 && std::signbit(x))) code |= 0x8000;
  *out = uint16_t(code);
  return true;
}

static int mp_kind(double u) { return u >= 0x1p-11 ? 16 : u >= 0x1p-24 ? 32 : 64; }

bool unit_params(int fmt, const double *a, int64_t n, double u, AflParams *p) {
  if (fmt == HLR_FMT_MP) {
    const int bits = mp_kind(u);
    for (int64_t j = 0; j < n; ++j) {
      uint16_t h;
      if (bits == 16 && !half_bits(a[j], &h)) return false;
      if (bits == 32 && !std::isfinite(float(a[j]))) return false;
      if (!std::isfinite(a[j])) return false;
    }
    p->kind = VF_MP;
    p->m_min = 1.0;
    p->e = bits == 16 ? 5 : bits == 32 ? 8 : 11;
    p->m = bits == 16 ? 10 : bits == 32 ? 23 : 52;
    p->w = bits;
    return true;
  }
  const int m = mantissa_bits(u);
  if (fmt == HLR_FMT_AFL_APLR) return afl_params_m(a, n, m, p);
  if (fmt == HLR_FMT_AFLP) {
    for (int mm = m;; ++mm) {
      if (!afl_params_m(a, n, mm, p)) return false;
      if (p->w % 8 == 0 || mm == 52) return true;
    }
  }
  if (fmt == HLR_FMT_BFL) {
    const int mp = m <= 7 ? 7 : m <= 15 ? 15 : 23;
    for (int64_t j = 0; j < n; ++j) {
      const float x = float(a[j]);
      if (!std::isfinite(a[j]) || !std::isfinite(x)) return false;
      uint64_t b = fbits(x);
      if (mp < 23) b = (b + (uint64_t(1) << (22 - mp))) & ~((uint64_t(1) << (23 - mp)) - 1);
      if (((b >> 23) & 0xFF) == 0xFF) return false;
    }
    p->kind = VF_BFL;
    p->m_min = 1.0;
    p->e = 8;
    p->m = mp;
    p->w = 9 + mp;
    return true;
  }
  if (fmt == HLR_FMT_DFL) {
    int mp = 4;
    while (mp < m) mp += 8;
    for (int64_t j = 0; j < n; ++j) {
      if (!std::isfinite(a[j])) return false;
      if (((round_bits(a[j], mp) >> 52) & 0x7FF) == 0x7FF) return false;
    }
    p->kind = VF_DFL;
    p->m_min = 1.0;
    p->e = 11;
    p->m = mp;
    p->w = 12 + mp;
    return true;
  }
  return false;
}

void unit_pack(const double *a, int64_t n, const AflParams &p, uint8_t *out) {
  if (p.kind == VF_AFL) {
    afl_pack(a, n, p, out);
    return;
  }
  uint64_t *words = reinterpret_cast<uint64_t *>(out);
  const int w = p.w;
  for (int64_t j = 0; j < n; ++j) {
    uint64_t code;
    if (p.kind == VF_MP) {
      uint16_t h = 0;
      if (w == 16) half_bits(a[j], &h);
      code = w == 16 ? uint64_t(h) : w == 32 ? uint64_t(fbits(float(a[j]))) : dbits(a[j]);
    } else if (p.kind == VF_BFL) {
      uint64_t b = fbits(float(a[j]));
      if (p.m < 23) b = (b + (uint64_t(1) << (22 - p.m))) & ~((uint64_t(1) << (23 - p.m)) - 1);
      code = b >> (23 - p.m);
    } else {
      code = round_bits(a[j], p.m) >> (52 - p.m);
    }
    const uint64_t bit = uint64_t(j) * uint64_t(w);
    const uint64_t wi = bit >> 6;
    const unsigned off = unsigned(bit & 63);
    words[wi] |= code << off;
    if (off + unsigned(w) > 64) words[wi + 1] |= code >> (64 - off);
  }
}

}  // namespace hlr

extern "C" int hlr_encode(int32_t fmt, const double *a, int64_t n, double u, double *m_min, int32_t *e, int32_t *m,
                          uint8_t *out, size_t cap, size_t *nbytes) {
  using namespace hlr;
  if (n < 0 || (n > 0 && !a) || !m_min || !e || !m || !nbytes)
    return set_error(HLR_ERR_INVALID, "hlr_encode: null argument or negative n");
  if (!(u > 0.0) || !std::isfinite(u))
    return set_error(HLR_ERR_INVALID, "hlr_encode: precision must be positive and finite");
  if (fmt != HLR_FMT_AFL_APLR && fmt != HLR_FMT_AFLP && fmt != HLR_FMT_BFL && fmt != HLR_FMT_DFL &&
      fmt != HLR_FMT_MP)
    return set_error(HLR_ERR_INVALID, "hlr_encode: unknown format");
  AflParams p;
  if (!unit_params(fmt, a, n, u, &p)) return set_error(HLR_ERR_INVALID, "hlr_encode: value not representable");
  const size_t need = padded16(afl_bytes(n, p.w));
  *m_min = p.m_min;
  *e = p.e;
  *m = p.m;
  *nbytes = need;
  if (cap < need) return set_error(HLR_ERR_OOM, "hlr_encode: output buffer too small");
  if (need == 0) return HLR_OK;
  std::vector<uint64_t> tmp(need / 8 + 1, 0);
  unit_pack(a, n, p, reinterpret_cast<uint8_t *>(tmp.data()));
  std::memcpy(out, tmp.data(), need);
  return HLR_OK;
}

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
