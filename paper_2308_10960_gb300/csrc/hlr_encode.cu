// GPU encoder (Section 3.2 per unit, with the per-column precisions of AFL-APLR, Section 3.3,
// supplied by the caller): hlr_encode_device. Writes, for every unit, exactly the stream the
// host encoder hlr_encode writes, so that data built on the GPU is compressed where it lives
// instead of being copied to the host first (the paper's advice to compress during
// construction, Section 5.3).
//
// Five launches on the caller's stream, none of which allocates:
//   k_params_w / _b : parameters (m_min, e, m) of every unit and its padded stream size,
//              written to out_off[u + 1]; a warp per unit of at most kSmall values, a CTA per
//              larger unit;
//   k_scan   : one CTA: in-place inclusive scan of the sizes into stream offsets;
//   k_pack_w / _b : the codes, 32 values at a time per warp: the 32 codes of a group fill
//              exactly w 32-bit words, assembled in shared memory and stored whole (a warp per
//              small unit, the warps of a CTA taking turns on a large one).
// The results equal the host encoder's operation by operation: |a| / m_min + 1 in two IEEE
// round-to-nearest steps, half-up rounding of the FP64 pattern to m mantissa bits, FP32 / FP16
// casts by the round-to-nearest-even conversions. GB300's FP64 pipe is narrow, so the AFL
// codes take the quotient from a per-unit reciprocal and fall back to the IEEE division only
// where that approximation could round differently (see afl_rounded).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hlr_internal.h"

namespace hlr {
namespace {

constexpr int kEncThreads = 256;
constexpr int kEncWarps = kEncThreads / 32;

__device__ __forceinline__ uint64_t d2u(double x) { return static_cast<uint64_t>(__double_as_longlong(x)); }
__device__ __forceinline__ double u2d(uint64_t b) { return __longlong_as_double(static_cast<long long>(b)); }

// ceil(-log2 u) clamped to [0, 52] (u > 0 finite): u = f 2^E, f in [1/2, 1) gives 1 - E; for
// a normal u with biased exponent b, E = b - 1022
__device__ __forceinline__ int mbits_of(double u) {
  const int b = int((d2u(u) >> 52) & 0x7ff);
  if (b == 0) return 52;  // subnormal precision: all mantissa bits
  const int m = 1023 - b;
  return m < 0 ? 0 : m > 52 ? 52 : m;
}
// FP64 pattern b rounded half up to m mantissa bits (a carry runs into the exponent)
__device__ __forceinline__ uint64_t round_pattern(uint64_t b, int m) {
  if (m < 52) {
    b += uint64_t(1) << (51 - m);
    b &= ~((uint64_t(1) << (52 - m)) - 1);
  }
  return b;
}
__device__ __forceinline__ uint32_t f32_bits_rn(double x) { return __float_as_uint(__double2float_rn(x)); }
__device__ __forceinline__ uint32_t f16_bits_rn(double x) {
  unsigned short h;
  asm("cvt.rn.f16.f64 %0, %1;" : "=h"(h) : "d"(x));
  return h;
}
// BFL: the FP32 pattern rounded half up to m' mantissa bits
__device__ __forceinline__ uint32_t bfl_bits(double x, int mp) {
  uint32_t b = f32_bits_rn(x);
  if (mp < 23) b = (b + (1u << (22 - mp))) & ~((1u << (23 - mp)) - 1u);
  return b;
}
// MP: IEEE width (16, 32, 64) of the cheapest format with unit roundoff <= u (Table 1)
__device__ __forceinline__ int mp_bits(double u) { return u >= 0x1p-11 ? 16 : u >= 0x1p-24 ? 32 : 64; }

// v = RN(RN(av / m_min) + 1), exactly as the host computes it (av = |a| > 0 finite).
__device__ __forceinline__ double afl_v_exact(double av, double m_min) {
  return __dadd_rn(__ddiv_rn(av, m_min), 1.0);
}
// The pattern of v rounded half up to m bits, from the reciprocal r = RN(1 / m_min). The
// quotient q0 = RN(av r) is within 3 ulps of RN(av / m_min) (r and the product each add at most
// half an ulp of relative error), so RN(q0 + 1) is within 4 ulps of v (ulp(v) >= ulp(q)) and
// its pattern within 8 units of v's (16 across a binade edge). The half-up rounding to m bits
// only changes where the low 52 - m bits cross 2^(51 - m); when q0 + 1 lands farther than 32
// units from that point (and m <= 46, so the low bits have room), both round alike. Elsewhere
// the exact division decides: for m = 20 that is about one value in 2^26.
__device__ __forceinline__ uint64_t afl_rounded(double av, double m_min, double r, int m) {
  // (r must be a normal number for the error bound; a quotient that overflows goes the exact way)
  const uint32_t re = uint32_t(d2u(r) >> 52) & 0x7ffu;
  if (m <= 46 && re != 0 && re != 0x7ffu) {
    const uint64_t b = d2u(__dadd_rn(__dmul_rn(av, r), 1.0));
    const uint64_t low = b & ((uint64_t(1) << (52 - m)) - 1);
    const uint64_t half = uint64_t(1) << (51 - m);
    const uint64_t dist = low > half ? low - half : half - low;
    if (dist > 32 && ((b >> 52) & 0x7ff) != 0x7ff) return round_pattern(b, m);
  }
  return round_pattern(d2u(afl_v_exact(av, m_min)), m);
}

// Reductions over a group of NT threads that handles one unit: a warp (NT = 32: shuffles only)
// or the whole CTA (NT = kEncThreads: shuffles, then one slot per warp in shared memory). Every
// thread of the group gets the result.
struct RedShared {
  unsigned long long a[kEncWarps], b[kEncWarps];
  int i[kEncWarps];
};
template <int NT>
__device__ __forceinline__ int grp_rank() {
  return NT == 32 ? int(threadIdx.x & 31) : int(threadIdx.x);
}
// (min of a, max of b) over the group
template <int NT>
__device__ void grp_minmax(unsigned long long &a, unsigned long long &b, RedShared *sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a = min(a, (unsigned long long)__shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, (unsigned long long)__shfl_xor_sync(0xffffffffu, b, o));
  }
  if constexpr (NT != 32) {
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      sh->a[threadIdx.x >> 5] = a;
      sh->b[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    a = sh->a[0];
    b = sh->b[0];
    for (int k = 1; k < NT / 32; ++k) {
      a = min(a, sh->a[k]);
      b = max(b, sh->b[k]);
    }
    __syncthreads();
  }
}
template <int NT>
__device__ int grp_or(int v, RedShared *sh) {
  v = int(__reduce_or_sync(0xffffffffu, unsigned(v)));
  if constexpr (NT != 32) {
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh->i[threadIdx.x >> 5] = v;
    __syncthreads();
    v = 0;
    for (int k = 0; k < NT / 32; ++k) v |= sh->i[k];
    __syncthreads();
  }
  return v;
}

__device__ __forceinline__ int bit_length(unsigned long long x) { return x ? 64 - __clzll(x) : 0; }

// Units of at most kSmall values are handled by one warp each, larger ones by a whole CTA; both
// kernels see every unit and take exactly the units of their class.
constexpr int64_t kSmall = 2048;
__device__ __forceinline__ bool small_unit(const int64_t *off, int64_t u) { return off[u + 1] - off[u] <= kSmall; }

// parameters and padded stream size of unit u, computed by a group of NT threads
template <int NT>
__device__ void unit_params_dev(int fmt, int64_t u, int64_t total, const int64_t *__restrict__ off,
                                const double *__restrict__ a, const double *__restrict__ uprec, double *m_min_out,
                                int32_t *e_out, int32_t *m_out, int64_t *out_off, RedShared *sh) {
  const int64_t j0 = off[u], n = off[u + 1] - j0;
  const double uu = uprec[u];
  // a unit whose precision is not positive and finite, or whose offsets decrease or leave
  // [0, total], is rejected (and its values are not read)
  bool bad = !(uu > 0.0) || !(uu <= 1.7976931348623157e308) || n < 0 || j0 < 0 || off[u + 1] > total;
  const double *x = a + (bad ? 0 : j0);
  double m_min = 1.0;
  int e = 0, m = 0, w = 1;
  if (!bad && (fmt == HLR_FMT_AFL_APLR || fmt == HLR_FMT_AFLP)) {
    // Every rounding step of a code is monotone in |a|, so the largest exponent field is the
    // field of the largest magnitude: one pass finds the smallest nonzero and the largest
    // magnitude (non-negative doubles order like their bit patterns), one division per unit
    // gives the field.
    m = mbits_of(uu);
    unsigned long long mn = ~0ull, mx = 0;
    int nf = 0;
    for (int64_t j = grp_rank<NT>(); j < n; j += NT) {
      const unsigned long long b = d2u(x[j]) & 0x7fffffffffffffffull;
      if (b >= 0x7ff0000000000000ull) nf = 1;
      if (b != 0) mn = min(mn, b);
      mx = max(mx, b);
    }
    bad = grp_or<NT>(nf, sh) != 0;
    grp_minmax<NT>(mn, mx, sh);
    if (!bad) {
      if (mx == 0) {  // all zero: e = 0 (AFLP still aligns 1 + m)
        m_min = 0.0;
        e = 0;
        while (fmt == HLR_FMT_AFLP && (1 + m) % 8 != 0 && m < 52) ++m;
      } else {
        m_min = u2d(mn);
        const uint64_t vb = d2u(afl_v_exact(u2d(mx), m_min));
        for (;; ++m) {
          e = bit_length((unsigned long long)((round_pattern(vb, m) >> 52) - 1023));
          if (fmt == HLR_FMT_AFL_APLR || (1 + e + m) % 8 == 0 || m == 52) break;
        }
      }
      w = 1 + e + m;
    }
  } else if (!bad) {
    int over = 0;
    if (fmt == HLR_FMT_BFL) {
      const int mb = mbits_of(uu);
      m = mb <= 7 ? 7 : mb <= 15 ? 15 : 23;
      e = 8;
      for (int64_t j = grp_rank<NT>(); j < n; j += NT) {
        const double v = x[j];
        if (!(fabs(v) <= 1.7976931348623157e308) || ((bfl_bits(v, m) >> 23) & 0xffu) == 0xffu) over = 1;
      }
    } else if (fmt == HLR_FMT_DFL) {
      const int mb = mbits_of(uu);
      m = 4;
      while (m < mb) m += 8;
      e = 11;
      for (int64_t j = grp_rank<NT>(); j < n; j += NT)
        if (((round_pattern(d2u(x[j]), m) >> 52) & 0x7ff) == 0x7ff) over = 1;  // also NaN / Inf input
    } else {  // HLR_FMT_MP
      const int bits = mp_bits(uu);
      e = bits == 16 ? 5 : bits == 32 ? 8 : 11;
      m = bits == 16 ? 10 : bits == 32 ? 23 : 52;
      for (int64_t j = grp_rank<NT>(); j < n; j += NT) {
        const double v = x[j];
        if (!(fabs(v) <= 1.7976931348623157e308)) over = 1;
        if (bits == 32 && (f32_bits_rn(v) & 0x7f800000u) == 0x7f800000u) over = 1;
        if (bits == 16 && (f16_bits_rn(v) & 0x7c00u) == 0x7c00u) over = 1;
      }
    }
    bad = grp_or<NT>(over, sh) != 0;
    w = 1 + e + m;
  }
  if (grp_rank<NT>() == 0) {
    m_min_out[u] = bad ? 0.0 : m_min;
    e_out[u] = bad ? -1 : e;
    m_out[u] = bad ? 0 : m;
    out_off[u + 1] = bad ? 0 : int64_t(((uint64_t(n) * uint64_t(w) + 7) / 8 + 15) & ~uint64_t(15));
  }
}

// small units: one warp each
__global__ void __launch_bounds__(kEncThreads) k_params_w(int fmt, int64_t nunits, int64_t total,
                                                           const int64_t *__restrict__ off, const double *__restrict__ a,
                                                           const double *__restrict__ uprec, double *m_min_out,
                                                           int32_t *e_out, int32_t *m_out, int64_t *out_off) {
  const int64_t nwarps = int64_t(gridDim.x) * kEncWarps;
  for (int64_t u = int64_t(blockIdx.x) * kEncWarps + (threadIdx.x >> 5); u < nunits; u += nwarps)
    if (small_unit(off, u)) unit_params_dev<32>(fmt, u, total, off, a, uprec, m_min_out, e_out, m_out, out_off, nullptr);
}
// large units: one CTA each
__global__ void __launch_bounds__(kEncThreads) k_params_b(int fmt, int64_t nunits, int64_t total,
                                                           const int64_t *__restrict__ off, const double *__restrict__ a,
                                                           const double *__restrict__ uprec, double *m_min_out,
                                                           int32_t *e_out, int32_t *m_out, int64_t *out_off) {
  __shared__ RedShared sh;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    if (small_unit(off, u)) continue;
    unit_params_dev<kEncThreads>(fmt, u, total, off, a, uprec, m_min_out, e_out, m_out, out_off, &sh);
  }
}

// in-place inclusive scan of out_off[1..nunits] into stream offsets (out_off[0] = 0), by one
// CTA of kScanThreads threads walking tiles of kScanThreads * 4 entries: coalesced loads, a
// scan of the tile in shared memory, the running total carried from tile to tile
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan(int64_t nunits, int64_t *out_off) {
  __shared__ int64_t wsum[kScanThreads / 32];
  __shared__ int64_t carry;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) {
    carry = 0;
    out_off[0] = 0;
  }
  __syncthreads();
  for (int64_t base = 1; base <= nunits; base += int64_t(kScanThreads) * 4) {
    // thread t owns entries base + 4t .. base + 4t + 3
    int64_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = base + 4 * int64_t(t) + k;
      v[k] = i <= nunits ? out_off[i] : 0;
      s += v[k];
    }
    // inclusive scan of the threads' sums: within the warp, then over the warps
    int64_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t w = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < kScanThreads / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t run = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - s;  // exclusive prefix of thread t
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = base + 4 * int64_t(t) + k;
      run += v[k];
      if (i <= nunits) out_off[i] = run;
    }
    __syncthreads();
    if (t == kScanThreads - 1) carry = run;
    __syncthreads();
  }
}

// AFL code of x for a unit with w = 1 + e + m <= 32 in 32-bit integer operations (64-bit ones
// would share GB300's narrow FP64 pipe with the two FP64 operations of the quotient), by the
// reasoning of afl_rounded: the pattern b of RN(|x| r + 1) rounds like v unless (b + half + 32)
// mod L <= 64 (L = 2^(52 - m), half = L / 2); then, and when the unit cannot take the fast path
// (fast = false: m >= 46, r not normal), the IEEE division decides.
__device__ __forceinline__ uint32_t afl_code32(double x, double m_min, double r, bool fast, int e, int m) {
  const uint32_t xh = uint32_t(__double2hiint(x)), xl = uint32_t(__double2loint(x));
  const uint32_t ah = xh & 0x7fffffffu;
  if ((ah | xl) == 0u) return 0u;  // v = 1: field 0, mantissa 0, no sign
  const double av = __hiloint2double(int(ah), int(xl));
  uint32_t bh = 0, bl = 0;
  bool near = !fast;
  if (fast) {
    const double v0 = __dadd_rn(__dmul_rn(av, r), 1.0);
    bh = uint32_t(__double2hiint(v0));
    bl = uint32_t(__double2loint(v0));
    if ((bh >> 20) >= 0x7ffu) {
      near = true;  // the approximate quotient overflowed
    } else if (m < 20) {
      // L > 2^32: the low bits are (bh mod 2^(20 - m), bl); half = 2^(19 - m) in the high word
      const uint32_t cl = bl + 32u;
      const uint32_t ch = (bh + (1u << (19 - m)) + (cl < 32u ? 1u : 0u)) & ((1u << (20 - m)) - 1u);
      near = ch == 0u && cl <= 64u;
      bh = (bh + (1u << (19 - m))) & ~((1u << (20 - m)) - 1u);
      bl = 0u;
    } else {
      const int sh = 52 - m;  // 21 .. 32 (m <= 31 here)
      const uint32_t lmask = sh >= 32 ? 0xffffffffu : (1u << sh) - 1u;
      const uint32_t half = 1u << (sh - 1);
      near = ((bl + half + 32u) & lmask) <= 64u;
      const uint32_t t = bl + half;
      bh += t < bl ? 1u : 0u;
      bl = t & ~lmask;
    }
  }
  if (near) {
    const uint64_t b = round_pattern(d2u(afl_v_exact(av, m_min)), m);
    bh = uint32_t(b >> 32);
    bl = uint32_t(b);
  }
  const uint32_t field = (bh >> 20) - 1023u;
  const uint32_t mant = m <= 20 ? (bh & 0xfffffu) >> (20 - m) : ((bh & 0xfffffu) << (m - 20)) | (bl >> (52 - m));
  return ((xh >> 31) << (e + m)) | (field << m) | mant;
}

// code of value x of a unit (w = 1 + e + m bits, low bits of the result); r = RN(1 / m_min)
__device__ __forceinline__ uint64_t code_of(int fmt, double x, double m_min, double r, int e, int m) {
  if (fmt == HLR_FMT_AFL_APLR || fmt == HLR_FMT_AFLP) {
    const double av = fabs(x);
    if (m_min == 0.0 || av == 0.0) return 0;  // v = 1: field 0, mantissa 0, no sign
    const uint64_t b = afl_rounded(av, m_min, r, m);
    const uint64_t field = (b >> 52) - 1023;
    const uint64_t mant = (b & ((uint64_t(1) << 52) - 1)) >> (52 - m);
    const uint64_t sign = x < 0.0 ? 1 : 0;
    return (sign << (e + m)) | (field << m) | mant;
  }
  if (fmt == HLR_FMT_BFL) return uint64_t(bfl_bits(x, m) >> (23 - m));
  if (fmt == HLR_FMT_DFL) return round_pattern(d2u(x), m) >> (52 - m);
  // HLR_FMT_MP
  if (e == 5) return f16_bits_rn(x);
  if (e == 8) return f32_bits_rn(x);
  return d2u(x);
}

// Groups g0, g0 + gs, ... of 32 values of unit u, one warp: lane l builds the code of value
// 32 g + l, ORs its (up to three) word parts into the warp's buffer of w words, and the warp
// stores the w words (clipped to the unit's padded stream, whose tail words are zeroed).
__device__ void pack_groups(int fmt, int64_t u, int64_t g0, int64_t gs, const int64_t *__restrict__ off,
                            const double *__restrict__ a, const double *__restrict__ m_min_in,
                            const int32_t *__restrict__ e_in, const int32_t *__restrict__ m_in,
                            const int64_t *__restrict__ out_off, uint8_t *out, uint64_t cap, uint32_t *buf) {
  const int lane = threadIdx.x & 31;
  const int e = e_in[u];
  if (e < 0) return;
  const int m = m_in[u], w = 1 + e + m;
  const double m_min = m_min_in[u];
  const double r = m_min != 0.0 ? __drcp_rn(m_min) : 0.0;
  const bool afl = fmt == HLR_FMT_AFL_APLR || fmt == HLR_FMT_AFLP;
  const bool narrow = w <= 32 && fmt != HLR_FMT_DFL && !(afl && m_min == 0.0);
  const uint32_t re = uint32_t(d2u(r) >> 52) & 0x7ffu;
  const bool fast = m <= 45 && re != 0 && re != 0x7ffu;
  const int64_t j0 = off[u], n = off[u + 1] - j0;
  const uint64_t o0 = uint64_t(out_off[u]), o1 = uint64_t(out_off[u + 1]);
  if (o1 > cap || o1 < o0) return;  // unreachable when cap holds the bound the host checked
  const double *x = a + j0;
  uint32_t *dst = reinterpret_cast<uint32_t *>(out + o0);
  const int64_t nw = int64_t((o1 - o0) / 4);
  const int64_t ngroups = (n + 31) / 32;
  for (int64_t g = g0; g < ngroups; g += gs) {
    for (int k = lane; k < w; k += 32) buf[k] = 0;
    __syncwarp();
    const int64_t j = 32 * g + lane;
    if (j < n) {
      const int bit = lane * w;  // within the group's w words
      const int q = bit >> 5, s = bit & 31;
      if (narrow) {  // a 32-bit code: at most two words
        const uint32_t code = afl ? afl_code32(x[j], m_min, r, fast, e, m) : uint32_t(code_of(fmt, x[j], m_min, r, e, m));
        const uint32_t p0 = code << s, p1 = s ? code >> (32 - s) : 0u;
        if (p0) atomicOr(&buf[q], p0);
        if (p1) atomicOr(&buf[q + 1], p1);
      } else {
        const uint64_t code = code_of(fmt, x[j], m_min, r, e, m);
        const uint64_t lo = code << s;
        const uint32_t p0 = uint32_t(lo), p1 = uint32_t(lo >> 32), p2 = s ? uint32_t(code >> (64 - s)) : 0u;
        if (p0) atomicOr(&buf[q], p0);
        if (p1) atomicOr(&buf[q + 1], p1);
        if (p2) atomicOr(&buf[q + 2], p2);
      }
    }
    __syncwarp();
    const int64_t wbase = g * w;
    for (int k = lane; k < w; k += 32)
      if (wbase + k < nw) dst[wbase + k] = buf[k];
    __syncwarp();
  }
  // words of the padded stream past the last group (written by the group-0 warp)
  if (g0 == 0)
    for (int64_t k = ngroups * w + lane; k < nw; k += 32) dst[k] = 0u;
}

__global__ void __launch_bounds__(kEncThreads) k_pack_w(int fmt, int64_t nunits, const int64_t *__restrict__ off,
                                                         const double *__restrict__ a, const double *__restrict__ m_min_in,
                                                         const int32_t *__restrict__ e_in, const int32_t *__restrict__ m_in,
                                                         const int64_t *__restrict__ out_off, uint8_t *out, uint64_t cap) {
  __shared__ uint32_t bufs[kEncWarps][68];
  uint32_t *buf = bufs[threadIdx.x >> 5];
  const int64_t nwarps = int64_t(gridDim.x) * kEncWarps;
  for (int64_t u = int64_t(blockIdx.x) * kEncWarps + (threadIdx.x >> 5); u < nunits; u += nwarps)
    if (small_unit(off, u)) pack_groups(fmt, u, 0, 1, off, a, m_min_in, e_in, m_in, out_off, out, cap, buf);
}
__global__ void __launch_bounds__(kEncThreads) k_pack_b(int fmt, int64_t nunits, const int64_t *__restrict__ off,
                                                         const double *__restrict__ a, const double *__restrict__ m_min_in,
                                                         const int32_t *__restrict__ e_in, const int32_t *__restrict__ m_in,
                                                         const int64_t *__restrict__ out_off, uint8_t *out, uint64_t cap) {
  __shared__ uint32_t bufs[kEncWarps][68];
  uint32_t *buf = bufs[threadIdx.x >> 5];
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x)
    if (!small_unit(off, u))
      pack_groups(fmt, u, threadIdx.x >> 5, kEncWarps, off, a, m_min_in, e_in, m_in, out_off, out, cap, buf);
}

}  // namespace
}  // namespace hlr

using namespace hlr;

extern "C" int hlr_encode_device(int32_t fmt, int64_t nunits, const int64_t *off_dev, int64_t total_values,
                                 const double *a_dev, const double *u_dev, double *m_min_dev, int32_t *e_dev,
                                 int32_t *m_dev, int64_t *out_off_dev, uint8_t *out_dev, size_t cap,
                                 void *cuda_stream) {
  if (fmt != HLR_FMT_AFL_APLR && fmt != HLR_FMT_AFLP && fmt != HLR_FMT_BFL && fmt != HLR_FMT_DFL &&
      fmt != HLR_FMT_MP)
    return set_error(HLR_ERR_INVALID, "hlr_encode_device: unknown format");
  if (nunits < 0 || total_values < 0) return set_error(HLR_ERR_INVALID, "hlr_encode_device: negative size");
  if (nunits == 0) return HLR_OK;
  if (!off_dev || !u_dev || !m_min_dev || !e_dev || !m_dev || !out_off_dev || !out_dev || (total_values > 0 && !a_dev))
    return set_error(HLR_ERR_INVALID, "hlr_encode_device: null pointer");
  if (reinterpret_cast<uintptr_t>(out_dev) & 15)
    return set_error(HLR_ERR_INVALID, "hlr_encode_device: out_dev must be 16-byte aligned");
  const double need = 8.0 * double(total_values) + 16.0 * double(nunits);
  if (double(cap) < need) return set_error(HLR_ERR_OOM, "hlr_encode_device: cap below 8 total_values + 16 nunits");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaGetLastError();
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  // grid-stride launches: 8 CTAs per SM (a warp per small unit), 4 CTAs per SM (a CTA per
  // large unit), capped by the units
  const unsigned gw = unsigned(std::min<int64_t>((nunits + kEncWarps - 1) / kEncWarps, int64_t(sms) * 8));
  const unsigned gb = unsigned(std::min<int64_t>(nunits, int64_t(sms) * 4));
  k_params_w<<<gw, kEncThreads, 0, st>>>(fmt, nunits, total_values, off_dev, a_dev, u_dev, m_min_dev, e_dev, m_dev,
                                         out_off_dev);
  k_params_b<<<gb, kEncThreads, 0, st>>>(fmt, nunits, total_values, off_dev, a_dev, u_dev, m_min_dev, e_dev, m_dev,
                                         out_off_dev);
  k_scan<<<1, kScanThreads, 0, st>>>(nunits, out_off_dev);
  k_pack_w<<<gw, kEncThreads, 0, st>>>(fmt, nunits, off_dev, a_dev, m_min_dev, e_dev, m_dev, out_off_dev, out_dev,
                                       uint64_t(cap));
  k_pack_b<<<gb, kEncThreads, 0, st>>>(fmt, nunits, off_dev, a_dev, m_min_dev, e_dev, m_dev, out_off_dev, out_dev,
                                       uint64_t(cap));
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string("hlr_encode_device: ") + cudaGetErrorString(err));
  return HLR_OK;
}
