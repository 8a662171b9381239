// GPU encoder (Section 3.2 per unit, with the per-column precisions of AFL-APLR, Section 3.3,
// supplied by the caller): hlr_encode_device. Writes, for every unit, exactly the stream the
// host encoder hlr_encode writes, so that data built on the GPU is compressed where it lives
// instead of being copied to the host first (the paper's advice to compress during
// construction, Section 5.3).
//
// Three launches on the caller's stream, none of which allocates:
//   k_params : one CTA per unit: parameters (m_min, e, m) from two or more reductions over the
//              unit's values, and its padded stream size written to out_off[u + 1];
//   k_scan   : one CTA: in-place inclusive scan of the sizes into stream offsets;
//   k_pack   : one CTA per unit, one thread per 32-bit output word: the codes overlapping the
//              word are built and OR-ed together, so no two threads write the same word.
// Arithmetic follows the host encoder operation by operation: |a| / m_min + 1 in two IEEE
// round-to-nearest steps (__ddiv_rn, __dadd_rn), half-up rounding of the FP64 pattern to m
// mantissa bits, FP32 / FP16 casts by the round-to-nearest-even conversions.
#include <cuda_runtime.h>

#include <cstdint>

#include "hlr_internal.h"

namespace hlr {
namespace {

constexpr int kEncThreads = 256;

__device__ __forceinline__ uint64_t d2u(double x) { return static_cast<uint64_t>(__double_as_longlong(x)); }

// ceil(-log2 u) clamped to [0, 52] (u > 0 finite): u = f 2^E, f in [1/2, 1) gives 1 - E; for
// a normal u with biased exponent b, E = b - 1022
__device__ __forceinline__ int mbits_of(double u) {
  const int b = int((d2u(u) >> 52) & 0x7ff);
  if (b == 0) return 52;  // subnormal precision: all mantissa bits
  const int m = 1023 - b;
  return m < 0 ? 0 : m > 52 ? 52 : m;
}
// FP64 pattern of v rounded half up to m mantissa bits (a carry runs into the exponent)
__device__ __forceinline__ uint64_t round_bits(double v, int m) {
  uint64_t b = d2u(v);
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

// block-wide reductions (kEncThreads threads)
__device__ double block_min(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = sh[0];
  for (int k = 1; k < kEncThreads / 32; ++k) v = fmin(v, sh[k]);
  return v;
}
__device__ long long block_max(long long v, long long *sh) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = sh[0];
  for (int k = 1; k < kEncThreads / 32; ++k) v = max(v, sh[k]);
  return v;
}
__device__ int block_or(int v, int *sh) {
  v = __reduce_or_sync(0xffffffffu, unsigned(v));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0;
  for (int k = 0; k < kEncThreads / 32; ++k) v |= sh[k];
  return v;
}

__device__ __forceinline__ int bit_length(unsigned long long x) { return x ? 64 - __clzll(x) : 0; }

// largest exponent field of the AFL codes of a unit at m mantissa bits
__device__ long long afl_fmax(const double *a, int64_t n, double m_min, int m, long long *sh) {
  long long f = 0;
  for (int64_t j = threadIdx.x; j < n; j += kEncThreads) {
    const double v = __dadd_rn(__ddiv_rn(fabs(a[j]), m_min), 1.0);
    f = max(f, (long long)(round_bits(v, m) >> 52) - 1023);
  }
  return block_max(f, sh);
}

__global__ void __launch_bounds__(kEncThreads) k_params(int fmt, int64_t nunits, int64_t total,
                                                         const int64_t *__restrict__ off,
                                                         const double *__restrict__ a, const double *__restrict__ uprec,
                                                         double *m_min_out, int32_t *e_out, int32_t *m_out,
                                                         int64_t *out_off) {
  __shared__ double shd[kEncThreads / 32];
  __shared__ long long shl[kEncThreads / 32];
  __shared__ int shi[kEncThreads / 32];
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t j0 = off[u], n = off[u + 1] - j0;
    const double *x = a + j0;
    const double uu = uprec[u];
    // a unit whose precision is not positive and finite, or whose offsets decrease or leave
    // [0, total], is rejected (and its values are not read)
    bool bad = !(uu > 0.0) || !(uu <= 1.7976931348623157e308) || n < 0 || j0 < 0 || off[u + 1] > total;
    double m_min = 1.0;
    int e = 0, m = 0, w = 1;
    if (!bad && (fmt == HLR_FMT_AFL_APLR || fmt == HLR_FMT_AFLP)) {
      m = mbits_of(uu);
      double mn = __longlong_as_double(0x7ff0000000000000ll);  // +inf
      int nf = 0;
      for (int64_t j = threadIdx.x; j < n; j += kEncThreads) {
        const double v = x[j];
        const double av = fabs(v);
        if (!(av <= 1.7976931348623157e308)) nf = 1;
        if (av != 0.0) mn = fmin(mn, av);
      }
      bad = block_or(nf, shi) != 0;
      mn = block_min(mn, shd);
      if (!bad) {
        if (!(mn <= 1.7976931348623157e308)) {  // all zero: e = 0 (AFLP still aligns 1 + m)
          m_min = 0.0;
          e = 0;
          while (fmt == HLR_FMT_AFLP && (1 + m) % 8 != 0 && m < 52) ++m;
        } else {
          m_min = mn;
          for (;; ++m) {
            e = bit_length((unsigned long long)afl_fmax(x, n, mn, m, shl));
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
        for (int64_t j = threadIdx.x; j < n; j += kEncThreads) {
          const double v = x[j];
          if (!(fabs(v) <= 1.7976931348623157e308) || ((bfl_bits(v, m) >> 23) & 0xffu) == 0xffu) over = 1;
        }
      } else if (fmt == HLR_FMT_DFL) {
        const int mb = mbits_of(uu);
        m = 4;
        while (m < mb) m += 8;
        e = 11;
        for (int64_t j = threadIdx.x; j < n; j += kEncThreads)
          if (((round_bits(x[j], m) >> 52) & 0x7ff) == 0x7ff) over = 1;  // also NaN / Inf input
      } else {  // HLR_FMT_MP
        const int bits = mp_bits(uu);
        e = bits == 16 ? 5 : bits == 32 ? 8 : 11;
        m = bits == 16 ? 10 : bits == 32 ? 23 : 52;
        for (int64_t j = threadIdx.x; j < n; j += kEncThreads) {
          const double v = x[j];
          if (!(fabs(v) <= 1.7976931348623157e308)) over = 1;
          if (bits == 32 && (f32_bits_rn(v) & 0x7f800000u) == 0x7f800000u) over = 1;
          if (bits == 16 && (f16_bits_rn(v) & 0x7c00u) == 0x7c00u) over = 1;
        }
      }
      bad = block_or(over, shi) != 0;
      w = 1 + e + m;
    }
    if (threadIdx.x == 0) {
      m_min_out[u] = bad ? 0.0 : m_min;
      e_out[u] = bad ? -1 : e;
      m_out[u] = bad ? 0 : m;
      out_off[u + 1] = bad ? 0 : int64_t(((uint64_t(n) * uint64_t(w) + 7) / 8 + 15) & ~uint64_t(15));
    }
    __syncthreads();
  }
}

// in-place inclusive scan of out_off[1..nunits] (one CTA of kEncThreads threads; out_off[0] = 0)
__global__ void __launch_bounds__(kEncThreads) k_scan(int64_t nunits, int64_t *out_off) {
  __shared__ int64_t part[kEncThreads];
  const int64_t per = (nunits + kEncThreads - 1) / kEncThreads;
  const int64_t b = 1 + int64_t(threadIdx.x) * per, e = min(nunits + 1, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += out_off[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int k = 0; k < kEncThreads; ++k) {
      const int64_t t = part[k];
      part[k] = run;
      run += t;
    }
    out_off[0] = 0;
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) {
    run += out_off[i];
    out_off[i] = run;
  }
}

// code of value x of a unit (w = 1 + e + m bits, low bits of the result)
__device__ __forceinline__ uint64_t code_of(int fmt, double x, double m_min, int e, int m) {
  if (fmt == HLR_FMT_AFL_APLR || fmt == HLR_FMT_AFLP) {
    if (m_min == 0.0) return 0;
    const double v = __dadd_rn(__ddiv_rn(fabs(x), m_min), 1.0);
    const uint64_t b = round_bits(v, m);
    const uint64_t field = (b >> 52) - 1023;
    const uint64_t mant = (b & ((uint64_t(1) << 52) - 1)) >> (52 - m);
    const uint64_t sign = x < 0.0 ? 1 : 0;
    return (sign << (e + m)) | (field << m) | mant;
  }
  if (fmt == HLR_FMT_BFL) return uint64_t(bfl_bits(x, m) >> (23 - m));
  if (fmt == HLR_FMT_DFL) return round_bits(x, m) >> (52 - m);
  // HLR_FMT_MP
  if (e == 5) return f16_bits_rn(x);
  if (e == 8) return f32_bits_rn(x);
  return d2u(x);
}

__global__ void __launch_bounds__(kEncThreads) k_pack(int fmt, int64_t nunits, const int64_t *__restrict__ off,
                                                       const double *__restrict__ a, const double *__restrict__ m_min_in,
                                                       const int32_t *__restrict__ e_in, const int32_t *__restrict__ m_in,
                                                       const int64_t *__restrict__ out_off, uint8_t *out, uint64_t cap) {
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int e = e_in[u];
    if (e < 0) continue;
    const int m = m_in[u], w = 1 + e + m;
    const double m_min = m_min_in[u];
    const int64_t j0 = off[u], n = off[u + 1] - j0;
    const uint64_t o0 = uint64_t(out_off[u]), o1 = uint64_t(out_off[u + 1]);
    if (o1 > cap || o1 < o0) continue;  // unreachable when cap holds the bound the host checked
    const double *x = a + j0;
    uint32_t *dst = reinterpret_cast<uint32_t *>(out + o0);
    const uint64_t nw = (o1 - o0) / 4;
    const uint64_t nbits = uint64_t(n) * uint64_t(w);
    for (uint64_t k = threadIdx.x; k < nw; k += kEncThreads) {
      const uint64_t lo = 32 * k;
      uint32_t word = 0;
      if (lo < nbits) {
        const uint64_t jb = lo / uint64_t(w);
        const uint64_t je = min((lo + 31) / uint64_t(w), uint64_t(n) - 1);
        for (uint64_t j = jb; j <= je; ++j) {
          const uint64_t code = code_of(fmt, x[j], m_min, e, m);
          const int64_t sh = int64_t(j * uint64_t(w)) - int64_t(lo);  // code bit 0 relative to the word
          word |= sh >= 0 ? uint32_t(code << sh) : uint32_t(code >> (-sh));
        }
      }
      dst[k] = word;
    }
  }
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
  const unsigned grid = unsigned(nunits < (int64_t(1) << 30) ? nunits : (int64_t(1) << 30));
  k_params<<<grid, kEncThreads, 0, st>>>(fmt, nunits, total_values, off_dev, a_dev, u_dev, m_min_dev, e_dev, m_dev, out_off_dev);
  k_scan<<<1, kEncThreads, 0, st>>>(nunits, out_off_dev);
  k_pack<<<grid, kEncThreads, 0, st>>>(fmt, nunits, off_dev, a_dev, m_min_dev, e_dev, m_dev, out_off_dev, out_dev,
                                       uint64_t(cap));
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string("hlr_encode_device: ") + cudaGetErrorString(err));
  return HLR_OK;
}
