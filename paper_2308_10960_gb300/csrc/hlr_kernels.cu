// CUDA kernels of the compressed H-matrix-vector product y += A~ x (Section 5.4) over AFL /
// AFL-APLR streams (Sections 3.2, 3.3), decoded inside the product.
//
//   k_permute : x_perm = x[perm] (FP64 and FP32 copies)
//   k_phase1  : for every lowrank block b, t_b = Sigma_b (X~_b^T x|sigma) -- one warp per item
//               of <= 256 rows of X, warp-shuffle sums, partial sums of a block combined in
//               chunk order by the last item to finish (no spin waits, deterministic)
//   k_phase2  : one CTA per leaf row interval (<= 64 rows): y|l += sum over the blocks that
//               cover l of W~_b|l t_b or D~_b|l x|sigma, columns spread over 8 warps, one fixed
//               order, one owner per row (no atomics on y)
//
// Storage formats: FMT_AFL32 decodes to FP32 with integer ops and sums in FP32 inside a block
// and FP64 across blocks; FMT_AFL64 decodes and sums in FP64; FMT_RAW64 reads plain FP64
// factors (the uncompressed baseline).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hlr_internal.h"

namespace hlr {

enum { FMT_AFL32 = 0, FMT_AFL64 = 1, FMT_RAW64 = 2 };
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ const uint32_t *unit_words(const uint8_t *base, const UnitHdr &h) {
  const uint64_t o16 = uint64_t(h.off_lo) | (uint64_t(h.off_hi) << 32);
  return reinterpret_cast<const uint32_t *>(base + (o16 << 4));
}

__device__ __forceinline__ UnitHdr load_hdr(const UnitHdr *p) {
  const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
  UnitHdr h;
  h.m_min = __hiloint2double(int(v.y), int(v.x));
  h.off_lo = v.z;
  h.e = uint8_t(v.w & 0xff);
  h.m = uint8_t((v.w >> 8) & 0xff);
  h.w = uint8_t((v.w >> 16) & 0xff);
  h.off_hi = uint8_t(v.w >> 24);
  return h;
}

// Per-column decode constants.
struct ColDec {
  uint32_t em_mask;   // (1 << (e+m)) - 1, e+m <= 31
  uint32_t scale;     // 1 << (23 - m)     (FP32 fast path)
  uint32_t sshift;    // 31 - (e + m): moves the sign bit to bit 31
  uint32_t e, m, w;
  bool fast32;        // w <= 32, m <= 23, e <= 7: FP32 bit pattern built with integer ops
};

__device__ __forceinline__ ColDec col_dec(const UnitHdr &h) {
  ColDec c;
  c.e = h.e;
  c.m = h.m;
  c.w = h.w;
  const uint32_t em = c.e + c.m;
  c.em_mask = em >= 32 ? 0xffffffffu : ((1u << em) - 1u);
  c.scale = c.m <= 23 ? (1u << (23 - c.m)) : 0u;
  c.sshift = em <= 31 ? 31 - em : 0;
  c.fast32 = (c.w <= 32) && (c.m <= 23) && (c.e <= 7);
  return c;
}

// 32-bit code window starting at bit sh of p[0..1] (w <= 32).
__device__ __forceinline__ uint32_t code32(const uint32_t *p, uint32_t sh) {
  return __funnelshift_r(__ldg(p), __ldg(p + 1), sh);
}

// 64-bit code window starting at bit sh of p[0..2] (w <= 64).
__device__ __forceinline__ uint64_t code64(const uint32_t *p, uint32_t sh) {
  const uint32_t a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  const uint32_t lo = __funnelshift_r(a, b, sh), hi = __funnelshift_r(b, c, sh);
  return (uint64_t(hi) << 32) | lo;
}

// FP32 value +-(v - 1) from a code (fast path).
__device__ __forceinline__ float dec_f32(uint32_t code, const ColDec &c) {
  const uint32_t mag = (code & c.em_mask) * c.scale + 0x3F800000u;
  const float v = __uint_as_float(mag) - 1.0f;
  const uint32_t s = (code << c.sshift) & 0x80000000u;
  return __uint_as_float(__float_as_uint(v) ^ s);
}

// FP64 value +-(v - 1) from a code (any width).
__device__ __forceinline__ double dec_f64(uint64_t code, const ColDec &c) {
  const uint64_t em = code & ((c.e + c.m >= 64) ? ~0ull : ((1ull << (c.e + c.m)) - 1ull));
  const uint64_t b = (em << (52 - c.m)) + (1023ull << 52);
  double v = __longlong_as_double(static_cast<long long>(b)) - 1.0;
  const uint64_t s = (code >> (c.e + c.m)) & 1ull;
  return s ? -v : v;
}

template <int FMT>
struct Acc;
template <>
struct Acc<FMT_AFL32> {
  using T = float;
};
template <>
struct Acc<FMT_AFL64> {
  using T = double;
};
template <>
struct Acc<FMT_RAW64> {
  using T = double;
};

// value(at value index vi of the unit) * mult, added to acc. p/sh address the value's bits.
template <int FMT>
__device__ __forceinline__ void fma_value(typename Acc<FMT>::T &acc, const uint32_t *p, uint32_t sh,
                                          const ColDec &c, typename Acc<FMT>::T mult) {
  if constexpr (FMT == FMT_AFL32) {
    if (c.fast32) {
      acc = fmaf(dec_f32(code32(p, sh), c), mult, acc);
    } else {
      const double v = dec_f64(c.w <= 32 ? uint64_t(code32(p, sh)) : code64(p, sh), c);
      acc = fmaf(float(v), mult, acc);
    }
  } else {
    const double v = dec_f64(c.w <= 32 ? uint64_t(code32(p, sh)) : code64(p, sh), c);
    acc = fma(v, mult, acc);
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__global__ void k_permute(const int64_t *__restrict__ perm, int64_t n, const double *__restrict__ x,
                          double *__restrict__ x64, float *__restrict__ x32) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
    const double v = __ldg(x + __ldg(perm + p));
    x64[p] = v;
    x32[p] = float(v);
  }
}

// ---------------------------------------------------------------------------------------------
// Phase 1: t_b = Sigma_b (X~_b^T x|sigma)
// ---------------------------------------------------------------------------------------------
template <int FMT>
__global__ void __launch_bounds__(kThreads) k_phase1(DevLayout L) {
  using T = typename Acc<FMT>::T;
  const int lane = threadIdx.x & 31;
  uint32_t *work = L.counters + L.nlr;
  for (;;) {
    uint32_t ii = 0;
    if (lane == 0) ii = atomicAdd(work, 1u);
    ii = __shfl_sync(kFull, ii, 0);
    if (ii >= uint32_t(L.nitems)) break;
    const P1Item it = L.items[ii];
    const LRBlock B = L.lrb[it.blk];
    const int nr = it.nrows;
    T xr[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int r = lane + 32 * v;
      if constexpr (FMT == FMT_AFL32)
        xr[v] = r < nr ? __ldg(L.xperm32 + it.xoff + r) : 0.0f;
      else
        xr[v] = r < nr ? __ldg(L.xperm64 + it.xoff + r) : 0.0;
    }
    const bool single = B.nchunks == 1;
    for (int i = 0; i < B.k; ++i) {
      const UnitHdr h = load_hdr(L.units + B.xunit0 + i);
      const uint32_t *base = unit_words(L.base, h);
      T a = T(0);
      if constexpr (FMT == FMT_RAW64) {
        const double *col = reinterpret_cast<const double *>(base) + it.row0;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int r = lane + 32 * v;
          if (r < nr) a = fma(__ldg(col + r), xr[v], a);
        }
      } else {
        const ColDec c = col_dec(h);
        const uint64_t bit0 = uint64_t(it.row0 + lane) * c.w;
        const uint32_t *p = base + (bit0 >> 5);
        const uint32_t sh = uint32_t(bit0 & 31);
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          const int r = lane + 32 * v;
          if (r < nr) fma_value<FMT>(a, p + v * c.w, sh, c, xr[v]);
        }
      }
      a = warp_sum(a);
      if (lane == 0) {
        const double s = (FMT == FMT_RAW64) ? double(a) : double(a) * h.m_min;
        if (single)
          L.t[B.tbase + i] = __ldg(L.sigma + B.tbase + i) * s;
        else
          L.partial[B.part0 + uint32_t(it.chunk) * B.k + i] = s;
      }
    }
    if (!single) {
      uint32_t old = 0;
      if (lane == 0) {
        __threadfence();
        old = atomicAdd(L.counters + it.blk, 1u);
      }
      old = __shfl_sync(kFull, old, 0);
      if (old == uint32_t(B.nchunks) - 1) {
        __threadfence();
        for (int i = lane; i < B.k; i += 32) {
          double s = 0.0;
          for (int c = 0; c < B.nchunks; ++c) s += __ldcg(L.partial + B.part0 + uint32_t(c) * B.k + i);
          L.t[B.tbase + i] = __ldg(L.sigma + B.tbase + i) * s;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Phase 2: y|l += sum_b A~_b|l x   (per leaf row interval l)
// ---------------------------------------------------------------------------------------------
template <int FMT>
__global__ void __launch_bounds__(kThreads) k_phase2(DevLayout L, double *__restrict__ y) {
  using T = typename Acc<FMT>::T;
  __shared__ double red[kWarps][64];
  __shared__ uint32_t s_leaf;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *work = L.counters + L.nlr + 1;
  const double *t = L.t;
  for (;;) {
    if (threadIdx.x == 0) s_leaf = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t li = s_leaf;
    __syncthreads();
    if (li >= uint32_t(L.nleaves)) break;
    const Leaf lf = L.leaves[li];
    const int nr = int(lf.nrows);
    const bool ok0 = lane < nr, ok1 = lane + 32 < nr;
    double acc0 = 0.0, acc1 = 0.0;
    for (uint32_t ci = lf.c0; ci < lf.c1; ++ci) {
      const Contrib cb = L.contribs[ci];
      T a0 = T(0), a1 = T(0);
      const bool dense = cb.kind == CONTRIB_DENSE;
      uint32_t j = uint32_t(warp - int(cb.colbase & 7) + 8) & 7u;
      const UnitHdr hd = load_hdr(L.units + cb.unit);
      for (; j < cb.ncols; j += kWarps) {
        const UnitHdr h = dense ? hd : load_hdr(L.units + cb.unit + j);
        const uint64_t vstart = dense ? uint64_t(j) * cb.ld + cb.rowoff : uint64_t(cb.rowoff);
        const double m64 = dense ? __ldg(L.xperm64 + cb.mbase + j) : __ldcg(t + cb.mbase + j);
        const uint32_t *base = unit_words(L.base, h);
        if constexpr (FMT == FMT_RAW64) {
          const double *col = reinterpret_cast<const double *>(base) + vstart;
          if (ok0) a0 = fma(__ldg(col + lane), m64, a0);
          if (ok1) a1 = fma(__ldg(col + lane + 32), m64, a1);
        } else {
          const ColDec c = col_dec(h);
          const T mult = T(m64 * h.m_min);
          const uint64_t bit0 = (vstart + lane) * c.w;
          const uint32_t *p = base + (bit0 >> 5);
          const uint32_t sh = uint32_t(bit0 & 31);
          if (ok0) fma_value<FMT>(a0, p, sh, c, mult);
          if (ok1) fma_value<FMT>(a1, p + c.w, sh, c, mult);
        }
      }
      acc0 += double(a0);
      acc1 += double(a1);
    }
    red[warp][lane] = acc0;
    red[warp][lane + 32] = acc1;
    __syncthreads();
    if (threadIdx.x < nr) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
      const int64_t gi = L.perm[lf.row0 + threadIdx.x];
      y[gi] += s;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Bit-exact decoding (test path): a = (v - 1) * m_min in IEEE FP64, no contraction.
// ---------------------------------------------------------------------------------------------
__device__ double decode_exact(const uint32_t *words, uint64_t nwords, uint64_t j, int e, int m, double m_min) {
  const int w = 1 + e + m;
  const uint64_t bit = j * uint64_t(w);
  const uint64_t q = bit >> 5;
  const int sh = int(bit & 31);
  const int need = (sh + w + 31) >> 5;  // words touched: 1..3
  uint64_t lo = words[q];
  uint64_t hi = 0;
  if (need >= 2 && q + 1 < nwords) lo |= uint64_t(words[q + 1]) << 32;
  if (need >= 3 && q + 2 < nwords) hi = words[q + 2];
  uint64_t code = lo >> sh;
  if (sh) code |= hi << (64 - sh);
  if (w < 64) code &= (1ull << w) - 1ull;
  const uint64_t mant = code & ((1ull << m) - 1ull);
  const uint64_t field = (code >> m) & ((1ull << e) - 1ull);
  const uint64_t sign = (code >> (e + m)) & 1ull;
  const uint64_t b = ((field + 1023ull) << 52) | (mant << (52 - m));
  const double v = __longlong_as_double(static_cast<long long>(b));
  const double a = __dmul_rn(__dsub_rn(v, 1.0), m_min);
  return sign ? -a : a;
}

__global__ void k_decode_stream(const uint32_t *words, int64_t n, double m_min, int e, int m, double *out) {
  const uint64_t nwords = (uint64_t(n) * uint64_t(1 + e + m) + 31) / 32;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x)
    out[j] = decode_exact(words, nwords, uint64_t(j), e, m, m_min);
}

__global__ void k_decode_units(const uint8_t *base, const UnitHdr *units, const int64_t *voff, int64_t nunits,
                               int raw, double *out) {
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const UnitHdr h = units[u];
    const int64_t o = voff[u], len = voff[u + 1] - voff[u];
    const uint32_t *wd = unit_words(base, h);
    if (raw) {
      const double *src = reinterpret_cast<const double *>(wd);
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x) out[o + j] = src[j];
    } else {
      const uint64_t nwords = (uint64_t(len) * h.w + 31) / 32;
      for (int64_t j = threadIdx.x; j < len; j += blockDim.x)
        out[o + j] = decode_exact(wd, nwords, uint64_t(j), h.e, h.m, h.m_min);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------
namespace {

struct DevProps {
  int sms = 0;
  int occ1[3] = {0, 0, 0};
  int occ2[3] = {0, 0, 0};
};

std::mutex g_props_mu;
DevProps g_props[64];

template <int FMT>
void query_occ(DevProps &P) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.occ1[FMT], k_phase1<FMT>, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.occ2[FMT], k_phase2<FMT>, kThreads, 0);
  if (P.occ1[FMT] < 1) P.occ1[FMT] = 1;
  if (P.occ2[FMT] < 1) P.occ2[FMT] = 1;
}

const DevProps &props(int dev) {
  std::lock_guard<std::mutex> lk(g_props_mu);
  DevProps &P = g_props[dev & 63];
  if (P.sms == 0) {
    cudaDeviceGetAttribute(&P.sms, cudaDevAttrMultiProcessorCount, dev);
    query_occ<FMT_AFL32>(P);
    query_occ<FMT_AFL64>(P);
    query_occ<FMT_RAW64>(P);
  }
  return P;
}

int cuda_status(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return HLR_OK;
}

template <int FMT>
void launch_phases(const Handle &H, double *y, cudaStream_t st, cudaEvent_t *ev) {
  const DevProps &P = props(H.device);
  const DevLayout &L = H.L;
  if (ev) cudaEventRecord(ev[1], st);
  if (L.nitems > 0) {
    int grid = P.sms * P.occ1[FMT];
    grid = std::min(grid, (L.nitems + kWarps - 1) / kWarps);
    k_phase1<FMT><<<grid, kThreads, 0, st>>>(L);
  }
  if (ev) cudaEventRecord(ev[2], st);
  int grid2 = std::min(P.sms * P.occ2[FMT], L.nleaves);
  k_phase2<FMT><<<grid2, kThreads, 0, st>>>(L, y);
  if (ev) cudaEventRecord(ev[3], st);
}

// Events of the next profiled product (nullptr if not profiling or the ring is full).
cudaEvent_t *profile_slot(Handle &H, int flags) {
  if (!(flags & HLR_PROFILE)) return nullptr;
  if (H.prof_ev.empty()) {
    H.prof_ev.resize(4 * size_t(kProfileCap), nullptr);
    for (auto &e : H.prof_ev) {
      cudaEvent_t ev;
      cudaEventCreate(&ev);
      e = ev;
    }
  }
  if (H.prof_n >= kProfileCap) return nullptr;
  return reinterpret_cast<cudaEvent_t *>(&H.prof_ev[4 * size_t(H.prof_n++)]);
}

}  // namespace

int launch_matvec(Handle &H, const double *x, double *y, int flags, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DevLayout &L = H.L;
  cudaGetLastError();
  cudaEvent_t *ev = profile_slot(H, flags);
  const int acc = flags & 0xff;
  if (cudaMemsetAsync(L.counters, 0, sizeof(uint32_t) * (size_t(L.nlr) + 8), st) != cudaSuccess)
    return cuda_status("hlr_matvec: counter reset");
  const DevProps &P = props(H.device);
  int gp = int(std::min<int64_t>((L.n + kThreads - 1) / kThreads, int64_t(P.sms) * 8));
  if (ev) cudaEventRecord(ev[0], st);
  k_permute<<<gp, kThreads, 0, st>>>(L.perm, L.n, x, L.xperm64, L.xperm32);
  if (H.format == HLR_FMT_FP64)
    launch_phases<FMT_RAW64>(H, y, st, ev);
  else if (acc == HLR_ACC_FP32)
    launch_phases<FMT_AFL32>(H, y, st, ev);
  else
    launch_phases<FMT_AFL64>(H, y, st, ev);
  return cuda_status("hlr_matvec: launch");
}

int profile_read(Handle &H, double *ms, int *calls) {
  ms[0] = ms[1] = ms[2] = 0.0;
  for (int i = 0; i < H.prof_n; ++i) {
    cudaEvent_t *ev = reinterpret_cast<cudaEvent_t *>(&H.prof_ev[4 * size_t(i)]);
    if (cudaEventSynchronize(ev[3]) != cudaSuccess) return cuda_status("hlr_profile_read");
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      ms[k] += t;
    }
  }
  *calls = H.prof_n;
  H.prof_n = 0;
  return HLR_OK;
}

int launch_decode_units(const Handle &H, double *out, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  int64_t *voff = nullptr;
  const size_t bytes = sizeof(int64_t) * H.unit_value_offset.size();
  if (cudaMalloc(&voff, bytes) != cudaSuccess) return set_error(HLR_ERR_OOM, "hlr_decode_units: temp allocation failed");
  cudaMemcpyAsync(voff, H.unit_value_offset.data(), bytes, cudaMemcpyHostToDevice, st);
  const int grid = int(std::min<int64_t>(H.nunits, 65535));
  if (grid > 0)
    k_decode_units<<<grid, 128, 0, st>>>(H.L.base, H.L.units, voff, H.nunits, H.format == HLR_FMT_FP64 ? 1 : 0, out);
  int rc = cuda_status("hlr_decode_units");
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(voff);
  if (rc == HLR_OK && e != cudaSuccess) rc = set_error(HLR_ERR_CUDA, std::string("hlr_decode_units: ") + cudaGetErrorString(e));
  return rc;
}

int launch_decode_stream(const uint8_t *stream, int64_t n, double m_min, int e, int m, double *out, void *stream_) {
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  cudaGetLastError();
  const int grid = int(std::min<int64_t>((n + 255) / 256, 4096));
  k_decode_stream<<<grid, 256, 0, st>>>(reinterpret_cast<const uint32_t *>(stream), n, m_min, e, m, out);
  return cuda_status("hlr_afl_decode_device");
}

}  // namespace hlr
