// CUDA kernels of the compressed H-matrix-vector product y += A~ x (Section 5.4) over AFL /
// AFL-APLR codes (Sections 3.2, 3.3), decoded inside the product.
//
//   k_permute : x_perm = x[perm] (FP64 and FP32 copies)
//   k_product<FMT, 0> (phase 1): for every lowrank block b and column i,
//               t_b,i m_min(W_b,i) = sigma_i m_min(X_i) m_min(W_i) sum_r X~code_r,i x_r;
//               a block wider than 256 rows is split into items whose partial sums are
//               written to scratch and summed in chunk order by k_combine
//   k_combine : deterministic sum of those partial sums, times the column factor
//   k_product<FMT, 1> (phase 2): per leaf row interval l (<= 64 rows), the sum over the blocks
//               covering l of W~_b|l t_b and D~_b|l x|sigma in one fixed order, by the one CTA
//               that owns the leaf; the AFL paths write it as a row total in cluster order and
//   k_scatter : y[perm[p]] += total[p] (the other formats add into y at the leaf's end): no
//               atomics on y, a deterministic result
//   multi-column passes (R = 8 or 32 right-hand sides): the same two phases with R dot
//               products per value (phase 1) and a tensor-core contraction (phase 2)
//
// Both phases are persistent kernels over the work-ordered piece streams (hlr_internal.h):
// one producer warp per CTA issues TMA bulk copies (cp.async.bulk) of the next pieces and of
// their multipliers into a ring of shared-memory slots guarded by mbarriers; every lane of a
// consumer warp fences its reads against the async proxy before the warp hands a slot back. In
// the consumer warps of the compressed paths every lane owns one column slice of the current
// piece (phase 1: a <= 64-row part of an X column; phase 2: a column of the leaf). Phase 2 keeps
// 64 row sums per lane in registers over the leaf's pieces and reduces them over the warp with a
// butterfly at the leaf's end; the FP64 route of the plain FP64 format lets lanes be rows. Every
// wait is bounded (about 2 s of clock cycles), after which the kernel records an error word and
// returns.
//
// FMT_AFL32: codes -> FP32 bit patterns with integer ops (two codes per 32- or 64-bit window);
//            FP32 sums over a slice (phase 1) or over a lane's slices of a leaf and the warp's
//            lanes (phase 2); FP64 over the four warps and into y.
// FMT_AFL64: codes -> FP64 (one FP64 fused multiply-add per value), FP64 sums.
// FMT_RAW64: plain FP64 factors (uncompressed baseline). FMT_BFL32 / DFL32 / MP32: the
//            byte-aligned and mixed-precision formats with FP32 accumulation.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "hlr_internal.h"

namespace hlr {

// Kernel formats: the stored values (AFL family, BFL, DFL, plain FP64) and the accumulation.
enum { FMT_AFL32 = 0, FMT_AFL64 = 1, FMT_RAW64 = 2, FMT_BFL32 = 3, FMT_DFL32 = 4, FMT_MP32 = 5 };
template <int FMT>
constexpr bool kFP32 = FMT == FMT_AFL32 || FMT == FMT_BFL32 || FMT == FMT_DFL32 || FMT == FMT_MP32;
template <int FMT>
constexpr int kVF = FMT == FMT_BFL32 ? VF_BFL : FMT == FMT_DFL32 ? VF_DFL : FMT == FMT_MP32 ? VF_MP : VF_AFL;
constexpr int kThreads = kConsumers + 32;
constexpr int kCWarps = kConsumers / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at the GB300 SM clock

template <int FMT>
struct Tr {
  using A = double;  // multiplier / accumulator type
  static constexpr int esz = 8;
};
template <>
struct Tr<FMT_AFL32> {
  using A = float;
  static constexpr int esz = 4;
};
template <>
struct Tr<FMT_BFL32> : Tr<FMT_AFL32> {};
template <>
struct Tr<FMT_DFL32> : Tr<FMT_AFL32> {};
template <>
struct Tr<FMT_MP32> : Tr<FMT_AFL32> {};
constexpr int kRB = 32;         // right-hand sides per pass of the multi-RHS product (widest pass)
constexpr int kRN = 8;          // width of the narrow pass, for requests of at most 8 columns
// B-fragment column swizzle of a warp's multipliers in a multi-RHS phase 2 (rows of R floats):
// with R = 32, row k keeps column n at n ^ 8 (k % 4), so that the fragment loads (rows 8 kg + tq
// and + 4, columns 8 nt + g) hit 32 different banks; with R = 8 the plain layout already does
template <int R>
__host__ __device__ constexpr int kSwz(int k) {
  return R == 32 ? (k & 3) << 3 : 0;
}
constexpr int kMaxBatch = 64;   // products per launch of the batched path

// One product of a launch. Single right-hand side (R = 1): y += A~ x with the handle's scratch.
// Multi-RHS pass (R = kRN or kRB): Y(:, 0:nrhs) += A~ X(:, 0:nrhs) for nrhs <= R columns, with the
// pass's own scratch (xp, tw, part).
struct Job {
  DevLayout L;
  const double *x;   // x (R = 1) or the pass's first column of X (column-major, leading dim ldx)
  double *y;         // y (R = 1) or the pass's first column of Y (leading dim ldy)
  int64_t ldx, ldy;
  int32_t nrhs, pad;
  float *xp;         // R > 1: X in cluster order, R floats per row          [n + 8][R]
  float *tw;         // R > 1: t m_min(W), R per lowrank column              [rank_sum + 8][R]
  double *part;      // R > 1: phase-1 chunk partial sums, R per entry       [part_total + 1][R]
};
// A launch's products, passed by value as a kernel parameter (no device-side descriptor copy,
// so a batched launch needs no allocation and can be captured in a graph).
template <int NB>
struct Jobs {
  int32_t n, pad;
  Job j[NB];
};
static_assert(sizeof(Jobs<kMaxBatch>) < 30000, "kernel parameter size");

// ring slot: piece, pad, staged multipliers (phase 1 stages more: x of the items' rows); the
// multi-RHS kernels read their multipliers from global memory and stage none. The pad covers
// the words a lane reads past its column (at most two rows of 32 words beyond the last region).
constexpr size_t kSlotPad = 272;
template <int FMT, int PH, int R = 1>
__host__ __device__ constexpr size_t slot_bytes() {
  return size_t(kPieceMax) + kSlotPad + (R == 1 ? size_t(PH == 0 ? kAuxMax1 : kAuxMax2) * Tr<FMT>::esz : 0);
}
// phase-2 tiles of one warp: 16 rows x 33 (single RHS, accumulation type) or, for a multi-RHS
// pass, a 16 x 36 decode tile and the 32 slices' R multipliers split into TF32 hi and lo parts
template <int FMT, int R>
__host__ __device__ constexpr size_t tile_bytes() {
  return R > 1 ? (size_t(16) * 36 + 2 * 32 * R) * 4 : FMT == FMT_RAW64 ? 0 : size_t(16) * 33 * Tr<FMT>::esz;
}
// dynamic shared memory: ring, mbarriers; phase 2 adds the leaf reduction buffers (single RHS:
// two halves; multi-RHS: the tiles, and in the same space, once a leaf is done, each warp's
// 64 x R row sums at stride R + 8)
template <int FMT, int PH, int R = 1>
__host__ __device__ constexpr size_t smem_bytes() {
  return size_t(kStages) * slot_bytes<FMT, PH, R>() + 2 * kStages * 8 + 16 +
         (PH == 0 ? (R > kRN ? size_t(kCWarps) * (32 * 65 + 64) * 4 : 0)
          : R > 1 ? (tile_bytes<FMT, R>() > size_t(64) * (R + 8) * 4 ? size_t(kCWarps) * tile_bytes<FMT, R>()
                                                                     : size_t(kCWarps) * 64 * (R + 8) * 4)
                  : 2 * kCWarps * 64 * 8 + size_t(kCWarps) * tile_bytes<FMT, R>());
}

// ---------------------------------------------------------------------------------------------
// PTX helpers: shared-memory addresses, mbarriers, TMA bulk copies, consumer barrier
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// A consumer warp hands its ring slot back to the producer (empty barrier, one arrival per warp).
// The lanes read the slot with ordinary shared loads (the generic proxy) and the next TMA copy
// writes it through the async proxy: each lane's proxy fence orders its reads before the copy
// the producer issues after its wait, without which a copy can overtake reads still in flight
// (observed: the first rows of a leaf decoding the next piece's bytes, when other kernels share
// the SMs).
__device__ __forceinline__ void release_slot(uint64_t *b) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(b);
}
// try_wait with a suspend-time hint: a waiting warp sleeps (up to ~20 us per try) until the
// phase completes instead of spinning on issue slots
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete; false after `limit` clock cycles (~2 s
// by default).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, long long limit = kWaitCycles) {
  if (mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bar_consumers() { asm volatile("bar.sync 1, %0;" ::"r"(kConsumers) : "memory"); }


// ---------------------------------------------------------------------------------------------
// Decoding
// ---------------------------------------------------------------------------------------------
struct ColDec {
  uint32_t em_mask;  // (1 << (e+m)) - 1 (all ones if e+m >= 32)
  uint32_t scale;    // 1 << (23 - m)   (FP32 fast path)
  uint32_t sshift;   // 31 - (e + m): moves the sign bit to bit 31
  uint32_t e, m, w;
  bool fast32;       // w <= 32, m <= 23, e <= 7: FP32 bit pattern built with integer ops
  bool narrow;       // w <= 32: a code fits a two-word window
  bool mid32;        // w <= 32 and (fast32 or e <= 4): dec_mid32 gives the FP64 route's value
};

__device__ __forceinline__ ColDec col_dec(uint32_t e, uint32_t m) {
  ColDec c;
  c.e = e;
  c.m = m;
  c.w = 1 + e + m;
  const uint32_t em = e + m;
  c.em_mask = em >= 32 ? 0xffffffffu : ((1u << em) - 1u);
  c.scale = m <= 23 ? (1u << (23 - m)) : 0u;
  c.sshift = em <= 31 ? 31 - em : 0;
  c.fast32 = (c.w <= 32) && (m <= 23) && (e <= 7);
  c.narrow = c.w <= 32;
  c.mid32 = c.fast32 || (c.narrow && e <= 4);
  return c;
}

// +-(v - 1) rounded once to FP32 (the value the FP64 route float(dec_f64(code)) gives) for a
// code of w <= 32 bits whose mantissa may be wider than FP32's (m up to 31): v's top 23
// mantissa bits form an FP32 v_hi, v_hi - 1 is exact while the field is below 2^4 (e <= 4; for
// m <= 23, v_hi = v and any e of fast32 works), and the remaining m - 23 bits, an exact FP32
// lo * 2^(field - m), are added with the one rounding.
__device__ __forceinline__ float dec_mid32(uint32_t code, const ColDec &c) {
  const uint32_t m = c.m;
  const uint32_t mant = code & (m ? 0xffffffffu >> (32 - m) : 0u);
  const uint32_t field = (code >> m) & ((1u << c.e) - 1u);
  const uint32_t k = m > 23 ? m - 23 : 0u;
  const uint32_t hi = m > 23 ? mant >> k : mant << (23 - m);
  const float lo = __uint2float_rn(mant & ((1u << k) - 1u)) * __uint_as_float((field + 127u - m) << 23);
  const float r = (__uint_as_float(((field + 127u) << 23) | hi) - 1.0f) + lo;
  return ((code >> (c.e + m)) & 1u) ? -r : r;
}

// +-(v - 1) as FP32 (fast path: integer ops build the FP32 pattern of v)
__device__ __forceinline__ float dec_f32(uint32_t code, const ColDec &c) {
  const uint32_t mag = (code & c.em_mask) * c.scale + 0x3F800000u;
  const float v = __uint_as_float(mag) - 1.0f;
  const uint32_t s = (code << c.sshift) & 0x80000000u;
  return __uint_as_float(__float_as_uint(v) ^ s);
}

// +-(v - 1) * mult as one fused multiply-add v * s - s with s = +-mult (fast path)
__device__ __forceinline__ float dec_mul_f32(uint32_t code, const ColDec &c, float mult) {
  const uint32_t mag = (code & c.em_mask) * c.scale + 0x3F800000u;
  const float sm = __uint_as_float(__float_as_uint(mult) ^ ((code << c.sshift) & 0x80000000u));
  return fmaf(__uint_as_float(mag), sm, -sm);
}

// +-(v - 1) as FP64 (any width)
__device__ __forceinline__ double dec_f64(uint64_t code, const ColDec &c) {
  const uint32_t em = c.e + c.m;
  const uint64_t mag = code & (em >= 64 ? ~0ull : ((1ull << em) - 1ull));
  const uint64_t b = (mag << (52 - c.m)) + (1023ull << 52);
  const double v = __longlong_as_double(static_cast<long long>(b)) - 1.0;
  return ((code >> em) & 1ull) ? -v : v;
}

// Decode parameters of a lane: e and m from its header; bit 7 of the header's e marks a DFL
// slice whose values are all FP32 normal numbers (the packer checks), decoded with integer ops.
__device__ __forceinline__ ColDec lane_dec(const LaneHdr &h) {
  ColDec c = col_dec(h.e & 0x7fu, h.m);
  if (h.e & 0x80u) c.fast32 = c.narrow;
  return c;
}

// BFL / DFL codes (Section 3.2): the code is the top of an FP32 / FP64 bit pattern, so it is
// shifted back into place; the bits above the code leave the word. DFL as FP32 needs w <= 32.
__device__ __forceinline__ float dec_bfl(uint32_t code, const ColDec &c) { return __uint_as_float(code << (23 - c.m)); }
// (slices marked by the packer: all values FP32 normal numbers; rebias the exponent 1023 -> 127
// and widen the mantissa, exact)
__device__ __forceinline__ float dec_dfl32(uint32_t code, const ColDec &c) {
  const uint32_t x = code << (20 - c.m);
  return __uint_as_float((((x & 0x7fffffffu) - 0x38000000u) << 3) | (x & 0x80000000u));
}
// MP codes (Section 3.3): IEEE patterns, FP16 (e = 5) widened by the hardware conversion, FP32
// (e = 8) as they are; the bits above a 16-bit code are dropped
__device__ __forceinline__ float dec_mp32(uint32_t code, const ColDec &c) {
  return c.e == 5 ? __half2float(__ushort_as_half(static_cast<unsigned short>(code & 0xffffu))) : __uint_as_float(code);
}
__device__ __forceinline__ double dec_mp64(uint64_t code, const ColDec &c) {
  if (c.e == 11) return __longlong_as_double(static_cast<long long>(code));
  return double(dec_mp32(uint32_t(code), c));
}
// value of a code of any width and value format in FP64: AFL family +-(v - 1) (to be scaled by
// m_min), BFL, DFL and MP the stored value itself
__device__ __forceinline__ double dec_any64(uint64_t code, const ColDec &c, int vf) {
  if (vf == VF_BFL) return double(__uint_as_float(uint32_t(code << (23 - c.m))));
  if (vf == VF_DFL) return __longlong_as_double(static_cast<long long>(code << (52 - c.m)));
  if (vf == VF_MP) return dec_mp64(code, c);
  return dec_f64(code, c);
}
// FP32 family: the value entering the phase-1 dot product, and value times multiplier
template <int FMT>
__device__ __forceinline__ float val32(uint32_t code, const ColDec &c) {
  if constexpr (FMT == FMT_BFL32)
    return dec_bfl(code, c);
  else if constexpr (FMT == FMT_DFL32)
    return dec_dfl32(code, c);
  else if constexpr (FMT == FMT_MP32)
    return dec_mp32(code, c);
  else
    return dec_f32(code, c);
}
template <int FMT>
__device__ __forceinline__ float valmul32(uint32_t code, const ColDec &c, float mult) {
  if constexpr (FMT == FMT_AFL32)
    return dec_mul_f32(code, c, mult);
  else
    return val32<FMT>(code, c) * mult;
}
// whether val32 applies to this column (else the FP64 decode of a 64-bit window)
template <int FMT>
__device__ __forceinline__ bool fast_dec(const ColDec &c) {
  if constexpr (FMT == FMT_BFL32)
    return true;
  else if constexpr (FMT == FMT_MP32)
    return c.narrow;  // FP16 and FP32 columns (FP64 ones take the 64-bit window)
  else
    return c.fast32;  // DFL: set by lane_dec for marked slices
}

// code (w <= 32) starting at an arbitrary bit of a shared-memory word array
__device__ __forceinline__ uint32_t code32_at(const uint32_t *p, uint32_t bit) {
  const uint32_t q = bit >> 5;
  return __funnelshift_r(p[q], p[q + 1], bit);
}

// 64-bit window of a shared-memory word array at an arbitrary bit
__device__ __forceinline__ uint64_t code64_at(const uint32_t *p, uint32_t bit) {
  const uint32_t q = bit >> 5;
  const uint32_t a = p[q], b = p[q + 1], c = p[q + 2];
  return (uint64_t(__funnelshift_r(b, c, bit)) << 32) | __funnelshift_r(a, b, bit);
}

// Bank-column pieces: first word of the column of lane t, and codes of the column (word k of
// the column is col[32 k]).
__device__ __forceinline__ uint32_t bc_column(const PieceHdr *ph, int t) {
  const uint32_t hdr_w = (16u + 32u * ph->nseg + ((4u * ph->ncols + 15u) & ~15u)) / 4u;
  const int w = t >> 5;
  uint32_t rows = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < w) rows += ph->h[k];
  return hdr_w + 32u * rows + uint32_t(t & 31);
}
__device__ __forceinline__ uint32_t bc_code32(const uint32_t *col, uint32_t bit) {
  const uint32_t q = bit >> 5;
  return __funnelshift_r(col[32 * q], col[32 * q + 32], bit);
}
__device__ __forceinline__ uint64_t bc_code64(const uint32_t *col, uint32_t bit) {
  const uint32_t q = bit >> 5;
  const uint32_t a = col[32 * q], b = col[32 * q + 32], c = col[32 * q + 64];
  return (uint64_t(__funnelshift_r(b, c, bit)) << 32) | __funnelshift_r(a, b, bit);
}
// The same with 32-bit shared-memory addresses (col_s: byte address of the column's word 0,
// x_s: of an FP32 staged multiplier), for the phase-1 inner loop.
__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float ld_shared_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t bc_code32_s(uint32_t col_s, uint32_t bit) {
  const uint32_t a = col_s + ((bit >> 5) << 7);
  return __funnelshift_r(ld_shared_u32(a), ld_shared_u32(a + 128), bit);
}
__device__ __forceinline__ const LaneHdr *lane_hdrs(const uint8_t *slot, const PieceHdr *ph) {
  return reinterpret_cast<const LaneHdr *>(slot + 16 + 32 * size_t(ph->nseg));
}

// ---------------------------------------------------------------------------------------------
// Two codes per window. For AFL codes whose FP32 bit pattern can be built with integer operations
// (w <= 31, m <= 23, e <= 7; the FP32 fast path of dec_mul_f32), two consecutive codes of a lane
// column come from one funnel-shifted window: for w <= 16 a 32-bit window of two shared words,
// else a 64-bit window of three, so a code costs one and a half shared loads or fewer.
// ---------------------------------------------------------------------------------------------
// shared-memory word at byte address a + OFF
template <int OFF>
__device__ __forceinline__ uint32_t lds_at(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
  return v;
}
// Codes 2p and 2p + 1 of a bank column (word k at col_s + 128 k) of width w, starting at bit
// b = 2p w; each at bit 0 of its word (other bits above it).
//  WIDE = false: w <= 16, one 32-bit window; WIDE = true: w <= 31, a 64-bit window.
template <bool WIDE>
__device__ __forceinline__ void code_pair(uint32_t col_s, uint32_t b, uint32_t w, uint32_t &c0, uint32_t &c1) {
  const uint32_t a = col_s + ((b >> 5) << 7);
  const uint32_t w0 = lds_at<0>(a), w1 = lds_at<128>(a);
  c0 = __funnelshift_r(w0, w1, b);
  if constexpr (WIDE)
    c1 = __funnelshift_r(c0, __funnelshift_r(w1, lds_at<256>(a), b), w);
  else
    c1 = c0 >> w;
}

// Value r of a slice (FP32 / FP64 accumulation types) for the generic (wide) path.
template <typename A>
__device__ __forceinline__ A dec_at(const uint32_t *p, uint32_t bit, const ColDec &c) {
  return A(dec_f64(code64_at(p, bit), c));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Accumulation across pieces: compensated FP32 pair (about 48 significant bits) for the FP32
// path, plain FP64 otherwise.
struct Comp32 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a) {
    const float s = hi + a;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (a - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
  __device__ __forceinline__ void reset() { hi = lo = 0.f; }
};
struct Sum64 {
  double s = 0.0;
  __device__ __forceinline__ void add(double a) { s += a; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void reset() { s = 0.0; }
};

// x_perm = x[perm] in FP64 and FP32 for every single-RHS product of the launch (blockIdx.y)
template <int NB>
__global__ void k_permute(const __grid_constant__ Jobs<NB> J) {
  const Job &jb = J.j[blockIdx.y];
  const DevLayout &L = jb.L;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < L.n; p += int64_t(gridDim.x) * blockDim.x) {
    const double v = __ldg(jb.x + __ldg(L.perm + p));
    L.xperm64[p] = v;
    L.xperm32[p] = float(v);
  }
}

// X_perm for a multi-RHS pass: row p holds X(perm[p], 0:R) in FP32, zero beyond nrhs
template <int R, int NB>
__global__ void k_permute_multi(const __grid_constant__ Jobs<NB> J) {
  const Job &jb = J.j[blockIdx.y];
  const DevLayout &L = jb.L;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < L.n; p += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = __ldg(L.perm + p);
    float v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = q < jb.nrhs ? float(__ldg(jb.x + q * jb.ldx + g)) : 0.f;
    float4 *dst = reinterpret_cast<float4 *>(jb.xp + p * R);
#pragma unroll
    for (int q = 0; q < R / 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
}

// y[perm[p]] += ysum[p] for every single-RHS product of the launch (blockIdx.y) whose phase 2
// leaves its row totals in ysum (AFL value format), in cluster order, one update per row
// (deterministic)
template <int NB>
__global__ void k_scatter(const __grid_constant__ Jobs<NB> J) {
  const Job &jb = J.j[blockIdx.y];
  const DevLayout &L = jb.L;
  if (L.vfmt != VF_AFL) return;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < L.n; p += int64_t(gridDim.x) * blockDim.x) {
    double *yp = jb.y + __ldg(L.perm + p);
    *yp = *yp + L.ysum[p];
  }
}

// ---------------------------------------------------------------------------------------------
// Producer: TMA bulk copies of the CTA's pieces and their multipliers into the slot ring
// ---------------------------------------------------------------------------------------------
// Issue the TMA copies of one product's pieces for this CTA (entries [e0, e1) of its issue
// stream). The stream is read 32 entries per coalesced load, one load ahead, and lane k holds
// entry k: the piece entries are taken in order by lane 0 (wait for the slot, post the bytes the
// slot expects, copy the piece), and the aux entries (multiplier ranges) that follow a piece are
// issued by their own lanes at once into that piece's slot. i counts the pieces this CTA issued
// during the launch (ring slot i % kStages) and cur is the slot of the latest one. The multi-RHS
// kernels (R > 1) skip the aux copies. Returns false when a wait for a free slot gave up
// (status bit 2 set).
template <int FMT, int PH, int R>
__device__ bool produce(const DevLayout &L, uint32_t e0, uint32_t e1, uint8_t *smem, uint64_t *full,
                        uint64_t *empty, uint32_t &i, uint32_t &cur) {
  constexpr uint32_t esz = Tr<FMT>::esz;
  constexpr size_t slot = slot_bytes<FMT, PH, R>();
  const int lane = threadIdx.x & 31;
  const uint8_t *xsrc = kFP32<FMT> ? reinterpret_cast<const uint8_t *>(L.xperm32)
                                         : reinterpret_cast<const uint8_t *>(L.xperm64);
  const uint8_t *tsrc = kFP32<FMT> ? reinterpret_cast<const uint8_t *>(L.tw32)
                                         : reinterpret_cast<const uint8_t *>(L.tw64);
  const uint8_t *fsrc = kFP32<FMT> ? reinterpret_cast<const uint8_t *>(L.fac32)
                                         : reinterpret_cast<const uint8_t *>(L.fac64);
  const uint4 *ent = reinterpret_cast<const uint4 *>(L.ph[PH].ent);
  // this lane's aux entry into slot `sl` (lane of an aux entry only)
  auto aux_copy = [&](const uint4 &en, uint32_t sl) {
    const uint32_t nelem = en.y & 0xffffu, which = en.y >> 16;
    const uint8_t *src = (which == 0 ? xsrc : which == 1 ? tsrc : fsrc) + size_t(en.x) * esz;
    tma_load(smem + size_t(sl) * slot + kPieceMax + kSlotPad + size_t(en.z) * esz, src, nelem * esz, &full[sl]);
  };
  uint4 nxt = e0 + lane < e1 ? __ldg(ent + e0 + lane) : make_uint4(0, 0, 0, 0);
  for (uint32_t e = e0; e < e1; e += 32) {
    const uint4 mine = nxt;
    if (e + 32 + lane < e1) nxt = __ldg(ent + e + 32 + lane);
    const uint32_t cnt = min(32u, e1 - e);
    const bool valid = uint32_t(lane) < cnt;
    const bool is_piece = valid && (mine.y & kIssuePiece);
    uint32_t pmask = __ballot_sync(kFull, is_piece);
    // aux entries continuing the latest piece of the previous batch
    const uint32_t first = pmask ? uint32_t(__ffs(pmask) - 1) : cnt;
    if (R == 1 && valid && !is_piece && uint32_t(lane) < first) aux_copy(mine, cur);
    while (pmask) {
      const uint32_t p = __ffs(pmask) - 1;
      pmask &= pmask - 1;
      const uint32_t next = pmask ? uint32_t(__ffs(pmask) - 1) : cnt;
      const uint32_t a = __shfl_sync(kFull, mine.x, p), b = __shfl_sync(kFull, mine.y, p);
      const uint32_t c = __shfl_sync(kFull, mine.z, p), d = __shfl_sync(kFull, mine.w, p);
      const uint32_t s = i % kStages;
      uint32_t good = 1;
      if (lane == 0) {
        if (i >= uint32_t(kStages) && !mbar_wait(&empty[s], ((i / kStages) - 1) & 1)) {
          atomicOr(L.status, 2u);
          good = 0;
        } else {
          const uint64_t off = (uint64_t(b & ~kIssuePiece) << 32) | a;
          mbar_expect_tx(&full[s], R == 1 ? c + d * esz : c);
          tma_load(smem + size_t(s) * slot, L.base + off, c, &full[s]);
        }
      }
      if (!__shfl_sync(kFull, good, 0)) return false;
      cur = s;
      ++i;
      if (R == 1 && uint32_t(lane) > p && uint32_t(lane) < next) aux_copy(mine, cur);
    }
  }
  return true;
}

template <int FMT, int PH, int R, int NB>
__device__ void producer(const Jobs<NB> &J, uint8_t *smem, uint64_t *full, uint64_t *empty) {
  const int lane = threadIdx.x & 31;
  uint32_t i = 0, cur = 0;
  int m = 0;
  bool ok = true;
  for (; m < J.n && ok; ++m) {
    const PhaseDev &P = J.j[m].L.ph[PH];
    // the work lists of CTA slots q = blockIdx.x, blockIdx.x + gridDim.x, ... (all of them when
    // the launch has a CTA per work list)
    for (int q = blockIdx.x; q < P.nct && ok; q += gridDim.x) {
      const uint32_t e0 = __ldg(P.cta_e0 + q), e1 = __ldg(P.cta_e0 + q + 1);
      ok = produce<FMT, PH, R>(J.j[m].L, e0, e1, smem, full, empty, i, cur);
    }
    if (!ok) break;
  }
  // the last copy issued into every slot has landed before the CTA exits
  if (lane == 0) {
    uint32_t *status = J.j[m < J.n ? m : J.n - 1].L.status;
    const uint32_t first = i > uint32_t(kStages) ? i - kStages : 0;
    for (uint32_t j = first; j < i; ++j)
      if (!mbar_wait(&full[j % kStages], (j / kStages) & 1)) {
        atomicOr(status, 4u);
        break;
      }
  }
}

// segment of column slice c of a piece (largest q with cstart <= c)
__device__ __forceinline__ int find_seg(const Seg *segs, int nseg, int c) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (int(segs[mid].cstart) <= c)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------------
// Phase 1 consumers: one lane per X column slice, t_i m_min(W_i) (or a partial sum)
// ---------------------------------------------------------------------------------------------
template <int FMT>
__device__ bool consume_phase1(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                               uint64_t *empty) {
  using A = typename Tr<FMT>::A;
  constexpr size_t slot = slot_bytes<FMT, 0>();
  const int t = threadIdx.x;
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const A *aux = reinterpret_cast<const A *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    A dot = A(0);
    uint32_t G = 1;
    const Seg *sgp = nullptr;
    int j = 0;
    bool lead = false;
    if (t < int(ph->ncols)) {
      if constexpr (FMT == FMT_RAW64) {
        // contiguous pieces: the lane's segment by binary search over the segments' first lanes
        const Seg &sg = segs[find_seg(segs, ph->nseg, t)];
        const int rel = t - int(sg.cstart);
        const int jj = rel >> sg.lg;
        if (jj < int(sg.nc)) {
          sgp = &sg;
          j = jj;
          G = 1u << sg.lg;
          const int sub = rel & int(G - 1);
          lead = sub == 0;
          const uint32_t ch = Wd[sg.col_w + j];
          const uint32_t *Dc = Wd + sg.data_w + (ch & 0xffffu);
          const int r0 = sub * kSubRows;
          const int rc = min(kSubRows, int(sg.nr) - r0);  // rows of this lane (may be <= 0)
          const A *xr = aux + sg.xs + r0;
          const double *Dd = reinterpret_cast<const double *>(Dc) + r0;
#pragma unroll 4
          for (int r = 0; r < rc; ++r) dot = fma(Dd[r], xr[r], dot);
        }
      } else {
        // bank-column pieces: the lane's slice is column (t & 31) of its warp's region; value i
        // of it is row sub + i G of the X column
        const LaneHdr h = lane_hdrs(sl, ph)[t];
        if (h.seg != 0xff) {
          const Seg &sg = segs[h.seg];
          sgp = &sg;
          j = h.j;
          G = 1u << sg.lg;
          const int sub = t & int(G - 1);
          lead = sub == 0;
          const int rc = (int(sg.nr) - sub + int(G) - 1) >> sg.lg;
          const A *xr = aux + sg.xs + sub;
          const int xs = int(G);
          const uint32_t *col = Wd + bc_column(ph, t);
          const ColDec c = lane_dec(h);
          if (c.narrow) {
            uint32_t bit = 0;
            if constexpr (kFP32<FMT>) {
              if (fast_dec<FMT>(c)) {
                const uint32_t col_s = smem_u32(col);
                const uint32_t xstep = uint32_t(xs) * 4u;
                uint32_t xa = smem_u32(xr);
#pragma unroll 8
                for (int r = 0; r < rc; ++r, bit += c.w, xa += xstep)
                  dot = fmaf(val32<FMT>(bc_code32_s(col_s, bit), c), ld_shared_f32(xa), dot);
              } else if (FMT == FMT_AFL32 && c.mid32) {
                // mantissas wider than FP32's: the FP64 route's values from FP32 operations
                const uint32_t col_s = smem_u32(col);
                const uint32_t xstep = uint32_t(xs) * 4u;
                uint32_t xa = smem_u32(xr);
#pragma unroll 4
                for (int r = 0; r < rc; ++r, bit += c.w, xa += xstep)
                  dot = fmaf(dec_mid32(bc_code32_s(col_s, bit), c), ld_shared_f32(xa), dot);
              } else {
                for (int r = 0; r < rc; ++r, bit += c.w)
                  dot = fmaf(float(dec_any64(bc_code32(col, bit), c, kVF<FMT>)), xr[r * xs], dot);
              }
            } else {
#pragma unroll 4
              for (int r = 0; r < rc; ++r, bit += c.w) dot = fma(dec_any64(bc_code32(col, bit), c, L.vfmt), xr[r * xs], dot);
            }
          } else {
            const int vf = kFP32<FMT> ? kVF<FMT> : L.vfmt;
            for (int r = 0; r < rc; ++r) dot += A(dec_any64(bc_code64(col, uint32_t(r) * c.w), c, vf)) * xr[r * xs];
          }
        }
      }
    }
    // the G lanes of a column (an aligned group) sum their row parts in a fixed order
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const A v = __shfl_xor_sync(kFull, dot, o);
      if (o < G) dot += v;
    }
    if (lead) {
      const Seg &sg = *sgp;
      const A f = aux[sg.fs + j];
      if (sg.x.nchunks == 1) {
        if constexpr (kFP32<FMT>)
          L.tw32[sg.tidx + j] = dot * f;
        else
          L.tw64[sg.tidx + j] = dot * f;
      } else {
        L.partial[size_t(sg.x.pbase) + size_t(j) * sg.x.nchunks + sg.x.chunk] = double(dot);
      }
    }
    release_slot(&empty[s]);
  }
  return true;
}

// Phase 1, AFL codes, FP32 accumulation with two codes per window (code_pair): the lane's rc
// values (rows sub, sub + G, ... of its X column), decoded as dec_f32 does, times the staged x
// of their rows, summed in two FP32 partial sums (even and odd values). An odd last value comes
// with the next (unused) code of its window; windows read at most two rows of 32 words past the
// slice (inside the pad).
template <bool WIDE, bool MID = false>
__device__ __forceinline__ float p1_pairs(int rc, uint32_t col_s, const ColDec &c, uint32_t xa, uint32_t xstep) {
  float s0 = 0.f, s1 = 0.f;
  uint32_t b = 0;
  int r = 0;
#pragma unroll 2
  for (; r + 2 <= rc; r += 2, b += 2 * c.w, xa += 2 * xstep) {
    uint32_t c0, c1;
    code_pair<WIDE>(col_s, b, c.w, c0, c1);
    s0 = fmaf(MID ? dec_mid32(c0, c) : dec_f32(c0, c), ld_shared_f32(xa), s0);
    s1 = fmaf(MID ? dec_mid32(c1, c) : dec_f32(c1, c), ld_shared_f32(xa + xstep), s1);
  }
  if (r < rc) {
    uint32_t c0, c1;
    code_pair<WIDE>(col_s, b, c.w, c0, c1);
    s0 = fmaf(MID ? dec_mid32(c0, c) : dec_f32(c0, c), ld_shared_f32(xa), s0);
  }
  return s0 + s1;
}

__device__ bool consume_phase1_pairs(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                     uint64_t *empty) {
  constexpr int FMT = FMT_AFL32;
  constexpr size_t slot = slot_bytes<FMT, 0>();
  const int t = threadIdx.x;
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const float *aux = reinterpret_cast<const float *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    LaneHdr h{0xff, 0, 0, 0};
    if (t < int(ph->ncols)) h = lane_hdrs(sl, ph)[t];
    const bool active = h.seg != 0xff;
    const ColDec c = col_dec(h.e & 0x7fu, h.m);
    const bool narrow = __all_sync(kFull, !active || (c.fast32 && c.w <= 16));
    float dot = 0.f;
    uint32_t G = 1;
    const Seg *sgp = nullptr;
    bool lead = false;
    if (active) {
      const Seg &sg = segs[h.seg];
      sgp = &sg;
      G = 1u << sg.lg;
      const int sub = t & int(G - 1);
      lead = sub == 0;
      const int rc = (int(sg.nr) - sub + int(G) - 1) >> sg.lg;  // rows sub, sub + G, ...
      const uint32_t *col = Wd + bc_column(ph, t);
      const uint32_t xa = smem_u32(aux + sg.xs + sub), xstep = 4u * G;
      if (c.fast32) {
        dot = narrow ? p1_pairs<false>(rc, smem_u32(col), c, xa, xstep) : p1_pairs<true>(rc, smem_u32(col), c, xa, xstep);
      } else if (c.mid32 && c.w <= 31) {  // mantissas wider than FP32's, two codes per window
        dot = p1_pairs<true, true>(rc, smem_u32(col), c, xa, xstep);
      } else {
        const float *xr = aux + sg.xs + sub;
        uint32_t bit = 0;
        if (c.mid32) {
          // mantissas wider than FP32's: the FP64 route's values from FP32 operations
          for (int r = 0; r < rc; ++r, bit += c.w) dot = fmaf(dec_mid32(bc_code32(col, bit), c), xr[r * int(G)], dot);
        } else if (c.narrow) {
          for (int r = 0; r < rc; ++r, bit += c.w)
            dot = fmaf(float(dec_f64(bc_code32(col, bit), c)), xr[r * int(G)], dot);
        } else {
          for (int r = 0; r < rc; ++r, bit += c.w)
            dot = fmaf(float(dec_f64(bc_code64(col, bit), c)), xr[r * int(G)], dot);
        }
      }
    }
    // the G lanes of a column (an aligned group) sum their row parts in a fixed order
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const float v = __shfl_xor_sync(kFull, dot, o);
      if (o < G) dot += v;
    }
    if (lead) {
      const Seg &sg = *sgp;
      const float f = aux[sg.fs + h.j];
      if (sg.x.nchunks == 1)
        L.tw32[sg.tidx + h.j] = dot * f;
      else
        L.partial[size_t(sg.x.pbase) + size_t(h.j) * sg.x.nchunks + sg.x.chunk] = double(dot);
    }
    release_slot(&empty[s]);
  }
  return true;
}

// Columns of blocks whose phase-1 work is split into chunks: sum the partial sums in chunk
// order and apply the column factor (deterministic, no atomics). One product per blockIdx.y;
// R > 1 handles the R right-hand sides of a multi-RHS pass.
template <int FMT, int R, int NB>
__global__ void k_combine(const __grid_constant__ Jobs<NB> J) {
  const Job &jb = J.j[blockIdx.y];
  const DevLayout &L = jb.L;
  const int64_t total = int64_t(L.ncnt) * R;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const Combine c = L.comb[i / R];
    const int q = int(i % R);
    double sum = 0.0;
    if constexpr (R == 1) {
      for (uint32_t k = 0; k < c.nchunks; ++k) sum += L.partial[size_t(c.pbase) + k];
      if constexpr (kFP32<FMT>)
        L.tw32[c.tidx] = float(sum * double(L.fac32[c.tidx]));
      else
        L.tw64[c.tidx] = sum * L.fac64[c.tidx];
    } else {
      for (uint32_t k = 0; k < c.nchunks; ++k) sum += jb.part[(size_t(c.pbase) + k) * R + q];
      jb.tw[size_t(c.tidx) * R + q] = float(sum * double(L.fac32[c.tidx]));
    }
  }
}

// Setup of this lane's column slice j of segment sg: bit offset of row 0, e, m, multiplier.
template <int FMT>
__device__ __forceinline__ void slice_setup(const Seg &sg, int j, int nr, const uint32_t *Wd,
                                            const typename Tr<FMT>::A *aux, uint32_t &start, uint32_t &e,
                                            uint32_t &m, typename Tr<FMT>::A &mult) {
  using A = typename Tr<FMT>::A;
  if (sg.kind == SEG_DENSE) {
    e = sg.col_w & 0xffu;
    m = (sg.col_w >> 8) & 0xffu;
    const uint32_t w = FMT == FMT_RAW64 ? 64u : 1u + e + m;
    start = uint32_t(sg.data_w) * 32u + uint32_t(j * nr) * w;
    mult = aux[sg.xs + j] * A(sg.m_min);
  } else {
    const uint32_t ch = Wd[sg.col_w + j];
    e = (ch >> 16) & 0xffu;
    m = ch >> 24;
    start = (uint32_t(sg.data_w) + (ch & 0xffffu)) * 32u;
    mult = aux[sg.xs + j];
  }
}

// ---------------------------------------------------------------------------------------------
// Phase 2, FP32 accumulation: one lane per column slice of the leaf (its lane column of the
// bank-column piece). A lane keeps the FP32 sums of its columns' products for all rows of the
// leaf in registers, over all pieces of the leaf; at the end of the leaf each warp reduces its
// 32 lanes' row sums with a butterfly of shuffles (fixed order) and the four warps' sums are
// added in FP64, in fixed order, into y.
// ---------------------------------------------------------------------------------------------
// rows [0, nr) of the lane's slice into acc[r]; rows past the leaf decode the slice's first value
// (in bounds) and are dropped. MODE 0: the FP32 bit-pattern decode; 1: dec_mid32 (the FP64
// route's values, for warps with mantissas wider than FP32's); 2 (GEN): the generic FP64 decode
// (codes wider than 32 bits, large e).
template <int MODE, int FMT>
__device__ __forceinline__ void p2_rows(float (&acc)[64], int nr, const uint32_t *col, const ColDec &c, float mult) {
  constexpr bool GEN = MODE == 2;
  const uint32_t col_s = smem_u32(col);  // 32-bit shared-memory address of the lane column
  // chunks of 8 rows: leaves of the cluster tree hold 32..64 rows, so a row count that is not a
  // multiple of the chunk costs at most 7 predicated decodes
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (8 * k >= nr) break;
    if (!GEN && 8 * k + 8 <= nr) {  // a whole chunk of the leaf: no row checks
      uint32_t bit = uint32_t(8 * k) * c.w;
#pragma unroll
      for (int rr = 0; rr < 8; ++rr, bit += c.w) {
        const uint32_t code = bc_code32_s(col_s, bit);
        acc[8 * k + rr] += MODE == 1 ? dec_mid32(code, c) * mult : valmul32<FMT>(code, c, mult);
      }
    } else {
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int r = 8 * k + rr;
        const bool ok = r < nr;
        const uint32_t bit = uint32_t(ok ? r : 0) * c.w;
        const float p = GEN         ? float(dec_any64(bc_code64(col, bit), c, kVF<FMT>)) * mult
                        : MODE == 1 ? dec_mid32(bc_code32_s(col_s, bit), c) * mult
                                    : valmul32<FMT>(bc_code32_s(col_s, bit), c, mult);
        if (ok) acc[r] += p;
      }
    }
  }
}

template <int FMT>
__device__ bool consume_phase2_reg(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                   uint64_t *empty, double *red, double *__restrict__ y, uint32_t &parity) {
  constexpr size_t slot = slot_bytes<FMT, 1>();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float acc[64];
#pragma unroll
  for (int r = 0; r < 64; ++r) acc[r] = 0.f;
  int64_t gi = 0;
  double yold = 0.0;  // y of this thread's row, read when the leaf starts
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const float *aux = reinterpret_cast<const float *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    const int nr = ph->nr;
    const uint32_t flags = ph->flags;
    if (flags & PF_START_LEAF) {
#pragma unroll
      for (int r = 0; r < 64; ++r) acc[r] = 0.f;
      if (t < nr) {
        gi = __ldg(L.perm + ph->row0 + uint32_t(t));
        yold = y[gi];
      }
    }
    // idle lanes (no slice) skip the rows
    float mult = 0.f;
    LaneHdr hd{0xff, 0, 0, 0};
    const uint32_t *col = Wd;
    bool active = false;
    if (t < int(ph->ncols)) {
      const LaneHdr h = lane_hdrs(sl, ph)[t];
      if (h.seg != 0xff) {
        const Seg &sg = segs[h.seg];
        mult = sg.kind == SEG_DENSE ? aux[sg.xs + h.j] * float(sg.m_min) : aux[sg.xs + h.j];
        hd = h;
        col = Wd + bc_column(ph, t);
        active = true;
      }
    }
    const ColDec c = lane_dec(hd);
    const bool fast = __all_sync(kFull, !active || fast_dec<FMT>(c));  // FP32 bit-pattern decode
    // AFL codes with mantissas wider than FP32's: the FP64 route's values from FP32 operations
    const bool mid = FMT == FMT_AFL32 && !fast && __all_sync(kFull, !active || c.mid32);
    if (active) {
      if (fast)
        p2_rows<0, FMT>(acc, nr, col, c, mult);
      else if (mid)
        p2_rows<1, FMT>(acc, nr, col, c, mult);
      else
        p2_rows<2, FMT>(acc, nr, col, c, mult);
    }
    if (flags & PF_END_LEAF) {
      // reduce-scatter over the warp: 5 halving stages (stage s keeps the upper half of the
      // vector when lane bit 4 - s is set); afterwards lane l holds the sums of rows 2l, 2l + 1
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const int half = 32 >> st;      // current vector length / 2
        const int mask = 16 >> st;
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
          const float send = up ? acc[q] : acc[q + half];
          const float keep = up ? acc[q + half] : acc[q];
          acc[q] = keep + __shfl_xor_sync(kFull, send, mask);
        }
      }
      const int rb = 2 * lane;
      double *buf = red + parity * (kCWarps * 64);
      buf[warp * 64 + rb] = double(acc[0]);
      buf[warp * 64 + rb + 1] = double(acc[1]);
      bar_consumers();
      if (t < nr) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < kCWarps; ++w) sum += buf[w * 64 + t];
        y[gi] = yold + sum;  // the only update of this row (its leaf has one owner CTA)
      }
      parity ^= 1u;
    }
    release_slot(&empty[s]);
  }
  return true;
}

// Phase 2, AFL codes, FP32 accumulation with two codes per window: as consume_phase2_reg (the
// same products dec_mul_f32 forms, the same row sums), but a warp whose lanes all have FP32-
// pattern codes takes two rows per window (code_pair), and a leaf's row totals go to ysum in
// cluster order (one store per row; k_scatter then adds them into y, so no register holds y or
// the permutation during the leaf). The row after an odd row count decodes the next code of its
// window (at most two rows of 32 words past the last warp region, inside the slot's pad) into a
// row sum that is never stored.
static_assert(8 * 128 <= kSlotPad + kAuxMax2 * 4, "phase-2 window reads stay inside the slot");

template <bool WIDE>
__device__ __forceinline__ void p2_pairs(float (&acc)[64], int nr, uint32_t col_s, const ColDec &c, float mult) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (8 * k >= nr) break;
    const bool whole = 8 * k + 8 <= nr;  // the leaf's rows cover the chunk: no row checks
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = 4 * k + q;  // rows 2p, 2p + 1
      if (!whole && 2 * p >= nr) break;
      uint32_t c0, c1;
      code_pair<WIDE>(col_s, uint32_t(2 * p) * c.w, c.w, c0, c1);
      acc[2 * p] += dec_mul_f32(c0, c, mult);
      acc[2 * p + 1] += dec_mul_f32(c1, c, mult);
    }
  }
}

__device__ bool consume_phase2_pairs(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                     uint64_t *empty, double *red, uint32_t &parity) {
  constexpr int FMT = FMT_AFL32;
  constexpr size_t slot = slot_bytes<FMT, 1>();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float acc[64];
#pragma unroll
  for (int r = 0; r < 64; ++r) acc[r] = 0.f;
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const float *aux = reinterpret_cast<const float *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    const int nr = ph->nr;
    const uint32_t flags = ph->flags;
    if (flags & PF_START_LEAF) {
#pragma unroll
      for (int r = 0; r < 64; ++r) acc[r] = 0.f;
    }
    float mult = 0.f;
    uint32_t e = 0, m = 0;
    const uint32_t *col = Wd;
    bool active = false;
    if (t < int(ph->ncols)) {
      const LaneHdr h = lane_hdrs(sl, ph)[t];
      if (h.seg != 0xff) {
        const Seg &sg = segs[h.seg];
        mult = sg.kind == SEG_DENSE ? aux[sg.xs + h.j] * float(sg.m_min) : aux[sg.xs + h.j];
        e = h.e & 0x7fu;
        m = h.m;
        col = Wd + bc_column(ph, t);
        active = true;
      }
    }
    const ColDec c = col_dec(e, m);
    if (__all_sync(kFull, !active || (c.fast32 && c.w <= 16))) {
      if (active) p2_pairs<false>(acc, nr, smem_u32(col), c, mult);
    } else if (__all_sync(kFull, !active || c.fast32)) {
      if (active) p2_pairs<true>(acc, nr, smem_u32(col), c, mult);
    } else {
      // mantissas wider than FP32's: the FP64 route's values from FP32 operations
      const bool mid = __all_sync(kFull, !active || c.mid32);
      if (active) {
        if (mid)
          p2_rows<1, FMT>(acc, nr, col, c, mult);
        else
          p2_rows<2, FMT>(acc, nr, col, c, mult);
      }
    }
    // the slot is not read after this point: hand it back before the leaf's reduction
    const uint32_t row0 = ph->row0;
    release_slot(&empty[s]);
    if (flags & PF_END_LEAF) {
      // reduce-scatter over the warp (as consume_phase2_reg): lane l ends with rows 2l, 2l + 1
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const int half = 32 >> st;
        const int mask = 16 >> st;
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
          const float send = up ? acc[q] : acc[q + half];
          const float keep = up ? acc[q + half] : acc[q];
          acc[q] = keep + __shfl_xor_sync(kFull, send, mask);
        }
      }
      const int rb = 2 * lane;
      double *buf = red + parity * (kCWarps * 64);
      buf[warp * 64 + rb] = double(acc[0]);
      buf[warp * 64 + rb + 1] = double(acc[1]);
      bar_consumers();
      if (t < nr) {
        double sum = 0.0;
#pragma unroll
        for (int w4 = 0; w4 < kCWarps; ++w4) sum += buf[w4 * 64 + t];
        L.ysum[row0 + uint32_t(t)] = sum;  // the row's total (its leaf has one owner CTA)
      }
      parity ^= 1u;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// FP64 accumulation over AFL codes with one FP64 multiply-add per value. For a code of the FP32
// fast path, v - 1 is exact in FP32 (at most 24 significant bits, 0 or >= 1), so its FP64
// pattern follows from the FP32 one by integer operations (rebias the exponent by
// 1023 - 127, widen the mantissa); the value is then fma(v - 1, +-mult, acc) in FP64 with the
// code's sign on the multiplier. Other codes take the FP64 route: v - 1.0 in FP64, then the
// multiply-add.
// ---------------------------------------------------------------------------------------------
// FP64 value of a nonnegative FP32 bit pattern P of a normal number or zero
__device__ __forceinline__ double f32pat_to_f64(uint32_t P) {
  const uint32_t hi = P != 0u ? (P >> 3) + 0x38000000u : 0u;
  return __hiloint2double(int(hi), int(P << 29));
}
// v - 1 of a code (fast path, code at bit 0, other bits above) as FP64
__device__ __forceinline__ double vm1_f64(uint32_t code, const ColDec &c) {
  const float v = __uint_as_float((code & c.em_mask) * c.scale + 0x3F800000u) - 1.0f;
  return f32pat_to_f64(__float_as_uint(v));
}
// v - 1 exactly in FP64, with integer operations only, for a code of w <= 31 bits whose field is
// below 16 (e <= 4) and whose mantissa may be wider than FP32's (m up to 30): N = (v - 1) 2^m =
// (2^m + mant) 2^field - 2^m is an integer below 2^47, so normalising it gives the exact pattern
// (the value the FP64 route RN(v - 1) gives, since fewer than 53 bits are significant)
__device__ __forceinline__ double vm1_f64_mid(uint32_t code, const ColDec &c) {
  const uint32_t m = c.m;
  const uint32_t mant = m ? (code & (0xffffffffu >> (32 - m))) : 0u;
  const uint32_t field = (code >> m) & ((1u << c.e) - 1u);
  const uint64_t N = (((uint64_t(1) << m) + mant) << field) - (uint64_t(1) << m);
  if (N == 0) return 0.0;
  const int msb = 63 - __clzll(static_cast<long long>(N));
  const uint64_t frac = (N << (52 - msb)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double(static_cast<long long>((uint64_t(msb - int(m) + 1023) << 52) | frac));
}
// +-s with the code's sign
__device__ __forceinline__ double signed_f64(uint32_t code, const ColDec &c, double s) {
  return __hiloint2double(__double2hiint(s) ^ int((code << c.sshift) & 0x80000000u), __double2loint(s));
}

// Phase 2, FP64 accumulation, AFL codes: one lane per column slice of the leaf, FP64 row sums
// in registers (one multiply-add per value), a butterfly over the warp and the four warps'
// sums into ysum at the end of the leaf (as consume_phase2_pairs).
template <bool WIDE>
__device__ __forceinline__ void p2_pairs64(double (&acc)[64], int nr, uint32_t col_s, const ColDec &c, double mult) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (8 * k >= nr) break;
    const bool whole = 8 * k + 8 <= nr;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = 4 * k + q;
      if (!whole && 2 * p >= nr) break;
      uint32_t c0, c1;
      code_pair<WIDE>(col_s, uint32_t(2 * p) * c.w, c.w, c0, c1);
      acc[2 * p] = fma(vm1_f64(c0, c), signed_f64(c0, c, mult), acc[2 * p]);
      acc[2 * p + 1] = fma(vm1_f64(c1, c), signed_f64(c1, c, mult), acc[2 * p + 1]);
    }
  }
}
// the FP64 route for codes outside the fast path (rows past the leaf decode the slice's first
// value and are dropped)
__device__ __forceinline__ void p2_rows64(double (&acc)[64], int nr, const uint32_t *col, const ColDec &c, double mult) {
#pragma unroll
  for (int r = 0; r < 64; ++r) {
    if (r >= nr) break;
    acc[r] = fma(dec_f64(bc_code64(col, uint32_t(r) * c.w), c), mult, acc[r]);
  }
}

__device__ bool consume_phase2_f64(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                   uint64_t *empty, double *red, uint32_t &parity) {
  constexpr int FMT = FMT_AFL64;
  constexpr size_t slot = slot_bytes<FMT, 1>();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double acc[64];
#pragma unroll
  for (int r = 0; r < 64; ++r) acc[r] = 0.0;
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const double *aux = reinterpret_cast<const double *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    const int nr = ph->nr;
    const uint32_t flags = ph->flags;
    if (flags & PF_START_LEAF) {
#pragma unroll
      for (int r = 0; r < 64; ++r) acc[r] = 0.0;
    }
    double mult = 0.0;
    uint32_t e = 0, m = 0;
    const uint32_t *col = Wd;
    bool active = false;
    if (t < int(ph->ncols)) {
      const LaneHdr h = lane_hdrs(sl, ph)[t];
      if (h.seg != 0xff) {
        const Seg &sg = segs[h.seg];
        mult = sg.kind == SEG_DENSE ? aux[sg.xs + h.j] * sg.m_min : aux[sg.xs + h.j];
        e = h.e & 0x7fu;
        m = h.m;
        col = Wd + bc_column(ph, t);
        active = true;
      }
    }
    const ColDec c = col_dec(e, m);
    if (__all_sync(kFull, !active || (c.fast32 && c.w <= 16))) {
      if (active) p2_pairs64<false>(acc, nr, smem_u32(col), c, mult);
    } else if (__all_sync(kFull, !active || c.fast32)) {
      if (active) p2_pairs64<true>(acc, nr, smem_u32(col), c, mult);
    } else if (active) {
      p2_rows64(acc, nr, col, c, mult);
    }
    // the slot is not read after this point: hand it back before the leaf's reduction
    const uint32_t row0 = ph->row0;
    release_slot(&empty[s]);
    if (flags & PF_END_LEAF) {
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const int half = 32 >> st;
        const int mask = 16 >> st;
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
          const double send = up ? acc[q] : acc[q + half];
          const double keep = up ? acc[q + half] : acc[q];
          acc[q] = keep + __shfl_xor_sync(kFull, send, mask);
        }
      }
      const int rb = 2 * lane;
      double *buf = red + parity * (kCWarps * 64);
      buf[warp * 64 + rb] = acc[0];
      buf[warp * 64 + rb + 1] = acc[1];
      bar_consumers();
      if (t < nr) {
        double sum = 0.0;
#pragma unroll
        for (int w4 = 0; w4 < kCWarps; ++w4) sum += buf[w4 * 64 + t];
        L.ysum[row0 + uint32_t(t)] = sum;  // the row's total (its leaf has one owner CTA)
      }
      parity ^= 1u;
    }
  }
  return true;
}

// Phase 1, FP64 accumulation, AFL codes: the lane's values times the staged FP64 x of their rows,
// one multiply-add per value into two FP64 partial sums.
template <bool WIDE, bool MID = false>
__device__ __forceinline__ double p1_pairs64(int rc, uint32_t col_s, const ColDec &c, const double *xr, int xs) {
  double s0 = 0.0, s1 = 0.0;
  uint32_t b = 0;
  int r = 0;
#pragma unroll 2
  for (; r + 2 <= rc; r += 2, b += 2 * c.w) {
    uint32_t c0, c1;
    code_pair<WIDE>(col_s, b, c.w, c0, c1);
    s0 = fma(MID ? vm1_f64_mid(c0, c) : vm1_f64(c0, c), signed_f64(c0, c, xr[r * xs]), s0);
    s1 = fma(MID ? vm1_f64_mid(c1, c) : vm1_f64(c1, c), signed_f64(c1, c, xr[(r + 1) * xs]), s1);
  }
  if (r < rc) {
    uint32_t c0, c1;
    code_pair<WIDE>(col_s, b, c.w, c0, c1);
    s0 = fma(MID ? vm1_f64_mid(c0, c) : vm1_f64(c0, c), signed_f64(c0, c, xr[r * xs]), s0);
  }
  return s0 + s1;
}

__device__ bool consume_phase1_f64(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                   uint64_t *empty) {
  constexpr int FMT = FMT_AFL64;
  constexpr size_t slot = slot_bytes<FMT, 0>();
  const int t = threadIdx.x;
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const double *aux = reinterpret_cast<const double *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    LaneHdr h{0xff, 0, 0, 0};
    if (t < int(ph->ncols)) h = lane_hdrs(sl, ph)[t];
    const bool active = h.seg != 0xff;
    const ColDec c = col_dec(h.e & 0x7fu, h.m);
    const bool narrow = __all_sync(kFull, !active || (c.fast32 && c.w <= 16));
    double dot = 0.0;
    uint32_t G = 1;
    const Seg *sgp = nullptr;
    bool lead = false;
    if (active) {
      const Seg &sg = segs[h.seg];
      sgp = &sg;
      G = 1u << sg.lg;
      const int sub = t & int(G - 1);
      lead = sub == 0;
      const int rc = (int(sg.nr) - sub + int(G) - 1) >> sg.lg;  // rows sub, sub + G, ...
      const uint32_t *col = Wd + bc_column(ph, t);
      const double *xr = aux + sg.xs + sub;
      if (c.fast32) {
        dot = narrow ? p1_pairs64<false>(rc, smem_u32(col), c, xr, int(G)) : p1_pairs64<true>(rc, smem_u32(col), c, xr, int(G));
      } else if (c.mid32 && c.w <= 31) {  // mantissas wider than FP32's: exact v - 1 by integer ops
        dot = p1_pairs64<true, true>(rc, smem_u32(col), c, xr, int(G));
      } else {
        uint32_t bit = 0;
        for (int r = 0; r < rc; ++r, bit += c.w) dot = fma(dec_f64(bc_code64(col, bit), c), xr[r * int(G)], dot);
      }
    }
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const double v = __shfl_xor_sync(kFull, dot, o);
      if (o < G) dot += v;
    }
    if (lead) {
      const Seg &sg = *sgp;
      const double f = aux[sg.fs + h.j];
      if (sg.x.nchunks == 1)
        L.tw64[sg.tidx + h.j] = dot * f;
      else
        L.partial[size_t(sg.x.pbase) + size_t(h.j) * sg.x.nchunks + sg.x.chunk] = dot;
    }
    release_slot(&empty[s]);
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// Phase 2 consumers, AFL formats: one lane per column slice of the leaf (its lane column of the
// bank-column piece); every 16 rows the lanes write their products to a padded shared-memory
// tile and sum it transposed (two lanes per row, one shuffle). FP32 path: FP32 products and
// tile sums, compensated FP32 pairs across pieces; FP64 path: the same in FP64.
// ---------------------------------------------------------------------------------------------
template <int FMT>
__device__ bool consume_phase2(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                               uint64_t *empty, double *red, typename Tr<FMT>::A *tiles, double *__restrict__ y,
                               uint32_t &parity) {
  using A = typename Tr<FMT>::A;
  using Acc = typename std::conditional<FMT == FMT_AFL32, Comp32, Sum64>::type;
  constexpr size_t slot = slot_bytes<FMT, 1>();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  Acc acc[4];  // rows lane + 16 k (lanes 0..15) of the leaf: this warp's columns so far
  int64_t gi = 0;
  double yold = 0.0;  // y of this thread's row, read when the leaf starts
  A *tile = tiles + warp * (16 * 33);
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const A *aux = reinterpret_cast<const A *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    const int nr = ph->nr;
    const uint32_t flags = ph->flags;
    if (flags & PF_START_LEAF) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k].reset();
      if (t < nr) {
        gi = __ldg(L.perm + ph->row0 + uint32_t(t));
        yold = y[gi];
      }
    }
    // idle lanes (no slice) write zeros
    A mult = A(0);
    uint32_t e = 0, m = 0;
    const uint32_t *col = Wd;
    bool active = false;
    if (t < int(ph->ncols)) {
      const LaneHdr h = lane_hdrs(sl, ph)[t];
      if (h.seg != 0xff) {
        const Seg &sg = segs[h.seg];
        mult = sg.kind == SEG_DENSE ? aux[sg.xs + h.j] * A(sg.m_min) : aux[sg.xs + h.j];
        e = h.e & 0x7fu;
        m = h.m;
        col = Wd + bc_column(ph, t);
        active = true;
      }
    }
    const ColDec c = col_dec(e, m);
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // 16-row chunks (nr <= 64)
      const int r0 = 16 * k;
      if (r0 >= nr) break;
      const int rows = min(16, nr - r0);
      const uint32_t bit0 = uint32_t(r0) * c.w;
      if constexpr (FMT == FMT_AFL32) {
        if (rows == 16 && c.fast32) {
#pragma unroll
          for (int rr = 0; rr < 16; ++rr) tile[rr * 33 + lane] = dec_mul_f32(bc_code32(col, bit0 + rr * c.w), c, mult);
        } else if (c.fast32) {
          for (int rr = 0; rr < rows; ++rr) tile[rr * 33 + lane] = dec_mul_f32(bc_code32(col, bit0 + rr * c.w), c, mult);
        } else if (c.narrow) {
          for (int rr = 0; rr < rows; ++rr)
            tile[rr * 33 + lane] = float(dec_f64(bc_code32(col, bit0 + rr * c.w), c)) * mult;
        } else {
          for (int rr = 0; rr < rows; ++rr)
            tile[rr * 33 + lane] = float(dec_f64(bc_code64(col, bit0 + rr * c.w), c)) * mult;
        }
      } else {
        if (!active) {
          for (int rr = 0; rr < rows; ++rr) tile[rr * 33 + lane] = A(0);
        } else if (c.narrow) {
#pragma unroll 4
          for (int rr = 0; rr < rows; ++rr)
            tile[rr * 33 + lane] = dec_any64(bc_code32(col, bit0 + rr * c.w), c, L.vfmt) * mult;
        } else {
          for (int rr = 0; rr < rows; ++rr)
            tile[rr * 33 + lane] = dec_any64(bc_code64(col, bit0 + rr * c.w), c, L.vfmt) * mult;
        }
      }
      __syncwarp();
      // transposed sum: lane l adds row (l & 15) over columns 16 (l >> 4) .. + 15; the two
      // halves are combined with one shuffle
      const int row = lane & 15;
      A sum = A(0);
      if (row < rows) {
        const A *tr = tile + row * 33 + (lane >> 4) * 16;
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) sum += tr[cc];
      }
      sum += __shfl_xor_sync(kFull, sum, 16);
      if (lane < rows) acc[k].add(sum);
      __syncwarp();
    }
    if (flags & PF_END_LEAF) {
      // per-warp row sums; the two halves of red alternate between leaves, so one barrier
      // suffices (a half is rewritten only after the next leaf's barrier)
      double *buf = red + parity * (kCWarps * 64);
      if (lane < 16) {
#pragma unroll
        for (int k = 0; k < 4; ++k) buf[warp * 64 + 16 * k + lane] = acc[k].value();
      }
      bar_consumers();
      if (t < nr) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < kCWarps; ++w) sum += buf[w * 64 + t];
        y[gi] = yold + sum;  // the only update of this row (its leaf has one owner CTA)
      }
      parity ^= 1u;
    }
    release_slot(&empty[s]);
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// Phase 2 consumers, FP64 paths: lanes are the rows of the leaf (lane, lane + 32); the warps
// take the piece's column slices in turn; one FP64 fused multiply-add per value
// ---------------------------------------------------------------------------------------------
template <int FMT>
__device__ bool consume_phase2_rows(const DevLayout &L, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                    uint64_t *empty, double *red, double *__restrict__ y, uint32_t &parity) {
  constexpr size_t slot = slot_bytes<FMT, 1>();
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double a0 = 0.0, a1 = 0.0;
  int64_t gi = 0;
  double yold = 0.0;  // y of this thread's row, read when the leaf starts
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const double *aux = reinterpret_cast<const double *>(sl + kPieceMax + kSlotPad);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    const int nr = ph->nr;
    const uint32_t flags = ph->flags;
    if (flags & PF_START_LEAF) {
      a0 = a1 = 0.0;
      if (t < nr) {
        gi = __ldg(L.perm + ph->row0 + uint32_t(t));
        yold = y[gi];
      }
    }
    const bool ok0 = lane < nr, ok1 = lane + 32 < nr;
    const int ncols = ph->ncols;
    for (int col = warp; col < ncols; col += kCWarps) {
      const Seg &sg = segs[find_seg(segs, ph->nseg, col)];
      double mult;
      uint32_t start, e, m;
      slice_setup<FMT>(sg, col - int(sg.cstart), nr, Wd, aux, start, e, m, mult);
      if constexpr (FMT == FMT_RAW64) {
        const double *Dd = reinterpret_cast<const double *>(Wd + (start >> 5));
        if (ok0) a0 = fma(Dd[lane], mult, a0);
        if (ok1) a1 = fma(Dd[lane + 32], mult, a1);
      } else {
        const ColDec c = col_dec(e, m);
        if (ok0) a0 = fma(dec_f64(code64_at(Wd, start + uint32_t(lane) * c.w), c), mult, a0);
        if (ok1) a1 = fma(dec_f64(code64_at(Wd, start + uint32_t(lane + 32) * c.w), c), mult, a1);
      }
    }
    if (flags & PF_END_LEAF) {
      double *buf = red + parity * (kCWarps * 64);
      buf[warp * 64 + lane] = a0;
      buf[warp * 64 + 32 + lane] = a1;
      bar_consumers();
      if (t < nr) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < kCWarps; ++w) sum += buf[w * 64 + t];
        y[gi] = yold + sum;
      }
      parity ^= 1u;
    }
    release_slot(&empty[s]);
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// Tensor-core helpers of the multi-RHS passes: TF32 parts of an FP32 operand and the warp-level
// m16n8k8 TF32 product with FP32 accumulation (fragment layouts of the PTX ISA: A row-major
// a0 = (g, tq), a1 = (g + 8, tq), a2 = (g, tq + 4), a3 = (g + 8, tq + 4); B column-major
// b0 = (tq, g), b1 = (tq + 4, g); C c0 = (g, 2 tq), c1 = (g, 2 tq + 1), c2 = (g + 8, 2 tq),
// c3 = (g + 8, 2 tq + 1), with g = lane / 4 and tq = lane % 4). An FP32 operand x is split into
// hi = tf32(x) and lo = tf32(x - hi); a product is hi hi + hi lo + lo hi (the lo lo term is
// below 2^-22 relative), so the contraction keeps FP32 accuracy.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d = a b (a fresh C fragment of zeros)
__device__ __forceinline__ void mma_tf32_z(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}
// acc += the three part products of one k step, formed in a fresh fragment and added with FP32
// rounding, so that no tensor-core accumulation chain is longer than three products
__device__ __forceinline__ void mma3_add(float (&acc)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                         uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
  float d[4];
  mma_tf32_z(d, al, bh0, bh1);
  mma_tf32(d, ah, bl0, bl1);
  mma_tf32(d, ah, bh0, bh1);
#pragma unroll
  for (int e = 0; e < 4; ++e) acc[e] += d[e];
}

__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

// ---------------------------------------------------------------------------------------------
// Multi-RHS pass of at most 8 columns, phase 1 (FP32): as consume_phase1, but every lane keeps R
// dot products; the x rows come from the pass's X_perm in global memory (R floats per row,
// through L1) and the column factors from fac32. (For 32 columns the x rows would cost 128
// bytes of L1 traffic per value; that pass uses the tensor cores, below.)
// ---------------------------------------------------------------------------------------------
template <int R>
__device__ bool consume_phase1_multi_fma(const Job &jb, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                     uint64_t *empty) {
  const DevLayout &L = jb.L;
  constexpr size_t slot = slot_bytes<FMT_AFL32, 0, R>();
  const int t = threadIdx.x;
  const float4 *xp4 = reinterpret_cast<const float4 *>(jb.xp);
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    float acc[R];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = 0.f;
    uint32_t G = 1;
    const Seg *sgp = nullptr;
    int j = 0;
    bool lead = false;
    if (t < int(ph->ncols)) {
      const LaneHdr h = lane_hdrs(sl, ph)[t];
      if (h.seg != 0xff) {
        const Seg &sg = segs[h.seg];
        sgp = &sg;
        j = h.j;
        G = 1u << sg.lg;
        const int sub = t & int(G - 1);
        lead = sub == 0;
        const int rc = (int(sg.nr) - sub + int(G) - 1) >> sg.lg;   // rows sub, sub + G, ...
        const float4 *xr = xp4 + (size_t(sg.gx) + sub) * (R / 4);
        const int xs = int(G) * (R / 4);
        const uint32_t *col = Wd + bc_column(ph, t);
        const ColDec c = lane_dec(h);
#pragma unroll 4
        for (int r = 0; r < rc; ++r) {
          float v;
          if (c.fast32)
            v = dec_f32(bc_code32(col, uint32_t(r) * c.w), c);
          else if (c.narrow)
            v = float(dec_f64(bc_code32(col, uint32_t(r) * c.w), c));
          else
            v = float(dec_f64(bc_code64(col, uint32_t(r) * c.w), c));
#pragma unroll
          for (int hh = 0; hh < R / 4; ++hh) {
            const float4 xv = __ldg(xr + r * xs + hh);
            acc[4 * hh] = fmaf(v, xv.x, acc[4 * hh]);
            acc[4 * hh + 1] = fmaf(v, xv.y, acc[4 * hh + 1]);
            acc[4 * hh + 2] = fmaf(v, xv.z, acc[4 * hh + 2]);
            acc[4 * hh + 3] = fmaf(v, xv.w, acc[4 * hh + 3]);
          }
        }
      }
    }
    // the G lanes of a column (an aligned group) sum their row parts in a fixed order
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const float v = __shfl_xor_sync(kFull, acc[q], o);
        if (o < G) acc[q] += v;
      }
    }
    if (lead) {
      const Seg &sg = *sgp;
      if (sg.x.nchunks == 1) {
        const float f = __ldg(L.fac32 + sg.tidx + j);
        float4 *dst = reinterpret_cast<float4 *>(jb.tw + (size_t(sg.tidx) + j) * R);
#pragma unroll
        for (int hh = 0; hh < R / 4; ++hh)
          dst[hh] = make_float4(acc[4 * hh] * f, acc[4 * hh + 1] * f, acc[4 * hh + 2] * f, acc[4 * hh + 3] * f);
      } else {
        double *dst = jb.part + (size_t(sg.x.pbase) + size_t(j) * sg.x.nchunks + sg.x.chunk) * R;
#pragma unroll
        for (int q = 0; q < R; ++q) dst[q] = double(acc[q]);
      }
    }
    release_slot(&empty[s]);
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// Multi-RHS pass of up to 32 columns, phase 1: every lane decodes its slice (rows sub, sub + G,
// ... of one column) into a padded shared-memory tile of its warp (64 values per lane and
// round). Then, per segment present in the warp (the X columns of one item of a lowrank block),
// the warp's lanes take (column, row phase, group of 16 right-hand sides) triples: a lane walks
// the rows p, p + P, ... of its column, reads each decoded value from the tile and the row's 16
// x values from X_perm, and keeps 16 FP32 dot products. All lanes of a step read few distinct x
// rows (every column of the segment shares them), so an x row is loaded once per warp and step
// instead of once per value; the P row phases of a column are added with xor-shuffles in fixed
// order. Every column's G lanes lie in one warp, so a warp completes its columns. The result,
// times the column factor (one chunk) or as a chunk partial sum, is written per column.
// ---------------------------------------------------------------------------------------------
template <int R>
__device__ bool consume_phase1_multi(const Job &jb, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                     uint64_t *empty, float *tiles) {
  static_assert(R % 16 == 0, "wide pass: groups of 16 right-hand sides");
  const DevLayout &L = jb.L;
  constexpr size_t slot = slot_bytes<FMT_AFL32, 0, R>();
  constexpr int kVS = 65;           // values per lane in the tile (64) + 1: conflict-free stores by row
  constexpr int NQ = R / 16;        // groups of 16 right-hand sides
  constexpr int SL = 32 / NQ;       // (column, row phase) slots of a warp
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int q = lane % NQ, sl = lane / NQ;
  float *tv = tiles + warp * (32 * kVS + 64);                 // [32 lanes][kVS] decoded values
  int *clane = reinterpret_cast<int *>(tv + 32 * kVS);        // [32] lanes of a segment's columns
  int *cj = clane + 32;                                       // [32] their column indices j
  const float4 *xp4 = reinterpret_cast<const float4 *>(jb.xp);
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl_p = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl_p);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl_p);
    const Seg *segs = reinterpret_cast<const Seg *>(sl_p + 16);
    LaneHdr h{0xff, 0, 0, 0};
    if (t < int(ph->ncols)) h = lane_hdrs(sl_p, ph)[t];
    const bool active = h.seg != 0xff;
    int sub = 0, rc = 0;
    const uint32_t *col = Wd;
    if (active) {
      const Seg &sg = segs[h.seg];
      sub = t & ((1 << sg.lg) - 1);
      rc = (int(sg.nr) - sub + (1 << sg.lg) - 1) >> sg.lg;   // rows sub, sub + G, ...
      col = Wd + bc_column(ph, t);
    }
    const ColDec c = lane_dec(h);
    // this lane's values at positions [r0, r0 + 64) of its slice into its tile row
    auto decode_round = [&](int r0) {
      const int r1 = min(rc, r0 + 64);
#pragma unroll 4
      for (int r = r0; r < r1; ++r) {
        float v;
        if (c.fast32)
          v = dec_f32(bc_code32(col, uint32_t(r) * c.w), c);
        else if (c.narrow)
          v = float(dec_f64(bc_code32(col, uint32_t(r) * c.w), c));
        else
          v = float(dec_f64(bc_code64(col, uint32_t(r) * c.w), c));
        tv[lane * kVS + (r - r0)] = v;
      }
    };
    decode_round(0);
    __syncwarp();
    const int segme = active ? int(h.seg) : -1;
    const bool lead = active && sub == 0;
    uint32_t todo = __ballot_sync(kFull, lead);
    while (todo) {  // warp-uniform: the segments whose columns lead in this warp
      const int s0 = __shfl_sync(kFull, segme, __ffs(todo) - 1);
      const bool mine = lead && segme == s0;
      const uint32_t mask = __ballot_sync(kFull, mine);
      todo &= ~mask;
      const Seg &sg = segs[s0];
      const int lg = sg.lg, gm = (1 << lg) - 1, nr = sg.nr;
      const int ncol = __popc(mask);
      if (mine) {
        const int k = __popc(mask & ((1u << lane) - 1));
        clane[k] = lane;
        cj[k] = h.j;
      }
      __syncwarp();
      for (int c0 = 0; c0 < ncol; c0 += SL) {  // columns in chunks of SL (more than one only if G = 1)
        const int cc = min(SL, ncol - c0);
        int lcp = 0;
        while ((1 << lcp) < cc) ++lcp;       // column slots: the next power of two >= cc
        const int cp = 1 << lcp, P = SL >> lcp;
        const int cl = sl & (cp - 1), p = sl >> lcp;
        const bool on = cl < cc;
        const int lc = on ? clane[c0 + cl] : 0;
        float acc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = 0.f;
        for (int rb = 0; rb < nr; rb += 64 << lg) {  // rounds of 64 positions per lane
          if (rb > 0) {  // slices longer than 64 rows (one column chunk then): decode the next round
            __syncwarp();
            if (segme == s0) decode_round(rb >> lg);
            __syncwarp();
          }
          const int rend = min(nr, rb + (64 << lg));
          if (on) {
#pragma unroll 4
            for (int rho = rb + p; rho < rend; rho += P) {  // unrolled: loads of 4 rows in flight
              const float v = tv[(lc + (rho & gm)) * kVS + ((rho - rb) >> lg)];
              const float4 *xr = xp4 + (size_t(sg.gx) + rho) * (R / 4) + 4 * q;
              const float4 x0 = __ldg(xr), x1 = __ldg(xr + 1), x2 = __ldg(xr + 2), x3 = __ldg(xr + 3);
              acc[0] = fmaf(v, x0.x, acc[0]);
              acc[1] = fmaf(v, x0.y, acc[1]);
              acc[2] = fmaf(v, x0.z, acc[2]);
              acc[3] = fmaf(v, x0.w, acc[3]);
              acc[4] = fmaf(v, x1.x, acc[4]);
              acc[5] = fmaf(v, x1.y, acc[5]);
              acc[6] = fmaf(v, x1.z, acc[6]);
              acc[7] = fmaf(v, x1.w, acc[7]);
              acc[8] = fmaf(v, x2.x, acc[8]);
              acc[9] = fmaf(v, x2.y, acc[9]);
              acc[10] = fmaf(v, x2.z, acc[10]);
              acc[11] = fmaf(v, x2.w, acc[11]);
              acc[12] = fmaf(v, x3.x, acc[12]);
              acc[13] = fmaf(v, x3.y, acc[13]);
              acc[14] = fmaf(v, x3.z, acc[14]);
              acc[15] = fmaf(v, x3.w, acc[15]);
            }
          }
        }
        // the P row phases of a column (lanes whose slot differs in the bits above lcp)
        for (int o = cp * NQ; o < 32; o <<= 1) {
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[e] += __shfl_xor_sync(kFull, acc[e], o);
        }
        if (on && p == 0) {
          const int j = cj[c0 + cl];
          if (sg.x.nchunks == 1) {
            const float f = __ldg(L.fac32 + sg.tidx + j);
            float4 *dst = reinterpret_cast<float4 *>(jb.tw + (size_t(sg.tidx) + j) * R + 16 * q);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              dst[e] = make_float4(acc[4 * e] * f, acc[4 * e + 1] * f, acc[4 * e + 2] * f, acc[4 * e + 3] * f);
          } else {
            double *dst = jb.part + (size_t(sg.x.pbase) + size_t(j) * sg.x.nchunks + sg.x.chunk) * R + 16 * q;
#pragma unroll
            for (int e = 0; e < 16; ++e) dst[e] = double(acc[e]);
          }
        }
      }
      __syncwarp();  // clane / cj are rewritten for the next segment
    }
    release_slot(&empty[s]);
  }
  return true;
}

// ---------------------------------------------------------------------------------------------
// Multi-RHS pass, phase 2 on the tensor cores: per warp and piece, Y|leaf (rows x R) +=
// W~(rows x 32 slices) T(32 slices x R) as mma.sync m16n8k8 TF32 products. Every lane decodes
// its slice (its bank column) 16 rows at a time into a padded shared-memory tile, from which the
// A fragments are read; the R multipliers of the 32 slices form the B fragments of the R / 8
// column tiles (three TF32 part products per step, mma3_add). Each step's products (8 slices) are
// added with FP32 rounding to the leaf's sums in registers; at the end of the leaf the warps'
// sums are added in FP64, in fixed order, into Y.
// ---------------------------------------------------------------------------------------------
template <int R>
__device__ bool consume_phase2_multi_mma(const Job &jb, uint32_t np, uint32_t &it, uint8_t *smem, uint64_t *full,
                                         uint64_t *empty, float *tiles) {
  const DevLayout &L = jb.L;
  constexpr size_t slot = slot_bytes<FMT_AFL32, 1, R>();
  constexpr int kTS = 36;  // tile row stride (floats): conflict-free stores by lane and fragment loads
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int g = lane >> 2, tq = lane & 3;  // mma fragment coordinates
  const float4 *xp4 = reinterpret_cast<const float4 *>(jb.xp);
  const float4 *tw4 = reinterpret_cast<const float4 *>(jb.tw);
  float *tile = tiles + warp * (16 * kTS + 2 * 32 * R);
  uint32_t *mhi = reinterpret_cast<uint32_t *>(tile + 16 * kTS);  // [32 slices][R] TF32 hi parts (swizzled)
  uint32_t *mlo = mhi + 32 * R;                                    // [32 slices][R] TF32 lo parts
  const int swz = kSwz<R>(tq);  // this lane's B rows are 8 kg + tq and 8 kg + tq + 4
  float *red = tiles;  // [kCWarps][64 rows][R + 8] leaf sums, over the tiles once every warp is done
  float c[4][R / 8][4];  // per 16-row tile and 8-column tile: C fragment (rows g, g + 8; columns 2 tq, 2 tq + 1)
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < R / 8; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) c[a][b][e] = 0.f;
  for (uint32_t i = 0; i < np; ++i, ++it) {
    const uint32_t s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1)) {
      atomicOr(L.status, 1u);
      return false;
    }
    const uint8_t *sl = smem + size_t(s) * slot;
    const uint32_t *Wd = reinterpret_cast<const uint32_t *>(sl);
    const PieceHdr *ph = reinterpret_cast<const PieceHdr *>(sl);
    const Seg *segs = reinterpret_cast<const Seg *>(sl + 16);
    const int nr = ph->nr;
    const uint32_t flags = ph->flags;
    const uint32_t row0 = ph->row0;
    if (flags & PF_START_LEAF) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < R / 8; ++b)
#pragma unroll
          for (int e = 0; e < 4; ++e) c[a][b][e] = 0.f;
    }
    // the lane's slice and its R multipliers (zero for idle lanes), split once into the TF32
    // parts the B fragments take
    LaneHdr hd{0xff, 0, 0, 0};
    const uint32_t *col = Wd;
    bool active = false;
    const Seg *sgp = nullptr;
    if (t < int(ph->ncols)) {
      const LaneHdr h = lane_hdrs(sl, ph)[t];
      if (h.seg != 0xff) {
        sgp = &segs[h.seg];
        hd = h;
        col = Wd + bc_column(ph, t);
        active = true;
      }
    }
    {
      const int rs = kSwz<R>(lane);  // this lane writes row `lane` of the multipliers
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        float4 mv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active) {
          if (sgp->kind == SEG_DENSE) {
            const float mm = float(sgp->m_min);
            const float4 xv = __ldg(xp4 + (size_t(sgp->gx) + hd.j) * (R / 4) + q);
            mv = make_float4(xv.x * mm, xv.y * mm, xv.z * mm, xv.w * mm);
          } else {
            mv = __ldg(tw4 + (size_t(sgp->gx) + hd.j) * (R / 4) + q);
          }
        }
        uint4 hi, lo;
        tf32_split(mv.x, hi.x, lo.x);
        tf32_split(mv.y, hi.y, lo.y);
        tf32_split(mv.z, hi.z, lo.z);
        tf32_split(mv.w, hi.w, lo.w);
        const int cidx = lane * R + ((4 * q) ^ rs);
        *reinterpret_cast<uint4 *>(mhi + cidx) = hi;
        *reinterpret_cast<uint4 *>(mlo + cidx) = lo;
      }
    }
    const ColDec cd = lane_dec(hd);
    const bool fast = __all_sync(kFull, !active || cd.fast32);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {  // 16-row tiles of the leaf
      if (16 * mt >= nr) break;
      // this lane's slice, rows 16 mt .. + 15 (rows past the leaf and idle lanes give 0)
      if (fast) {
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const int r = 16 * mt + rr;
          const bool ok = active && r < nr;
          const float v = dec_f32(bc_code32(col, uint32_t(ok ? r : 0) * cd.w), cd);
          tile[rr * kTS + lane] = ok ? v : 0.f;
        }
      } else {  // codes wider than the FP32 fast path: rare, kept out of line of the unrolled loop
#pragma unroll 1
        for (int rr = 0; rr < 16; ++rr) {
          const int r = 16 * mt + rr;
          const bool ok = active && r < nr;
          const float v = float(dec_any64(bc_code64(col, uint32_t(ok ? r : 0) * cd.w), cd, VF_AFL));
          tile[rr * kTS + lane] = ok ? v : 0.f;
        }
      }
      __syncwarp();
#pragma unroll 1
      for (int kg = 0; kg < 4; ++kg) {  // slices 8 kg .. 8 kg + 7 (a loop, to keep the code small)
        const float av[4] = {tile[g * kTS + 8 * kg + tq], tile[(g + 8) * kTS + 8 * kg + tq],
                             tile[g * kTS + 8 * kg + tq + 4], tile[(g + 8) * kTS + 8 * kg + tq + 4]};
        uint32_t ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ah[q] = tf32_of(av[q]);
          al[q] = tf32_of(av[q] - __uint_as_float(ah[q]));
        }
#pragma unroll
        for (int nt = 0; nt < R / 8; ++nt) {
          // B[k][n] = multiplier n of slice 8 kg + k, columns 8 nt .. 8 nt + 7
          const int i0 = (8 * kg + tq) * R + ((8 * nt + g) ^ swz), i1 = i0 + 4 * R;
          mma3_add(c[mt][nt], ah, al, mhi[i0], mhi[i1], mlo[i0], mlo[i1]);
        }
      }
      __syncwarp();  // the tile is rewritten for the next rows
    }
    release_slot(&empty[s]);  // the slot is not read after this point
    if (flags & PF_END_LEAF) {
      bar_consumers();  // every warp is past its tile reads
      float *wr = red + warp * (64 * (R + 8));
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < R / 8; ++nt) {
          *reinterpret_cast<float2 *>(wr + (16 * mt + g) * (R + 8) + 8 * nt + 2 * tq) = make_float2(c[mt][nt][0], c[mt][nt][1]);
          *reinterpret_cast<float2 *>(wr + (16 * mt + g + 8) * (R + 8) + 8 * nt + 2 * tq) =
              make_float2(c[mt][nt][2], c[mt][nt][3]);
        }
      bar_consumers();
      for (int idx = t; idx < nr * jb.nrhs; idx += kConsumers) {
        const int row = idx / jb.nrhs, q = idx - row * jb.nrhs;
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < kCWarps; ++w) sum += double(red[(w * 64 + row) * (R + 8) + q]);
        double *yp = jb.y + size_t(q) * size_t(jb.ldy) + __ldg(L.perm + row0 + uint32_t(row));
        *yp += sum;  // the only update of this entry (its leaf has one owner CTA)
      }
      bar_consumers();
    }
  }
  return true;
}

// resident CTAs per SM the product kernels are compiled for: the FP64-accumulation kernels keep
// 64 FP64 row sums per thread in phase 2
template <int FMT, int R>
constexpr int kMinBlocks = FMT == FMT_AFL64 ? 2 : R > kRN ? 3 : 4;

template <int FMT, int PH, int R, int NB>
__global__ void __launch_bounds__(kThreads, (kMinBlocks<FMT, R>)) k_product(const __grid_constant__ Jobs<NB> J) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr size_t slot = slot_bytes<FMT, PH, R>();
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + size_t(kStages) * slot);
  uint64_t *empty = full + kStages;
  double *red = reinterpret_cast<double *>(empty + kStages);
  using A = typename Tr<FMT>::A;
  A *tiles = reinterpret_cast<A *>(red + 2 * kCWarps * 64);
  uint32_t np_all = 0;
  for (int m = 0; m < J.n; ++m)
    for (int q = blockIdx.x; q < J.j[m].L.ph[PH].nct; q += gridDim.x) np_all += __ldg(J.j[m].L.ph[PH].cta_np + q);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kCWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (np_all == 0) return;
  if (threadIdx.x >= kConsumers) {
    producer<FMT, PH, R, NB>(J, smem, full, empty);
    return;
  }
  uint32_t it = 0, parity = 0;
  for (int m = 0; m < J.n; ++m)
  for (int q = blockIdx.x; q < J.j[m].L.ph[PH].nct; q += gridDim.x) {
    const Job &jb = J.j[m];
    const uint32_t np = __ldg(jb.L.ph[PH].cta_np + q);
    bool ok;
    if constexpr (R > 1) {
      if constexpr (PH == 0)
        if constexpr (R > kRN)
          ok = consume_phase1_multi<R>(jb, np, it, smem, full, empty, reinterpret_cast<float *>(red));
        else
          ok = consume_phase1_multi_fma<R>(jb, np, it, smem, full, empty);
      else
        ok = consume_phase2_multi_mma<R>(jb, np, it, smem, full, empty, reinterpret_cast<float *>(red));
    } else if constexpr (PH == 0 && FMT == FMT_AFL32) {
      ok = consume_phase1_pairs(jb.L, np, it, smem, full, empty);
    } else if constexpr (PH == 0 && FMT == FMT_AFL64) {
      ok = jb.L.vfmt == VF_AFL ? consume_phase1_f64(jb.L, np, it, smem, full, empty)
                               : consume_phase1<FMT>(jb.L, np, it, smem, full, empty);
    } else if constexpr (PH == 0) {
      ok = consume_phase1<FMT>(jb.L, np, it, smem, full, empty);
    } else if constexpr (FMT == FMT_AFL32) {
      ok = consume_phase2_pairs(jb.L, np, it, smem, full, empty, red, parity);
    } else if constexpr (kFP32<FMT>) {
      ok = consume_phase2_reg<FMT>(jb.L, np, it, smem, full, empty, red, jb.y, parity);
    } else if constexpr (FMT == FMT_AFL64) {
      ok = jb.L.vfmt == VF_AFL ? consume_phase2_f64(jb.L, np, it, smem, full, empty, red, parity)
                               : consume_phase2<FMT>(jb.L, np, it, smem, full, empty, red, tiles, jb.y, parity);
    } else {
      ok = consume_phase2_rows<FMT>(jb.L, np, it, smem, full, empty, red, jb.y, parity);
    }
    if (!ok) return;
  }
}

// ---------------------------------------------------------------------------------------------
// Bit-exact decoding (test path): a = (v - 1) * m_min in IEEE FP64, no contraction.
// ---------------------------------------------------------------------------------------------
__device__ double decode_code_exact(uint64_t code, int e, int m, double m_min) {
  const int w = 1 + e + m;
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
  const int w = 1 + e + m;
  const uint64_t nwords = (uint64_t(n) * uint64_t(w) + 31) / 32;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
    const uint64_t bit = uint64_t(j) * uint64_t(w);
    const uint64_t q = bit >> 5;
    const int sh = int(bit & 31);
    const int need = (sh + w + 31) >> 5;  // words touched: 1..3
    uint64_t lo = words[q], hi = 0;
    if (need >= 2 && q + 1 < nwords) lo |= uint64_t(words[q + 1]) << 32;
    if (need >= 3 && q + 2 < nwords) hi = words[q + 2];
    uint64_t code = lo >> sh;
    if (sh) code |= hi << (64 - sh);
    out[j] = decode_code_exact(code, e, m, m_min);
  }
}

// exact FP64 value of a code in value format vf (the decode of Section 3.2 for AFL, the FP32 /
// FP64 pattern for BFL / DFL)
__device__ double decode_exact_vf(uint64_t code, int e, int m, double m_min, int vf) {
  const int w = 1 + e + m;
  if (w < 64) code &= (1ull << w) - 1ull;
  if (vf == VF_BFL) return double(__uint_as_float(uint32_t(code << (23 - m))));
  if (vf == VF_DFL) return __longlong_as_double(static_cast<long long>(code << (52 - m)));
  if (vf == VF_MP) {
    if (e == 5) return double(__half2float(__ushort_as_half(static_cast<unsigned short>(code))));
    if (e == 8) return double(__uint_as_float(uint32_t(code)));
    return __longlong_as_double(static_cast<long long>(code));
  }
  return decode_code_exact(code, e, m, m_min);
}

__global__ void k_decode_slices(const uint8_t *base, const uint64_t *src, const uint64_t *dst, const uint32_t *nv,
                                const uint32_t *unit, const double *mmin, const uint8_t *ue, const uint8_t *um,
                                int64_t nslices, int raw, int vf, double *out) {
  for (int64_t s = blockIdx.x; s < nslices; s += gridDim.x) {
    const uint32_t u = unit[s];
    const int e = ue[u], m = um[u];
    const int w = raw ? 64 : 1 + e + m;
    const uint64_t s0 = src[s];
    const bool strided = (s0 & kStridedSlice) != 0;  // a lane column: word k at 32 k
    const uint64_t b0 = s0 & (kStridedSlice - 1);
    const uint32_t cnt = nv[s] & 0xffffffu, step = max(1u, nv[s] >> 24);  // values, their stride in the unit
    for (uint32_t v = threadIdx.x; v < cnt; v += blockDim.x) {
      if (raw) {
        const uint64_t bit = b0 + uint64_t(v) * uint64_t(w);
        out[dst[s] + v] = *reinterpret_cast<const double *>(base + bit / 8);
      } else if (strided) {
        const uint32_t *col = reinterpret_cast<const uint32_t *>(base) + (b0 >> 5);
        const uint64_t bit = uint64_t(v) * uint64_t(w);
        const uint64_t q = bit >> 5;
        const uint32_t sh = uint32_t(bit & 31);
        const uint32_t a = col[32 * q], b = col[32 * q + 32], c = col[32 * q + 64];
        const uint64_t code = (uint64_t(__funnelshift_r(b, c, sh)) << 32) | __funnelshift_r(a, b, sh);
        out[dst[s] + uint64_t(v) * step] = decode_exact_vf(code, e, m, mmin[u], vf);
      } else {
        const uint64_t bit = b0 + uint64_t(v) * uint64_t(w);
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(base) + (bit >> 5);
        const uint32_t sh = uint32_t(bit & 31);
        const uint64_t code = (uint64_t(__funnelshift_r(wp[1], wp[2], sh)) << 32) | __funnelshift_r(wp[0], wp[1], sh);
        out[dst[s] + v] = decode_exact_vf(code, e, m, mmin[u], vf);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------------
namespace {

struct DevProps {
  int sms = 0;
  int occ[2] = {0, 0};    // resident CTAs per SM of the phase-1 / phase-2 kernels (FP32 path)
  int occ64[2] = {0, 0};  // the same for the FP64-accumulation kernels
  int occN[2] = {0, 0};   // the same for the narrow multi-RHS pass kernels (R = kRN)
  int occR[2] = {0, 0};   // the same for the wide multi-RHS pass kernels (R = kRB)
};
std::mutex g_props_mu;
DevProps g_props[64];

template <int FMT, int PH, int R, int NB>
void set_smem_attr() {
  cudaFuncSetAttribute(k_product<FMT, PH, R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(smem_bytes<FMT, PH, R>()));
}
template <int NB>
void set_smem_attrs() {
  set_smem_attr<FMT_AFL32, 0, 1, NB>();
  set_smem_attr<FMT_AFL32, 1, 1, NB>();
  set_smem_attr<FMT_AFL64, 0, 1, NB>();
  set_smem_attr<FMT_AFL64, 1, 1, NB>();
  set_smem_attr<FMT_RAW64, 0, 1, NB>();
  set_smem_attr<FMT_RAW64, 1, 1, NB>();
  set_smem_attr<FMT_AFL32, 0, kRN, NB>();
  set_smem_attr<FMT_AFL32, 1, kRN, NB>();
  set_smem_attr<FMT_AFL32, 0, kRB, NB>();
  set_smem_attr<FMT_AFL32, 1, kRB, NB>();
  set_smem_attr<FMT_BFL32, 0, 1, NB>();
  set_smem_attr<FMT_BFL32, 1, 1, NB>();
  set_smem_attr<FMT_DFL32, 0, 1, NB>();
  set_smem_attr<FMT_DFL32, 1, 1, NB>();
  set_smem_attr<FMT_MP32, 0, 1, NB>();
  set_smem_attr<FMT_MP32, 1, 1, NB>();
}

const DevProps &props(int dev) {
  std::lock_guard<std::mutex> lk(g_props_mu);
  DevProps &P = g_props[dev & 63];
  if (P.sms == 0) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceGetAttribute(&P.sms, cudaDevAttrMultiProcessorCount, dev);
    set_smem_attrs<1>();
    set_smem_attrs<kMaxBatch>();
    int o0 = 0, o1 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_product<FMT_AFL32, 0, 1, 1>, kThreads,
                                                  smem_bytes<FMT_AFL32, 0>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_product<FMT_AFL32, 1, 1, 1>, kThreads,
                                                  smem_bytes<FMT_AFL32, 1>());
    P.occ[0] = o0 < 1 ? 1 : o0;
    P.occ[1] = o1 < 1 ? 1 : o1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_product<FMT_AFL64, 0, 1, 1>, kThreads,
                                                  smem_bytes<FMT_AFL64, 0>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_product<FMT_AFL64, 1, 1, 1>, kThreads,
                                                  smem_bytes<FMT_AFL64, 1>());
    P.occ64[0] = o0 < 1 ? 1 : o0;
    P.occ64[1] = o1 < 1 ? 1 : o1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_product<FMT_AFL32, 0, kRB, 1>, kThreads,
                                                  smem_bytes<FMT_AFL32, 0, kRB>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_product<FMT_AFL32, 1, kRB, 1>, kThreads,
                                                  smem_bytes<FMT_AFL32, 1, kRB>());
    P.occR[0] = o0 < 1 ? 1 : o0;
    P.occR[1] = o1 < 1 ? 1 : o1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_product<FMT_AFL32, 0, kRN, 1>, kThreads,
                                                  smem_bytes<FMT_AFL32, 0, kRN>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_product<FMT_AFL32, 1, kRN, 1>, kThreads,
                                                  smem_bytes<FMT_AFL32, 1, kRN>());
    P.occN[0] = o0 < 1 ? 1 : o0;
    P.occN[1] = o1 < 1 ? 1 : o1;
    if (cur != dev) cudaSetDevice(cur);
  }
  return P;
}

int cuda_status(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return HLR_OK;
}

// Launch the kernels of the products in J (all of one device, so all share the persistent grid
// sizes): permute, phase 1, combine of split blocks, phase 2 and, for the single-RHS AFL FP32
// product, the scatter of the row totals into y. ev (optional): kProfileEv events.
template <int FMT, int R, int NB>
void launch_jobs(const Jobs<NB> &J, cudaStream_t st, cudaEvent_t *ev, int share = 0) {
  if (J.n <= 0) return;
  int64_t nmax = 0, ncnt = 0;
  uint32_t np0 = 0, np1 = 0;
  for (int m = 0; m < J.n; ++m) {
    const DevLayout &L = J.j[m].L;
    nmax = std::max<int64_t>(nmax, L.n);
    ncnt = std::max<int64_t>(ncnt, L.ncnt);
    np0 += uint32_t(L.ph[0].np);
    np1 += uint32_t(L.ph[1].np);
  }
  // share (1..7): about share/8 of the CTA slots of the persistent kernels, each CTA walking the
  // work lists of several slots, so that concurrent work keeps the rest of every SM
  auto cap = [share](int nct) { return share > 0 && share < 8 ? std::max(1, (nct * share + 7) / 8) : nct; };
  int nct0 = cap(J.j[0].L.ph[0].nct), nct1 = cap(J.j[0].L.ph[1].nct);
  if constexpr (FMT == FMT_AFL64 || R > 1) {
    // fewer of these are resident than there are work lists (made for the single-RHS FP32
    // kernels): one wave of CTAs, each walking several work lists
    int dev = 0;
    cudaGetDevice(&dev);
    const DevProps &P = props(dev);
    const int *occ = R > kRN ? P.occR : R > 1 ? P.occN : P.occ64;
    nct0 = std::min(nct0, P.sms * occ[0]);
    nct1 = std::min(nct1, P.sms * occ[1]);
  }
  const dim3 gp(unsigned(std::min<int64_t>((nmax + 255) / 256, 4096)), unsigned(J.n));
  if (ev) cudaEventRecord(ev[0], st);
  if constexpr (R == 1)
    k_permute<NB><<<gp, 256, 0, st>>>(J);
  else
    k_permute_multi<R, NB><<<gp, 256, 0, st>>>(J);
  if (ev) cudaEventRecord(ev[1], st);
  if (np0 > 0) k_product<FMT, 0, R, NB><<<nct0, kThreads, smem_bytes<FMT, 0, R>(), st>>>(J);
  if (ncnt > 0) {
    const dim3 gc(unsigned(std::min<int64_t>((ncnt * R + 255) / 256, 1024)), unsigned(J.n));
    k_combine<FMT, R, NB><<<gc, 256, 0, st>>>(J);
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (np1 > 0) k_product<FMT, 1, R, NB><<<nct1, kThreads, smem_bytes<FMT, 1, R>(), st>>>(J);
  if (ev) cudaEventRecord(ev[3], st);
  if constexpr ((FMT == FMT_AFL32 || FMT == FMT_AFL64) && R == 1)
    if (np1 > 0) k_scatter<NB><<<gp, 256, 0, st>>>(J);
  if (ev) cudaEventRecord(ev[4], st);
}

// Events of the next profiled product (nullptr if not profiling or the ring is full).
cudaEvent_t *profile_slot(Handle &H, int flags) {
  if (!(flags & HLR_PROFILE)) return nullptr;
  if (H.prof_ev.empty()) {
    H.prof_ev.resize(kProfileEv * size_t(kProfileCap), nullptr);
    for (auto &e : H.prof_ev) {
      cudaEvent_t ev;
      cudaEventCreate(&ev);
      e = ev;
    }
  }
  if (H.prof_n >= kProfileCap) return nullptr;
  return reinterpret_cast<cudaEvent_t *>(&H.prof_ev[kProfileEv * size_t(H.prof_n++)]);
}

Job single_job(const Handle &H, const double *x, double *y) {
  Job j{};
  j.L = H.L;
  j.x = x;
  j.y = y;
  j.nrhs = 1;
  return j;
}

}  // namespace

int ctas_per_phase(int device, int nct[2]) {
  const DevProps &P = props(device);
  if (P.sms <= 0) return 0;
  nct[0] = P.sms * P.occ[0];
  nct[1] = P.sms * P.occ[1];
  return nct[1];
}

int launch_matvec(Handle &H, const double *x, double *y, int flags, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  props(H.device);
  cudaEvent_t *ev = profile_slot(H, flags);
  const int acc = flags & 0xff;
  const int share = (flags >> 16) & 15;
  Jobs<1> J{};
  J.n = 1;
  J.j[0] = single_job(H, x, y);
  if (H.L.raw)
    launch_jobs<FMT_RAW64, 1, 1>(J, st, ev, share);
  else if (acc != HLR_ACC_FP32)
    launch_jobs<FMT_AFL64, 1, 1>(J, st, ev, share);  // FP64 decode of every value format
  else if (H.L.vfmt == VF_BFL)
    launch_jobs<FMT_BFL32, 1, 1>(J, st, ev, share);
  else if (H.L.vfmt == VF_DFL)
    launch_jobs<FMT_DFL32, 1, 1>(J, st, ev, share);
  else if (H.L.vfmt == VF_MP)
    launch_jobs<FMT_MP32, 1, 1>(J, st, ev, share);
  else
    launch_jobs<FMT_AFL32, 1, 1>(J, st, ev, share);
  return cuda_status("hlr_matvec: launch");
}

// Scratch of multi-RHS passes: `passes` sets of (X_perm, t m_min(W), partial sums) per handle,
// allocated on first use and grown when a request needs more passes.
static int multi_scratch(Handle &H, int passes, float **xp, float **tw, double **part, size_t *stride) {
  const size_t n = size_t(H.L.n), rs = size_t(H.info.rank_sum);
  const size_t b_xp = (((n + 8) * kRB * 4) + 255) & ~size_t(255);
  const size_t b_tw = (((rs + 8) * kRB * 4) + 255) & ~size_t(255);
  const size_t b_pt = (((size_t(H.part_total) + 1) * kRB * 8) + 255) & ~size_t(255);
  const size_t per = b_xp + b_tw + b_pt;
  if (H.multi_passes < passes) {
    if (H.multi_ws) {
      cudaFree(H.multi_ws);
      H.multi_ws = nullptr;
      H.multi_passes = 0;
    }
    if (cudaMalloc(&H.multi_ws, per * size_t(passes)) != cudaSuccess) {
      cudaGetLastError();
      H.multi_ws = nullptr;
      return set_error(HLR_ERR_OOM, "hlr_matvec_batched: multi-RHS scratch allocation failed");
    }
    H.multi_passes = passes;
  }
  uint8_t *b = static_cast<uint8_t *>(H.multi_ws);
  *xp = reinterpret_cast<float *>(b);
  *tw = reinterpret_cast<float *>(b + b_xp);
  *part = reinterpret_cast<double *>(b + b_xp + b_tw);
  *stride = per;
  return HLR_OK;
}

// Single-RHS scratch sets of HLR_MULTI columns: set k of a handle holds what the arena's scratch
// holds for hlr_matvec (x_perm FP64/FP32, t m_min(W) FP64/FP32, chunk partial sums, row totals),
// so that columns of one call, and concurrent hlr_matvec / hlr_solve_cg calls on the handle, never
// share scratch. Sets are allocated one by one when a call needs more and are kept until
// hlr_free (no cudaFree, which would wait for the whole device, while the handle is in use).
static int column_scratch(Handle &H, int sets) {
  const size_t n = size_t(H.L.n), rs = size_t(H.info.rank_sum);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t bytes = al(8 * (n + 8)) + al(4 * (n + 8)) + al(8 * (rs + 8)) + al(4 * (rs + 8)) +
                       al(8 * size_t(H.part_total) + 8) + al(8 * (n + 8));
  while (int(H.col_ws.size()) < sets) {
    void *w = nullptr;
    if (cudaMalloc(&w, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(HLR_ERR_OOM, "hlr_matvec_batched: column scratch allocation failed");
    }
    H.col_ws.push_back(w);
  }
  return HLR_OK;
}
static DevLayout column_layout(const Handle &H, int k) {
  const size_t n = size_t(H.L.n), rs = size_t(H.info.rank_sum);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  uint8_t *b = static_cast<uint8_t *>(H.col_ws[size_t(k)]);
  DevLayout L = H.L;
  L.xperm64 = reinterpret_cast<double *>(b);
  b += al(8 * (n + 8));
  L.xperm32 = reinterpret_cast<float *>(b);
  b += al(4 * (n + 8));
  L.tw64 = reinterpret_cast<double *>(b);
  b += al(8 * (rs + 8));
  L.tw32 = reinterpret_cast<float *>(b);
  b += al(4 * (rs + 8));
  L.partial = reinterpret_cast<double *>(b);
  b += al(8 * size_t(H.part_total) + 8);
  L.ysum = reinterpret_cast<double *>(b);
  return L;
}

namespace {
// Accumulates the products of one kernel class and launches them in groups of <= kMaxBatch.
// Two products of one group must not share scratch: the same handle appears at most once among
// the single-RHS products of a group and each (handle, pass) at most once among the passes.
template <int FMT, int R>
struct Batcher {
  Jobs<kMaxBatch> J{};
  std::vector<std::pair<const Handle *, int>> keys;
  cudaStream_t st;
  int share;
  explicit Batcher(cudaStream_t s, int sh) : st(s), share(sh) { J.n = 0; }
  void flush() {
    if (J.n > 0) launch_jobs<FMT, R, kMaxBatch>(J, st, nullptr, share);
    J.n = 0;
    keys.clear();
  }
  void add(const Handle *H, int pass, const Job &jb) {
    const auto key = std::make_pair(H, pass);
    bool clash = J.n >= kMaxBatch;
    for (const auto &k : keys) clash = clash || k == key;
    if (clash) flush();
    J.j[J.n++] = jb;
    keys.push_back(key);
  }
};
}  // namespace

int launch_batch(int nreq, Handle *const *H, const int32_t *nrhs, const double *const *X, const int64_t *ldx,
                 double *const *Y, const int64_t *ldy, int flags, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (nreq <= 0) return HLR_OK;
  const int dev = H[0]->device;
  for (int q = 0; q < nreq; ++q)
    if (H[q]->device != dev) return set_error(HLR_ERR_INVALID, "hlr_matvec_batched: handles of different devices");
  props(dev);
  const bool fp32 = (flags & 0xff) == HLR_ACC_FP32;
  const bool percol = (flags & HLR_MULTI) != 0;  // every column a single-RHS product of its own
  const int multi_from = percol ? (1 << 30) : 2;  // fewest columns that take the multi-RHS passes
  const int share = (flags >> 16) & 15;
  Batcher<FMT_AFL32, 1> b32(st, share);
  Batcher<FMT_BFL32, 1> bbfl(st, share);
  Batcher<FMT_DFL32, 1> bdfl(st, share);
  Batcher<FMT_MP32, 1> bmp(st, share);
  Batcher<FMT_AFL64, 1> b64(st, share);
  Batcher<FMT_RAW64, 1> braw(st, share);
  // multi-column passes decode the AFL family only; a pass of at most kRN columns takes the
  // narrow kernels (a column's arithmetic is the same in both, so are its bits)
  Batcher<FMT_AFL32, kRN> bmn(st, share);
  Batcher<FMT_AFL32, kRB> bm(st, share);
  // pass scratch first (growing it frees the old one, which no pending product may still use)
  for (int q = 0; q < nreq; ++q) {
    if (nrhs[q] < multi_from || !fp32 || H[q]->L.raw || H[q]->L.vfmt != VF_AFL) continue;
    int passes = 0;
    for (int k = 0; k < nreq; ++k)
      if (H[k] == H[q] && nrhs[k] >= multi_from) passes = std::max(passes, (nrhs[k] + kRB - 1) / kRB);
    float *xp, *tw;
    double *part;
    size_t stride;
    if (int rc = multi_scratch(*H[q], passes, &xp, &tw, &part, &stride)) return rc;
  }
  // HLR_MULTI: column scratch sets, numbered per handle over the whole call
  std::vector<std::pair<const Handle *, int>> colbase;  // handle -> sets taken so far
  if (percol)
    for (int q = 0; q < nreq; ++q) {
      if (nrhs[q] <= 0) continue;
      int need = 0;
      for (int k = 0; k < nreq; ++k)
        if (H[k] == H[q] && nrhs[k] > 0) need += nrhs[k];
      if (int rc = column_scratch(*H[q], need)) return rc;
    }
  auto take_sets = [&](const Handle *h, int cnt) {
    for (auto &cb : colbase)
      if (cb.first == h) {
        const int k = cb.second;
        cb.second += cnt;
        return k;
      }
    colbase.push_back({h, cnt});
    return 0;
  };
  for (int q = 0; q < nreq; ++q) {
    Handle &Hq = *H[q];
    const int r = nrhs[q];
    if (r <= 0) continue;
    if (percol) {
      // one product per column, each on its own scratch set: the kernels and arithmetic of
      // hlr_matvec, so a column's bits are those of hlr_matvec of that column
      const int k0 = take_sets(&Hq, r);
      for (int c = 0; c < r; ++c) {
        Job jb = single_job(Hq, X[q] + size_t(c) * size_t(ldx[q]), Y[q] + size_t(c) * size_t(ldy[q]));
        jb.L = column_layout(Hq, k0 + c);
        if (Hq.L.raw)
          braw.add(&Hq, k0 + c, jb);
        else if (!fp32)
          b64.add(&Hq, k0 + c, jb);
        else if (Hq.L.vfmt == VF_BFL)
          bbfl.add(&Hq, k0 + c, jb);
        else if (Hq.L.vfmt == VF_DFL)
          bdfl.add(&Hq, k0 + c, jb);
        else if (Hq.L.vfmt == VF_MP)
          bmp.add(&Hq, k0 + c, jb);
        else
          b32.add(&Hq, k0 + c, jb);
      }
      continue;
    }
    if (r >= multi_from && fp32 && !Hq.L.raw && Hq.L.vfmt == VF_AFL) {
      const int passes = (r + kRB - 1) / kRB;
      float *xp, *tw;
      double *part;
      size_t stride;
      if (int rc = multi_scratch(Hq, passes, &xp, &tw, &part, &stride)) return rc;
      for (int p = 0; p < passes; ++p) {
        Job jb = single_job(Hq, X[q] + size_t(p) * kRB * size_t(ldx[q]), Y[q] + size_t(p) * kRB * size_t(ldy[q]));
        jb.ldx = ldx[q];
        jb.ldy = ldy[q];
        jb.nrhs = std::min(kRB, r - p * kRB);
        jb.xp = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(xp) + p * stride);
        jb.tw = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(tw) + p * stride);
        jb.part = reinterpret_cast<double *>(reinterpret_cast<uint8_t *>(part) + p * stride);
        if (jb.nrhs <= kRN)
          bmn.add(&Hq, p, jb);
        else
          bm.add(&Hq, p, jb);
      }
    } else {
      for (int c = 0; c < r; ++c) {
        const Job jb = single_job(Hq, X[q] + size_t(c) * size_t(ldx[q]), Y[q] + size_t(c) * size_t(ldy[q]));
        if (Hq.L.raw)
          braw.add(&Hq, -1, jb);
        else if (!fp32)
          b64.add(&Hq, -1, jb);
        else if (Hq.L.vfmt == VF_BFL)
          bbfl.add(&Hq, -1, jb);
        else if (Hq.L.vfmt == VF_DFL)
          bdfl.add(&Hq, -1, jb);
        else if (Hq.L.vfmt == VF_MP)
          bmp.add(&Hq, -1, jb);
        else
          b32.add(&Hq, -1, jb);
      }
    }
  }
  b32.flush();
  bbfl.flush();
  bdfl.flush();
  bmp.flush();
  b64.flush();
  braw.flush();
  bmn.flush();
  bm.flush();
  return cuda_status("hlr_matvec_batched: launch");
}

int profile_read(Handle &H, double *ms, int *calls) {
  for (int k = 0; k < kProfileEv - 1; ++k) ms[k] = 0.0;
  for (int i = 0; i < H.prof_n; ++i) {
    cudaEvent_t *ev = reinterpret_cast<cudaEvent_t *>(&H.prof_ev[kProfileEv * size_t(i)]);
    if (cudaEventSynchronize(ev[kProfileEv - 1]) != cudaSuccess) return cuda_status("hlr_profile_read");
    for (int k = 0; k < kProfileEv - 1; ++k) {
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
  const int64_t ns = int64_t(H.slice_src.size());
  const int64_t nu = H.nunits;
  if (ns == 0) return HLR_OK;
  const size_t bytes = ns * (8 + 8 + 4 + 4) + nu * (8 + 1 + 1) + 64;
  uint8_t *tmp = nullptr;
  if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_error(HLR_ERR_OOM, "hlr_decode_units: temporary allocation failed");
  }
  uint64_t *d_src = reinterpret_cast<uint64_t *>(tmp);
  uint64_t *d_dst = d_src + ns;
  double *d_mmin = reinterpret_cast<double *>(d_dst + ns);
  uint32_t *d_n = reinterpret_cast<uint32_t *>(d_mmin + nu);
  uint32_t *d_unit = d_n + ns;
  uint8_t *d_e = reinterpret_cast<uint8_t *>(d_unit + ns);
  uint8_t *d_m = d_e + nu;
  cudaMemcpyAsync(d_src, H.slice_src.data(), 8 * ns, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_dst, H.slice_dst.data(), 8 * ns, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_mmin, H.unit_mmin.data(), 8 * nu, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_n, H.slice_n.data(), 4 * ns, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_unit, H.slice_unit.data(), 4 * ns, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_e, H.unit_e.data(), nu, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_m, H.unit_m.data(), nu, cudaMemcpyHostToDevice, st);
  const int grid = int(std::min<int64_t>(ns, 65535));
  k_decode_slices<<<grid, 64, 0, st>>>(H.L.base, d_src, d_dst, d_n, d_unit, d_mmin, d_e, d_m, ns, H.L.raw, H.L.vfmt, out);
  int rc = cuda_status("hlr_decode_units");
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (rc == HLR_OK && e != cudaSuccess) rc = set_error(HLR_ERR_CUDA, std::string("hlr_decode_units: ") + cudaGetErrorString(e));
  return rc;
}

// ---------------------------------------------------------------------------------------------
// Unit decoding without any allocation (hlr_decode_units_static): the slice map is staged in a
// fixed array of this library instead of a temporary device allocation.
// ---------------------------------------------------------------------------------------------

// Every device on which the library's kernels are loaded holds these 4 MiB until the process
// exits. All calls share them, so two calls whose work overlaps on the GPU race.
constexpr size_t kStaticScratchBytes = size_t(4) << 20;
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_static_mu;
void *g_static_ptr[64] = {};

// Device address of g_static_scratch on `dev`, looked up once per device with that device current.
int static_scratch(int dev, uint8_t **p) {
  if (dev < 0 || dev >= 64) return set_error(HLR_ERR_UNSUPPORTED, "hlr_decode_units_static: device index above 63");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return cuda_status("hlr_decode_units_static: cudaGetDevice");
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return cuda_status("hlr_decode_units_static: cudaSetDevice");
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_static_scratch);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return set_error(HLR_ERR_CUDA, std::string("hlr_decode_units_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_static_ptr[dev] = ptr;
  }
  *p = static_cast<uint8_t *>(g_static_ptr[dev]);
  return HLR_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

int launch_decode_units_static(const Handle &H, double *out, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  const int64_t ns = int64_t(H.slice_src.size());
  const int64_t nu = H.nunits;
  // map layout in the scratch: src, dst [ns] u64 | m_min [nu] f64 | n, unit [ns] u32 | e, m [nu] u8
  const size_t o_dst = align256(8 * size_t(ns));
  const size_t o_mmin = o_dst + align256(8 * size_t(ns));
  const size_t o_n = o_mmin + align256(8 * size_t(nu));
  const size_t o_unit = o_n + align256(4 * size_t(ns));
  const size_t o_e = o_unit + align256(4 * size_t(ns));
  const size_t o_m = o_e + align256(size_t(nu));
  const size_t total = o_m + align256(size_t(nu));
  if (total > kStaticScratchBytes)
    return set_error(HLR_ERR_UNSUPPORTED, "hlr_decode_units_static: the slice map of this matrix needs " +
                                              std::to_string(total) + " bytes, more than the " +
                                              std::to_string(kStaticScratchBytes) +
                                              " bytes of static scratch (use hlr_decode_units)");
  uint8_t *base = nullptr;
  if (int rc = static_scratch(H.device, &base)) return rc;
  if (ns == 0) return HLR_OK;
  struct Cp {
    size_t off;
    const void *src;
    size_t bytes;
  } cps[] = {{0, H.slice_src.data(), 8 * size_t(ns)},        {o_dst, H.slice_dst.data(), 8 * size_t(ns)},
             {o_mmin, H.unit_mmin.data(), 8 * size_t(nu)},   {o_n, H.slice_n.data(), 4 * size_t(ns)},
             {o_unit, H.slice_unit.data(), 4 * size_t(ns)},  {o_e, H.unit_e.data(), size_t(nu)},
             {o_m, H.unit_m.data(), size_t(nu)}};
  for (const Cp &c : cps)
    if (c.bytes && cudaMemcpyAsync(base + c.off, c.src, c.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return cuda_status("hlr_decode_units_static: map copy");
  const int grid = int(std::min<int64_t>(ns, 65535));
  k_decode_slices<<<grid, 64, 0, st>>>(H.L.base, reinterpret_cast<const uint64_t *>(base),
                                       reinterpret_cast<const uint64_t *>(base + o_dst),
                                       reinterpret_cast<const uint32_t *>(base + o_n),
                                       reinterpret_cast<const uint32_t *>(base + o_unit),
                                       reinterpret_cast<const double *>(base + o_mmin), base + o_e, base + o_m, ns,
                                       H.L.raw, H.L.vfmt, out);
  return cuda_status("hlr_decode_units_static");
}

// Failure-detection self-test: thread 0 initialises an mbarrier on which nothing ever arrives
// and waits for its first phase with the product kernels' bounded wait, limited to `cycles`;
// when the wait gives up it records the failure in the status word as a product kernel does.
__global__ void k_wait_expire(uint32_t *status, long long cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait(&bar, 0, cycles)) atomicOr(status, 1u);
  }
}

int launch_wait_expire(const Handle &H, long long cycles, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  k_wait_expire<<<1, 32, 0, st>>>(H.L.status, cycles);
  return cuda_status("hlr_selftest_wait");
}

int launch_decode_stream(const uint8_t *stream, int64_t n, double m_min, int e, int m, double *out, void *stream_) {
  cudaStream_t st = static_cast<cudaStream_t>(stream_);
  cudaGetLastError();
  const int grid = int(std::min<int64_t>((n + 255) / 256, 4096));
  k_decode_stream<<<grid, 256, 0, st>>>(reinterpret_cast<const uint32_t *>(stream), n, m_min, e, m, out);
  return cuda_status("hlr_afl_decode_device");
}

}  // namespace hlr

extern "C" int hlr_decode_units_static(hlr_handle h, double *out, int64_t cap, void *stream) {
  using namespace hlr;
  Handle *H = lookup(h);
  if (!H || !out) return set_error(HLR_ERR_INVALID, "hlr_decode_units_static: unknown handle or null output");
  if (cap < H->values) return set_error(HLR_ERR_INVALID, "hlr_decode_units_static: output too small");
  if (H->values > 0 && H->slice_src.empty())
    return set_error(HLR_ERR_UNSUPPORTED, "hlr_decode_units_static: only for matrices of at most 2^26 values");
  return launch_decode_units_static(*H, out, stream);
}
