// Internal device layout of an uploaded H-matrix and host-side handle state.
// Shared by the host packer (hlr_upload.cpp) and the CUDA kernels (hlr_kernels.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hlr.h"

namespace hlr {

// One encoded data unit (a dense block, or one column of W or X). 16 bytes.
// Stream start = arena + 16 * (off_lo + 2^32 * off_hi). For HLR_FMT_FP64 the unit is plain
// FP64 values (w = 64, e = m = 0, m_min unused).
struct UnitHdr {
  double m_min;
  uint32_t off_lo;
  uint8_t e, m, w;
  uint8_t off_hi;
};
static_assert(sizeof(UnitHdr) == 16, "UnitHdr must be 16 bytes");

// Per lowrank block with rank > 0: offsets of its Sigma/t values and of its partial sums.
struct LRBlock {
  uint32_t tbase;    // sigma[tbase + i], t[tbase + i]
  uint32_t part0;    // partial[part0 + c * k + i] for chunk c
  uint16_t k;
  uint16_t nchunks;
  uint32_t xunit0;   // unit index of X column 0 (X column i = xunit0 + i)
};
static_assert(sizeof(LRBlock) == 16, "LRBlock must be 16 bytes");

// Phase-1 work item: rows [row0, row0 + nrows) of X of one lowrank block (nrows <= 256).
struct P1Item {
  uint32_t blk;      // index into LRBlock array
  uint32_t row0;     // first row of X (relative to the block's sigma cluster)
  uint32_t xoff;     // position of x|sigma[row0] in the permuted x
  uint16_t nrows;
  uint16_t chunk;    // chunk index c
};
static_assert(sizeof(P1Item) == 16, "P1Item must be 16 bytes");

// Phase-2 owner: a leaf row interval [row0, row0 + nrows), nrows <= 64, with the
// contributions [c0, c1) that cover it.
struct Leaf {
  uint32_t row0;
  uint32_t nrows;
  uint32_t c0, c1;
};
static_assert(sizeof(Leaf) == 16, "Leaf must be 16 bytes");

enum : uint32_t { CONTRIB_DENSE = 0, CONTRIB_LOWRANK = 1 };

// A block restricted to one leaf row interval.
//  dense  : unit = the block's unit; column j starts at value index j * ld + rowoff;
//           multiplier of column j = x_perm[mbase + j] * m_min.
//  lowrank: unit = W column 0 (column i = unit + i); value index rowoff + r;
//           multiplier of column i = t[mbase + i] * m_min_i.
struct Contrib {
  uint32_t unit;
  uint32_t ncols;
  uint32_t rowoff;
  uint32_t ld;
  uint32_t mbase;
  uint32_t kind;
  uint32_t colbase;  // running column count of the leaf before this contribution (for warp rotation)
  uint32_t pad;
};
static_assert(sizeof(Contrib) == 32, "Contrib must be 32 bytes");

// Device pointers into an arena (all set by the host after upload).
struct DevLayout {
  const uint8_t *base;       // arena base (unit streams are addressed from here)
  const UnitHdr *units;
  const double *sigma;       // [rank_sum]
  const LRBlock *lrb;        // [nlr]
  const P1Item *items;       // [nitems]
  const Leaf *leaves;        // [nleaves]
  const Contrib *contribs;   // [ncontribs]
  const int64_t *perm;       // [n]
  // scratch
  double *xperm64;           // [n * rhs_cap]
  float *xperm32;            // [n * rhs_cap]
  double *t;                 // [rank_sum * rhs_cap]
  double *partial;           // [part_total * rhs_cap]
  uint32_t *counters;        // [nlr] arrival counters + 4 work counters
  double *xdev;              // [n] device copy of a host x (hlr_matvec_host)
  double *ydev;              // [n] device copy of a host y (hlr_matvec_host)
  int64_t n;
  int32_t nlr, nitems, nleaves, format;
};

struct Handle {
  int device = 0;
  int format = HLR_FMT_AFL_APLR;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  DevLayout L{};
  hlr_info info{};
  int64_t ncontribs = 0;
  int64_t part_total = 0;
  int64_t nunits = 0;
  int64_t values = 0;
  std::vector<int64_t> unit_value_offset;  // host copy: start of unit u in the decode output
  std::vector<int64_t> unit_len;           // host copy: number of values of unit u
  std::vector<UnitHdr> unit_hdr;           // host copy of the headers
  size_t scratch_bytes = 0;                // bytes of the scratch region
  size_t scratch_off = 0;                  // offset of the scratch region in the arena
  void *cg_ws = nullptr;                   // CG work vectors (allocated on first solve)
  std::vector<void *> prof_ev;             // cudaEvent_t ring: 4 per profiled product
  int prof_n = 0;                          // profiled products since the last read
};
constexpr int kProfileCap = 4096;

// Error reporting (thread-local message).
int set_error(int code, const std::string &msg);
Handle *lookup(hlr_handle h);

// Kernel launchers (hlr_kernels.cu).
int launch_matvec(Handle &H, const double *x, double *y, int flags, void *stream);
int launch_decode_units(const Handle &H, double *out, void *stream);
int profile_read(Handle &H, double *ms, int *calls);
int launch_decode_stream(const uint8_t *stream, int64_t n, double m_min, int e, int m, double *out,
                         void *stream_);

// Host codec (hlr_codec.cpp).
int mantissa_bits(double u);
struct AflParams {
  double m_min;
  int e, m, w;
};
// Scan values: m_min, e, m for precision u. Returns false on non-finite input.
bool afl_params(const double *a, int64_t n, double u, AflParams *p);
// Pack the codes of a at params p into out (zeroed, >= padded size bytes).
void afl_pack(const double *a, int64_t n, const AflParams &p, uint8_t *out);
inline size_t padded16(size_t b) { return (b + 15) & ~size_t(15); }
inline size_t afl_bytes(int64_t n, int w) { return (size_t(n) * size_t(w) + 7) / 8; }

}  // namespace hlr
