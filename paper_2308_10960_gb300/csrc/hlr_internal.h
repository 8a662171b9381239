// Internal device layout of an uploaded H-matrix and host-side handle state.
// Shared by the host packer (hlr_upload.cpp, hlr_pack.cpp) and the CUDA kernels.
//
// Work-ordered layout. The compressed codes of every AFL unit are re-placed (not re-encoded)
// so that each CTA of a product kernel streams ONE contiguous byte range: a sequence of
// pieces (<= kPieceMax bytes, <= kMaxCols column slices) copied into shared memory by TMA bulk
// copies. A column slice is a run of consecutive values of one unit (a column of a dense
// block, of W or of X restricted to a task's rows); in the kernels every lane owns one slice of
// the current piece and decodes it sequentially.
//  phase 1 (t = Sigma X~^T x): task = item = rows [row0, row0+R) (R <= 256) of the X columns
//           of one lowrank block; a lane forms one column's dot product with x.
//  phase 2 (y += W~ t + D~ x): task = leaf = a row interval of <= 64 rows; its slices are the
//           columns of the dense blocks and of the W factors of the lowrank blocks covering it,
//           in block order; lanes combine their slices row by row.
// Segments group consecutive slices of one block inside a piece. The multipliers of a piece
// (x|sigma, t m_min(W), phase-1 column factors) are staged by extra TMA ("aux") copies into the
// same ring slot.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hlr.h"

namespace hlr {

constexpr int kPieceMax = 16384;  // bytes of one piece (header, segments, column headers, data)
constexpr int kMaxCols = 128;     // column slices per piece (one per consumer lane)
constexpr int kAuxMax1 = 1024;    // phase 1: staged elements per piece (x of the rows, factors)
constexpr int kAuxMax2 = 512;     // phase 2: staged multipliers per piece
constexpr int kAuxMax = kAuxMax1; // the larger of the two
constexpr int kStages = 2;        // ring slots per CTA
constexpr int kConsumers = 128;   // consumer threads (4 warps) per CTA, plus one producer warp
constexpr int kRowsPerItem = 256;
constexpr int kSubRows = 64;      // phase 1: rows of an X column read by one lane
constexpr int kLeafRows = 64;

enum : uint8_t { SEG_DENSE = 0, SEG_W = 1, SEG_X = 2 };
// value formats of the stored codes; VF_MP: IEEE FP16 / FP32 / FP64 patterns, the lane's e
// (5, 8, 11) telling which
enum { VF_AFL = 0, VF_BFL = 1, VF_DFL = 2, VF_MP = 3 };
enum : uint8_t { PF_START_LEAF = 1, PF_END_LEAF = 2 };

struct PieceHdr {
  uint16_t nseg;
  uint16_t ncols;    // column slices (lanes) in the piece (<= kMaxCols)
  uint16_t nr;       // phase 2: rows of the leaf
  uint8_t flags;     // PF_START_LEAF, PF_END_LEAF (phase 2)
  uint8_t pad0;
  uint32_t row0;     // phase 2: first row of the leaf (cluster order)
  uint8_t h[4];      // bank-column pieces: words per lane column in the region of warp 0..3
};
static_assert(sizeof(PieceHdr) == 16, "PieceHdr");

// One segment (32 bytes): slices [cstart, cstart + nc) of the piece, all of one block.
//  dense: nc columns x nr rows, codes column-major and contiguous at width w from word data_w;
//         multiplier of column j = aux[xs + j] * m_min.
//  W    : nc column slices of nr rows; slice i starts at word data_w + colhdr[i].wordoff;
//         multiplier = aux[xs + i] (t_i m_min(W_i), computed by phase 1).
//  X    : nc column slices of nr (= R) rows of one item; x of row r at aux[xs + r]; column
//         factor sigma_i m_min(X_i) m_min(W_i) at aux[fs + i]; result for t index tidx + i, or
//         for blocks of several chunks the partial sum partial[pbase + i nchunks + chunk]
//         (combined in chunk order by k_combine).
struct Seg {
  uint8_t kind;
  uint8_t lg;        // X: log2 of the lanes per column (a column of R rows uses 2^lg lanes)
  uint16_t nc;
  uint16_t cstart;   // first lane of the segment (aligned to 2^lg)
  uint16_t nr;
  uint16_t xs;
  uint16_t data_w;   // data start, 32-bit words from the piece start
  uint16_t col_w;    // W/X: column headers, words from the piece start; dense: e | m << 8
  uint16_t fs;       // X: aux offset of the first column factor
  uint32_t tidx;     // X: t index of the segment's first column
  uint32_t gx;       // global index of the first multiplier: x column (dense), t index (W),
                     // x row of row 0 of the item (X); read by the multi-RHS kernels
  union {
    double m_min;    // dense: m_min of the block's unit
    struct {
      uint32_t pbase;    // X: partial index of the first column's chunk 0
      uint16_t chunk;    // X: chunk index of the item
      uint16_t nchunks;  // X: chunks of the block
    } x;
  };
};
static_assert(sizeof(Seg) == 32, "Seg");

// Bank-column pieces (the AFL formats). After the segments come one LaneHdr per lane and then
// the data as four warp regions: region w is an array of h[w] rows of 32 words, and lane
// t = 32 w + l owns column l of it, so its k-th word is at region + 32 k + l. A warp's 32 lanes
// thus read 32 different shared-memory banks whatever their positions in their slices. Each
// lane column holds one slice from bit 0 (value r at bits [r w, r w + w)). Lanes are ordered by
// slice length (X: whole aligned groups of 2^lg lanes) so that the columns of a warp are about
// equally long. An X column of an item of nr rows is read by G = 2^lg lanes (the smallest G
// with 64 G >= nr), lane g of the group taking rows g, g + G, g + 2G, ... (value i of its
// column is row g + i G). The FP64 format keeps the contiguous layout (ColHdr below).
struct LaneHdr {
  uint8_t seg;       // segment of the lane's slice (0xff: idle lane)
  uint8_t j;         // column of the slice within its segment
  uint8_t e, m;      // AFL parameters of the slice's unit
};
static_assert(sizeof(LaneHdr) == 4, "LaneHdr");
constexpr uint64_t kStridedSlice = uint64_t(1) << 62;  // decode map: slice stored as a lane column

// Column header of a W or X slice: word offset from the segment data start, e, m.
struct ColHdr {
  uint16_t wordoff;
  uint8_t e;
  uint8_t m;
};
static_assert(sizeof(ColHdr) == 4, "ColHdr");

// A multiplier range copied into a slot: elements [elem0, elem0 + nelem) of x (which = 0), of
// t m_min(W) (which = 1) or of the phase-1 column factors (which = 2) to slot aux element soff.
// elem0 and nelem are multiples of 4.
struct AuxCopy {
  uint32_t elem0;
  uint16_t nelem;
  uint8_t which;
  uint8_t pad;
  uint32_t soff;
  uint32_t pad2;
};
static_assert(sizeof(AuxCopy) == 16, "AuxCopy");

// A column of a lowrank block whose phase-1 work is split into several chunks.
struct Combine {
  uint32_t tidx;     // t index of the column
  uint32_t pbase;    // partial[pbase + c], c < nchunks
  uint32_t nchunks;
  uint32_t pad;
};
static_assert(sizeof(Combine) == 16, "Combine");

// Issue stream of a CTA's producer: for every piece one entry
//   {offset_lo, offset_hi | 1 << 31, bytes, aux elements}
// followed by one entry per aux copy {elem0, nelem | which << 16, soff, 0}.
struct IssueEnt {
  uint32_t a, b, c, d;
};
static_assert(sizeof(IssueEnt) == 16, "IssueEnt");
constexpr uint32_t kIssuePiece = 1u << 31;

struct PhaseDev {
  const IssueEnt *ent;        // issue streams of all CTAs, back to back
  const uint32_t *cta_e0;     // [nct + 1] entry ranges
  const uint32_t *cta_np;     // [nct] pieces per CTA
  int32_t nct, np;
};

// Device pointers into an arena (set by the host after upload).
struct DevLayout {
  const uint8_t *base;
  const int64_t *perm;       // [n]
  const double *fac64;       // [rank_sum + 8] sigma_i m_min(X_i) m_min(W_i)
  const float *fac32;        // [rank_sum + 8] the same in FP32
  PhaseDev ph[2];
  // scratch
  double *xperm64;           // [n + 8]
  float *xperm32;            // [n + 8]
  double *tw64;              // [rank_sum + 8]  t_i m_min(W_i)
  float *tw32;               // [rank_sum + 8]
  double *partial;           // [part_total]
  double *ysum;              // [n + 8] phase-2 row sums in cluster order (single-RHS AFL FP32
                             // path), added into y by k_scatter
  const Combine *comb;       // [ncnt] columns of blocks with several phase-1 chunks
  uint32_t *status;          // [4] error words (0 = ok)
  double *xdev;              // [n] device copy of a host x (hlr_matvec_host)
  double *ydev;              // [n]
  int64_t n;
  int32_t ncnt, raw;         // raw = 1 for HLR_FMT_FP64
  int32_t vfmt, pad;         // value format of the codes: VF_AFL (AFL, AFLP), VF_BFL, VF_DFL, VF_MP
};

struct Handle {
  int device = 0;
  int format = HLR_FMT_AFL_APLR;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  DevLayout L{};
  hlr_info info{};
  int64_t nunits = 0;
  int64_t values = 0;
  std::vector<uint64_t> slice_src;   // decode map: arena bit address of each unit slice
  std::vector<uint64_t> slice_dst;   // ... its first value index in the unit-order output
  std::vector<uint32_t> slice_n;     // ... its number of values
  std::vector<uint32_t> slice_unit;  // ... its unit
  std::vector<double> unit_mmin;     // per unit: m_min
  std::vector<uint8_t> unit_e, unit_m;
  void *cg_ws = nullptr;             // CG work vectors (allocated on first solve)
  void *multi_ws = nullptr;          // multi-RHS pass scratch (allocated on first use)
  int multi_passes = 0;              // passes multi_ws holds
  std::vector<void *> col_ws;        // HLR_MULTI: one single-RHS scratch set per column of a
                                     // batched call (allocated on first use, never freed early)
  int64_t part_total = 0;            // phase-1 chunk partial sums of one product
  std::vector<void *> prof_ev;       // cudaEvent_t ring: 4 per profiled product
  int prof_n = 0;
};
constexpr int kProfileCap = 4096;
constexpr int kProfileEv = 5;  // events per profiled product: around permute, phase 1, phase 2, scatter

// Error reporting (thread-local message).
int set_error(int code, const std::string &msg);
Handle *lookup(hlr_handle h);

// Kernel side (hlr_kernels.cu).
int launch_matvec(Handle &H, const double *x, double *y, int flags, void *stream);
// Products of many handles (hlr_matvec_batched); arguments validated by the caller.
int launch_batch(int nreq, Handle *const *H, const int32_t *nrhs, const double *const *X, const int64_t *ldx,
                 double *const *Y, const int64_t *ldy, int flags, void *stream);
int launch_decode_units(const Handle &H, double *out, void *stream);
int launch_decode_stream(const uint8_t *stream, int64_t n, double m_min, int e, int m, double *out,
                         void *stream_);
int profile_read(Handle &H, double *ms, int *calls);
int launch_wait_expire(const Handle &H, long long cycles, void *stream);  // hlr_selftest_wait
int ctas_per_phase(int device, int nct[2]);  // persistent grid sizes of the two product kernels

// Host codec (hlr_codec.cpp).
int mantissa_bits(double u);
struct AflParams {
  double m_min;
  int e, m, w;
  int kind;  // value format of the codes: VF_AFL (AFL, AFLP), VF_BFL, VF_DFL, VF_MP
};
bool afl_params(const double *a, int64_t n, double u, AflParams *p);
void afl_pack(const double *a, int64_t n, const AflParams &p, uint8_t *out);
// Parameters and codes of one unit in format fmt (HLR_FMT_AFL_APLR, _AFLP, _BFL, _DFL, _MP);
// false for non-finite input (or values that overflow the BFL / DFL / MP layout). MP with
// u = 0 selects FP64.
bool unit_params(int fmt, const double *a, int64_t n, double u, AflParams *p);
void unit_pack(const double *a, int64_t n, const AflParams &p, uint8_t *out);
inline size_t padded16(size_t b) { return (b + 15) & ~size_t(15); }
inline size_t afl_bytes(int64_t n, int w) { return (size_t(n) * size_t(w) + 7) / 8; }

}  // namespace hlr
