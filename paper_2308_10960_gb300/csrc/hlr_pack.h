// Work-ordered packing of an encoded H-matrix (see hlr_internal.h for the device layout).
#pragma once
#include <cstdint>
#include <vector>

#include "hlr_internal.h"

namespace hlr {

struct PackInput {
  int64_t n = 0;
  bool raw = false;                        // plain FP64 values instead of AFL codes
  const hlr_block_desc *blocks = nullptr;  // cluster order
  int64_t nblocks = 0;
  std::vector<int64_t> blk_unit0;          // first unit of each block (-1: none)
  std::vector<int64_t> unit_len;           // values per unit
  std::vector<AflParams> prm;              // per unit
  std::vector<uint64_t> uoff;              // canonical stream byte offset per unit (+ end)
  const uint8_t *canon = nullptr;          // canonical streams (64 bytes readable past the end)
  const std::vector<std::vector<int64_t>> *cover = nullptr;  // blocks covering each row interval
  const std::vector<int64_t> *brk = nullptr;                 // row interval breakpoints
  int sub_rows = kSubRows;      // AFL phase 1: rows of an X column per lane
  int leaf_rows = kLeafRows;    // phase-2 task rows
  int piece_max = kPieceMax;    // AFL piece bytes
};

struct PhaseOut {
  std::vector<uint8_t> bytes;        // pieces, back to back (16-byte aligned)
  std::vector<uint64_t> piece_off;   // [np + 1], relative to the phase region
  std::vector<uint32_t> aux_idx;     // [np + 1]
  std::vector<AuxCopy> aux;
  std::vector<uint32_t> cta_p0;      // [nct + 1]
};

struct PackOutput {
  PhaseOut ph[2];
  std::vector<double> fac;           // per lowrank column: sigma_i m_min(X_i) m_min(W_i)
  int64_t part_total = 0;            // partial sums of blocks with several phase-1 chunks
  int64_t ncnt = 0;                  // their columns
  std::vector<Combine> comb;         // one entry per such column
  int64_t nleaves = 0, nitems = 0;
  // decode map (optional): per slice of a unit placed in a piece
  std::vector<uint64_t> slice_src;   // bit address relative to its phase region; bit 63 = region of phase 2
  std::vector<uint64_t> slice_dst;   // value index in the unit-order output
  std::vector<uint32_t> slice_n;
  std::vector<uint32_t> slice_unit;
};

// Build both phases' piece streams for nct[0] (phase 1) and nct[1] (phase 2) CTAs. Returns HLR_OK or an HLR_ERR_* code.
int pack_work(const PackInput &in, const int nct[2], bool want_map, PackOutput *out);

}  // namespace hlr
