// Work-ordered packing: re-places the AFL codes (or FP64 values) of every unit into the piece
// streams read by the persistent product kernels. Codes are copied bit for bit; nothing is
// re-encoded, so every stored value decodes exactly as in its canonical unit stream.
//
//  phase 1 (index 0): items = rows [c 256, c 256 + R) of the X columns of lowrank block b;
//  phase 2 (index 1): leaves = row intervals of <= 64 rows with their covering blocks in block
//                     order (dense: the leaf's rows of every column; lowrank: the leaf's rows of
//                     every W column). Pieces never span two leaves.
// Tasks are assigned longest-first to the least loaded of the nct CTAs; each CTA's pieces are
// contiguous. Pieces of one CTA are built independently (in parallel) and concatenated.
#include "hlr_pack.h"

#include <omp.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <queue>

namespace hlr {
namespace {

inline uint32_t words_of(uint64_t bits) { return uint32_t((bits + 31) / 32); }
inline size_t a16(size_t b) { return (b + 15) & ~size_t(15); }
inline int64_t aligned_span(int64_t start, int64_t cnt) {
  return ((start + cnt + 3) & ~int64_t(3)) - (start & ~int64_t(3));
}

// OR nbits bits from bit `so` of src into dst from bit `dof` (dst zeroed; src readable 8 bytes
// past the copied range).
void copy_bits(const uint8_t *srcb, uint64_t so, uint32_t *dst, uint64_t dof, uint64_t nbits) {
  while (nbits) {
    const uint64_t sw = so >> 6;
    const unsigned sb = unsigned(so & 63);
    uint64_t v;
    std::memcpy(&v, srcb + 8 * sw, 8);
    if (sb) {
      uint64_t v2;
      std::memcpy(&v2, srcb + 8 * (sw + 1), 8);
      v = (v >> sb) | (v2 << (64 - sb));
    }
    const unsigned db = unsigned(dof & 31);
    const uint64_t take = std::min<uint64_t>(nbits, 32 - db);
    const uint32_t part = uint32_t(v & ((uint64_t(1) << take) - 1));
    dst[dof >> 5] |= part << db;
    so += take;
    dof += take;
    nbits -= take;
  }
}

// Codes of values v0, v0 + step, v0 + 2 step, ... (count values of w bits) of a canonical
// stream, packed back to back from bit 0 of dst (zeroed; src readable 8 bytes past the end).
void gather_codes(const uint8_t *src, uint64_t v0, uint64_t step, uint64_t count, int w, uint32_t *dst) {
  if (w > 56) {
    for (uint64_t i = 0; i < count; ++i) copy_bits(src, (v0 + i * step) * uint64_t(w), dst, i * uint64_t(w), uint64_t(w));
    return;
  }
  const uint64_t mask = (uint64_t(1) << w) - 1;
  for (uint64_t i = 0; i < count; ++i) {
    const uint64_t sb = (v0 + i * step) * uint64_t(w);
    uint64_t v;
    std::memcpy(&v, src + (sb >> 3), 8);
    const uint64_t code = (v >> (sb & 7)) & mask;
    const uint64_t db = i * uint64_t(w);
    const uint64_t q = db >> 5;
    const unsigned sh = unsigned(db & 31);
    const uint64_t part = code << sh;  // sh + w <= 31 + 56 < 96: at most three words
    dst[q] |= uint32_t(part);
    if (sh + unsigned(w) > 32) dst[q + 1] |= uint32_t(part >> 32);
    if (sh + unsigned(w) > 64) dst[q + 2] |= uint32_t(code >> (64 - sh));
  }
}

struct LR {  // host view of a lowrank block with rank > 0
  uint32_t tbase, part0, cbase;
  uint16_t k, nchunks;
};

struct Task {
  int64_t a, b, c;  // item: block, chunk, R ; leaf: interval index, row0, nr
  double cost;
};

struct Frag {  // one CTA's pieces
  std::vector<uint8_t> bytes;
  std::vector<uint64_t> piece_off;  // relative to the fragment
  std::vector<uint32_t> aux_idx;    // relative to the fragment's aux list
  std::vector<AuxCopy> aux;
  std::vector<uint64_t> s_src, s_dst;
  std::vector<uint32_t> s_n, s_unit;
};

class Builder {
 public:
  Builder(const PackInput &in, const std::vector<int64_t> &uvoff, Frag &f, bool want_map, int aux_max)
      : in_(in), uvoff_(uvoff), f_(f), map_(want_map), aux_max_(aux_max) {}

  int w_of(int64_t u) const { return in_.raw ? 64 : in_.prm[u].w; }

  void begin_leaf(int64_t nr, int64_t row0) {
    leaf_nr_ = uint16_t(nr);
    leaf_row0_ = uint32_t(row0);
    leaf_start_ = true;
  }
  void end_leaf() {
    flush(PF_END_LEAF);
  }

  // phase 2, dense block b: the leaf's nr rows (from rowoff) of every column
  void dense(int64_t b, int64_t nr, int64_t rowoff) {
    const hlr_block_desc &B = in_.blocks[b];
    const int64_t u = in_.blk_unit0[b];
    const int w = w_of(u);
    int64_t j0 = 0;
    while (j0 < B.ncols) {
      int64_t fit = 0;
      for (;;) {
        const int64_t c = fit + 1;
        if (j0 + c > B.ncols || ncols_ + c > kMaxCols) break;
        const size_t bytes = 16 + 32 * (segs_.size() + 1) + a16(4 * cols_.size()) +
                             4 * (data_.size() + words_of(uint64_t(c) * nr * w));
        if (bytes > size_t(kPieceMax) || aux_elems_ + aligned_span(B.col0 + j0, c) > aux_max_) break;
        fit = c;
      }
      if (fit == 0) {
        flush(0);
        continue;
      }
      Seg s{};
      s.kind = SEG_DENSE;
      s.nc = uint16_t(fit);
      s.cstart = uint16_t(ncols_);
      s.nr = uint16_t(nr);
      s.xs = add_aux(0, B.col0 + j0, fit);
      s.gx = uint32_t(B.col0 + j0);
      s.data_w = uint16_t(data_.size());
      s.col_w = uint16_t((in_.raw ? 0 : in_.prm[u].e) | ((in_.raw ? 0 : in_.prm[u].m) << 8));
      s.m_min = in_.raw ? 1.0 : in_.prm[u].m_min;
      const uint64_t bits = uint64_t(fit) * nr * w;
      const uint32_t base_w = uint32_t(data_.size());
      data_.resize(data_.size() + words_of(bits), 0);
      const uint8_t *src = in_.canon + in_.uoff[u];
      if (rowoff == 0 && nr == B.nrows) {
        copy_bits(src, uint64_t(j0) * nr * w, data_.data() + base_w, 0, bits);
        slice(base_w, 0, u, j0 * nr, fit * nr);
      } else {
        for (int64_t j = 0; j < fit; ++j) {
          const uint64_t so = (uint64_t(j0 + j) * B.nrows + rowoff) * w;
          copy_bits(src, so, data_.data() + base_w, uint64_t(j) * nr * w, uint64_t(nr) * w);
          slice(base_w, uint64_t(j) * nr * w, u, (j0 + j) * B.nrows + rowoff, nr);
        }
      }
      segs_.push_back(s);
      ncols_ += uint32_t(fit);
      j0 += fit;
    }
  }

  // column slices of units u0 + i (i < k), rows [rowoff, rowoff + nr) of each.
  //  W (phase 2): multipliers t m_min(W) at [L.tbase + i, ...).
  //  X (phase 1): x of the rows at [xoff, xoff + nr), factors at [L.tbase + i, ...).
  void slices(uint8_t kind, int64_t u0, const LR &L, int64_t nr, int64_t rowoff, int64_t xoff, uint16_t chunk) {
    const int k = L.k;
    // X: a column of nr rows is read by G = 2^lg lanes of 64 rows each (aligned lane groups)
    int lg = 0;
    if (kind == SEG_X)
      while ((kSubRows << lg) < nr) ++lg;
    const uint32_t G = 1u << lg;
    int i0 = 0;
    while (i0 < k) {
      const uint32_t lane0 = (ncols_ + G - 1) & ~(G - 1);
      int fit = 0;
      uint64_t wsum = 0;
      for (;;) {
        const int c = fit + 1;
        if (i0 + c > k || lane0 + uint32_t(c) * G > uint32_t(kMaxCols)) break;
        const uint64_t wi = words_of(uint64_t(nr) * w_of(u0 + i0 + c - 1));
        const size_t bytes = 16 + 32 * (segs_.size() + 1) + a16(4 * (cols_.size() + c)) + 4 * (data_.size() + wsum + wi);
        int64_t need = aux_elems_;
        if (kind == SEG_X)
          need += aligned_span(xoff, nr) + aligned_span(L.tbase + i0, c);
        else
          need += aligned_span(L.tbase + i0, c);
        if (bytes > size_t(kPieceMax) || need > aux_max_) break;
        wsum += wi;
        fit = c;
      }
      if (fit == 0) {
        flush(0);
        continue;
      }
      Seg s{};
      s.kind = kind;
      s.lg = uint8_t(lg);
      s.nc = uint16_t(fit);
      s.cstart = uint16_t(lane0);
      s.nr = uint16_t(nr);
      s.data_w = uint16_t(data_.size());
      s.col_w = uint16_t(cols_.size());
      if (kind == SEG_X) {
        s.xs = add_aux(0, xoff, nr);
        s.fs = add_aux(2, L.tbase + i0, fit);
        s.tidx = L.tbase + uint32_t(i0);
        s.gx = uint32_t(xoff);
        s.x.pbase = L.part0 + uint32_t(i0) * L.nchunks;
        s.x.chunk = chunk;
        s.x.nchunks = L.nchunks;
      } else {
        s.xs = add_aux(1, L.tbase + i0, fit);
        s.gx = L.tbase + uint32_t(i0);
      }
      uint32_t woff = 0;
      for (int i = i0; i < i0 + fit; ++i) {
        const int64_t u = u0 + i;
        const int w = w_of(u);
        const uint64_t bits = uint64_t(nr) * w;
        ColHdr ch;
        ch.wordoff = uint16_t(woff);
        ch.e = uint8_t(in_.raw ? 0 : in_.prm[u].e);
        ch.m = uint8_t(in_.raw ? 0 : in_.prm[u].m);
        cols_.push_back(ch);
        const uint32_t base_w = uint32_t(data_.size());
        data_.resize(data_.size() + words_of(bits), 0);
        copy_bits(in_.canon + in_.uoff[u], uint64_t(rowoff) * w, data_.data() + base_w, 0, bits);
        slice(base_w, 0, u, rowoff, nr);
        woff += words_of(bits);
      }
      segs_.push_back(s);
      ncols_ = lane0 + uint32_t(fit) * G;
      i0 += fit;
    }
  }

  void flush(uint8_t end_flags) {
    if (segs_.empty()) return;
    const size_t nseg = segs_.size();
    const uint32_t col_words = uint32_t(16 + 32 * nseg) / 4;
    const uint32_t hdr_bytes = uint32_t(16 + 32 * nseg + a16(4 * cols_.size()));
    const uint32_t hdr_words = hdr_bytes / 4;
    for (auto &s : segs_) {
      s.data_w = uint16_t(s.data_w + hdr_words);
      if (s.kind != SEG_DENSE) s.col_w = uint16_t(s.col_w + col_words);
    }
    PieceHdr ph{};
    ph.nseg = uint16_t(nseg);
    ph.ncols = uint16_t(ncols_);
    ph.nr = leaf_nr_;
    ph.flags = uint8_t((leaf_start_ ? PF_START_LEAF : 0) | end_flags);
    ph.row0 = leaf_row0_;
    leaf_start_ = false;
    const size_t total = a16(hdr_bytes + 4 * data_.size());
    const size_t start = f_.bytes.size();
    f_.piece_off.push_back(start);
    f_.aux_idx.push_back(uint32_t(f_.aux.size()));
    f_.bytes.resize(start + total, 0);
    uint8_t *p = f_.bytes.data() + start;
    std::memcpy(p, &ph, 16);
    std::memcpy(p + 16, segs_.data(), 32 * nseg);
    if (!cols_.empty()) std::memcpy(p + 16 + 32 * nseg, cols_.data(), 4 * cols_.size());
    if (!data_.empty()) std::memcpy(p + hdr_bytes, data_.data(), 4 * data_.size());
    for (auto &a : auxs_) f_.aux.push_back(a);
    for (size_t i = 0; i < ps_src_.size(); ++i) {
      f_.s_src.push_back(8 * (start + hdr_bytes) + ps_src_[i]);
      f_.s_dst.push_back(ps_dst_[i]);
      f_.s_n.push_back(ps_n_[i]);
      f_.s_unit.push_back(ps_unit_[i]);
    }
    segs_.clear();
    cols_.clear();
    data_.clear();
    auxs_.clear();
    aux_elems_ = 0;
    ncols_ = 0;
    ps_src_.clear();
    ps_dst_.clear();
    ps_n_.clear();
    ps_unit_.clear();
  }

 private:
  uint16_t add_aux(int which, int64_t start, int64_t cnt) {
    const int64_t a0 = start & ~int64_t(3);
    AuxCopy a{};
    a.elem0 = uint32_t(a0);
    a.nelem = uint16_t(aligned_span(start, cnt));
    a.which = uint8_t(which);
    a.soff = aux_elems_;
    auxs_.push_back(a);
    const uint16_t xs = uint16_t(aux_elems_ + (start - a0));
    aux_elems_ += a.nelem;
    return xs;
  }
  void slice(uint32_t base_w, uint64_t bitoff, int64_t u, int64_t v0, int64_t nv) {
    if (!map_) return;
    ps_src_.push_back(uint64_t(base_w) * 32 + bitoff);
    ps_dst_.push_back(uint64_t(uvoff_[u] + v0));
    ps_n_.push_back(uint32_t(nv));
    ps_unit_.push_back(uint32_t(u));
  }

  const PackInput &in_;
  const std::vector<int64_t> &uvoff_;
  Frag &f_;
  bool map_;
  int aux_max_;
  uint16_t leaf_nr_ = 0;
  uint32_t leaf_row0_ = 0;
  bool leaf_start_ = false;
  std::vector<Seg> segs_;
  std::vector<ColHdr> cols_;
  std::vector<uint32_t> data_;
  std::vector<AuxCopy> auxs_;
  uint32_t aux_elems_ = 0;
  uint32_t ncols_ = 0;
  std::vector<uint64_t> ps_src_, ps_dst_;
  std::vector<uint32_t> ps_n_, ps_unit_;
};

// Pieces in the bank-column layout (hlr_internal.h, LaneHdr): the same tasks, segments and aux
// copies as Builder, but every slice becomes one lane column of a warp region.
class BcBuilder {
 public:
  BcBuilder(const PackInput &in, const std::vector<int64_t> &uvoff, Frag &f, bool want_map, int aux_max)
      : in_(in), uvoff_(uvoff), f_(f), map_(want_map), aux_max_(aux_max) {}

  void begin_leaf(int64_t nr, int64_t row0) {
    leaf_nr_ = uint16_t(nr);
    leaf_row0_ = uint32_t(row0);
    leaf_start_ = true;
  }
  void end_leaf() { flush(PF_END_LEAF); }

  // phase 2, dense block b: the leaf's nr rows (from rowoff) of every column, one lane each
  void dense(int64_t b, int64_t nr, int64_t rowoff) {
    const hlr_block_desc &B = in_.blocks[b];
    const int64_t u = in_.blk_unit0[b];
    int64_t j0 = 0;
    while (j0 < B.ncols) {
      const size_t l0 = lanes_.size();
      Seg s{};
      s.kind = SEG_DENSE;
      s.nr = uint16_t(nr);
      s.m_min = in_.prm[u].m_min;
      s.gx = uint32_t(B.col0 + j0);
      segs_.push_back(s);
      int64_t fit = 0;
      for (;;) {
        const int64_t c = fit + 1;
        if (j0 + c > B.ncols || c > kMaxCols) break;
        lanes_.push_back(lane(u, uint64_t(j0 + fit) * B.nrows + rowoff, nr, uint16_t(segs_.size() - 1), uint8_t(fit), 1, 0));
        if (!fits(aux_elems_ + aligned_span(B.col0 + j0, c))) {
          lanes_.pop_back();
          break;
        }
        fit = c;
      }
      if (fit == 0) {
        segs_.pop_back();
        if (segs_.empty()) {  // not even one column fits an empty piece
          failed = true;
          return;
        }
        flush(0);
        continue;
      }
      Seg &sg = segs_.back();
      sg.nc = uint16_t(fit);
      sg.xs = add_aux(0, B.col0 + j0, fit);
      j0 += fit;
      if (j0 < B.ncols) flush(0);
    }
  }

  // column slices of units u0 + i (i < k), rows [rowoff, rowoff + nr) of each (see Builder)
  void slices(uint8_t kind, int64_t u0, const LR &L, int64_t nr, int64_t rowoff, int64_t xoff, uint16_t chunk) {
    const int k = L.k;
    int lg = 0;
    if (kind == SEG_X) {
      int wmax = 1;
      for (int i = 0; i < k; ++i) wmax = std::max(wmax, int(in_.prm[u0 + i].w));
      // a lane column must leave room in a piece: one warp region of 32 such columns
      const int64_t max_words = std::max<int64_t>(8, (in_.piece_max - 1024) / 128);
      while ((in_.sub_rows << lg) < nr || int64_t((nr + (1 << lg) - 1) >> lg) * wmax > max_words * 32) ++lg;
    }
    const int G = 1 << lg;
    int i0 = 0;
    while (i0 < k) {
      Seg s{};
      s.kind = kind;
      s.lg = uint8_t(lg);
      s.nr = uint16_t(nr);
      if (kind == SEG_X) {
        s.tidx = L.tbase + uint32_t(i0);
        s.gx = uint32_t(xoff);
        s.x.pbase = L.part0 + uint32_t(i0) * L.nchunks;
        s.x.chunk = chunk;
        s.x.nchunks = L.nchunks;
      } else {
        s.gx = L.tbase + uint32_t(i0);
      }
      segs_.push_back(s);
      const uint16_t si = uint16_t(segs_.size() - 1);
      int fit = 0;
      for (;;) {
        const int c = fit + 1;
        if (i0 + c > k || c * G > kMaxCols) break;
        const int64_t u = u0 + i0 + fit;
        for (int g = 0; g < G; ++g) {
          // X: lane g of the G lanes of a column takes rows g, g + G, g + 2G, ... of its nr rows,
          // so that at every step the group's lanes read consecutive x rows (distinct banks)
          const int64_t nv = kind == SEG_X ? (nr - g + G - 1) / G : nr;
          lanes_.push_back(lane(u, uint64_t(rowoff + (kind == SEG_X ? g : 0)), nv, si, uint8_t(fit), uint8_t(G),
                                uint8_t(g), kind == SEG_X ? uint32_t(G) : 1u));
        }
        int64_t need = aux_elems_;
        if (kind == SEG_X)
          need += aligned_span(xoff, nr) + aligned_span(L.tbase + i0, c);
        else
          need += aligned_span(L.tbase + i0, c);
        if (!fits(need)) {
          lanes_.resize(lanes_.size() - G);
          break;
        }
        fit = c;
      }
      if (fit == 0) {
        segs_.pop_back();
        if (segs_.empty()) {
          failed = true;
          return;
        }
        flush(0);
        continue;
      }
      Seg &sg = segs_.back();
      sg.nc = uint16_t(fit);
      if (kind == SEG_X) {
        sg.xs = add_aux(0, xoff, nr);
        sg.fs = add_aux(2, L.tbase + i0, fit);
      } else {
        sg.xs = add_aux(1, L.tbase + i0, fit);
      }
      i0 += fit;
      if (i0 < k) flush(0);
    }
  }

  void flush(uint8_t end_flags) {
    if (segs_.empty()) return;
    Layout lay;
    layout(lanes_, &lay);
    const size_t nseg = segs_.size();
    const uint32_t nl = uint32_t(lay.nl);
    const uint32_t hdr_bytes = uint32_t(16 + 32 * nseg + a16(4 * nl));
    const uint32_t data_w0 = hdr_bytes / 4;
    PieceHdr ph{};
    ph.nseg = uint16_t(nseg);
    ph.ncols = uint16_t(nl);
    ph.nr = leaf_nr_;
    ph.flags = uint8_t((leaf_start_ ? PF_START_LEAF : 0) | end_flags);
    ph.row0 = leaf_row0_;
    for (int w = 0; w < 4; ++w) ph.h[w] = uint8_t(lay.h[w]);
    leaf_start_ = false;
    const size_t total = a16(hdr_bytes + 4 * lay.data_words);
    const size_t start = f_.bytes.size();
    f_.piece_off.push_back(start);
    f_.aux_idx.push_back(uint32_t(f_.aux.size()));
    f_.bytes.resize(start + total, 0);
    uint8_t *p = f_.bytes.data() + start;
    std::memcpy(p, &ph, 16);
    std::memcpy(p + 16, segs_.data(), 32 * nseg);
    std::vector<LaneHdr> lh(nl, LaneHdr{0xff, 0, 0, 0});
    uint32_t *data = reinterpret_cast<uint32_t *>(p + hdr_bytes);
    uint32_t region[4] = {0, 0, 0, 0};
    for (int w = 1; w < 4; ++w) region[w] = region[w - 1] + 32 * lay.h[w - 1];
    std::vector<uint32_t> tmp;
    for (size_t i = 0; i < lanes_.size(); ++i) {
      const Lane &L = lanes_[i];
      const int pos = lay.pos[i];
      lh[pos] = LaneHdr{uint8_t(L.seg), L.j, L.e, L.m};
      const uint32_t col = region[pos >> 5] + uint32_t(pos & 31);
      const uint64_t bits = uint64_t(L.nv) * L.w;
      tmp.assign(L.words + 3, 0);
      if (L.step == 1)
        copy_bits(in_.canon + in_.uoff[L.u], L.v0 * L.w, tmp.data(), 0, bits);
      else
        gather_codes(in_.canon + in_.uoff[L.u], L.v0, L.step, L.nv, L.w, tmp.data());
      for (uint32_t k = 0; k < L.words; ++k) data[col + 32 * k] = tmp[k];
      if (in_.prm[L.u].kind == VF_DFL && L.m <= 20 && L.nv > 0) {
        // all values FP32 normal numbers (biased FP64 exponent 897..1150): integer decode
        bool fast = true;
        for (uint32_t v = 0; v < L.nv && fast; ++v) {
          const uint64_t bit = uint64_t(v) * L.w;
          const uint64_t code = ((uint64_t(tmp[bit >> 5]) | (uint64_t(tmp[(bit >> 5) + 1]) << 32)) >> (bit & 31)) &
                                ((uint64_t(1) << L.w) - 1);
          const uint32_t ex = uint32_t(code >> L.m) & 0x7ffu;
          fast = ex >= 897 && ex <= 1150;
        }
        if (fast) lh[pos].e = uint8_t(lh[pos].e | 0x80);
      }
      if (map_ && L.nv > 0) {
        f_.s_src.push_back((8 * start + 32 * uint64_t(data_w0 + col)) | kStridedSlice);
        f_.s_dst.push_back(uint64_t(uvoff_[L.u]) + L.v0);
        f_.s_n.push_back(L.nv | (L.step << 24));  // values | value stride in the unit << 24
        f_.s_unit.push_back(uint32_t(L.u));
      }
    }
    std::memcpy(p + 16 + 32 * nseg, lh.data(), 4 * nl);
    for (auto &a : auxs_) f_.aux.push_back(a);
    segs_.clear();
    lanes_.clear();
    auxs_.clear();
    aux_elems_ = 0;
  }

 private:
  struct Lane {
    int64_t u;
    uint64_t v0;      // first value within the unit
    uint32_t step;    // distance of consecutive values of the slice within the unit
    uint32_t nv;      // values
    uint32_t words;   // ceil(nv w / 32)
    uint16_t seg;
    uint8_t j, e, m, w, G, sub;
  };
  struct Layout {
    std::vector<int> pos;   // position (lane index in the piece) of every lane
    int nl = 0;
    uint32_t h[4] = {0, 0, 0, 0};
    size_t data_words = 0;
  };

  Lane lane(int64_t u, uint64_t v0, int64_t nv, uint16_t seg, uint8_t j, uint8_t G, uint8_t sub,
            uint32_t step = 1) const {
    Lane L{};
    L.u = u;
    L.v0 = v0;
    L.step = step;
    L.nv = uint32_t(nv);
    L.e = uint8_t(in_.prm[u].e);
    L.m = uint8_t(in_.prm[u].m);
    L.w = uint8_t(in_.prm[u].w);
    L.words = words_of(uint64_t(nv) * L.w);
    L.seg = seg;
    L.j = j;
    L.G = G;
    L.sub = sub;
    return L;
  }

  // Groups (the G lanes of one X column, or single lanes) by decreasing G, then decreasing
  // length; positions are consecutive, so every group stays aligned to its size.
  static void layout(const std::vector<Lane> &lanes, Layout *out) {
    std::vector<int> gs;
    for (size_t i = 0; i < lanes.size(); ++i)
      if (lanes[i].sub == 0) gs.push_back(int(i));
    std::stable_sort(gs.begin(), gs.end(), [&](int a, int b) {
      if (lanes[a].G != lanes[b].G) return lanes[a].G > lanes[b].G;
      return lanes[a].words > lanes[b].words;
    });
    out->pos.assign(lanes.size(), 0);
    int p = 0;
    for (int g : gs) {
      const int G = lanes[g].G;
      p = (p + G - 1) / G * G;
      for (int s = 0; s < G; ++s) out->pos[g + s] = p + s;
      p += G;
    }
    out->nl = p;
    for (int w = 0; w < 4; ++w) out->h[w] = 0;
    for (size_t i = 0; i < lanes.size(); ++i) {
      const int w = out->pos[i] >> 5;
      if (w < 4) out->h[w] = std::max(out->h[w], lanes[i].words);
    }
    out->data_words = 32 * size_t(out->h[0] + out->h[1] + out->h[2] + out->h[3]);
  }

  bool fits(int64_t aux_need) const {
    if (aux_need > aux_max_) return false;
    Layout lay;
    layout(lanes_, &lay);
    if (lay.nl > kMaxCols) return false;
    for (int w = 0; w < 4; ++w)
      if (lay.h[w] > 255) return false;
    const size_t bytes = 16 + 32 * segs_.size() + a16(4 * size_t(lay.nl)) + 4 * lay.data_words;
    return bytes <= size_t(in_.piece_max);
  }

  uint16_t add_aux(int which, int64_t start, int64_t cnt) {
    const int64_t a0 = start & ~int64_t(3);
    AuxCopy a{};
    a.elem0 = uint32_t(a0);
    a.nelem = uint16_t(aligned_span(start, cnt));
    a.which = uint8_t(which);
    a.soff = aux_elems_;
    auxs_.push_back(a);
    const uint16_t xs = uint16_t(aux_elems_ + (start - a0));
    aux_elems_ += a.nelem;
    return xs;
  }

 public:
  bool failed = false;  // a column did not fit an empty piece

 private:
  const PackInput &in_;
  const std::vector<int64_t> &uvoff_;
  Frag &f_;
  bool map_;
  int aux_max_;
  uint16_t leaf_nr_ = 0;
  uint32_t leaf_row0_ = 0;
  bool leaf_start_ = false;
  std::vector<Seg> segs_;
  std::vector<Lane> lanes_;
  std::vector<AuxCopy> auxs_;
  uint32_t aux_elems_ = 0;
};

// Longest task first onto the least loaded CTA; returns each CTA's tasks in assignment order.
std::vector<std::vector<int64_t>> assign(const std::vector<Task> &tasks, int nct) {
  std::vector<int64_t> ord(tasks.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return tasks[a].cost > tasks[b].cost; });
  using E = std::pair<double, int>;
  std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
  for (int q = 0; q < nct; ++q) pq.push({0.0, q});
  std::vector<std::vector<int64_t>> out(nct);
  for (int64_t t : ord) {
    E e = pq.top();
    pq.pop();
    out[e.second].push_back(t);
    pq.push({e.first + tasks[t].cost, e.second});
  }
  return out;
}

void concat(std::vector<Frag> &frags, PhaseOut &po, bool phase2, PackOutput *out) {
  size_t total = 0;
  for (auto &f : frags) total += f.bytes.size();
  po.bytes.reserve(total);
  for (auto &f : frags) {
    po.cta_p0.push_back(uint32_t(po.piece_off.size()));
    const uint64_t boff = po.bytes.size();
    const uint32_t aoff = uint32_t(po.aux.size());
    for (auto v : f.piece_off) po.piece_off.push_back(boff + v);
    for (auto v : f.aux_idx) po.aux_idx.push_back(aoff + v);
    po.aux.insert(po.aux.end(), f.aux.begin(), f.aux.end());
    po.bytes.insert(po.bytes.end(), f.bytes.begin(), f.bytes.end());
    for (size_t i = 0; i < f.s_src.size(); ++i) {
      out->slice_src.push_back((8 * boff + f.s_src[i]) | (phase2 ? (uint64_t(1) << 63) : 0));
      out->slice_dst.push_back(f.s_dst[i]);
      out->slice_n.push_back(f.s_n[i]);
      out->slice_unit.push_back(f.s_unit[i]);
    }
    std::vector<uint8_t>().swap(f.bytes);
  }
  po.cta_p0.push_back(uint32_t(po.piece_off.size()));
  po.piece_off.push_back(po.bytes.size());
  po.aux_idx.push_back(uint32_t(po.aux.size()));
}

}  // namespace

int pack_work(const PackInput &in, const int nct2[2], bool want_map, PackOutput *out) {
  const int64_t nb = in.nblocks;
  const int64_t nunits = int64_t(in.unit_len.size());
  std::vector<int64_t> uvoff(nunits + 1, 0);
  for (int64_t u = 0; u < nunits; ++u) uvoff[u + 1] = uvoff[u] + in.unit_len[u];
  auto wbits = [&](int64_t u) -> int { return in.raw ? 64 : in.prm[u].w; };

  // ---- lowrank blocks: column factors, partial-sum and counter offsets
  std::vector<LR> lr(nb);
  std::vector<char> has_lr(nb, 0);
  uint32_t tbase = 0;
  int64_t part = 0, ncnt = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = in.blocks[b];
    if (B.kind != HLR_LOWRANK || B.rank == 0) continue;
    LR L{};
    L.tbase = tbase;
    L.k = uint16_t(B.rank);
    const int64_t nch = (B.ncols + kRowsPerItem - 1) / kRowsPerItem;
    if (nch > 65535) return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: lowrank block too wide");
    L.nchunks = uint16_t(nch);
    L.part0 = uint32_t(part);
    L.cbase = uint32_t(ncnt);
    if (nch > 1) {
      for (int i = 0; i < B.rank; ++i) {
        Combine c{};
        c.tidx = tbase + uint32_t(i);
        c.pbase = uint32_t(part + int64_t(i) * nch);
        c.nchunks = uint32_t(nch);
        out->comb.push_back(c);
      }
      part += nch * B.rank;
      ncnt += B.rank;
    }
    if (part > (int64_t(1) << 32) - 1) return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: too many partial sums");
    lr[b] = L;
    has_lr[b] = 1;
    const int64_t u0 = in.blk_unit0[b];
    for (int i = 0; i < B.rank; ++i) {
      const double wmin = in.raw ? 1.0 : in.prm[u0 + i].m_min;
      const double xmin = in.raw ? 1.0 : in.prm[u0 + B.rank + i].m_min;
      out->fac.push_back((B.sigma[i] * xmin) * wmin);
    }
    tbase += uint32_t(B.rank);
  }
  out->part_total = part;
  out->ncnt = ncnt;

  // ---- tasks
  std::vector<Task> items, leaves;
  for (int64_t b = 0; b < nb; ++b) {
    if (!has_lr[b]) continue;
    const hlr_block_desc &B = in.blocks[b];
    const int64_t u0 = in.blk_unit0[b];
    for (int64_t c = 0; c < lr[b].nchunks; ++c) {
      const int64_t R = std::min<int64_t>(kRowsPerItem, B.ncols - c * kRowsPerItem);
      double cost = 64;
      for (int i = 0; i < B.rank; ++i) cost += 4.0 * words_of(uint64_t(R) * wbits(u0 + B.rank + i)) + 8;
      items.push_back({b, c, R, cost});
    }
  }
  const auto &cover = *in.cover;
  const auto &brk = *in.brk;
  for (size_t iv = 0; iv < cover.size(); ++iv) {
    for (int64_t r0 = brk[iv]; r0 < brk[iv + 1]; r0 += in.leaf_rows) {
      const int64_t nr = std::min<int64_t>(in.leaf_rows, brk[iv + 1] - r0);
      double cost = 64;
      int nc = 0;
      for (int64_t b : cover[iv]) {
        const hlr_block_desc &B = in.blocks[b];
        const int64_t u0 = in.blk_unit0[b];
        if (B.kind == HLR_DENSE) {
          cost += 4.0 * words_of(uint64_t(B.ncols) * nr * wbits(u0)) + 40 + 8.0 * B.ncols;
          ++nc;
        } else if (B.rank > 0) {
          for (int i = 0; i < B.rank; ++i) cost += 4.0 * words_of(uint64_t(nr) * wbits(u0 + i)) + 12;
          cost += 40;
          ++nc;
        }
      }
      if (nc) leaves.push_back({int64_t(iv), r0, nr, cost});
    }
  }
  out->nitems = int64_t(items.size());
  out->nleaves = int64_t(leaves.size());
  std::atomic<int> failed{0};

  // ---- phase 1 (items)
  {
    const int nct = nct2[0];
    auto per = assign(items, nct);
    std::vector<Frag> frags(nct);
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nct; ++q) {
      auto run = [&](auto &bld) {
        for (int64_t t : per[q]) {
          const Task &T = items[t];
          const int64_t b = T.a;
          const hlr_block_desc &B = in.blocks[b];
          const int64_t row0 = T.b * kRowsPerItem;
          bld.slices(SEG_X, in.blk_unit0[b] + B.rank, lr[b], T.c, row0, B.col0 + row0, uint16_t(T.b));
        }
        bld.flush(0);
      };
      if (in.raw) {
        Builder bld(in, uvoff, frags[q], want_map, kAuxMax1);
        run(bld);
      } else {
        BcBuilder bld(in, uvoff, frags[q], want_map, kAuxMax1);
        run(bld);
        if (bld.failed) failed.store(1);
      }
    }
    concat(frags, out->ph[0], false, out);
  }
  // ---- phase 2 (leaves)
  {
    const int nct = nct2[1];
    auto per = assign(leaves, nct);
    std::vector<Frag> frags(nct);
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nct; ++q) {
      auto run = [&](auto &bld) {
        for (int64_t t : per[q]) {
          const Task &T = leaves[t];
          std::vector<int64_t> bl = cover[T.a];
          std::sort(bl.begin(), bl.end());
          bld.begin_leaf(T.c, T.b);
          for (int64_t b : bl) {
            const hlr_block_desc &B = in.blocks[b];
            const int64_t rowoff = T.b - B.row0;
            if (B.kind == HLR_DENSE)
              bld.dense(b, T.c, rowoff);
            else if (has_lr[b])
              bld.slices(SEG_W, in.blk_unit0[b], lr[b], T.c, rowoff, 0, 0);
          }
          bld.end_leaf();
        }
      };
      if (in.raw) {
        Builder bld(in, uvoff, frags[q], want_map, kAuxMax2);
        run(bld);
      } else {
        BcBuilder bld(in, uvoff, frags[q], want_map, kAuxMax2);
        run(bld);
        if (bld.failed) failed.store(1);
      }
    }
    concat(frags, out->ph[1], true, out);
  }
  if (failed) return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: a column does not fit one piece of this work layout");
  return HLR_OK;
}

}  // namespace hlr
