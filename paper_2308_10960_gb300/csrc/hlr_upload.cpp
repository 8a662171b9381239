// hlr_upload / hlr_free / hlr_get_info / hlr_last_error and the handle registry.
//
// Upload flattens the block tree's leaves (Def. 2.2) into the work lists of the product:
//  * every dense block is one AFL unit at precision eps; every lowrank block contributes one
//    unit per column of W and of X at precision eps sigma_0 / sigma_i (APLR, Section 3.3);
//  * phase-1 items: rows of X of a lowrank block in chunks of <= 256 rows (t = Sigma X^T x);
//  * phase-2 owners: the leaf row intervals (finest row partition induced by the blocks,
//    cut to <= 64 rows); each owner lists every block whose row cluster contains it, in block
//    order, so y is accumulated by exactly one owner per row, in a fixed order.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "hlr_internal.h"

namespace hlr {

static thread_local std::string g_err;
static std::mutex g_mu;
static std::unordered_map<uint64_t, std::unique_ptr<Handle>> g_handles;
static uint64_t g_next = 1;

int set_error(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

Handle *lookup(hlr_handle h) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_handles.find(h);
  return it == g_handles.end() ? nullptr : it->second.get();
}

namespace {

constexpr int kRowsPerItem = 256;
constexpr int kLeafRows = 64;

struct UnitSrc {
  const double *a;
  int64_t n;
  double u;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct HostBuf {
  uint8_t *p = nullptr;
  ~HostBuf() { std::free(p); }
};

}  // namespace
}  // namespace hlr

using namespace hlr;

extern "C" const char *hlr_last_error(void) { return g_err.c_str(); }

extern "C" int hlr_upload(const hlr_hmatrix_desc *d, void *cuda_stream, hlr_handle *out,
                          size_t *device_bytes) {
  if (!d || !out) return set_error(HLR_ERR_INVALID, "hlr_upload: null descriptor or output");
  *out = 0;
  const int64_t n = d->n;
  if (n <= 0 || n > (int64_t(1) << 31)) return set_error(HLR_ERR_INVALID, "hlr_upload: n out of range");
  if (d->nblocks <= 0 || !d->blocks) return set_error(HLR_ERR_INVALID, "hlr_upload: no blocks");
  if (d->format != HLR_FMT_AFL_APLR && d->format != HLR_FMT_FP64)
    return set_error(HLR_ERR_INVALID, "hlr_upload: unknown format");
  if (d->reserved != 0) return set_error(HLR_ERR_INVALID, "hlr_upload: reserved must be 0");
  if (d->format == HLR_FMT_AFL_APLR && !(d->eps > 0.0 && d->eps < 1.0))
    return set_error(HLR_ERR_INVALID, "hlr_upload: eps must be in (0, 1)");
  const bool afl = d->format == HLR_FMT_AFL_APLR;

  // ---- permutation
  std::vector<int64_t> perm(n);
  if (d->perm) {
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
      int64_t p = d->perm[i];
      if (p < 0 || p >= n || seen[p]) return set_error(HLR_ERR_INVALID, "hlr_upload: perm is not a permutation");
      seen[p] = 1;
      perm[i] = p;
    }
  } else {
    std::iota(perm.begin(), perm.end(), 0);
  }

  // ---- block checks
  const int64_t nb = d->nblocks;
  int64_t ndense = 0, nlr = 0, rank_sum = 0, values = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.row0 < 0 || B.col0 < 0 || B.nrows <= 0 || B.ncols <= 0 || B.row0 + B.nrows > n ||
        B.col0 + B.ncols > n)
      return set_error(HLR_ERR_INVALID, "hlr_upload: block " + std::to_string(b) + " out of range");
    if (B.kind == HLR_DENSE) {
      if (!B.D) return set_error(HLR_ERR_INVALID, "hlr_upload: dense block without data");
      if (B.nrows * B.ncols > (int64_t(1) << 31))
        return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: dense block too large");
      ++ndense;
      values += B.nrows * B.ncols;
    } else if (B.kind == HLR_LOWRANK) {
      if (B.rank < 0 || B.rank > 65535 || B.rank > std::min(B.nrows, B.ncols))
        return set_error(HLR_ERR_INVALID, "hlr_upload: bad rank in block " + std::to_string(b));
      if (B.rank > 0) {
        if (!B.W || !B.X || !B.sigma) return set_error(HLR_ERR_INVALID, "hlr_upload: lowrank block without factors");
        for (int i = 0; i < B.rank; ++i) {
          double s = B.sigma[i];
          if (!(s > 0.0) || !std::isfinite(s) || s > B.sigma[0])
            return set_error(HLR_ERR_INVALID, "hlr_upload: sigma must be positive, finite and led by its maximum");
        }
        ++nlr;
        rank_sum += B.rank;
        values += int64_t(B.rank) * (B.nrows + B.ncols);
      }
    } else {
      return set_error(HLR_ERR_INVALID, "hlr_upload: unknown block kind");
    }
  }

  // ---- elementary row intervals and coverage check
  std::vector<int64_t> brk;
  brk.reserve(2 * nb + 2);
  brk.push_back(0);
  brk.push_back(n);
  for (int64_t b = 0; b < nb; ++b) {
    brk.push_back(d->blocks[b].row0);
    brk.push_back(d->blocks[b].row0 + d->blocks[b].nrows);
  }
  std::sort(brk.begin(), brk.end());
  brk.erase(std::unique(brk.begin(), brk.end()), brk.end());
  const int64_t nint = int64_t(brk.size()) - 1;
  std::vector<std::vector<int64_t>> cover(nint);
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    int64_t i0 = std::lower_bound(brk.begin(), brk.end(), B.row0) - brk.begin();
    for (int64_t i = i0; i < nint && brk[i] < B.row0 + B.nrows; ++i) cover[i].push_back(b);
  }
  for (int64_t i = 0; i < nint; ++i) {
    std::vector<std::pair<int64_t, int64_t>> cols;
    cols.reserve(cover[i].size());
    for (int64_t b : cover[i]) cols.push_back({d->blocks[b].col0, d->blocks[b].ncols});
    std::sort(cols.begin(), cols.end());
    int64_t c = 0;
    for (auto &pc : cols) {
      if (pc.first != c) return set_error(HLR_ERR_INVALID, "hlr_upload: blocks do not cover the matrix exactly once");
      c += pc.second;
    }
    if (c != n) return set_error(HLR_ERR_INVALID, "hlr_upload: blocks do not cover the matrix exactly once");
  }

  // ---- units
  std::vector<UnitSrc> src;
  src.reserve(ndense + 2 * rank_sum);
  std::vector<int64_t> blk_unit0(nb, -1);
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.kind == HLR_DENSE) {
      blk_unit0[b] = int64_t(src.size());
      src.push_back({B.D, B.nrows * B.ncols, d->eps});
    } else if (B.rank > 0) {
      blk_unit0[b] = int64_t(src.size());
      const double delta = d->eps * B.sigma[0];
      for (int i = 0; i < B.rank; ++i) src.push_back({B.W + i * B.nrows, B.nrows, delta / B.sigma[i]});
      for (int i = 0; i < B.rank; ++i) src.push_back({B.X + i * B.ncols, B.ncols, delta / B.sigma[i]});
    }
  }
  const int64_t nunits = int64_t(src.size());
  std::vector<AflParams> prm(nunits);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t u = 0; u < nunits; ++u) {
    if (afl) {
      if (!afl_params(src[u].a, src[u].n, src[u].u, &prm[u])) bad |= 1;
    } else {
      for (int64_t j = 0; j < src[u].n; ++j)
        if (!std::isfinite(src[u].a[j])) bad |= 1;
      prm[u] = AflParams{0.0, 0, 0, 64};
    }
  }
  if (bad) return set_error(HLR_ERR_INVALID, "hlr_upload: NaN or Inf in block data");

  std::vector<uint64_t> uoff(nunits + 1, 0);
  uint64_t stream_bytes = 0;
  for (int64_t u = 0; u < nunits; ++u) {
    size_t bytes = afl ? afl_bytes(src[u].n, prm[u].w) : size_t(src[u].n) * 8;
    stream_bytes += bytes;
    uoff[u + 1] = uoff[u] + padded16(bytes);
  }

  // ---- phase-1 items (lowrank blocks), sorted by decreasing cost
  std::vector<LRBlock> lrb;
  std::vector<int64_t> lr_of_block(nb, -1);
  std::vector<P1Item> items;
  std::vector<double> item_cost;
  uint32_t tbase = 0, part = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.kind != HLR_LOWRANK || B.rank == 0) continue;
    int64_t nch = (B.ncols + kRowsPerItem - 1) / kRowsPerItem;
    if (nch > 65535) return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: lowrank block too wide");
    LRBlock L;
    L.tbase = tbase;
    L.part0 = part;
    L.k = uint16_t(B.rank);
    L.nchunks = uint16_t(nch);
    L.xunit0 = uint32_t(blk_unit0[b] + B.rank);
    lr_of_block[b] = int64_t(lrb.size());
    double wsum = 0;
    for (int i = 0; i < B.rank; ++i) wsum += prm[L.xunit0 + i].w;
    for (int64_t c = 0; c < nch; ++c) {
      P1Item it;
      it.blk = uint32_t(lrb.size());
      it.row0 = uint32_t(c * kRowsPerItem);
      it.xoff = uint32_t(B.col0 + c * kRowsPerItem);
      it.nrows = uint16_t(std::min<int64_t>(kRowsPerItem, B.ncols - c * kRowsPerItem));
      it.chunk = uint16_t(c);
      items.push_back(it);
      item_cost.push_back(double(it.nrows) * wsum + 64.0 * B.rank);
    }
    lrb.push_back(L);
    tbase += uint32_t(B.rank);
    part += uint32_t(nch * B.rank);
  }
  {
    std::vector<int64_t> ord(items.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return item_cost[a] > item_cost[b]; });
    std::vector<P1Item> s(items.size());
    for (size_t i = 0; i < ord.size(); ++i) s[i] = items[ord[i]];
    items.swap(s);
  }

  // ---- phase-2 owners (leaf row intervals <= 64 rows) and their contributions
  std::vector<Leaf> leaves;
  std::vector<Contrib> contribs;
  std::vector<double> leaf_cost;
  std::vector<std::vector<Contrib>> per_leaf;
  for (int64_t i = 0; i < nint; ++i) {
    std::vector<int64_t> bl = cover[i];
    std::sort(bl.begin(), bl.end());
    for (int64_t r0 = brk[i]; r0 < brk[i + 1]; r0 += kLeafRows) {
      int64_t nr = std::min<int64_t>(kLeafRows, brk[i + 1] - r0);
      std::vector<Contrib> cs;
      double cost = 0;
      uint32_t colbase = 0;
      for (int64_t b : bl) {
        const hlr_block_desc &B = d->blocks[b];
        Contrib c{};
        c.rowoff = uint32_t(r0 - B.row0);
        c.colbase = colbase;
        if (B.kind == HLR_DENSE) {
          c.kind = CONTRIB_DENSE;
          c.unit = uint32_t(blk_unit0[b]);
          c.ncols = uint32_t(B.ncols);
          c.ld = uint32_t(B.nrows);
          c.mbase = uint32_t(B.col0);
          cost += double(nr) * B.ncols * prm[c.unit].w;
        } else {
          if (B.rank == 0) continue;
          c.kind = CONTRIB_LOWRANK;
          c.unit = uint32_t(blk_unit0[b]);
          c.ncols = uint32_t(B.rank);
          c.ld = uint32_t(B.nrows);
          c.mbase = lrb[lr_of_block[b]].tbase;
          for (int k = 0; k < B.rank; ++k) cost += double(nr) * prm[c.unit + k].w;
        }
        colbase += c.ncols;
        cs.push_back(c);
      }
      Leaf L{uint32_t(r0), uint32_t(nr), 0, 0};
      leaves.push_back(L);
      leaf_cost.push_back(cost + 64.0 * cs.size());
      per_leaf.push_back(std::move(cs));
    }
  }
  {
    std::vector<int64_t> ord(leaves.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return leaf_cost[a] > leaf_cost[b]; });
    std::vector<Leaf> s;
    s.reserve(leaves.size());
    for (int64_t o : ord) {
      Leaf L = leaves[o];
      L.c0 = uint32_t(contribs.size());
      for (auto &c : per_leaf[o]) contribs.push_back(c);
      L.c1 = uint32_t(contribs.size());
      s.push_back(L);
    }
    leaves.swap(s);
  }

  // ---- arena layout
  auto H = std::make_unique<Handle>();
  cudaGetDevice(&H->device);
  H->format = d->format;
  size_t off = align_up(uoff[nunits] + 64, 256);
  size_t o_units = off;
  off = align_up(off + sizeof(UnitHdr) * nunits, 256);
  size_t o_sigma = off;
  off = align_up(off + 8 * size_t(rank_sum), 256);
  size_t o_lrb = off;
  off = align_up(off + sizeof(LRBlock) * lrb.size(), 256);
  size_t o_items = off;
  off = align_up(off + sizeof(P1Item) * items.size(), 256);
  size_t o_leaves = off;
  off = align_up(off + sizeof(Leaf) * leaves.size(), 256);
  size_t o_contribs = off;
  off = align_up(off + sizeof(Contrib) * contribs.size(), 256);
  size_t o_perm = off;
  off = align_up(off + 8 * size_t(n), 256);
  size_t image_bytes = off;  // everything above is copied from the host
  size_t o_x64 = off;
  off = align_up(off + 8 * size_t(n), 256);
  size_t o_x32 = off;
  off = align_up(off + 4 * size_t(n), 256);
  size_t o_t = off;
  off = align_up(off + 8 * size_t(rank_sum), 256);
  size_t o_part = off;
  off = align_up(off + 8 * size_t(part), 256);
  size_t o_cnt = off;
  off = align_up(off + 4 * (size_t(lrb.size()) + 8), 256);
  size_t o_xdev = off;
  off = align_up(off + 8 * size_t(n), 256);
  size_t o_ydev = off;
  off = align_up(off + 8 * size_t(n), 256);
  const size_t arena_bytes = off;
  if ((o_units >> 4) >= (uint64_t(1) << 40)) return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: arena too large");

  HostBuf img;
  img.p = static_cast<uint8_t *>(std::aligned_alloc(256, align_up(image_bytes, 256)));
  if (!img.p) return set_error(HLR_ERR_OOM, "hlr_upload: host staging allocation failed");
  uint8_t *P = img.p;
  std::memset(P + uoff[nunits], 0, o_units - uoff[nunits]);

  std::vector<UnitHdr> hdr(nunits);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t u = 0; u < nunits; ++u) {
    uint8_t *dst = P + uoff[u];
    std::memset(dst, 0, uoff[u + 1] - uoff[u]);
    if (afl)
      afl_pack(src[u].a, src[u].n, prm[u], dst);
    else
      std::memcpy(dst, src[u].a, size_t(src[u].n) * 8);
    UnitHdr h;
    h.m_min = prm[u].m_min;
    uint64_t o16 = uoff[u] >> 4;
    h.off_lo = uint32_t(o16 & 0xffffffffu);
    h.off_hi = uint8_t(o16 >> 32);
    h.e = uint8_t(prm[u].e);
    h.m = uint8_t(prm[u].m);
    h.w = uint8_t(prm[u].w);
    hdr[u] = h;
  }
  std::memcpy(P + o_units, hdr.data(), sizeof(UnitHdr) * nunits);
  {
    double *sg = reinterpret_cast<double *>(P + o_sigma);
    for (int64_t b = 0; b < nb; ++b) {
      const hlr_block_desc &B = d->blocks[b];
      if (lr_of_block[b] < 0) continue;
      std::memcpy(sg + lrb[lr_of_block[b]].tbase, B.sigma, 8 * size_t(B.rank));
    }
  }
  if (!lrb.empty()) std::memcpy(P + o_lrb, lrb.data(), sizeof(LRBlock) * lrb.size());
  if (!items.empty()) std::memcpy(P + o_items, items.data(), sizeof(P1Item) * items.size());
  std::memcpy(P + o_leaves, leaves.data(), sizeof(Leaf) * leaves.size());
  if (!contribs.empty()) std::memcpy(P + o_contribs, contribs.data(), sizeof(Contrib) * contribs.size());
  std::memcpy(P + o_perm, perm.data(), 8 * size_t(n));

  void *arena = nullptr;
  if (cudaMalloc(&arena, arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    return set_error(HLR_ERR_OOM, "hlr_upload: device allocation of " + std::to_string(arena_bytes) + " bytes failed");
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t ce = cudaMemcpyAsync(arena, P, image_bytes, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(static_cast<uint8_t *>(arena) + image_bytes, 0, arena_bytes - image_bytes, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    cudaFree(arena);
    return set_error(HLR_ERR_CUDA, std::string("hlr_upload: copy failed: ") + cudaGetErrorString(ce));
  }

  uint8_t *A = static_cast<uint8_t *>(arena);
  H->arena = arena;
  H->arena_bytes = arena_bytes;
  DevLayout &L = H->L;
  L.base = A;
  L.units = reinterpret_cast<const UnitHdr *>(A + o_units);
  L.sigma = reinterpret_cast<const double *>(A + o_sigma);
  L.lrb = reinterpret_cast<const LRBlock *>(A + o_lrb);
  L.items = reinterpret_cast<const P1Item *>(A + o_items);
  L.leaves = reinterpret_cast<const Leaf *>(A + o_leaves);
  L.contribs = reinterpret_cast<const Contrib *>(A + o_contribs);
  L.perm = reinterpret_cast<const int64_t *>(A + o_perm);
  L.xperm64 = reinterpret_cast<double *>(A + o_x64);
  L.xperm32 = reinterpret_cast<float *>(A + o_x32);
  L.t = reinterpret_cast<double *>(A + o_t);
  L.partial = reinterpret_cast<double *>(A + o_part);
  L.counters = reinterpret_cast<uint32_t *>(A + o_cnt);
  L.xdev = reinterpret_cast<double *>(A + o_xdev);
  L.ydev = reinterpret_cast<double *>(A + o_ydev);
  L.n = n;
  L.nlr = int32_t(lrb.size());
  L.nitems = int32_t(items.size());
  L.nleaves = int32_t(leaves.size());
  L.format = d->format;
  H->ncontribs = int64_t(contribs.size());
  H->part_total = part;
  H->nunits = nunits;
  H->values = values;
  H->scratch_off = o_x64;
  H->scratch_bytes = arena_bytes - o_x64;
  H->unit_hdr = hdr;
  H->unit_len.resize(nunits);
  H->unit_value_offset.resize(nunits + 1);
  H->unit_value_offset[0] = 0;
  for (int64_t u = 0; u < nunits; ++u) {
    H->unit_len[u] = src[u].n;
    H->unit_value_offset[u + 1] = H->unit_value_offset[u] + src[u].n;
  }

  hlr_info &I = H->info;
  I.n = n;
  I.nblocks = nb;
  I.ndense = ndense;
  I.nlowrank = nb - ndense;
  I.nunits = nunits;
  I.nleaves = int64_t(leaves.size());
  I.nitems = int64_t(items.size());
  I.rank_sum = rank_sum;
  I.values = values;
  I.fp64_bytes = uint64_t(values) * 8 + uint64_t(rank_sum) * 8;
  I.stream_bytes = stream_bytes;
  I.header_bytes = afl ? uint64_t(nunits) * sizeof(UnitHdr) : 0;
  I.algorithmic_bytes = stream_bytes + I.header_bytes + 8 * uint64_t(rank_sum) + 32 * uint64_t(n);
  I.device_bytes = arena_bytes;
  double fl = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.kind == HLR_DENSE)
      fl += 2.0 * double(B.nrows) * double(B.ncols);
    else
      fl += 2.0 * double(B.rank) * double(B.nrows + B.ncols);
  }
  I.flops = fl;
  {
    uint64_t xs = 0, nx = 0;
    for (const auto &L : lrb)
      for (int i = 0; i < L.k; ++i) {
        const int64_t u = int64_t(L.xunit0) + i;
        xs += afl ? afl_bytes(src[u].n, prm[u].w) : uint64_t(src[u].n) * 8;
        ++nx;
      }
    const uint64_t hb = afl ? sizeof(UnitHdr) : 0;
    I.phase1_bytes = xs + hb * nx + 16 * uint64_t(rank_sum) + 4 * uint64_t(n);
    I.phase2_bytes = (stream_bytes - xs) + hb * (uint64_t(nunits) - nx) + 8 * uint64_t(rank_sum) + 32 * uint64_t(n);
  }

  std::lock_guard<std::mutex> lk(g_mu);
  uint64_t id = g_next++;
  g_handles[id] = std::move(H);
  *out = id;
  if (device_bytes) *device_bytes = arena_bytes;
  return HLR_OK;
}

extern "C" int hlr_free(hlr_handle h) {
  std::unique_ptr<Handle> H;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_handles.find(h);
    if (it == g_handles.end()) return set_error(HLR_ERR_INVALID, "hlr_free: unknown handle");
    H = std::move(it->second);
    g_handles.erase(it);
  }
  cudaError_t ce = cudaDeviceSynchronize();
  if (H->arena) cudaFree(H->arena);
  if (H->cg_ws) cudaFree(H->cg_ws);
  for (void *e : H->prof_ev)
    if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
  if (ce != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string("hlr_free: ") + cudaGetErrorString(ce));
  return HLR_OK;
}

extern "C" int hlr_get_info(hlr_handle h, hlr_info *out) {
  Handle *H = lookup(h);
  if (!H || !out) return set_error(HLR_ERR_INVALID, "hlr_get_info: unknown handle or null output");
  *out = H->info;
  return HLR_OK;
}

extern "C" int hlr_matvec(hlr_handle h, const double *x, double *y, int flags, void *stream) {
  Handle *H = lookup(h);
  if (!H) return set_error(HLR_ERR_INVALID, "hlr_matvec: unknown handle");
  if (!x || !y) return set_error(HLR_ERR_INVALID, "hlr_matvec: null vector");
  const int acc = flags & ~HLR_PROFILE;
  if (acc != HLR_ACC_FP64 && acc != HLR_ACC_FP32) return set_error(HLR_ERR_INVALID, "hlr_matvec: bad flags");
  const int64_t n = H->L.n;
  const char *xb = reinterpret_cast<const char *>(x);
  const char *yb = reinterpret_cast<const char *>(y);
  if (xb < yb + 8 * n && yb < xb + 8 * n) return set_error(HLR_ERR_INVALID, "hlr_matvec: x and y overlap");
  return launch_matvec(*H, x, y, flags, stream);
}

extern "C" int hlr_decode_units(hlr_handle h, double *out, int64_t cap, void *stream) {
  Handle *H = lookup(h);
  if (!H || !out) return set_error(HLR_ERR_INVALID, "hlr_decode_units: unknown handle or null output");
  if (cap < H->values) return set_error(HLR_ERR_INVALID, "hlr_decode_units: output too small");
  return launch_decode_units(*H, out, stream);
}

extern "C" int hlr_afl_decode_device(const uint8_t *stream_dev, int64_t n, double m_min, int32_t e, int32_t m,
                                     double *out_dev, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!stream_dev || !out_dev))) return set_error(HLR_ERR_INVALID, "hlr_afl_decode_device: bad arguments");
  if (e < 0 || e > 11 || m < 0 || m > 52) return set_error(HLR_ERR_INVALID, "hlr_afl_decode_device: bad e or m");
  if (reinterpret_cast<uintptr_t>(stream_dev) & 15) return set_error(HLR_ERR_INVALID, "hlr_afl_decode_device: stream not 16-byte aligned");
  if (n == 0) return HLR_OK;
  return launch_decode_stream(stream_dev, n, m_min, e, m, out_dev, cuda_stream);
}

extern "C" int hlr_profile_read(hlr_handle h, double *kernel_ms, int *calls) {
  Handle *H = lookup(h);
  if (!H || !kernel_ms || !calls) return set_error(HLR_ERR_INVALID, "hlr_profile_read: bad arguments");
  return profile_read(*H, kernel_ms, calls);
}

extern "C" int hlr_matvec_host(hlr_handle h, const double *x, double *y, int flags, void *stream) {
  Handle *H = lookup(h);
  if (!H) return set_error(HLR_ERR_INVALID, "hlr_matvec_host: unknown handle");
  if (!x || !y) return set_error(HLR_ERR_INVALID, "hlr_matvec_host: null vector");
  const int acc = flags & ~HLR_PROFILE;
  if (acc != HLR_ACC_FP64 && acc != HLR_ACC_FP32) return set_error(HLR_ERR_INVALID, "hlr_matvec_host: bad flags");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = 8 * size_t(H->L.n);
  cudaError_t ce = cudaMemcpyAsync(H->L.xdev, x, bytes, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(H->L.ydev, y, bytes, cudaMemcpyHostToDevice, st);
  if (ce != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string("hlr_matvec_host: copy in: ") + cudaGetErrorString(ce));
  int rc = launch_matvec(*H, H->L.xdev, H->L.ydev, flags, stream);
  if (rc) return rc;
  ce = cudaMemcpyAsync(y, H->L.ydev, bytes, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string("hlr_matvec_host: ") + cudaGetErrorString(ce));
  return HLR_OK;
}
