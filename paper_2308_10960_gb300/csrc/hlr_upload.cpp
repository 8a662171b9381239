// hlr_upload / hlr_free / hlr_get_info / hlr_last_error / host entry points and the handle registry.
//
// Upload
//  1. validates the descriptor (shapes, exact coverage of I x I, permutation, finite data);
//  2. encodes every unit on the host: a dense block is one AFL unit at precision eps, a lowrank
//     block one unit per column of W and of X at precision eps sigma_0 / sigma_i (APLR, Section
//     3.3); the plain FP64 format stores the values as they are;
//  3. flattens the leaves of the block tree (Def. 2.2) into the two work lists of the product --
//     phase-1 items (<= 256 rows of the X columns of one lowrank block) and phase-2 leaves (row
//     intervals of <= 64 rows with every block covering them, in block order) -- assigns them to
//     the CTAs of the persistent kernels (longest task first onto the least loaded CTA) and
//     re-places the codes so that every CTA reads one contiguous run of pieces (hlr_pack.cpp);
//  4. copies the arena to the device.
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
#include "hlr_pack.h"

namespace hlr {

// Precision of a unit (Section 3.3). A dense leaf is one unit at the accuracy eps of Eq. 1 (the
// MP comparison format keeps dense leaves in FP64, i.e. any precision below 2^-53). Column i of
// a lowrank leaf W diag(sigma) X^T (W and X columns alike) gets the adaptive precision
// u_i = delta / sigma_i with delta = eps sigma_0, the truncation threshold of Eq. 1 in the
// spectral norm: the larger sigma_i, the more mantissa bits its columns keep.
double dense_precision(int format, double eps) { return format == HLR_FMT_MP ? 0x1p-60 : eps; }
double column_precision(double eps, double sigma0, double sigma_i) { return (eps * sigma0) / sigma_i; }

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

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct HostBuf {
  uint8_t *p = nullptr;
  ~HostBuf() { std::free(p); }
};

// Values up to which hlr_decode_units is available (its map costs 24 bytes per slice).
constexpr int64_t kDecodeMapMaxValues = int64_t(1) << 26;

// HLR_ENCODE_DEVICE: the units' parameters and canonical streams from the GPU encoder
// (hlr_encode_device) instead of the host's. The values go to the device through two pinned
// staging buffers (gathered by the host threads, copied while the next chunk is gathered); the
// parameters and streams come back into prm and a host buffer laid out as the host encoder
// lays it out (unit u at uoff[u], each stream padded to 16 bytes).
int encode_units_on_device(int fmt, const std::vector<const double *> &usrc, const std::vector<int64_t> &len,
                           const std::vector<double> &uprec, cudaStream_t st, std::vector<AflParams> *prm,
                           std::vector<uint64_t> *uoff, HostBuf *canon) {
  const int64_t nu = int64_t(usrc.size());
  std::vector<int64_t> voff(nu + 1, 0);
  for (int64_t u = 0; u < nu; ++u) voff[u + 1] = voff[u] + len[u];
  const int64_t total = voff[nu];
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t cap = 8 * size_t(total) + 16 * size_t(nu) + 64;
  const size_t b_a = al(8 * size_t(total) + 8), b_off = al(8 * size_t(nu + 1)), b_u = al(8 * size_t(nu)),
               b_mm = al(8 * size_t(nu)), b_e = al(4 * size_t(nu)), b_m = al(4 * size_t(nu)),
               b_oo = al(8 * size_t(nu + 1)), b_out = al(cap);
  uint8_t *d = nullptr;
  if (cudaMalloc(&d, b_a + b_off + b_u + b_mm + b_e + b_m + b_oo + b_out) != cudaSuccess) {
    cudaGetLastError();
    return set_error(HLR_ERR_OOM, "hlr_upload: device encoding buffers");
  }
  struct DevFree {
    uint8_t *p;
    ~DevFree() { cudaFree(p); }
  } dfree{d};
  double *a_dev = reinterpret_cast<double *>(d);
  int64_t *off_dev = reinterpret_cast<int64_t *>(d + b_a);
  double *u_dev = reinterpret_cast<double *>(d + b_a + b_off);
  double *mm_dev = reinterpret_cast<double *>(d + b_a + b_off + b_u);
  int32_t *e_dev = reinterpret_cast<int32_t *>(d + b_a + b_off + b_u + b_mm);
  int32_t *m_dev = reinterpret_cast<int32_t *>(d + b_a + b_off + b_u + b_mm + b_e);
  int64_t *oo_dev = reinterpret_cast<int64_t *>(d + b_a + b_off + b_u + b_mm + b_e + b_m);
  uint8_t *out_dev = d + b_a + b_off + b_u + b_mm + b_e + b_m + b_oo;
  // values, in chunks of kChunk doubles through two pinned buffers
  constexpr int64_t kChunk = int64_t(1) << 24;  // 128 MiB
  double *pin[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  auto release = [&]() {
    for (int k = 0; k < 2; ++k) {
      if (done[k]) cudaEventSynchronize(done[k]), cudaEventDestroy(done[k]);
      if (pin[k]) cudaFreeHost(pin[k]);
    }
  };
  for (int k = 0; k < 2; ++k)
    if (cudaMallocHost(reinterpret_cast<void **>(&pin[k]), size_t(kChunk) * 8) != cudaSuccess ||
        cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release();
      return set_error(HLR_ERR_OOM, "hlr_upload: pinned staging for device encoding");
    }
  int64_t u0 = 0;
  for (int64_t c0 = 0, k = 0; c0 < total; c0 += kChunk, k ^= 1) {
    const int64_t c1 = std::min(total, c0 + kChunk);
    cudaEventSynchronize(done[k]);  // the copy out of this buffer two chunks ago has finished
    while (voff[u0 + 1] <= c0) ++u0;
    int64_t u1 = u0;
    while (u1 < nu && voff[u1] < c1) ++u1;
    double *buf = pin[k];
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t u = u0; u < u1; ++u) {
      const int64_t lo = std::max(voff[u], c0), hi = std::min(voff[u + 1], c1);
      if (hi > lo) std::memcpy(buf + (lo - c0), usrc[u] + (lo - voff[u]), size_t(hi - lo) * 8);
    }
    if (cudaMemcpyAsync(a_dev + c0, buf, size_t(c1 - c0) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(done[k], st) != cudaSuccess) {
      release();
      return set_error(HLR_ERR_CUDA, "hlr_upload: copying values for device encoding");
    }
  }
  int rc = HLR_OK;
  if (cudaMemcpyAsync(off_dev, voff.data(), 8 * size_t(nu + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(u_dev, uprec.data(), 8 * size_t(nu), cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = set_error(HLR_ERR_CUDA, "hlr_upload: copying unit offsets for device encoding");
  if (!rc)
    rc = hlr_encode_device(fmt, nu, off_dev, total, a_dev, u_dev, mm_dev, e_dev, m_dev, oo_dev, out_dev, cap, st);
  std::vector<double> mm(nu);
  std::vector<int32_t> ee(nu), em(nu);
  std::vector<int64_t> oo(nu + 1);
  if (!rc && (cudaMemcpyAsync(mm.data(), mm_dev, 8 * size_t(nu), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaMemcpyAsync(ee.data(), e_dev, 4 * size_t(nu), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaMemcpyAsync(em.data(), m_dev, 4 * size_t(nu), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaMemcpyAsync(oo.data(), oo_dev, 8 * size_t(nu + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
              cudaStreamSynchronize(st) != cudaSuccess))
    rc = set_error(HLR_ERR_CUDA, "hlr_upload: reading device encoding results");
  release();
  if (rc) return rc;
  const int kind = fmt == HLR_FMT_BFL ? VF_BFL : fmt == HLR_FMT_DFL ? VF_DFL : fmt == HLR_FMT_MP ? VF_MP : VF_AFL;
  prm->resize(nu);
  uoff->assign(nu + 1, 0);
  for (int64_t u = 0; u < nu; ++u) {
    if (ee[u] < 0)
      return set_error(HLR_ERR_INVALID, "hlr_upload: NaN or Inf in block data (or beyond the format's range)");
    AflParams &q = (*prm)[u];
    q.m_min = mm[u];
    q.e = ee[u];
    q.m = em[u];
    q.w = 1 + ee[u] + em[u];
    q.kind = kind;
    (*uoff)[u + 1] = (*uoff)[u] + padded16(afl_bytes(len[u], q.w));
    if (int64_t((*uoff)[u]) != oo[u])
      return set_error(HLR_ERR_CUDA, "hlr_upload: device encoder offsets differ from the layout");
  }
  canon->p = static_cast<uint8_t *>(std::aligned_alloc(64, align_up((*uoff)[nu] + 64, 64)));
  if (!canon->p) return set_error(HLR_ERR_OOM, "hlr_upload: host allocation failed");
  std::memset(canon->p + (*uoff)[nu], 0, 64);
  if (cudaMemcpy(canon->p, out_dev, (*uoff)[nu], cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(HLR_ERR_CUDA, "hlr_upload: reading device encoded streams");
  return HLR_OK;
}

}  // namespace
}  // namespace hlr

using namespace hlr;

extern "C" const char *hlr_last_error(void) { return g_err.c_str(); }

extern "C" int hlr_upload(const hlr_hmatrix_desc *d, void *cuda_stream, hlr_handle *out,
                          size_t *device_bytes) {
  if (!d || !out) return set_error(HLR_ERR_INVALID, "hlr_upload: null descriptor or output");
  *out = 0;
  const int64_t n = d->n;
  if (n <= 0 || n > (int64_t(1) << 31) - 64) return set_error(HLR_ERR_INVALID, "hlr_upload: n out of range");
  if (d->nblocks <= 0 || !d->blocks) return set_error(HLR_ERR_INVALID, "hlr_upload: no blocks");
  if (d->format != HLR_FMT_AFL_APLR && d->format != HLR_FMT_FP64 && d->format != HLR_FMT_AFLP &&
      d->format != HLR_FMT_BFL && d->format != HLR_FMT_DFL && d->format != HLR_FMT_MP)
    return set_error(HLR_ERR_INVALID, "hlr_upload: unknown format");
  int sub_rows = kSubRows, leaf_rows = kLeafRows, piece_max = kPieceMax;
  if ((d->tuning >> 16) & ~0xf3) return set_error(HLR_ERR_INVALID, "hlr_upload: unknown tuning flags");
  const bool enc_dev = (d->tuning & HLR_ENCODE_DEVICE) != 0;
  const bool keep_map = (d->tuning & HLR_DECODE_MAP) != 0;
  const int ctas_sm = (d->tuning >> 20) & 15;  // HLR_CTAS_PER_SM; 0: as many as are resident
  if (ctas_sm > 8) return set_error(HLR_ERR_INVALID, "hlr_upload: bad tuning (HLR_CTAS_PER_SM above 8)");
  const int32_t layout = d->tuning & 0xffff;
  if (layout != 0) {
    const int sl = layout & 15, ll = (layout >> 4) & 15, kb = (layout >> 8) & 255;
    if (d->format == HLR_FMT_FP64 || sl < 5 || sl > 7 || ll < 5 || ll > 6 || kb < 4 || kb > kPieceMax / 1024)
      return set_error(HLR_ERR_INVALID, "hlr_upload: bad tuning (see HLR_TUNING; AFL format only)");
    sub_rows = 1 << sl;
    leaf_rows = 1 << ll;
    piece_max = kb * 1024;
  }
  const bool afl = d->format != HLR_FMT_FP64;  // one of the compressed formats
  if (afl && !(d->eps > 0.0 && d->eps < 1.0))
    return set_error(HLR_ERR_INVALID, "hlr_upload: eps must be in (0, 1)");

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
  int64_t ndense = 0, rank_sum = 0, values = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.row0 < 0 || B.col0 < 0 || B.nrows <= 0 || B.ncols <= 0 || B.row0 + B.nrows > n ||
        B.col0 + B.ncols > n)
      return set_error(HLR_ERR_INVALID, "hlr_upload: block " + std::to_string(b) + " out of range");
    if (B.kind == HLR_DENSE) {
      if (!B.D) return set_error(HLR_ERR_INVALID, "hlr_upload: dense block without data");
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
        rank_sum += B.rank;
        values += int64_t(B.rank) * (B.nrows + B.ncols);
      }
    } else {
      return set_error(HLR_ERR_INVALID, "hlr_upload: unknown block kind");
    }
  }
  if (rank_sum > (int64_t(1) << 31)) return set_error(HLR_ERR_UNSUPPORTED, "hlr_upload: total rank too large");

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

  // ---- units (canonical per-unit streams)
  PackInput in;
  in.n = n;
  in.raw = !afl;
  in.blocks = d->blocks;
  in.nblocks = nb;
  std::vector<const double *> usrc;
  std::vector<double> uprec;
  std::vector<char> rowside;  // dense and W units: their lanes hold a leaf's rows in phase 2
  in.blk_unit0.assign(nb, -1);
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.kind == HLR_DENSE) {
      in.blk_unit0[b] = int64_t(usrc.size());
      usrc.push_back(B.D);
      in.unit_len.push_back(B.nrows * B.ncols);
      uprec.push_back(dense_precision(d->format, d->eps));
      rowside.push_back(1);
    } else if (B.rank > 0) {
      in.blk_unit0[b] = int64_t(usrc.size());
      for (int i = 0; i < B.rank; ++i) {
        usrc.push_back(B.W + i * B.nrows);
        in.unit_len.push_back(B.nrows);
        uprec.push_back(column_precision(d->eps, B.sigma[0], B.sigma[i]));
        rowside.push_back(1);
      }
      for (int i = 0; i < B.rank; ++i) {
        usrc.push_back(B.X + i * B.ncols);
        in.unit_len.push_back(B.ncols);
        uprec.push_back(column_precision(d->eps, B.sigma[0], B.sigma[i]));
        rowside.push_back(0);
      }
    }
  }
  const int64_t nunits = int64_t(usrc.size());
  HostBuf canon;
  const bool on_device = afl && enc_dev && nunits > 0;
  if (on_device) {
    std::vector<uint64_t> uoff_dev;
    if (int rc = encode_units_on_device(d->format, usrc, in.unit_len, uprec, static_cast<cudaStream_t>(cuda_stream),
                                        &in.prm, &uoff_dev, &canon))
      return rc;
  } else {
    in.prm.resize(nunits);
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int64_t u = 0; u < nunits; ++u) {
    if (on_device) continue;
    if (afl) {
      if (!unit_params(d->format, usrc[u], in.unit_len[u], uprec[u], &in.prm[u])) bad |= 1;
    } else {
      for (int64_t j = 0; j < in.unit_len[u]; ++j)
        if (!std::isfinite(usrc[u][j])) bad |= 1;
      in.prm[u] = AflParams{1.0, 0, 0, 64, VF_AFL};
    }
  }
  if (bad) return set_error(HLR_ERR_INVALID, "hlr_upload: NaN or Inf in block data (or beyond the format's range)");
  // A phase-2 lane holds one column over the task's rows, in a warp region of 32 such lanes:
  // 64 rows of 64-bit codes (FP64 values of MP, DFL at m' = 52) make a 16 KiB region, more than
  // a piece holds with its headers, so the default layout then takes tasks of 32 rows.
  if (afl && layout == 0) {
    for (int64_t u = 0; u < nunits; ++u)
      if (rowside[u] && 64 + 128 * ((int64_t(in.prm[u].w) * kLeafRows + 31) / 32) > int64_t(piece_max)) {
        leaf_rows = kLeafRows / 2;
        break;
      }
  }
  in.uoff.assign(nunits + 1, 0);
  uint64_t stream_bytes = 0;
  for (int64_t u = 0; u < nunits; ++u) {
    size_t bytes = afl_bytes(in.unit_len[u], in.prm[u].w);
    stream_bytes += bytes;
    in.uoff[u + 1] = in.uoff[u] + padded16(bytes);
  }
  if (!on_device) {
    canon.p = static_cast<uint8_t *>(std::aligned_alloc(64, align_up(in.uoff[nunits] + 64, 64)));
    if (!canon.p) return set_error(HLR_ERR_OOM, "hlr_upload: host allocation failed");
    std::memset(canon.p + in.uoff[nunits], 0, 64);
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t u = 0; u < nunits; ++u) {
    if (on_device) continue;  // the device encoder wrote the streams, zero-padded to 16 bytes
    uint8_t *dst = canon.p + in.uoff[u];
    std::memset(dst, 0, in.uoff[u + 1] - in.uoff[u]);
    if (afl)
      unit_pack(usrc[u], in.unit_len[u], in.prm[u], dst);
    else
      std::memcpy(dst, usrc[u], size_t(in.unit_len[u]) * 8);
  }
  in.canon = canon.p;

  // ---- work lists
  in.cover = &cover;
  in.brk = &brk;
  in.sub_rows = sub_rows;
  in.leaf_rows = leaf_rows;
  in.piece_max = piece_max;
  int dev = 0;
  cudaGetDevice(&dev);
  int nct[2] = {0, 0};
  if (ctas_per_phase(dev, nct) <= 0) return set_error(HLR_ERR_CUDA, "hlr_upload: cannot query the device");
  if (ctas_sm > 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int p = 0; p < 2; ++p) nct[p] = std::min(nct[p], std::max(1, sms) * ctas_sm);
  }
  PackOutput po;
  const bool want_map = keep_map || values <= kDecodeMapMaxValues;
  int rc = pack_work(in, nct, want_map, &po);
  if (rc) return rc;

  // ---- arena layout
  auto H = std::make_unique<Handle>();
  H->device = dev;
  H->format = d->format;
  size_t off = 0;
  const size_t o_ph0 = off;
  off = align_up(off + po.ph[0].bytes.size() + 512, 256);  // lane-column reads run up to 252 B past a piece
  const size_t o_ph1 = off;
  off = align_up(off + po.ph[1].bytes.size() + 512, 256);
  // issue streams: per piece one descriptor, then its aux copies (offsets filled in below)
  std::vector<IssueEnt> ent[2];
  std::vector<uint32_t> cta_e0[2], cta_np[2];
  for (int p = 0; p < 2; ++p) {
    const PhaseOut &ph = po.ph[p];
    for (int q = 0; q < nct[p]; ++q) {
      cta_e0[p].push_back(uint32_t(ent[p].size()));
      cta_np[p].push_back(ph.cta_p0[q + 1] - ph.cta_p0[q]);
      for (uint32_t k = ph.cta_p0[q]; k < ph.cta_p0[q + 1]; ++k) {
        uint32_t nel = 0;
        for (uint32_t a = ph.aux_idx[k]; a < ph.aux_idx[k + 1]; ++a) nel += ph.aux[a].nelem;
        IssueEnt e{};
        const uint64_t rel = ph.piece_off[k];  // relative to the region; made absolute below
        e.a = uint32_t(rel & 0xffffffffu);
        e.b = uint32_t(rel >> 32) | kIssuePiece;
        e.c = uint32_t(ph.piece_off[k + 1] - ph.piece_off[k]);
        e.d = nel;
        ent[p].push_back(e);
        for (uint32_t a = ph.aux_idx[k]; a < ph.aux_idx[k + 1]; ++a) {
          const AuxCopy &c = ph.aux[a];
          ent[p].push_back(IssueEnt{c.elem0, uint32_t(c.nelem) | (uint32_t(c.which) << 16), c.soff, 0});
        }
      }
    }
    cta_e0[p].push_back(uint32_t(ent[p].size()));
  }
  size_t o_meta[2][3];
  for (int p = 0; p < 2; ++p) {
    o_meta[p][0] = off;
    off = align_up(off + sizeof(IssueEnt) * (ent[p].size() + 32), 256);
    o_meta[p][1] = off;
    off = align_up(off + 4 * cta_e0[p].size(), 256);
    o_meta[p][2] = off;
    off = align_up(off + 4 * cta_np[p].size(), 256);
  }
  const size_t o_fac64 = off;
  off = align_up(off + 8 * (size_t(rank_sum) + 8), 256);
  const size_t o_fac32 = off;
  off = align_up(off + 4 * (size_t(rank_sum) + 8), 256);
  const size_t o_comb = off;
  off = align_up(off + sizeof(Combine) * po.comb.size() + 16, 256);
  const size_t o_perm = off;
  off = align_up(off + 8 * size_t(n), 256);
  const size_t image_bytes = off;  // everything above is copied from the host
  const size_t o_x64 = off;
  off = align_up(off + 8 * (size_t(n) + 8), 256);
  const size_t o_x32 = off;
  off = align_up(off + 4 * (size_t(n) + 8), 256);
  const size_t o_tw64 = off;
  off = align_up(off + 8 * (size_t(rank_sum) + 8), 256);
  const size_t o_tw32 = off;
  off = align_up(off + 4 * (size_t(rank_sum) + 8), 256);
  const size_t o_part = off;
  off = align_up(off + 8 * size_t(po.part_total) + 8, 256);
  const size_t o_ysum = off;
  off = align_up(off + 8 * (size_t(n) + 8), 256);
  const size_t o_status = off;
  off = align_up(off + 64, 256);
  const size_t o_xdev = off;
  off = align_up(off + 8 * size_t(n), 256);
  const size_t o_ydev = off;
  off = align_up(off + 8 * size_t(n), 256);
  const size_t arena_bytes = off;

  HostBuf img;
  img.p = static_cast<uint8_t *>(std::aligned_alloc(256, align_up(image_bytes, 256)));
  if (!img.p) return set_error(HLR_ERR_OOM, "hlr_upload: host staging allocation failed");
  uint8_t *P = img.p;
  std::memset(P, 0, image_bytes);
  std::memcpy(P + o_ph0, po.ph[0].bytes.data(), po.ph[0].bytes.size());
  std::memcpy(P + o_ph1, po.ph[1].bytes.data(), po.ph[1].bytes.size());
  const size_t o_ph[2] = {o_ph0, o_ph1};
  for (int p = 0; p < 2; ++p) {
    for (auto &e : ent[p]) {
      if (!(e.b & kIssuePiece)) continue;
      const uint64_t abs = ((uint64_t(e.b & ~kIssuePiece) << 32) | e.a) + o_ph[p];
      e.a = uint32_t(abs & 0xffffffffu);
      e.b = uint32_t(abs >> 32) | kIssuePiece;
    }
    if (!ent[p].empty()) std::memcpy(P + o_meta[p][0], ent[p].data(), sizeof(IssueEnt) * ent[p].size());
    std::memcpy(P + o_meta[p][1], cta_e0[p].data(), 4 * cta_e0[p].size());
    std::memcpy(P + o_meta[p][2], cta_np[p].data(), 4 * cta_np[p].size());
  }
  if (rank_sum) {
    std::memcpy(P + o_fac64, po.fac.data(), 8 * po.fac.size());
    float *f32 = reinterpret_cast<float *>(P + o_fac32);
    for (size_t i = 0; i < po.fac.size(); ++i) f32[i] = float(po.fac[i]);
  }
  if (!po.comb.empty()) std::memcpy(P + o_comb, po.comb.data(), sizeof(Combine) * po.comb.size());
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
  L.perm = reinterpret_cast<const int64_t *>(A + o_perm);
  L.fac64 = reinterpret_cast<const double *>(A + o_fac64);
  L.fac32 = reinterpret_cast<const float *>(A + o_fac32);
  for (int p = 0; p < 2; ++p) {
    L.ph[p].ent = reinterpret_cast<const IssueEnt *>(A + o_meta[p][0]);
    L.ph[p].cta_e0 = reinterpret_cast<const uint32_t *>(A + o_meta[p][1]);
    L.ph[p].cta_np = reinterpret_cast<const uint32_t *>(A + o_meta[p][2]);
    L.ph[p].nct = nct[p];
    L.ph[p].np = int32_t(po.ph[p].piece_off.size()) - 1;
  }
  L.xperm64 = reinterpret_cast<double *>(A + o_x64);
  L.xperm32 = reinterpret_cast<float *>(A + o_x32);
  L.tw64 = reinterpret_cast<double *>(A + o_tw64);
  L.tw32 = reinterpret_cast<float *>(A + o_tw32);
  L.partial = reinterpret_cast<double *>(A + o_part);
  L.ysum = reinterpret_cast<double *>(A + o_ysum);
  L.comb = reinterpret_cast<const Combine *>(A + o_comb);
  L.status = reinterpret_cast<uint32_t *>(A + o_status);
  L.xdev = reinterpret_cast<double *>(A + o_xdev);
  L.ydev = reinterpret_cast<double *>(A + o_ydev);
  L.n = n;
  L.ncnt = int32_t(po.ncnt);
  L.raw = afl ? 0 : 1;
  L.vfmt = d->format == HLR_FMT_BFL ? VF_BFL : d->format == HLR_FMT_DFL ? VF_DFL : d->format == HLR_FMT_MP ? VF_MP : VF_AFL;
  H->nunits = nunits;
  H->values = values;
  H->part_total = po.part_total;
  if (want_map) {
    H->slice_src = std::move(po.slice_src);
    H->slice_dst = std::move(po.slice_dst);
    H->slice_n = std::move(po.slice_n);
    H->slice_unit = std::move(po.slice_unit);
    for (size_t i = 0; i < H->slice_src.size(); ++i) {
      const uint64_t v = H->slice_src[i];
      const uint64_t ph = v >> 63;                   // phase tag
      const uint64_t strided = v & kStridedSlice;    // lane-column slice (bank-column piece)
      const uint64_t addr = v & (kStridedSlice - 1);
      H->slice_src[i] = (addr + 8 * uint64_t(ph ? o_ph1 : o_ph0)) | strided;
    }
    H->unit_mmin.resize(nunits);
    H->unit_e.resize(nunits);
    H->unit_m.resize(nunits);
    for (int64_t u = 0; u < nunits; ++u) {
      H->unit_mmin[u] = in.prm[u].m_min;
      H->unit_e[u] = uint8_t(in.prm[u].e);
      H->unit_m[u] = uint8_t(in.prm[u].m);
    }
  }

  hlr_info &I = H->info;
  I.n = n;
  I.nblocks = nb;
  I.ndense = ndense;
  I.nlowrank = nb - ndense;
  I.nunits = nunits;
  I.nleaves = po.nleaves;
  I.nitems = po.nitems;
  I.rank_sum = rank_sum;
  I.values = values;
  I.fp64_bytes = uint64_t(values) * 8 + uint64_t(rank_sum) * 8;
  I.stream_bytes = stream_bytes;
  I.header_bytes = afl ? uint64_t(nunits) * 16 : 0;
  I.algorithmic_bytes = stream_bytes + I.header_bytes + 8 * uint64_t(rank_sum) + 32 * uint64_t(n);
  I.device_bytes = arena_bytes;
  double fl = 0;
  uint64_t xs = 0, nx = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.kind == HLR_DENSE) {
      fl += 2.0 * double(B.nrows) * double(B.ncols);
    } else {
      fl += 2.0 * double(B.rank) * double(B.nrows + B.ncols);
      for (int i = 0; i < B.rank; ++i) {
        const int64_t u = in.blk_unit0[b] + B.rank + i;
        xs += afl_bytes(in.unit_len[u], in.prm[u].w);
        ++nx;
      }
    }
  }
  I.flops = fl;
  const uint64_t hb = afl ? 16 : 0;
  I.phase1_bytes = xs + hb * nx + 16 * uint64_t(rank_sum) + 4 * uint64_t(n);
  // the FP32-accumulation product of the AFL and AFLP formats adds its phase-2 row sums into y
  // in one more kernel
  I.launches = 1 + (po.ph[0].piece_off.size() > 1) + (po.ncnt > 0) + (po.ph[1].piece_off.size() > 1) +
               ((afl && L.vfmt == VF_AFL && po.ph[1].piece_off.size() > 1) ? 1 : 0);
  I.phase2_bytes = (stream_bytes - xs) + hb * (uint64_t(nunits) - nx) + 8 * uint64_t(rank_sum) + 32 * uint64_t(n);

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
  if (H->multi_ws) cudaFree(H->multi_ws);
  for (void *w : H->col_ws) cudaFree(w);
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
  const int acc = flags & ~(HLR_PROFILE | HLR_SM_SHARE(15));
  if ((acc != HLR_ACC_FP64 && acc != HLR_ACC_FP32) || ((flags >> 16) & 15) > 8)
    return set_error(HLR_ERR_INVALID, "hlr_matvec: bad flags");
  const int64_t n = H->L.n;
  const char *xb = reinterpret_cast<const char *>(x);
  const char *yb = reinterpret_cast<const char *>(y);
  if (xb < yb + 8 * n && yb < xb + 8 * n) return set_error(HLR_ERR_INVALID, "hlr_matvec: x and y overlap");
  return launch_matvec(*H, x, y, flags, stream);
}

extern "C" int hlr_check(hlr_handle h, void *stream) {
  Handle *H = lookup(h);
  if (!H) return set_error(HLR_ERR_INVALID, "hlr_check: unknown handle");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t s[4] = {0, 0, 0, 0};
  cudaError_t ce = cudaMemcpyAsync(s, H->L.status, sizeof(s), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string("hlr_check: ") + cudaGetErrorString(ce));
  if (s[0] | s[1] | s[2] | s[3]) {
    cudaMemsetAsync(H->L.status, 0, sizeof(s), st);
    cudaStreamSynchronize(st);
    return set_error(HLR_ERR_TIMEOUT, "hlr_check: a device-side wait ran out of time (status " +
                                          std::to_string(s[0]) + ")");
  }
  return HLR_OK;
}

extern "C" int hlr_selftest_wait(hlr_handle h, int64_t cycles, void *stream) {
  Handle *H = lookup(h);
  if (!H) return set_error(HLR_ERR_INVALID, "hlr_selftest_wait: unknown handle");
  if (cycles < 1000 || cycles > (int64_t(1) << 31))
    return set_error(HLR_ERR_INVALID, "hlr_selftest_wait: cycles must be in [1000, 2^31]");
  return launch_wait_expire(*H, static_cast<long long>(cycles), stream);
}

extern "C" int hlr_decode_units(hlr_handle h, double *out, int64_t cap, void *stream) {
  Handle *H = lookup(h);
  if (!H || !out) return set_error(HLR_ERR_INVALID, "hlr_decode_units: unknown handle or null output");
  if (cap < H->values) return set_error(HLR_ERR_INVALID, "hlr_decode_units: output too small");
  if (H->values > 0 && H->slice_src.empty())
    return set_error(HLR_ERR_UNSUPPORTED, "hlr_decode_units: only for matrices of at most 2^26 values");
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
  const int acc = flags & ~(HLR_PROFILE | HLR_SM_SHARE(15));
  if ((acc != HLR_ACC_FP64 && acc != HLR_ACC_FP32) || ((flags >> 16) & 15) > 8)
    return set_error(HLR_ERR_INVALID, "hlr_matvec_host: bad flags");
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

extern "C" int hlr_unit_list(const hlr_hmatrix_desc *d, int64_t *off, double *prec, double *values, int64_t cap_units,
                             int64_t cap_values, int64_t *nunits, int64_t *nvalues) {
  using namespace hlr;
  if (!d || (d->nblocks > 0 && !d->blocks) || d->nblocks < 0 || !nunits || !nvalues)
    return set_error(HLR_ERR_INVALID, "hlr_unit_list: bad arguments");
  const bool afl = d->format != HLR_FMT_FP64;
  if (afl && !(d->eps > 0.0 && d->eps < 1.0)) return set_error(HLR_ERR_INVALID, "hlr_unit_list: eps must be in (0, 1)");
  int64_t nu = 0, nv = 0;
  for (int64_t b = 0; b < d->nblocks; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.nrows < 0 || B.ncols < 0) return set_error(HLR_ERR_INVALID, "hlr_unit_list: negative block size");
    if (B.kind == HLR_DENSE) {
      if (!B.D && B.nrows * B.ncols > 0) return set_error(HLR_ERR_INVALID, "hlr_unit_list: dense block without data");
      nu += 1;
      nv += B.nrows * B.ncols;
    } else if (B.kind == HLR_LOWRANK) {
      if (B.rank < 0 || B.rank > std::min(B.nrows, B.ncols))
        return set_error(HLR_ERR_INVALID, "hlr_unit_list: bad rank in block " + std::to_string(b));
      if (B.rank > 0 && (!B.W || !B.X || !B.sigma))
        return set_error(HLR_ERR_INVALID, "hlr_unit_list: lowrank block without factors");
      for (int i = 0; i < B.rank; ++i)
        if (!(B.sigma[i] > 0.0) || !std::isfinite(B.sigma[i]) || B.sigma[i] > B.sigma[0])
          return set_error(HLR_ERR_INVALID, "hlr_unit_list: sigma must be positive, finite and led by its maximum");
      nu += 2 * int64_t(B.rank);
      nv += int64_t(B.rank) * (B.nrows + B.ncols);
    } else {
      return set_error(HLR_ERR_INVALID, "hlr_unit_list: unknown block kind");
    }
  }
  *nunits = nu;
  *nvalues = nv;
  if ((off && cap_units < nu + 1) || (prec && cap_units < nu) || (values && cap_values < nv))
    return set_error(HLR_ERR_OOM, "hlr_unit_list: output arrays too small");
  int64_t u = 0, v = 0;
  auto put = [&](const double *src, int64_t len, double p) {
    if (off) off[u] = v;
    if (prec) prec[u] = p;
    if (values && len > 0) std::memcpy(values + v, src, size_t(len) * 8);
    ++u;
    v += len;
  };
  for (int64_t b = 0; b < d->nblocks; ++b) {
    const hlr_block_desc &B = d->blocks[b];
    if (B.kind == HLR_DENSE) {
      put(B.D, B.nrows * B.ncols, dense_precision(d->format, d->eps));
    } else {
      for (int i = 0; i < B.rank; ++i) put(B.W + i * B.nrows, B.nrows, column_precision(d->eps, B.sigma[0], B.sigma[i]));
      for (int i = 0; i < B.rank; ++i) put(B.X + i * B.ncols, B.ncols, column_precision(d->eps, B.sigma[0], B.sigma[i]));
    }
  }
  if (off) off[u] = v;
  return HLR_OK;
}
