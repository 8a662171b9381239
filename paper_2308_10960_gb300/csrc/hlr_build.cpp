// Host construction of kernel H-matrices (hlr_build): the input of hlr_upload.
//
//  * cluster tree (Def. 2.1): bounding-box bisection -- cut at the midpoint of the longest
//    box edge (first axis on ties), coordinate <= midpoint to the first son in the father's
//    order; if a side would be empty, split at the median of (coordinate, index); clusters of
//    at most leaf_size indices are leaves;
//  * block tree (Def. 2.2) with standard admissibility min(diam t, diam s) <= eta dist(t, s)
//    (Section 5.1), diam = box diagonal, dist = distance between boxes;
//  * dense leaves are evaluated; admissible leaves are approximated by ACA with partial
//    pivoting (first pivot row 0, next pivot row = largest entry of the newest column among
//    unused rows, stop after a term with ||u|| ||v|| <= eps/10 ||S||_F, at most
//    min(#t, #s)/2 terms, else a full SVD) and recompressed as in Algorithm 1 (QR of both
//    factors, SVD of R_U R_V^T) with sigma_i > eps sigma_0 kept; Sigma stays separate from W.
// Compiled with -ffp-contract=off so the geometric predicates round like plain IEEE code.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "hlr_internal.h"

struct hlr_host_hmatrix {
  int64_t n = 0;
  double eps = 0;
  std::vector<int64_t> perm;
  struct Blk {
    int64_t row0, nrows, col0, ncols;
    int kind, rank;
    std::vector<double> D, W, S, X;
  };
  std::vector<Blk> blocks;
  std::vector<hlr_block_desc> descs;
};

namespace {

using hlr::set_error;

struct Kern {
  int kind, dim;
  const double *P;
  double scale, diag;
  double operator()(int64_t i, int64_t j) const {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
      double df = P[i * dim + d] - P[j * dim + d];
      s += df * df;
    }
    const double r = std::sqrt(s);
    switch (kind) {
      case HLR_KERNEL_EXP:
        return std::exp(-r / scale) + (i == j ? diag : 0.0);
      case HLR_KERNEL_LAPLACE:
        return i == j ? diag : 1.0 / (4.0 * M_PI * r);
      default: {
        const double a = std::sqrt(3.0) * r / scale;
        return (1.0 + a) * std::exp(-a) + (i == j ? diag : 0.0);
      }
    }
  }
};

struct Cl {
  int64_t lo, hi;
  double bmin[3], bmax[3];
  int64_t son[2] = {-1, -1};
};

struct Tree {
  const double *P;
  int dim;
  int leaf;
  std::vector<int64_t> perm;
  std::vector<Cl> nodes;

  int64_t build(int64_t lo, int64_t hi) {
    Cl c;
    c.lo = lo;
    c.hi = hi;
    for (int d = 0; d < dim; ++d) {
      c.bmin[d] = INFINITY;
      c.bmax[d] = -INFINITY;
    }
    for (int64_t k = lo; k < hi; ++k)
      for (int d = 0; d < dim; ++d) {
        double v = P[perm[k] * dim + d];
        c.bmin[d] = std::min(c.bmin[d], v);
        c.bmax[d] = std::max(c.bmax[d], v);
      }
    int64_t id = int64_t(nodes.size());
    nodes.push_back(c);
    if (hi - lo <= leaf) return id;
    int dd = 0;
    double best = c.bmax[0] - c.bmin[0];
    for (int d = 1; d < dim; ++d) {
      double e = c.bmax[d] - c.bmin[d];
      if (e > best) {
        best = e;
        dd = d;
      }
    }
    const double mid = 0.5 * (c.bmin[dd] + c.bmax[dd]);
    std::vector<int64_t> a, b;
    a.reserve(hi - lo);
    b.reserve(hi - lo);
    for (int64_t k = lo; k < hi; ++k) (P[perm[k] * dim + dd] <= mid ? a : b).push_back(perm[k]);
    int64_t nfirst = int64_t(a.size());
    if (nfirst == 0 || nfirst == hi - lo) {
      std::vector<int64_t> idx(perm.begin() + lo, perm.begin() + hi);
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
        double cx = P[x * dim + dd], cy = P[y * dim + dd];
        if (cx != cy) return cx < cy;
        return x < y;
      });
      std::copy(idx.begin(), idx.end(), perm.begin() + lo);
      nfirst = (hi - lo) / 2;
    } else {
      std::copy(a.begin(), a.end(), perm.begin() + lo);
      std::copy(b.begin(), b.end(), perm.begin() + lo + nfirst);
    }
    int64_t s0 = build(lo, lo + nfirst);
    int64_t s1 = build(lo + nfirst, hi);
    nodes[id].son[0] = s0;
    nodes[id].son[1] = s1;
    return id;
  }

  double diam(const Cl &c) const {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
      double e = c.bmax[d] - c.bmin[d];
      s += e * e;
    }
    return std::sqrt(s);
  }
  double dist(const Cl &a, const Cl &b) const {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
      double g = std::max(0.0, std::max(b.bmin[d] - a.bmax[d], a.bmin[d] - b.bmax[d]));
      s += g * g;
    }
    return std::sqrt(s);
  }
};

struct Leaf {
  int64_t t, s;
  bool adm;
};

void block_tree(const Tree &T, double eta, int64_t t, int64_t s, std::vector<Leaf> &out) {
  const Cl &a = T.nodes[t], &b = T.nodes[s];
  if (std::min(T.diam(a), T.diam(b)) <= eta * T.dist(a, b)) {
    out.push_back({t, s, true});
  } else if (a.son[0] < 0 || b.son[0] < 0) {
    out.push_back({t, s, false});
  } else {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) block_tree(T, eta, a.son[i], b.son[j], out);
  }
}

// ---- small dense linear algebra (column-major) ------------------------------------------------

// Thin Householder QR of A (m x k, m >= k): Q (m x k) with orthonormal columns, R (k x k).
void qr_thin(int64_t m, int64_t k, std::vector<double> A, std::vector<double> &Q, std::vector<double> &R) {
  std::vector<double> vs(size_t(m) * k, 0.0), beta(k, 0.0);
  for (int64_t j = 0; j < k; ++j) {
    double *a = &A[size_t(j) * m];
    double nrm = 0.0;
    for (int64_t i = j; i < m; ++i) nrm += a[i] * a[i];
    nrm = std::sqrt(nrm);
    double *v = &vs[size_t(j) * m];
    if (nrm == 0.0) {
      beta[j] = 0.0;
      continue;
    }
    const double alpha = a[j] >= 0 ? -nrm : nrm;
    for (int64_t i = j; i < m; ++i) v[i] = a[i];
    v[j] -= alpha;
    double vn = 0.0;
    for (int64_t i = j; i < m; ++i) vn += v[i] * v[i];
    beta[j] = vn > 0 ? 2.0 / vn : 0.0;
    for (int64_t c = j; c < k; ++c) {
      double *ac = &A[size_t(c) * m];
      double dot = 0.0;
      for (int64_t i = j; i < m; ++i) dot += v[i] * ac[i];
      dot *= beta[j];
      for (int64_t i = j; i < m; ++i) ac[i] -= dot * v[i];
    }
  }
  R.assign(size_t(k) * k, 0.0);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r <= c; ++r) R[r + c * k] = A[r + size_t(c) * m];
  Q.assign(size_t(m) * k, 0.0);
  for (int64_t c = 0; c < k; ++c) Q[c + size_t(c) * m] = 1.0;
  for (int64_t j = k - 1; j >= 0; --j) {
    const double *v = &vs[size_t(j) * m];
    if (beta[j] == 0.0) continue;
    for (int64_t c = 0; c < k; ++c) {
      double *qc = &Q[size_t(c) * m];
      double dot = 0.0;
      for (int64_t i = j; i < m; ++i) dot += v[i] * qc[i];
      dot *= beta[j];
      for (int64_t i = j; i < m; ++i) qc[i] -= dot * v[i];
    }
  }
}

// One-sided Jacobi SVD of A (m x n, m >= n): A = U diag(s) V^T, s descending.
void svd_jacobi(int64_t m, int64_t n, std::vector<double> A, std::vector<double> &U, std::vector<double> &s,
                std::vector<double> &V) {
  V.assign(size_t(n) * n, 0.0);
  for (int64_t i = 0; i < n; ++i) V[i + size_t(i) * n] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int64_t p = 0; p < n - 1; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        double *ap = &A[size_t(p) * m], *aq = &A[size_t(q) * m];
        double al = 0, be = 0, ga = 0;
        for (int64_t i = 0; i < m; ++i) {
          al += ap[i] * ap[i];
          be += aq[i] * aq[i];
          ga += ap[i] * aq[i];
        }
        if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
        rotated = true;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int64_t i = 0; i < m; ++i) {
          const double x = ap[i], y = aq[i];
          ap[i] = c * x - sn * y;
          aq[i] = sn * x + c * y;
        }
        double *vp = &V[size_t(p) * n], *vq = &V[size_t(q) * n];
        for (int64_t i = 0; i < n; ++i) {
          const double x = vp[i], y = vq[i];
          vp[i] = c * x - sn * y;
          vq[i] = sn * x + c * y;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> nr(n);
  for (int64_t j = 0; j < n; ++j) {
    double ss = 0;
    for (int64_t i = 0; i < m; ++i) ss += A[i + size_t(j) * m] * A[i + size_t(j) * m];
    nr[j] = std::sqrt(ss);
  }
  std::vector<int64_t> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return nr[a] > nr[b]; });
  U.assign(size_t(m) * n, 0.0);
  s.assign(n, 0.0);
  std::vector<double> V2(size_t(n) * n);
  for (int64_t jj = 0; jj < n; ++jj) {
    const int64_t j = ord[jj];
    s[jj] = nr[j];
    for (int64_t i = 0; i < m; ++i) U[i + size_t(jj) * m] = nr[j] > 0 ? A[i + size_t(j) * m] / nr[j] : 0.0;
    for (int64_t i = 0; i < n; ++i) V2[i + size_t(jj) * n] = V[i + size_t(j) * n];
  }
  V.swap(V2);
}

int trunc_rank(const std::vector<double> &s, double eps) {
  if (s.empty() || s[0] == 0.0) return 0;
  int k = 0;
  for (double v : s)
    if (v > eps * s[0]) ++k;
  return k;
}

// Truncated SVD of a full block M (m x n): W (m x k), S, X (n x k).
void lowrank_dense_svd(int64_t m, int64_t n, const std::vector<double> &M, double eps, hlr_host_hmatrix::Blk &B) {
  std::vector<double> U, s, V;
  if (m >= n) {
    svd_jacobi(m, n, M, U, s, V);
  } else {
    std::vector<double> Mt(size_t(m) * n);
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) Mt[j + size_t(i) * n] = M[i + size_t(j) * m];
    svd_jacobi(n, m, Mt, V, s, U);  // M^T = V s U^T
  }
  const int k = trunc_rank(s, eps);
  const int64_t kk = int64_t(s.size());
  B.rank = k;
  B.S.assign(s.begin(), s.begin() + k);
  B.W.assign(U.begin(), U.begin() + size_t(m) * k);
  B.X.assign(V.begin(), V.begin() + size_t(n) * k);
  (void)kk;
}

// ACA with partial pivoting; returns false if the term cap was reached.
bool aca(const Kern &K, const int64_t *I, int64_t m, const int64_t *J, int64_t n, double eps_aca, int64_t cap,
         std::vector<std::vector<double>> &us, std::vector<std::vector<double>> &vs) {
  std::vector<char> used(m, 0);
  double norm2 = 0.0;
  int64_t i = 0;
  std::vector<double> row(n), col(m);
  for (;;) {
    if (int64_t(us.size()) >= cap) return false;
    used[i] = 1;
    for (int64_t j = 0; j < n; ++j) row[j] = K(I[i], J[j]);
    for (size_t l = 0; l < us.size(); ++l) {
      const double ui = us[l][i];
      const double *v = vs[l].data();
      for (int64_t j = 0; j < n; ++j) row[j] = row[j] - ui * v[j];
    }
    int64_t jp = 0;
    double best = std::fabs(row[0]);
    for (int64_t j = 1; j < n; ++j)
      if (std::fabs(row[j]) > best) {
        best = std::fabs(row[j]);
        jp = j;
      }
    if (row[jp] == 0.0) {
      int64_t nxt = -1;
      for (int64_t r = 0; r < m; ++r)
        if (!used[r]) {
          nxt = r;
          break;
        }
      if (nxt < 0) break;
      i = nxt;
      continue;
    }
    std::vector<double> v(n), u(m);
    const double piv = row[jp];
    for (int64_t j = 0; j < n; ++j) v[j] = row[j] / piv;
    for (int64_t r = 0; r < m; ++r) col[r] = K(I[r], J[jp]);
    for (size_t l = 0; l < us.size(); ++l) {
      const double vj = vs[l][jp];
      const double *ul = us[l].data();
      for (int64_t r = 0; r < m; ++r) col[r] = col[r] - vj * ul[r];
    }
    for (int64_t r = 0; r < m; ++r) u[r] = col[r];
    double cross = 0.0;
    for (size_t l = 0; l < us.size(); ++l) {
      double du = 0, dv = 0;
      for (int64_t r = 0; r < m; ++r) du += us[l][r] * u[r];
      for (int64_t j = 0; j < n; ++j) dv += vs[l][j] * v[j];
      cross += du * dv;
    }
    double uu = 0, vv = 0;
    for (int64_t r = 0; r < m; ++r) uu += u[r] * u[r];
    for (int64_t j = 0; j < n; ++j) vv += v[j] * v[j];
    const double nu2 = uu * vv;
    norm2 = norm2 + 2.0 * cross + nu2;
    us.push_back(std::move(u));
    vs.push_back(std::move(v));
    if (std::sqrt(nu2) <= eps_aca * std::sqrt(std::max(norm2, 0.0))) break;
    bool all = true;
    int64_t nxt = -1;
    double bu = -1.0;
    const std::vector<double> &ul = us.back();
    for (int64_t r = 0; r < m; ++r) {
      if (used[r]) continue;
      all = false;
      if (std::fabs(ul[r]) > bu) {
        bu = std::fabs(ul[r]);
        nxt = r;
      }
    }
    if (all) break;
    i = nxt;
  }
  return true;
}

void recompress(int64_t m, int64_t n, const std::vector<std::vector<double>> &us,
                const std::vector<std::vector<double>> &vs, double eps, hlr_host_hmatrix::Blk &B) {
  const int64_t k = int64_t(us.size());
  if (k == 0) {
    B.rank = 0;
    return;
  }
  std::vector<double> U(size_t(m) * k), V(size_t(n) * k);
  for (int64_t l = 0; l < k; ++l) {
    std::copy(us[l].begin(), us[l].end(), U.begin() + size_t(l) * m);
    std::copy(vs[l].begin(), vs[l].end(), V.begin() + size_t(l) * n);
  }
  std::vector<double> QU, RU, QV, RV;
  qr_thin(m, k, U, QU, RU);
  qr_thin(n, k, V, QV, RV);
  std::vector<double> M(size_t(k) * k, 0.0);  // RU * RV^T
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r < k; ++r) {
      double s = 0;
      for (int64_t l = 0; l < k; ++l) s += RU[r + l * k] * RV[c + l * k];
      M[r + c * k] = s;
    }
  std::vector<double> Us, s, Vs;
  svd_jacobi(k, k, M, Us, s, Vs);
  const int kk = trunc_rank(s, eps);
  B.rank = kk;
  B.S.assign(s.begin(), s.begin() + kk);
  B.W.assign(size_t(m) * kk, 0.0);
  B.X.assign(size_t(n) * kk, 0.0);
  for (int c = 0; c < kk; ++c) {
    for (int64_t l = 0; l < k; ++l) {
      const double a = Us[l + size_t(c) * k], b = Vs[l + size_t(c) * k];
      for (int64_t r = 0; r < m; ++r) B.W[r + size_t(c) * m] += QU[r + size_t(l) * m] * a;
      for (int64_t r = 0; r < n; ++r) B.X[r + size_t(c) * n] += QV[r + size_t(l) * n] * b;
    }
  }
}

}  // namespace

// block descriptors pointing into the matrix's own arrays
static void fill_descs(hlr_host_hmatrix &H) {
  const int64_t nb = int64_t(H.blocks.size());
  H.descs.resize(nb);
  for (int64_t b = 0; b < nb; ++b) {
    const auto &B = H.blocks[b];
    hlr_block_desc &d = H.descs[b];
    d.row0 = B.row0;
    d.nrows = B.nrows;
    d.col0 = B.col0;
    d.ncols = B.ncols;
    d.kind = B.kind;
    d.rank = B.rank;
    d.D = B.D.empty() ? nullptr : B.D.data();
    d.W = B.W.empty() ? nullptr : B.W.data();
    d.sigma = B.S.empty() ? nullptr : B.S.data();
    d.X = B.X.empty() ? nullptr : B.X.data();
  }
}

extern "C" int hlr_build(const hlr_kernel_problem *p, hlr_host_hmatrix **out) {
  if (!p || !out || !p->points) return set_error(HLR_ERR_INVALID, "hlr_build: null argument");
  *out = nullptr;
  if (p->n <= 0 || p->dim < 1 || p->dim > 3 || p->leaf_size < 1 || !(p->eps > 0 && p->eps < 1) || !(p->eta > 0))
    return set_error(HLR_ERR_INVALID, "hlr_build: bad problem parameters");
  if (p->kernel != HLR_KERNEL_EXP && p->kernel != HLR_KERNEL_LAPLACE && p->kernel != HLR_KERNEL_MATERN15)
    return set_error(HLR_ERR_INVALID, "hlr_build: unknown kernel");
  if (p->kernel != HLR_KERNEL_LAPLACE && !(p->scale > 0)) return set_error(HLR_ERR_INVALID, "hlr_build: scale must be > 0");
  for (int64_t i = 0; i < p->n * p->dim; ++i)
    if (!std::isfinite(p->points[i])) return set_error(HLR_ERR_INVALID, "hlr_build: non-finite point");

  auto H = std::make_unique<hlr_host_hmatrix>();
  H->n = p->n;
  H->eps = p->eps;
  Tree T;
  T.P = p->points;
  T.dim = p->dim;
  T.leaf = p->leaf_size;
  T.perm.resize(p->n);
  std::iota(T.perm.begin(), T.perm.end(), 0);
  T.build(0, p->n);
  std::vector<Leaf> leaves;
  block_tree(T, p->eta, 0, 0, leaves);

  const Kern K{p->kernel, p->dim, p->points, p->scale, p->diag};
  const int64_t nb = int64_t(leaves.size());
  H->blocks.resize(nb);
  std::vector<int64_t> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const Cl &ta = T.nodes[leaves[a].t], &sa = T.nodes[leaves[a].s];
    const Cl &tb = T.nodes[leaves[b].t], &sb = T.nodes[leaves[b].s];
    return (ta.hi - ta.lo) + (sa.hi - sa.lo) > (tb.hi - tb.lo) + (sb.hi - sb.lo);
  });
  const int nt = p->threads > 0 ? p->threads : omp_get_max_threads();
  const int64_t *perm = T.perm.data();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t oi = 0; oi < nb; ++oi) {
    const int64_t b = order[oi];
    const Cl &t = T.nodes[leaves[b].t], &s = T.nodes[leaves[b].s];
    hlr_host_hmatrix::Blk &B = H->blocks[b];
    B.row0 = t.lo;
    B.nrows = t.hi - t.lo;
    B.col0 = s.lo;
    B.ncols = s.hi - s.lo;
    B.rank = 0;
    const int64_t *I = perm + t.lo, *J = perm + s.lo;
    if (!leaves[b].adm) {
      B.kind = HLR_DENSE;
      B.D.resize(size_t(B.nrows) * B.ncols);
      for (int64_t c = 0; c < B.ncols; ++c)
        for (int64_t r = 0; r < B.nrows; ++r) B.D[r + size_t(c) * B.nrows] = K(I[r], J[c]);
      continue;
    }
    B.kind = HLR_LOWRANK;
    std::vector<std::vector<double>> us, vs;
    const int64_t cap = std::max<int64_t>(1, std::min(B.nrows, B.ncols) / 2);
    if (aca(K, I, B.nrows, J, B.ncols, p->eps / 10.0, cap, us, vs)) {
      recompress(B.nrows, B.ncols, us, vs, p->eps, B);
    } else {
      std::vector<double> M(size_t(B.nrows) * B.ncols);
      for (int64_t c = 0; c < B.ncols; ++c)
        for (int64_t r = 0; r < B.nrows; ++r) M[r + size_t(c) * B.nrows] = K(I[r], J[c]);
      lowrank_dense_svd(B.nrows, B.ncols, M, p->eps, B);
    }
  }
  H->perm = T.perm;
  fill_descs(*H);
  *out = H.release();
  return HLR_OK;
}

extern "C" int hlr_host_describe(const hlr_host_hmatrix *hm, hlr_hmatrix_desc *d) {
  if (!hm || !d) return set_error(HLR_ERR_INVALID, "hlr_host_describe: null argument");
  d->n = hm->n;
  d->perm = hm->perm.data();
  d->nblocks = int64_t(hm->descs.size());
  d->blocks = hm->descs.data();
  d->eps = hm->eps;
  d->format = HLR_FMT_AFL_APLR;
  d->tuning = 0;
  return HLR_OK;
}

extern "C" void hlr_host_free(hlr_host_hmatrix *hm) { delete hm; }

// ---- checkpoint: the FP64 host matrix in one file --------------------------------------------
// Layout (little-endian): "HLRHMAT\0", u32 version (1), u32 0, i64 n, i64 nblocks, f64 eps,
// i64 perm[n]; per block i64 row0, nrows, col0, ncols, i32 kind, i32 rank, then D (dense,
// column-major nrows x ncols) or W (nrows x rank), sigma (rank), X (ncols x rank); last, the
// FNV-1a 64-bit hash of every byte before it.
namespace {
constexpr char kMagic[8] = {'H', 'L', 'R', 'H', 'M', 'A', 'T', '\0'};
constexpr uint32_t kVersion = 1;

uint64_t fnv1a(const uint8_t *p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Streams the file through a small buffer, hashing every byte it writes (FNV-1a, updated as it
// goes), so that saving needs no second copy of the matrix.
struct Writer {
  FILE *f;
  uint64_t h = 1469598103934665603ull;
  bool ok = true;
  std::vector<uint8_t> buf;
  explicit Writer(FILE *file) : f(file) { buf.reserve(1 << 20); }
  void write(const void *src, size_t n) {
    const uint8_t *p = static_cast<const uint8_t *>(src);
    for (size_t i = 0; i < n; ++i) {
      h ^= p[i];
      h *= 1099511628211ull;
    }
    if (buf.size() + n > buf.capacity()) flush();
    if (n >= buf.capacity()) {
      ok = ok && std::fwrite(p, 1, n, f) == n;
    } else {
      buf.insert(buf.end(), p, p + n);
    }
  }
  void flush() {
    if (!buf.empty()) ok = ok && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    buf.clear();
  }
  template <typename T>
  void put(const T &v) {
    write(&v, sizeof(T));
  }
  void put_doubles(const std::vector<double> &v) { write(v.data(), 8 * v.size()); }
};

struct Reader {
  const uint8_t *p;
  size_t n, at = 0;
  bool ok = true;
  template <typename T>
  T get() {
    T v{};
    if (at + sizeof(T) > n) {
      ok = false;
      return v;
    }
    std::memcpy(&v, p + at, sizeof(T));
    at += sizeof(T);
    return v;
  }
  bool get_doubles(std::vector<double> &v, uint64_t count) {
    if (count > (n - at) / 8) return ok = false;
    v.resize(size_t(count));
    std::memcpy(v.data(), p + at, size_t(count) * 8);
    at += size_t(count) * 8;
    return true;
  }
};
}  // namespace

extern "C" int hlr_host_save(const hlr_host_hmatrix *hm, const char *path) {
  if (!hm || !path) return set_error(HLR_ERR_INVALID, "hlr_host_save: null argument");
  // written to path.tmp and renamed over path once complete, so a failed save leaves an
  // earlier file at path as it was
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "wb");
  if (!f) return set_error(HLR_ERR_INVALID, std::string("hlr_host_save: cannot open ") + tmp);
  Writer w(f);
  w.write(kMagic, 8);
  w.put(kVersion);
  w.put(uint32_t(0));
  w.put(int64_t(hm->n));
  w.put(int64_t(hm->blocks.size()));
  w.put(hm->eps);
  w.write(hm->perm.data(), 8 * hm->perm.size());
  for (const auto &B : hm->blocks) {
    w.put(B.row0);
    w.put(B.nrows);
    w.put(B.col0);
    w.put(B.ncols);
    w.put(int32_t(B.kind));
    w.put(int32_t(B.rank));
    if (B.kind == HLR_DENSE) {
      w.put_doubles(B.D);
    } else {
      w.put_doubles(B.W);
      w.put_doubles(B.S);
      w.put_doubles(B.X);
    }
  }
  const uint64_t h = w.h;
  w.flush();
  const bool wrote = w.ok && std::fwrite(&h, 1, 8, f) == 8;
  const int cl = std::fclose(f);
  if (!wrote || cl != 0 || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return set_error(HLR_ERR_INVALID, std::string("hlr_host_save: write failed: ") + path);
  }
  return HLR_OK;
}

extern "C" int hlr_host_load(const char *path, hlr_host_hmatrix **out) {
  if (!path || !out) return set_error(HLR_ERR_INVALID, "hlr_host_load: null argument");
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) return set_error(HLR_ERR_INVALID, std::string("hlr_host_load: cannot open ") + path);
  // one read into a buffer of the file's size
  long size = -1;
  if (std::fseek(f, 0, SEEK_END) == 0) size = std::ftell(f);
  if (size < 0 || std::fseek(f, 0, SEEK_SET) != 0) {
    std::fclose(f);
    return set_error(HLR_ERR_INVALID, std::string("hlr_host_load: cannot size ") + path);
  }
  std::vector<uint8_t> buf(static_cast<size_t>(size));
  const size_t got = size > 0 ? std::fread(buf.data(), 1, buf.size(), f) : 0;
  std::fclose(f);
  if (got != buf.size()) return set_error(HLR_ERR_INVALID, std::string("hlr_host_load: read failed: ") + path);
  if (buf.size() < 8 + 4 + 4 + 8 + 8 + 8 + 8 || std::memcmp(buf.data(), kMagic, 8) != 0)
    return set_error(HLR_ERR_INVALID, "hlr_host_load: not a saved H-matrix");
  const size_t body = buf.size() - 8;
  uint64_t h;
  std::memcpy(&h, buf.data() + body, 8);
  if (h != fnv1a(buf.data(), body)) return set_error(HLR_ERR_INVALID, "hlr_host_load: checksum mismatch");
  Reader r{buf.data(), body};
  r.at = 8;
  const uint32_t version = r.get<uint32_t>();
  r.get<uint32_t>();
  if (version != kVersion) return set_error(HLR_ERR_INVALID, "hlr_host_load: unsupported version");
  auto H = std::make_unique<hlr_host_hmatrix>();
  H->n = r.get<int64_t>();
  const int64_t nb = r.get<int64_t>();
  H->eps = r.get<double>();
  if (!r.ok || H->n <= 0 || nb <= 0 || uint64_t(H->n) > (body - r.at) / 8 || uint64_t(nb) > (body - r.at) / 40)
    return set_error(HLR_ERR_INVALID, "hlr_host_load: bad sizes");
  H->perm.resize(size_t(H->n));
  for (auto &v : H->perm) {
    v = r.get<int64_t>();
    if (v < 0 || v >= H->n) r.ok = false;
  }
  H->blocks.resize(size_t(nb));
  for (auto &B : H->blocks) {
    B.row0 = r.get<int64_t>();
    B.nrows = r.get<int64_t>();
    B.col0 = r.get<int64_t>();
    B.ncols = r.get<int64_t>();
    B.kind = r.get<int32_t>();
    B.rank = r.get<int32_t>();
    if (!r.ok || B.row0 < 0 || B.nrows <= 0 || B.col0 < 0 || B.ncols <= 0 || B.row0 > H->n - B.nrows ||
        B.col0 > H->n - B.ncols || B.rank < 0 || (B.kind != HLR_DENSE && B.kind != HLR_LOWRANK) ||
        (B.kind == HLR_DENSE && B.rank != 0)) {
      r.ok = false;
      break;
    }
    if (B.kind == HLR_DENSE) {
      r.get_doubles(B.D, uint64_t(B.nrows) * uint64_t(B.ncols));
    } else {
      r.get_doubles(B.W, uint64_t(B.nrows) * uint64_t(B.rank));
      r.get_doubles(B.S, uint64_t(B.rank));
      r.get_doubles(B.X, uint64_t(B.ncols) * uint64_t(B.rank));
    }
    if (!r.ok) break;
  }
  if (!r.ok || r.at != body) return set_error(HLR_ERR_INVALID, "hlr_host_load: truncated or malformed file");
  fill_descs(*H);
  *out = H.release();
  return HLR_OK;
}
