// hlr_solve_cg: unpreconditioned conjugate gradients on the compressed operator, with FP64
// vectors, FP64 inner products reduced in a fixed order (deterministic), and the products
// computed by the compressed H-matrix-vector kernels (Section 5.4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "hlr_internal.h"

namespace hlr {
namespace {

constexpr int kDotBlocks = 608;   // fixed grid of the reductions: 4 x 152 SMs (order is fixed)
constexpr int kDotThreads = 256;

enum { S_RR = 0, S_PAP = 1, S_RRNEW = 2, S_BB = 3, S_TMP = 4, S_IT = 5, S_N = 8 };
constexpr int kCheckEvery = 8;  // CG iterations launched between two reads of the residual by the host

__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kDotThreads / 32; ++i) s += sh[i];
  __syncthreads();
  return s;
}

// partial[b] = sum over the block's grid-stride share of a[i] * b[i]
__global__ void k_dot(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *partial) {
  __shared__ double sh[kDotThreads / 32];
  double v = 0.0;
  for (int64_t i = blockIdx.x * int64_t(kDotThreads) + threadIdx.x; i < n; i += int64_t(kDotBlocks) * kDotThreads)
    v = fma(a[i], b[i], v);
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_dot_final(const double *partial, double *out) {
  __shared__ double sh[kDotThreads / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) v += partial[i];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) *out = s;
}

// r = b - Ap ; p = r ; Ap = 0
__global__ void k_init(const double *__restrict__ b, double *__restrict__ r, double *__restrict__ p,
                       double *__restrict__ Ap, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double v = b[i] - Ap[i];
    r[i] = v;
    p[i] = v;
    Ap[i] = 0.0;
  }
}

// alpha = rr / pAp ; x += alpha p ; r -= alpha Ap ; partial of r.r. Once rr <= stop2 the iteration
// has converged: alpha = 0 leaves x and r as they are (the host reads the residual only every
// kCheckEvery iterations), and only unconverged iterations are counted in scal[S_IT].
__global__ void k_update_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ Ap, double *scal, int64_t n, double *partial, double stop2) {
  __shared__ double sh[kDotThreads / 32];
  const bool done = !(scal[S_RR] > stop2);
  const double alpha = done ? 0.0 : scal[S_RR] / scal[S_PAP];
  if (!done && blockIdx.x == 0 && threadIdx.x == 0) scal[S_IT] += 1.0;
  double v = 0.0;
  for (int64_t i = blockIdx.x * int64_t(kDotThreads) + threadIdx.x; i < n; i += int64_t(kDotBlocks) * kDotThreads) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, Ap[i], r[i]);
    r[i] = ri;
    v = fma(ri, ri, v);
  }
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// beta = rrnew / rr ; p = r + beta p ; Ap = 0
__global__ void k_update_p(double *__restrict__ p, const double *__restrict__ r, double *__restrict__ Ap,
                           double *scal, int64_t n, double stop2) {
  // a converged iteration keeps p finite (beta = 0) whatever rr is
  const double beta = !(scal[S_RR] > stop2) ? 0.0 : scal[S_RRNEW] / scal[S_RR];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    p[i] = fma(beta, p[i], r[i]);
    Ap[i] = 0.0;
  }
}

__global__ void k_copy_scalar(double *scal, int dst, int src) { scal[dst] = scal[src]; }

__global__ void k_residual(const double *__restrict__ b, double *__restrict__ Ax, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    Ax[i] = b[i] - Ax[i];
}

// x += d
__global__ void k_add(double *__restrict__ x, const double *__restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] += d[i];
}

struct CgWork {
  double *r, *p, *Ap, *rt, *d, *partial, *scal;
};

int ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) return set_error(HLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return HLR_OK;
}

}  // namespace

int cg_workspace(Handle &H, void **ws) {
  const size_t n = size_t(H.L.n);
  const size_t bytes = 8 * (5 * n + kDotBlocks + S_N) + 1024;
  if (!H.cg_ws) {
    if (cudaMalloc(&H.cg_ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      H.cg_ws = nullptr;
      return set_error(HLR_ERR_OOM, "hlr_solve_cg: workspace allocation failed");
    }
  }
  *ws = H.cg_ws;
  return HLR_OK;
}

namespace {

struct Cg {
  Handle &H;
  CgWork W;
  int64_t n;
  cudaStream_t st;
  int share;  // HLR_SM_SHARE bits of the products
  double h_scal[S_N];

  void dot(const double *a, const double *c, int slot) {
    k_dot<<<kDotBlocks, kDotThreads, 0, st>>>(a, c, n, W.partial);
    k_dot_final<<<1, kDotThreads, 0, st>>>(W.partial, W.scal + slot);
  }
  // the scalars, and the handle's status words: a product kernel that gave up a bounded wait
  // has left an incomplete product, so the solve stops with HLR_ERR_TIMEOUT
  int fetch() {
    uint32_t status[4] = {0, 0, 0, 0};
    int rc = ck(cudaMemcpyAsync(h_scal, W.scal, sizeof(h_scal), cudaMemcpyDeviceToHost, st), "hlr_solve_cg");
    if (!rc) rc = ck(cudaMemcpyAsync(status, H.L.status, sizeof(status), cudaMemcpyDeviceToHost, st), "hlr_solve_cg");
    if (!rc) rc = ck(cudaStreamSynchronize(st), "hlr_solve_cg");
    if (!rc && (status[0] | status[1] | status[2] | status[3]))
      rc = set_error(HLR_ERR_TIMEOUT, "hlr_solve_cg: a product kernel gave up a bounded wait (status " +
                                          std::to_string(status[0]) + ")");
    return rc;
  }
  // ||rhs - A sol|| with the FP64-accumulation product; the residual is left in W.rt
  int true_residual(const double *rhs, const double *sol, double *norm) {
    int rc = ck(cudaMemsetAsync(W.rt, 0, 8 * size_t(n), st), "hlr_solve_cg");
    if (!rc) rc = launch_matvec(H, sol, W.rt, HLR_ACC_FP64 | share, st);
    if (rc) return rc;
    k_residual<<<2 * kDotBlocks, 256, 0, st>>>(rhs, W.rt, n);
    dot(W.rt, W.rt, S_TMP);
    if ((rc = fetch())) return rc;
    *norm = std::sqrt(h_scal[S_TMP]);
    return HLR_OK;
  }
  // CG iterations for A sol = rhs with products of accumulation `acc`, from sol (zero_start: from
  // sol = 0, which is set here), until ||r|| <= stop or `maxit` iterations.
  int run(const double *rhs, double *sol, bool zero_start, double stop, int maxit, int acc, int *its, bool *conv) {
    int rc = ck(cudaMemsetAsync(W.Ap, 0, 8 * size_t(n), st), "hlr_solve_cg");
    if (rc) return rc;
    if (zero_start) {
      if ((rc = ck(cudaMemsetAsync(sol, 0, 8 * size_t(n), st), "hlr_solve_cg"))) return rc;
    } else if ((rc = launch_matvec(H, sol, W.Ap, acc | share, st))) {
      return rc;
    }
    k_init<<<2 * kDotBlocks, 256, 0, st>>>(rhs, W.r, W.p, W.Ap, n);
    dot(W.r, W.r, S_RR);
    if ((rc = ck(cudaMemsetAsync(W.scal + S_IT, 0, sizeof(double), st), "hlr_solve_cg"))) return rc;
    if ((rc = fetch())) return rc;
    double rr = h_scal[S_RR];
    int launched = 0, it = 0;
    bool ok = std::sqrt(rr) <= stop;
    const double stop2 = stop * stop;
    // iterations are launched kCheckEvery at a time without waiting; the device stops updating x
    // once the residual has dropped below stop, so the few iterations launched after that change
    // nothing and are not counted
    while (!ok && launched < maxit) {
      const int batch = std::min(kCheckEvery, maxit - launched);
      for (int k = 0; k < batch; ++k) {
        if ((rc = launch_matvec(H, W.p, W.Ap, acc | share, st))) return rc;
        dot(W.p, W.Ap, S_PAP);
        k_update_xr<<<kDotBlocks, kDotThreads, 0, st>>>(sol, W.r, W.p, W.Ap, W.scal, n, W.partial, stop2);
        k_dot_final<<<1, kDotThreads, 0, st>>>(W.partial, W.scal + S_RRNEW);
        k_update_p<<<2 * kDotBlocks, 256, 0, st>>>(W.p, W.r, W.Ap, W.scal, n, stop2);
        k_copy_scalar<<<1, 1, 0, st>>>(W.scal, S_RR, S_RRNEW);
      }
      launched += batch;
      if ((rc = fetch())) return rc;
      rr = h_scal[S_RR];
      it = int(h_scal[S_IT]);
      if (!std::isfinite(rr)) return set_error(HLR_ERR_NOCONV, "hlr_solve_cg: breakdown (non-finite residual)");
      ok = std::sqrt(rr) <= stop;
    }
    *its = it;
    *conv = ok;
    return HLR_OK;
  }
};

}  // namespace

// HLR_ACC_FP64: one CG run with FP64-accumulation products.
// HLR_ACC_FP32: iterative refinement. The true residual r = b - A~ x is formed with the FP64
// product; CG with the (about 7x faster) FP32-accumulation product solves A~ d = r to a relative
// 1e-3 (or to what the final step still needs), x += d, repeat. Every correction starts from
// d = 0, so the error of the FP32 products only limits how much one step gains.
int solve_cg(Handle &H, const double *b, double *x, double rtol, int maxit, int flags, void *stream, int *iters,
             double *relres) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *ws = nullptr;
  int rc = cg_workspace(H, &ws);
  if (rc) return rc;
  const int64_t n = H.L.n;
  double *base = static_cast<double *>(ws);
  Cg cg{H, CgWork{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n, base + 5 * n + kDotBlocks},
        n, st, flags & HLR_SM_SHARE(15), {}};
  cg.dot(b, b, S_BB);
  if ((rc = cg.fetch())) return rc;
  const double bnorm = std::sqrt(cg.h_scal[S_BB]);
  int total = 0;
  double rnorm = 0.0;
  if (bnorm == 0.0) {
    if ((rc = cg.true_residual(b, x, &rnorm))) return rc;
  } else if ((flags & 0xff) == HLR_ACC_FP64) {
    int it = 0;
    bool conv = false;
    if ((rc = cg.run(b, x, false, rtol * bnorm, maxit, HLR_ACC_FP64, &it, &conv))) return rc;
    total = it;
    if ((rc = cg.true_residual(b, x, &rnorm))) return rc;
  } else {
    if ((rc = cg.true_residual(b, x, &rnorm))) return rc;
    for (int outer = 0; rnorm > rtol * bnorm && total < maxit && outer < 64; ++outer) {
      const double eta = std::max(0.1 * rtol * bnorm / rnorm, 1e-3);
      int it = 0;
      bool conv = false;
      // W.rt holds the true residual, the right-hand side of the correction equation A~ d = r
      // (run() reads it once, in k_init, and never writes it)
      if ((rc = cg.run(cg.W.rt, cg.W.d, true, eta * rnorm, maxit - total, HLR_ACC_FP32, &it, &conv))) return rc;
      total += it;
      k_add<<<2 * kDotBlocks, 256, 0, st>>>(x, cg.W.d, n);
      if ((rc = cg.true_residual(b, x, &rnorm))) return rc;
      if (it == 0) break;
    }
  }
  if (iters) *iters = total;
  if (relres) *relres = bnorm > 0 ? rnorm / bnorm : 0.0;
  if (bnorm > 0 && !(rnorm <= rtol * bnorm)) return set_error(HLR_ERR_NOCONV, "hlr_solve_cg: maxit reached");
  return HLR_OK;
}

}  // namespace hlr

using namespace hlr;

extern "C" int hlr_solve_cg(hlr_handle h, const double *b, double *x, double rtol, int maxit, int flags,
                            void *stream, int *iters, double *relres) {
  Handle *H = lookup(h);
  if (!H) return set_error(HLR_ERR_INVALID, "hlr_solve_cg: unknown handle");
  if (!b || !x || !(rtol > 0) || maxit < 0) return set_error(HLR_ERR_INVALID, "hlr_solve_cg: bad arguments");
  const int acc = flags & ~HLR_SM_SHARE(15);
  if ((acc != HLR_ACC_FP64 && acc != HLR_ACC_FP32) || ((flags >> 16) & 15) > 8)
    return set_error(HLR_ERR_INVALID, "hlr_solve_cg: bad flags");
  return solve_cg(*H, b, x, rtol, maxit, flags, stream, iters, relres);
}

extern "C" int hlr_matvec_batched(int nreq, const hlr_handle *h, const int32_t *nrhs, const double *const *X,
                                  const int64_t *ldx, double *const *Y, const int64_t *ldy, int flags,
                                  void *stream) {
  if (nreq < 0 || (nreq > 0 && (!h || !nrhs || !X || !ldx || !Y || !ldy)))
    return set_error(HLR_ERR_INVALID, "hlr_matvec_batched: bad arguments");
  const int acc = flags & ~(HLR_MULTI | HLR_SM_SHARE(15));
  if ((acc != HLR_ACC_FP64 && acc != HLR_ACC_FP32) || ((flags & HLR_MULTI) && acc != HLR_ACC_FP32) ||
      ((flags >> 16) & 15) > 8)
    return set_error(HLR_ERR_INVALID, "hlr_matvec_batched: bad flags");
  for (int q = 0; q < nreq; ++q) {
    Handle *H = lookup(h[q]);
    if (!H) return set_error(HLR_ERR_INVALID, "hlr_matvec_batched: unknown handle");
    if (nrhs[q] < 0 || (nrhs[q] > 0 && (!X[q] || !Y[q])) || ldx[q] < H->L.n || ldy[q] < H->L.n)
      return set_error(HLR_ERR_INVALID, "hlr_matvec_batched: bad request " + std::to_string(q));
  }
  std::vector<Handle *> hs(nreq);
  for (int q = 0; q < nreq; ++q) hs[q] = lookup(h[q]);
  return launch_batch(nreq, hs.data(), nrhs, X, ldx, Y, ldy, flags, stream);
}
