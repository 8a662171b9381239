/*
 * hlr.h -- C ABI of the GB300 compressed H-matrix library.
 *
 * The library stores an H-matrix (Def. 2.3: a block partition of I x I whose admissible leaves
 * are lowrank and whose other leaves are dense, with eps-accurate lowrank leaves as in Eq. 1)
 * in the AFL binary compression of Section 3.2, every lowrank factor column at its own
 * precision (APLR, Section 3.3), and applies it to vectors on one GPU (Section 5.4), decoding
 * the bit streams inside the product kernels.
 *
 * Conventions for every call
 *  - All functions return HLR_OK (0) on success and a negative HLR_ERR_* code otherwise; the
 *    calling thread's message is then available from hlr_last_error(). No C++ exception
 *    crosses this boundary.
 *  - "_dev" pointers are device pointers of the current CUDA device; other pointers are host
 *    pointers. The caller keeps ownership of every buffer it passes.
 *  - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default stream). Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Vectors are FP64 in ORIGINAL index order; the cluster permutation is applied inside.
 *  - A handle may be used from several threads for read-only calls; calls that overlap on the
 *    GPU with the same handle and different streams race on the handle's scratch memory and
 *    must be serialised by the caller.
 */
#ifndef HLR_H
#define HLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define HLR_OK               0
#define HLR_ERR_INVALID     (-1)  /* bad argument, shape, coverage, NaN/Inf, unknown handle   */
#define HLR_ERR_OOM         (-2)  /* device or pinned host allocation failed                 */
#define HLR_ERR_CUDA        (-3)  /* a CUDA runtime call or kernel launch failed             */
#define HLR_ERR_TIMEOUT     (-4)  /* a bounded device-side wait expired                      */
#define HLR_ERR_NOCONV      (-5)  /* CG reached maxit; x holds the last iterate              */
#define HLR_ERR_UNSUPPORTED (-6)  /* valid request outside this library's limits             */

/* ---- block kinds and storage formats ---------------------------------------------------- */
#define HLR_DENSE   0
#define HLR_LOWRANK 1

#define HLR_FMT_AFL_APLR 1  /* dense leaves: one AFL unit at eps; lowrank: AFL-APLR columns  */
#define HLR_FMT_FP64     2  /* plain uncompressed FP64 factors (the baseline H-matvec)        */
/* Byte-aligned variants of AFL (Section 3.2), same per-unit precisions as HLR_FMT_AFL_APLR:  */
#define HLR_FMT_AFLP     3  /* AFL with m raised to the smallest m' making 1 + e + m' a multiple of 8 */
#define HLR_FMT_BFL      4  /* FP32 layout: FP32 cast, mantissa rounded to m' in {7, 15, 23}      */
#define HLR_FMT_DFL      5  /* FP64 layout: mantissa rounded to m' in {4, 12, ..., 52}             */
/* Mixed precision comparison format MP-D-S-H (Section 3.3): every lowrank column i is cast
 * (round to nearest even) to the cheapest of FP16, FP32, FP64 whose unit roundoff (2^-11,
 * 2^-24, 2^-53; Table 1) is <= its precision eps sigma_0 / sigma_i; dense leaves stay FP64.
 * Values beyond the chosen format's range are rejected (HLR_ERR_INVALID). */
#define HLR_FMT_MP       6

/* ---- product flags ---------------------------------------------------------------------- */
#define HLR_ACC_FP64 0  /* decode to FP64 and accumulate in FP64 everywhere                    */
#define HLR_ACC_FP32 1  /* decode to FP32, FP32 sums inside a block, FP64 across blocks into y */
#define HLR_PROFILE  0x100 /* OR-ed into flags: record CUDA events around each kernel launch of the
                              product on cuda_stream, for hlr_profile_read (adds no synchronisation) */
#define HLR_MULTI    0x200 /* OR-ed into hlr_matvec_batched flags: run every column of every
                              request as a product of its own (the kernels of hlr_matvec, many per
                              launch), each on a scratch set of its own, so that a column's result
                              is bit for bit that of hlr_matvec for it, whatever it is launched
                              with, and the call never shares scratch with hlr_matvec or
                              hlr_solve_cg running on the same matrix on another stream */

/* OR-ed into the flags of hlr_matvec, hlr_matvec_host, hlr_matvec_batched and hlr_solve_cg:
 * the persistent product kernels take about eighths/8 of their CTA slots (1..7; 0 or 8 = all),
 * each CTA then walking the work lists of several slots, so that work running concurrently on
 * other streams keeps the rest of every SM (e.g. served solves beside served products). The
 * result does not depend on it. */
#define HLR_SM_SHARE(eighths) ((eighths) << 16)

typedef uint64_t hlr_handle; /* 0 is never a valid handle */

/* One leaf block b = (tau, sigma) of the block tree (Def. 2.2) in CLUSTER order: rows
 * [row0, row0+nrows) and columns [col0, col0+ncols) are positions of the permutation perm.
 *  dense  : D, nrows x ncols, column-major.
 *  lowrank: W (nrows x rank) and X (ncols x rank) column-major with orthonormal columns and
 *           sigma[rank] > 0 descending, so that the block is W diag(sigma) X^T (Section 3.3).
 * Unused pointers may be NULL. */
typedef struct {
  int64_t row0, nrows, col0, ncols;
  int32_t kind;
  int32_t rank;
  const double *D;
  const double *W;
  const double *sigma;
  const double *X;
} hlr_block_desc;

/* A whole H-matrix. perm[p] is the original index of cluster position p (NULL = identity).
 * The leaves must cover {0..n-1} x {0..n-1} exactly once. eps is the accuracy of Eq. 1; it
 * sets the precision of every AFL unit (dense: eps; lowrank column i: eps sigma_0 / sigma_i). */
typedef struct {
  int64_t n;
  const int64_t *perm;
  int64_t nblocks;
  const hlr_block_desc *blocks;
  double eps;
  int32_t format;   /* HLR_FMT_AFL_APLR, _AFLP, _BFL, _DFL, _MP or HLR_FMT_FP64 */
  int32_t tuning;   /* 0: default work layout; else HLR_TUNING(sub, leaf, piece_kb), AFL only */
} hlr_hmatrix_desc;

/* Work layout of the AFL product kernels (chosen per matrix, e.g. by an autotuner; the stored
 * codes and the result up to FP32 rounding order do not depend on it):
 *  sub      rows of an X column one lane decodes in phase 1: 32, 64 (default) or 128
 *           (a column of an item of nr rows is read by the smallest power of two of lanes
 *           with lanes * sub >= nr);
 *  leaf     rows of a phase-2 task: 32 or 64 (default; longer leaves are split);
 *  piece_kb bytes of a piece, in KiB: 4 .. 16 (default 16). */
#define HLR_TUNING(sub_log2, leaf_log2, piece_kb) ((sub_log2) | ((leaf_log2) << 4) | ((piece_kb) << 8))
/* OR-ed into hlr_hmatrix_desc.tuning (any format): keep the decode map of hlr_decode_units
 * whatever the matrix size (it costs 24 bytes of host memory per column slice), e.g. to check
 * the stored codes of a large matrix against an independent decoder. */
#define HLR_DECODE_MAP (1 << 16)
/* OR-ed into hlr_hmatrix_desc.tuning (any format): the launch shape of the persistent product
 * kernels. Their work lists are made for k CTAs per SM (1..8; 0, the default, = as many as the
 * single-column FP32 kernels keep resident; values above that are treated as that). A kernel
 * variant that keeps fewer CTAs resident (FP64 accumulation, multi-column passes) runs one
 * wave of CTAs that each walk several lists, so a matrix used mostly with such a variant is
 * better balanced with k equal to that variant's residency. The result does not depend on k. */
#define HLR_CTAS_PER_SM(k) ((k) << 20)
/* OR-ed into hlr_hmatrix_desc.tuning (compressed formats): compress the blocks on the GPU as
 * they are uploaded (Section 5.3: compression where the data is placed, as part of building
 * the device matrix): the FP64 values go to the device through pinned staging, the unit
 * parameters and streams come from hlr_encode_device, and the host only re-places the codes.
 * The result is byte for byte the matrix the host encoder gives. Needs device memory for the
 * FP64 values and the streams during the call. */
#define HLR_ENCODE_DEVICE (1 << 17)

/* Sizes of an uploaded matrix (hlr_get_info). Byte counts exclude alignment padding. */
typedef struct {
  int64_t n, nblocks, ndense, nlowrank, nunits, nleaves, nitems;
  int64_t rank_sum, values;
  uint64_t fp64_bytes;        /* 8 per stored value + 8 per singular value                  */
  uint64_t stream_bytes;      /* compressed (or FP64) factor bytes, unpadded                */
  uint64_t header_bytes;      /* 16 per unit (m_min, offset, e, m, width)                    */
  uint64_t algorithmic_bytes; /* bytes one y += A x must move: streams + headers + 8 per
                                 singular value + 8n (x) + 16n (y read and write) + 8n (perm) */
  uint64_t device_bytes;      /* size of the device arena                                   */
  double flops;               /* 2 k (#tau + #sigma) per lowrank + 2 #tau #sigma per dense  */
  uint64_t phase1_bytes;      /* phase 1 (t = Sigma X~^T x): X streams + X headers + 16 per
                                 singular value (Sigma read, t written) + 4n (x, once)        */
  uint64_t phase2_bytes;      /* phase 2: W and dense streams + their headers + 8 per singular
                                 value (t) + 8n (x, once) + 16n (y) + 8n (perm)              */
  int64_t launches;           /* kernels one hlr_matvec with HLR_ACC_FP32 launches (permute,
                                 phase 1, combine of split blocks, phase 2 and, for the AFL and
                                 AFLP formats, the scatter of its row totals into y; a phase
                                 without work is not launched) */
} hlr_info;

/* Encode the matrix (AFL-APLR or FP64), build the work lists of the product (blocks grouped by
 * leaf row cluster) and copy everything to one device arena. Synchronous: returns after the
 * copy has completed on cuda_stream. The caller may free the descriptor on return.
 * Errors: HLR_ERR_INVALID (shape, coverage, perm, NaN/Inf, rank/sigma), HLR_ERR_OOM,
 * HLR_ERR_CUDA, HLR_ERR_UNSUPPORTED (arena > 16 TiB). Section 3, Section 3.3. */
int hlr_upload(const hlr_hmatrix_desc *d, void *cuda_stream, hlr_handle *out, size_t *device_bytes);

/* y_dev += A~ x_dev (Section 5.4) where A~ is the decoded stored matrix; x_dev and y_dev hold
 * n FP64 values in original order and must not overlap. flags: HLR_ACC_FP64 or HLR_ACC_FP32
 * (ignored for HLR_FMT_FP64, which always computes in FP64). Deterministic: the same inputs
 * give the same bits. Errors: HLR_ERR_INVALID, HLR_ERR_CUDA. */
int hlr_matvec(hlr_handle h, const double *x_dev, double *y_dev, int flags, void *cuda_stream);

/* y_host += A~ x_host with HOST buffers (n FP64 values each, original order): copies x and y to
 * the handle's device buffers on cuda_stream, computes the product there and copies y back, then
 * waits for the stream. Pinned host memory makes the copies asynchronous DMA. Same flags and
 * errors as hlr_matvec. */
int hlr_matvec_host(hlr_handle h, const double *x_host, double *y_host, int flags, void *cuda_stream);

/* Many products in one launch sequence: for request q, Y_q += A~_q X_q with X_q, Y_q holding
 * nrhs[q] columns (leading dimensions ldx[q], ldy[q] >= n_q, column-major). The pointer
 * arrays are host arrays of device pointers. Requests may repeat a handle only if their Y
 * blocks do not overlap. Products of the same kind go into persistent launches of up to 64
 * products each (permute, phase 1, combine, phase 2 per launch group; the job list is a kernel
 * parameter, so no device memory is allocated per call and the call can be captured in a CUDA
 * graph once the scratch below exists). With HLR_ACC_FP32, requests with several columns
 * run in passes of up to 32 columns that decode each value once (phase 2 on the tensor cores,
 * phase 1 with FP32 fused multiply-adds; a pass of more than 8 columns stages the decoded values
 * in shared memory so that the columns of a block share each x row); their pass scratch is
 * allocated per handle on first use and grown when a request needs more passes.
 * HLR_MULTI instead runs every column as its own product (see
 * there) on per-column scratch sets, allocated one by one on first use and kept until
 * hlr_free. Call once with the widest requests before capturing.
 * FP64 accumulation and plain FP64 storage run one product per column.
 * Errors: HLR_ERR_INVALID, HLR_ERR_OOM, HLR_ERR_CUDA. Section 5.4 (applied per column). */
int hlr_matvec_batched(int nreq, const hlr_handle *h, const int32_t *nrhs,
                       const double *const *X_dev, const int64_t *ldx,
                       double *const *Y_dev, const int64_t *ldy, int flags, void *cuda_stream);

/* Unpreconditioned conjugate gradients for A~ x = b (A~ symmetric positive definite), with
 * x_dev as initial guess on entry and the solution on return. The paper defines no solver: CG
 * is here as the repeated application of the product of Section 5.4 that a served solve
 * request needs (the textbook Hestenes-Stiefel iteration), not as a passage of the paper. Inner products (reduced in a
 * fixed order) and vector updates are FP64. flags:
 *  HLR_ACC_FP64: CG with FP64-accumulation products, stopped when the recursive residual has
 *                ||r|| <= rtol ||b||;
 *  HLR_ACC_FP32: iterative refinement: the true residual b - A~ x is formed with the FP64
 *                product, the correction A~ d = r is solved by CG with the FP32-accumulation
 *                product to a relative 1e-3 (or what the last step needs), x += d, until the
 *                TRUE residual has ||b - A~ x|| <= rtol ||b||.
 * Synchronous: iterations are launched eight at a time and the host reads the residual after
 * each group (a converged iterate is left unchanged by the rest of its group). Returns *iters (CG iterations,
 * all corrections together) and *relres, the relative TRUE residual ||b - A~ x|| / ||b|| of
 * the returned x (FP64 product). HLR_ERR_NOCONV when maxit is reached. Workspace of 5n doubles
 * is allocated per handle on the first solve. */
int hlr_solve_cg(hlr_handle h, const double *b_dev, double *x_dev, double rtol, int maxit,
                 int flags, void *cuda_stream, int *iters, double *relres);

/* Wait for cuda_stream and report whether a product kernel of h gave up a bounded device-side
 * wait since the previous check (HLR_ERR_TIMEOUT; the affected result is incomplete). Clears
 * the error word. The product kernels never spin without a limit: every wait on a TMA copy or
 * a shared-memory slot gives up after about 2 s. */
int hlr_check(hlr_handle h, void *cuda_stream);

/* Failure-detection self-test (no counterpart in the paper): launches on cuda_stream one small
 * kernel that waits, with the same bounded wait as the product kernels, on a shared-memory
 * barrier that nothing ever completes, and gives up after `cycles` SM clock cycles (1000 ..
 * 2^31, about 1 s at most). It then records the expired wait in h's status word, so that the
 * next hlr_check(h) returns HLR_ERR_TIMEOUT and clears it. Nothing faults or hangs: the
 * context, the handle and its data stay usable. Errors: HLR_ERR_INVALID (unknown handle,
 * cycles out of range), HLR_ERR_CUDA (launch). */
int hlr_selftest_wait(hlr_handle h, int64_t cycles, void *cuda_stream);

/* Release the device arena of h (synchronises the device first). */
int hlr_free(hlr_handle h);

/* Message of the calling thread's most recent failure ("" if none). Never NULL. */
const char *hlr_last_error(void);

/* Fill *out with the sizes of an uploaded matrix. */
int hlr_get_info(hlr_handle h, hlr_info *out);

/* Per-kernel device time of the products launched with HLR_PROFILE since the previous read:
 * kernel_ms[0] = x permutation, [1] = phase 1 (t = Sigma X~^T x), [2] = phase 2 (y += W~ t, D~ x),
 * [3] = the scatter of phase 2's row totals into y (0 for paths that update y in phase 2),
 * summed over *calls products (kernel_ms holds 4 values). Waits for the recorded events. At most 4096 products are kept
 * between reads; later ones are not recorded. */
int hlr_profile_read(hlr_handle h, double *kernel_ms, int *calls);

/* ---- codec entry points ----------------------------------------------------------------- */

/* AFL-encode n FP64 values (one unit, Section 3.2) at precision u on the HOST (no GPU needed).
 * Writes m_min, e, m and the packed stream (value j at bits [j w, (j+1) w), w = 1+e+m,
 * LSB-first, zero-padded to a multiple of 16 bytes) into out[cap]; *nbytes = padded size.
 * HLR_ERR_INVALID for NaN/Inf input or u <= 0; HLR_ERR_OOM if cap is too small. */
int hlr_afl_encode(const double *a, int64_t n, double u, double *m_min, int32_t *e, int32_t *m,
                   uint8_t *out, size_t cap, size_t *nbytes);

/* hlr_afl_encode for any compressed format (HLR_FMT_AFL_APLR, HLR_FMT_AFLP, HLR_FMT_BFL,
 * HLR_FMT_DFL, HLR_FMT_MP), Sections 3.2 and 3.3: same arguments and errors; for BFL, DFL and
 * MP *m_min is 1 and *e the exponent width of the layout (BFL 8, DFL 11; MP 5, 8 or 11 for the
 * FP16, FP32 or FP64 the precision u selects, *m then 10, 23 or 52). BFL and MP also fail
 * (HLR_ERR_INVALID) for values that are not finite after the cast and rounding. */
int hlr_encode(int32_t format, const double *a, int64_t n, double u, double *m_min, int32_t *e, int32_t *m,
               uint8_t *out, size_t cap, size_t *nbytes);

/* Encode nunits units on the GPU in format fmt (any compressed format; Section 3.2, and
 * Section 3.3 for the per-column precisions of AFL-APLR and the MP layout), writing for every
 * unit the very bytes hlr_encode writes for it. This is the device side of compressing data
 * where it is built (Section 5.3: compression as part of the construction).
 *   off_dev[nunits + 1] (device, int64): unit u is a_dev[off_dev[u] .. off_dev[u+1]);
 *   total_values       (host): off_dev[nunits], used to check cap;
 *   a_dev (device, FP64), u_dev[nunits] (device, FP64): the values and each unit's precision
 *     (dense leaf: eps, or for MP any u < 2^-53, i.e. FP64; column i of a lowrank block:
 *     eps sigma_0 / sigma_i);
 *   m_min_dev, e_dev, m_dev [nunits] (device, out): the unit parameters as hlr_encode returns
 *     them; e_dev[u] = -1 marks a rejected unit, which gets no stream: one hlr_encode would
 *     reject (NaN / Inf, a value beyond the format's range, a precision that is not positive
 *     and finite) or one whose offsets decrease or leave [0, total_values] (its values are
 *     then not read);
 *   out_off_dev[nunits + 1] (device, out): unit u's stream is out_dev[out_off_dev[u] ..
 *     out_off_dev[u+1]) (each padded to 16 bytes; out_off_dev[nunits] = total bytes);
 *   out_dev (device, 16-byte aligned, cap bytes >= 8 total_values + 16 nunits).
 * Asynchronous on cuda_stream (three kernels, no allocation, no synchronisation); capturable
 * into a CUDA graph. Errors: HLR_ERR_INVALID (format, null or misaligned pointers, negative
 * sizes), HLR_ERR_OOM (cap below the bound), HLR_ERR_CUDA (launch). */
int hlr_encode_device(int32_t fmt, int64_t nunits, const int64_t *off_dev, int64_t total_values, const double *a_dev,
                      const double *u_dev, double *m_min_dev, int32_t *e_dev, int32_t *m_dev, int64_t *out_off_dev,
                      uint8_t *out_dev, size_t cap, void *cuda_stream);

/* The units of a matrix as hlr_upload forms and encodes them (Section 3.3), in upload order:
 * a dense leaf is one unit, its column-major values, at the precision eps of Eq. 1 (for
 * HLR_FMT_MP 2^-60, which selects FP64); a lowrank leaf of rank k > 0 gives its k W columns,
 * then its k X columns, column i of either at the adaptive precision
 * u_i = eps sigma_0 / sigma_i (delta = eps sigma_0, the truncation threshold of Eq. 1). These
 * are the inputs hlr_encode / hlr_encode_device take for a unit. Host only.
 *   *nunits, *nvalues (out): the number of units and of their values (always set);
 *   off[nunits + 1] (out, optional): unit u holds values off[u] .. off[u+1]);
 *   prec[nunits]    (out, optional): the precision of unit u;
 *   values[nvalues] (out, optional): the values of all units, concatenated.
 * Pass NULL outputs to query the sizes first. Errors: HLR_ERR_INVALID (null descriptor, bad
 * rank or sigma, eps outside (0, 1) for a compressed format), HLR_ERR_OOM (cap_units below
 * nunits + 1 with off, below nunits with prec, or cap_values below nvalues with values). */
int hlr_unit_list(const hlr_hmatrix_desc *d, int64_t *off, double *prec, double *values, int64_t cap_units,
                  int64_t cap_values, int64_t *nunits, int64_t *nvalues);

/* Decode one AFL stream on the GPU into n FP64 values, bit-exact IEEE round-to-nearest
 * ((v - 1) * m_min without contraction, Section 3.2). stream_dev must be 16-byte aligned and
 * hold ceil(n (1+e+m) / 8) bytes rounded up to 16. */
int hlr_afl_decode_device(const uint8_t *stream_dev, int64_t n, double m_min, int32_t e, int32_t m,
                          double *out_dev, void *cuda_stream);

/* Decode every unit of an uploaded matrix to FP64 on the GPU, concatenated in unit order
 * (per block in block order: dense -> its column-major values; lowrank -> W columns then X
 * columns). cap is the capacity of out_dev in doubles (>= hlr_info.values). Available for
 * matrices of at most 2^26 stored values, or uploaded with HLR_DECODE_MAP in their tuning
 * (HLR_ERR_UNSUPPORTED otherwise); allocates a temporary device map and synchronises
 * cuda_stream. */
int hlr_decode_units(hlr_handle h, double *out_dev, int64_t cap, void *cuda_stream);

/* The paper has no counterpart of this call: it is hlr_decode_units for callers that must not
 * allocate device memory, e.g. code running under an allocator that owns all of the GPU's
 * memory, or code that must not stall other streams (cudaFree synchronises the whole device).
 * Same arguments, result and limits as hlr_decode_units, but it calls no cudaMalloc, cudaFree
 * or other allocating routine and does not synchronise: the slice map is copied from host
 * memory (cudaMemcpyAsync on cuda_stream) into a fixed 4 MiB device array of this library,
 * which every GPU that loads the library holds until the process exits, and the decoding
 * kernel reads it from there. The map takes 24 bytes per column slice plus 10 per unit
 * (each of its seven parts rounded up to 256 bytes); a matrix whose map does not fit is
 * rejected with HLR_ERR_UNSUPPORTED and a message giving the bytes it needs.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current).
 * All calls share the one array and it keeps the last call's map: every call rewrites all of
 * the map it reads before its kernel runs, so nothing has to start at zero, but calls whose
 * copies or kernels overlap on the GPU (different streams or threads without ordering between
 * them) race and may decode with another call's map. Calls on one stream are ordered.
 * Errors: HLR_ERR_INVALID (unknown handle, null or small output), HLR_ERR_UNSUPPORTED (map
 * above 4 MiB, more than 2^26 values, device index above 63), HLR_ERR_CUDA. */
int hlr_decode_units_static(hlr_handle h, double *out_dev, int64_t cap, void *cuda_stream);

/* ---- construction of kernel matrices (host, multithreaded) --------------------------------- */
#define HLR_KERNEL_EXP      1  /* exp(-|x-y| / scale) + diag * [i == j]                           */
#define HLR_KERNEL_LAPLACE  2  /* 1 / (4 pi |x-y|) for i != j, diag for i == j                     */
#define HLR_KERNEL_MATERN15 3  /* (1 + sqrt3 |x-y|/scale) exp(-sqrt3 |x-y|/scale) + diag [i == j]  */

typedef struct {
  int32_t kernel;
  int32_t dim;           /* 1..3 */
  int64_t n;
  const double *points;  /* n x dim, row-major */
  double scale;
  double diag;
  double eps;            /* Eq. 1 accuracy of the lowrank leaves */
  double eta;            /* standard admissibility parameter (Section 5.1) */
  int32_t leaf_size;
  int32_t threads;       /* 0 = all */
} hlr_kernel_problem;

typedef struct hlr_host_hmatrix hlr_host_hmatrix; /* opaque, owned by the library */

/* Build the FP64 H-matrix of a kernel problem: bounding-box bisection cluster tree (Def. 2.1),
 * block tree with standard admissibility (Def. 2.2), dense leaves evaluated, admissible
 * leaves by ACA with partial pivoting at eps/10 followed by SVD recompression (Algorithm 1)
 * truncated at sigma_i > eps sigma_0. Errors: HLR_ERR_INVALID, HLR_ERR_OOM. */
int hlr_build(const hlr_kernel_problem *p, hlr_host_hmatrix **out);

/* Describe a built matrix: fills *d with pointers into hm (valid until hlr_host_free). */
int hlr_host_describe(const hlr_host_hmatrix *hm, hlr_hmatrix_desc *d);

void hlr_host_free(hlr_host_hmatrix *hm);

/* Checkpoint (no counterpart in the paper): write a built matrix to the file `path` so that a
 * large construction runs once, and read it back. The file holds a versioned header, n, eps,
 * the permutation, every block's ranges, kind, rank and FP64 data (D, or W, sigma, X), and a
 * 64-bit FNV-1a hash of all preceding bytes. hlr_host_load returns a matrix owned by the
 * library (free with hlr_host_free) that describes, uploads and computes exactly like the
 * saved one. Errors: HLR_ERR_INVALID (null argument, unreadable or unwritable file, wrong
 * magic or version, checksum mismatch, truncated or malformed contents). Host only. */
int hlr_host_save(const hlr_host_hmatrix *hm, const char *path);
int hlr_host_load(const char *path, hlr_host_hmatrix **out);

#ifdef __cplusplus
}
#endif
#endif /* HLR_H */
