/*
 * rd.h -- C ABI of the GB300 (sm_103a) library for the Roman domination number
 * of cylinders P_m box C_n by (min,+) matrix powers (arXiv 2409.17658).
 *
 * Method (Sec. 4.A-4.B of the paper): the columns of a Roman dominating
 * function are "correct words" over {a,b,c,d} (Definition 4); the digraph G on
 * those words has an arc q -> p when p can follow q, labelled with the weight
 * 2 p(a) + p(b) of p.  With A = A(G), gamma_R(P_m box C_n) = min_p (A^n)_pp
 * (Corollary 6), and a relation A^(k+p) = q (x) A^k fixes gamma_R for every
 * larger n (Lemma 2, Prop. 7).
 *
 * Conventions shared by every entry point:
 *  - Matrices are dense, row-major int16 in device memory, with a leading
 *    dimension (ld, in elements) that must be a multiple of 8 and >= the
 *    number of columns; base pointers must be 16-byte aligned.
 *  - RD_INF (0x3FFF) encodes the tropical infinity.  Every other operand entry
 *    must be finite and lie in [0, RD_MAX_FINITE]; then a + b never wraps in
 *    int16 and a product entry is finite exactly when some finite + finite
 *    term exists.  Product entries are clamped to RD_INF.
 *  - The caller owns every buffer; unless stated otherwise a call allocates no
 *    device memory.  Device buffers may come from any allocator (PyTorch's
 *    caching allocator in the Python binding).
 *  - Calls are asynchronous on the given stream unless stated otherwise.
 *    Errors are returned as rd_status; no call aborts, throws or exits.
 *  - Word order: word p_1..p_m (row 1 first) has code sum_i letter(p_i) 4^(m-i)
 *    with a=0, b=1, c=2, d=3; states are numbered in increasing code order
 *    (lexicographic, a < b < c < d).  The paper fixes no order; gamma_R and
 *    the period do not depend on it.
 */
#ifndef RD_H
#define RD_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RD_OK = 0,
  RD_ERR_ARG = 1,     /* bad argument: size, pointer alignment, m or n out of range */
  RD_ERR_RANGE = 2,   /* an entry left [0, RD_MAX_FINITE] after normalisation: int16 no longer exact */
  RD_ERR_NOMEM = 3,   /* caller's work buffer too small (or, for rd_gamma_R, a failed allocation) */
  RD_ERR_CUDA = 4,    /* a CUDA runtime call failed; see rd_last_cuda_error() */
  RD_NOT_FOUND = 5,   /* no relation A^(k+p) = q (x) A^k with k + p <= kmax (Algorithm 2's "not found") */
  RD_ERR_TIMEOUT = 6  /* reserved for bounded device-side waits */
} rd_status;

#define RD_INF ((int16_t)0x3FFF)
#define RD_MAX_FINITE 0x1FFF
#define RD_MAX_M 15                 /* codes are 2 bits per row in a uint32 */
#define RD_GAMMA_UNSET INT64_MIN    /* gamma slots that were not computed */
#define RD_GAMMA_INF INT64_MAX      /* min diag(A^k) when every diagonal entry is infinite */

/* Text of the last CUDA error seen by this library in the calling thread ("" if none). */
const char *rd_last_cuda_error(void);

/*
 * rd_state_count -- C_m, the number of correct words of length m
 * (Definition 4; Table 1 of Sec. 4.C lists m = 2..11).  Host-only, exact.
 * m in [1, RD_MAX_M] else RD_ERR_ARG.
 */
rd_status rd_state_count(int m, int64_t *N);

/* rd_padded_dim -- the smallest leading dimension >= N accepted by the library (N rounded up to 8). */
rd_status rd_padded_dim(int64_t N, int64_t *Np);

/*
 * rd_enumerate_states -- the correct words of length m (Definition 4), in the
 * word order above: codes_dev[r] = code of the r-th word, weights_dev[r] =
 * 2 p(a) + p(b) (the arc label of Sec. 4.A).  Both device arrays hold C_m
 * entries.  One thread per word unranks its code directly (no scan, no
 * scratch).  RD_ERR_ARG for a bad m or null pointers.
 */
rd_status rd_enumerate_states(int m, uint32_t *codes_dev, uint8_t *weights_dev, cudaStream_t s);

/*
 * rd_build_transfer -- the transfer matrix A(G) of Corollary 6:
 * A[q][p] = 2 p(a) + p(b) when word p can follow word q under the row rules of
 * Sec. 4.A, else RD_INF.  Writes rows 0..C_m-1 and columns 0..lda-1 of A_dev
 * (columns C_m..lda-1 are RD_INF).  A_dev holds C_m x lda int16, lda a multiple
 * of 8 and >= C_m.  Readings where the paper is garbled or silent: the
 * intermediate-row rules' "or p_1 = d" is read as p_i = d; for m = 1 there is
 * no vertical neighbour, so "p_i = c and a neighbour is a" never holds.
 */
rd_status rd_build_transfer(int m, int16_t *A_dev, int64_t lda, cudaStream_t s);

/*
 * rd_build_transfer_loss -- the matrix of the Appendix (lower bound via the
 * loss of almost Roman dominating functions on the top m rows, m >= 2; the
 * paper uses m = 4).  Arcs follow Sec. 4.A except in the last row, where
 * q_m = d behaves like q_m = c (that row needs no domination); the label is
 * 10 p(a) + 5 p(b) - 2 nd(q,p) with nd from Algorithm 3 (including the vertex
 * below the strip when p_m = a), STORED PLUS 2m so that no entry is negative
 * (each row contributes at least -2).  Then A'^n = (2mn) (x) A^n:
 * 2 L_a(n) = min diag A'^n - 2mn, and a relation A'^(k+p) = q' (x) A'^k means
 * A^(k+p) = (q' - 2mp) (x) A^k.  Readings of two typos: the word factors are
 * those of Definition 4, and the last-row case q_m = b reads "or p_m = d".
 * Layout and errors as rd_build_transfer.
 */
rd_status rd_build_transfer_loss(int m, int16_t *A_dev, int64_t lda, cudaStream_t s);

/*
 * rd_minplus_gemm -- C = A (x) B, the (min,+) product of Sec. 3:
 * C[i][j] = min_t (A[i][t] + B[t][j]), for an M x K matrix A, a K x N matrix B
 * and an M x N result C (C may not alias A or B).  Operands follow the
 * conventions above; result entries with no finite term are RD_INF (K = 0
 * gives an all-RD_INF C).  Runs on the DPX add-min units (__viaddmin_s16x2).
 * min_out, if not null, is a device int32 that receives min_ij C[i][j]
 * (RD_INF when C has no finite entry); it is written by this call.
 * M = 1 goes to rd_minplus_gemv.  Products whose 128 x 256 output tiles fill
 * less than one wave of the GPU split K across a thread-block cluster (2, 4
 * or 8 CTAs per tile, partial tiles combined in distributed shared memory);
 * an RD_TUNE_GEMM_SPLITK entry of the tuning table (below) for the product's
 * size class chooses the split and the output tile (128 x 256 or 128 x 128)
 * instead.  The result does not depend on either choice.
 * RD_ERR_ARG for bad sizes, strides or alignment.
 */
rd_status rd_minplus_gemm(const int16_t *A, int64_t lda, const int16_t *B, int64_t ldb, int16_t *C, int64_t ldc,
                          int64_t M, int64_t N, int64_t K, int32_t *min_out, cudaStream_t s);

/*
 * rd_minplus_gemm_streamk -- the same product C = A (x) B as rd_minplus_gemm
 * (Sec. 3), for products with few 128 x 256 output tiles.  The work is cut
 * into (output tile, 32-deep k-tile) units, and exactly the resident CTAs (two
 * per SM) take equal contiguous runs of them, so every SM has the same share
 * whatever the tile count.  A CTA whose run starts or ends inside a tile leaves
 * that partial tile in the workspace; the last CTA to finish the tile takes the
 * minimum of the partials and writes C.  No CTA waits for another.  The result
 * is bit-identical to rd_minplus_gemm.
 * work_dev: caller-owned device memory, 256-byte aligned, at least
 * rd_minplus_gemm_streamk_work_bytes(M, N, K) bytes (about 40 MB on a 152-SM
 * GPU: partial tiles, then one counter per output tile).  It must be
 * zero-filled before its first use; every call leaves its counters at zero, so
 * the same workspace serves later calls of any shape whose size it covers.  One
 * call at a time per workspace: calls on different streams need separate
 * workspaces.  The size depends on the current device's SM count.
 * M = 1, N = 0 or K = 0, and products too large for 32-bit unit numbers
 * (units x grid >= 2^32, many waves of tiles), go to rd_minplus_gemm with the
 * same result, and the workspace is then not touched.  Other conventions,
 * min_out and errors as rd_minplus_gemm; RD_ERR_NOMEM for a short workspace.
 */
rd_status rd_minplus_gemm_streamk_work_bytes(int64_t M, int64_t N, int64_t K, size_t *bytes);
rd_status rd_minplus_gemm_streamk(const int16_t *A, int64_t lda, const int16_t *B, int64_t ldb, int16_t *C,
                                  int64_t ldc, int64_t M, int64_t N, int64_t K, void *work_dev, size_t work_bytes,
                                  int32_t *min_out, cudaStream_t s);

/*
 * rd_minplus_gemm_host -- rd_minplus_gemm (Sec. 3's product) for operands in
 * host memory: A (M x K, row stride lda elements) and B (K x N, ldb) are read
 * from host memory and C (M x N, ldc) is written to host memory.  Host strides
 * need only be >= the row length; host pointers have no alignment rule.  The
 * operands are staged in the caller's device buffer work_dev (256-byte aligned,
 * >= rd_minplus_gemm_host_work_bytes(M, N, K)): enqueued on s are the copies of
 * A and B in, the product (min_out as in rd_minplus_gemm), and the copy of C
 * out.  Asynchronous: the host buffers must stay valid and C must not be read
 * until s has passed this call.  With page-locked (pinned) host buffers the
 * copies run as DMA beside other streams' work, so a caller that alternates two
 * streams and two staging buffers overlaps one product's copies with another's
 * arithmetic; with pageable buffers CUDA stages the copies and may block.
 * RD_ERR_ARG for bad sizes or pointers, RD_ERR_NOMEM for a short work buffer.
 */
rd_status rd_minplus_gemm_host_work_bytes(int64_t M, int64_t N, int64_t K, size_t *bytes);
rd_status rd_minplus_gemm_host(const int16_t *A_host, int64_t lda, const int16_t *B_host, int64_t ldb, int16_t *C_host,
                               int64_t ldc, int64_t M, int64_t N, int64_t K, void *work_dev, size_t work_bytes,
                               int32_t *min_out, cudaStream_t s);

/*
 * rd_minplus_gemv -- y = x (x) B, the (min,+) product of a row vector x (K
 * entries, device, any alignment) with a K x N matrix B (ldb): y[j] =
 * min_k x[k] + B[k][j], y device (16-byte aligned), N entries; conventions and
 * min_out as rd_minplus_gemm.  B is read once, so this is bound by HBM
 * bandwidth; rd_minplus_gemm uses it when M = 1.  For N >= 4096 it runs as
 * thread-block clusters of 8 CTAs (one 256-column band each) whose partial
 * minima meet in distributed shared memory; no workspace.
 */
rd_status rd_minplus_gemv(const int16_t *x, const int16_t *B, int64_t ldb, int16_t *y, int64_t N, int64_t K,
                          int32_t *min_out, cudaStream_t s);

/*
 * rd_minplus_gemm_batched -- `count` (<= 128) independent products
 * C_i = A_i (x) B_i, each with the conventions of rd_minplus_gemm (min_out may
 * be null), in one persistent launch: two CTAs per SM walk the concatenated
 * tile list of all products, longest tiles (largest K) first, so small products
 * run side by side and the tail of a large one is filled by others.  The
 * problem table travels in the kernel's parameters (no device copy).
 */
typedef struct {
  const int16_t *A;
  int64_t lda;
  const int16_t *B;
  int64_t ldb;
  int16_t *C;
  int64_t ldc;
  int64_t M, N, K;
  int32_t *min_out;
} rd_gemm_problem;

rd_status rd_minplus_gemm_batched(const rd_gemm_problem *problems, int count, cudaStream_t s);

/*
 * rd_power_work_bytes -- size of the work buffer rd_power_until_periodic needs
 * to keep `slots` normalised powers (slots >= 2) of an N x N matrix with
 * leading dimension ld, for at most kmax powers.  A relation with period p
 * is verified only if slots > p.
 */
rd_status rd_power_work_bytes(int64_t N, int64_t ld, int kmax, int slots, size_t *bytes);

/*
 * rd_power_until_periodic -- Algorithm 2 of Sec. 4.B with the first-repeat
 * rule.  For k = 1, 2, ... it forms the normalised power P_k = A^k - o_k
 * (o_k = min A^k, kept exactly in int64; P_k has minimum 0), records
 * gamma_host[k] = min_p (A^k)_pp = o_k + min diag P_k (Corollary 6; it is
 * gamma_R(P_m box C_k) for k >= 3 when A is a transfer matrix), and stops at
 * the smallest j for which P_j = P_i for some i < j, i.e. A^j = q (x) A^i with
 * q = o_j - o_i (Lemma 2): then *k_out = i, *p_out = j - i, *q_out = q.
 *   A_dev: N x N operand (lda), entries in [0, RD_MAX_FINITE] or RD_INF.
 *   work_dev / work_bytes: caller-owned device scratch of at least
 *     rd_power_work_bytes(N, lda, kmax, 2) bytes, 256-byte aligned; the ring
 *     holds as many powers as fit.  Contents on entry are ignored.
 *   gamma_host: host array of kmax + 1 int64; entries 1..j are written (j =
 *     k + p, or kmax when no relation was found); the others are RD_GAMMA_UNSET.
 * Returns RD_OK (relation found), RD_NOT_FOUND (none with j <= kmax; gamma
 * entries 1..kmax are valid), RD_ERR_RANGE (a normalised power left
 * [0, RD_MAX_FINITE]), RD_ERR_NOMEM (the ring was too short to hold the
 * matching power P_i), RD_ERR_ARG or RD_ERR_CUDA.  The call synchronises the
 * stream before returning; all host outputs are valid on return.  For N <= 128
 * the whole search runs in one CTA (one launch; the same work-buffer contents
 * and results), also when reached through the _sparse and _split variants.
 */
rd_status rd_power_until_periodic(const int16_t *A_dev, int64_t N, int64_t lda, int kmax, void *work_dev,
                                  size_t work_bytes, int64_t *gamma_host, int32_t *k_out, int32_t *p_out,
                                  int64_t *q_out, cudaStream_t s);

/*
 * rd_power_slot -- byte offset, from the start of work_dev, of the normalised
 * power P_k left in the ring by rd_power_until_periodic (same N, lda, kmax and
 * work_bytes).  On return from that call the last `slots` powers computed are
 * resident: P_k for last - slots < k <= last, where last = k_out + p_out when a
 * relation was found.  The matrix there is N x lda int16 with min entry 0;
 * A^k = o_k (x) P_k.  k = 0 gives the slot the search writes only from its
 * second power on: a caller short of memory may build A itself there (A_dev
 * then points into work_dev), since A is read only for the first power.
 * RD_ERR_ARG when k < 0 or the arguments describe no ring.
 */
rd_status rd_power_slot(int64_t N, int64_t lda, int kmax, size_t work_bytes, int k, size_t *byte_offset);

/*
 * Dense x sparse power step (the left operand sparse).  A(G) has few finite
 * entries (0.55 % at m = 9) while its powers are dense; since A^k (x) A =
 * A (x) A^k, a power step can be R = A (x) P_k, whose row i is the entrywise
 * minimum over the arcs i -> t of A[i][t] + row t of P_k: N nnz(A) add-mins
 * instead of N^3 (Theorem 1: extend every walk by one arc).
 *
 * Block-sparse form of an M x K operand A: rows in blocks of R consecutive rows
 * (R in {1, 2, 4, 8}); for block b, entries block_start[b] .. block_start[b+1]-1
 * list, in increasing order, the columns t where some row of the block is
 * finite.  Entry e is a record of rd_sparse_record_words(R) uint32 words at
 * records[e * words]: word 0 = t, word 1 + r = A[b*R + r][t] in both halfwords
 * (RD_INF when that row has no arc to t), the rest zero.  Both arrays are
 * device memory owned by the caller: block_start has ceil(M/R) + 1 int64 and
 * records has entries * words uint32 (16-byte aligned).
 *
 * rd_sparse_count -- fills block_start (exclusive prefix sums of the per-block
 * entry counts; block_start[ceil(M/R)] = total) and returns the total in
 * *entries_host.  Synchronises the stream.
 */
rd_status rd_sparse_count(const int16_t *A, int64_t lda, int64_t M, int64_t K, int R, int64_t *block_start_dev,
                          int64_t *entries_host, cudaStream_t s);

/* rd_sparse_record_words -- 32-bit words per entry record for R (4, 4, 8 or 12); 0 for an invalid R. */
int rd_sparse_record_words(int R);

/* rd_sparse_build -- fills the records from A and the block_start of rd_sparse_count. */
rd_status rd_sparse_build(const int16_t *A, int64_t lda, int64_t M, int64_t K, int R, const int64_t *block_start_dev,
                          uint32_t *records_dev, cudaStream_t s);

/*
 * rd_sparse_minplus -- C = A (x) B (Sec. 3) with A (M x K) in block-sparse form
 * and B a dense K x N matrix (ldb), C dense M x N (ldc); same conventions and
 * min_out as rd_minplus_gemm.  C may not alias B.
 */
rd_status rd_sparse_minplus(int R, int64_t M, const int64_t *block_start, const uint32_t *records, const int16_t *B,
                            int64_t ldb, int64_t N, int16_t *C, int64_t ldc, int32_t *min_out, cudaStream_t s);

/*
 * rd_sparse_minplus_tma -- the same product as rd_sparse_minplus, with the rows
 * of B streamed into shared memory by bulk copies (cp.async.bulk) through a
 * 16-stage ring guarded by mbarriers: a producer warp per CTA issues the copies,
 * two consumer warps apply them.  Every device-side wait is bounded; if one runs
 * out, the value 8 is OR-ed into *err_dev (a device int32 the caller zeroes) and
 * C is not valid.  Measured on GB300 it is slower than rd_sparse_minplus (m = 9,
 * R = 2: 15.4 ms against 5.0 ms; one 2 KB row segment per stage does not amortise
 * the per-copy work), so the period searches use rd_sparse_minplus's kernel.
 */
rd_status rd_sparse_minplus_tma(int R, int64_t M, const int64_t *block_start, const uint32_t *records,
                                const int16_t *B, int64_t ldb, int64_t N, int16_t *C, int64_t ldc, int32_t *min_out,
                                int32_t *err_dev, cudaStream_t s);

/*
 * rd_sparse_minplus_tma_bounded -- rd_sparse_minplus_tma with its two
 * failure-handling knobs exposed, so that the timeout path can be exercised
 * without faulting or hanging a GPU: wait_limit (>= 1) is the number of
 * mbarrier try_wait rounds after which a wait gives up (rd_sparse_minplus_tma
 * uses 2^20), and stop_at (>= -1) makes each CTA's producer issue the copies of
 * entries [0, stop_at) of its block and then stop, as a lost copy would (-1:
 * never).  A consumer then waits for the missing entry, gives up after
 * wait_limit rounds with no copy in flight, ORs 8 (the timeout bit) into
 * *err_dev and ends its CTA; other CTAs see the bit and stop early.  Copies
 * already issued are waited for before a CTA exits.  C is not valid after a
 * timeout; the device and the context stay usable.
 */
rd_status rd_sparse_minplus_tma_bounded(int R, int64_t M, const int64_t *block_start, const uint32_t *records,
                                        const int16_t *B, int64_t ldb, int64_t N, int16_t *C, int64_t ldc,
                                        int32_t *min_out, int32_t *err_dev, uint32_t wait_limit, int32_t stop_at,
                                        cudaStream_t s);

/*
 * rd_power_until_periodic_sparse -- rd_power_until_periodic (same work buffer,
 * outputs and errors) with the power step R = A (x) P_k on the block-sparse form
 * of the same A (built from A_dev with rd_sparse_count / rd_sparse_build), run by
 * the kernel of rd_sparse_minplus.  A_dev is still read once, for the first power.
 */
rd_status rd_power_until_periodic_sparse(const int16_t *A_dev, int64_t N, int64_t lda, int R,
                                         const int64_t *block_start, const uint32_t *records, int kmax,
                                         void *work_dev, size_t work_bytes, int64_t *gamma_host, int32_t *k_out,
                                         int32_t *p_out, int64_t *q_out, cudaStream_t s);

/*
 * rd_sparse_tune -- autotuner for the rows per block R of the sparse step: for
 * R = 1, 2, 4, 8 it builds the block-sparse form of the N x N operand A in
 * scratch_dev, times three products A (x) A (the same bytes and DPX work as a
 * power step) with CUDA events, and returns the fastest R in *best_R;
 * ms_per_R[0..3] (nullable) receives the times (-1 for a candidate whose plan
 * did not fit).  scratch_dev (256-byte aligned) must hold an N x lda int16
 * result plus the plans; a power work buffer's ring is large enough.  The
 * fastest R is also recorded as the RD_TUNE_SPARSE_R entry for N's size class
 * in the tuning table (below).  Synchronous.
 */
rd_status rd_sparse_tune(const int16_t *A, int64_t lda, int64_t N, void *scratch_dev, size_t scratch_bytes,
                         int *best_R, float *ms_per_R, cudaStream_t s);

/*
 * Row-split power step (Sec. 4.A, Corollary 6): R = A(G) (x) B for the transfer
 * matrix of P_m box C_n, computed from the row rules without forming A(G).  The
 * label of an arc q -> p is the weight of p alone, and "p can follow q" is a
 * conjunction over the rows i of "the row type of p_i is admitted by q_i" (row
 * type = the letter, with c split by whether a vertical neighbour in p is an a).
 * Splitting the rows after row j turns the minimum over the followers of q into
 * two nested minima:
 *   X[pi][sigma] = min over the row-type prefixes rho admitted by pi of
 *                  w(p) + B[p],   p = (rho, sigma)                      (pass 1)
 *   R[q]         = min over the row-type suffixes sigma admitted by
 *                  q_{j+1..m} of X[q_{1..j}][sigma]                     (pass 2)
 * with pi a correct word of j letters.  Every entry is the minimum of the same
 * sums as A(G) (x) B, so the result is identical to rd_sparse_minplus /
 * rd_minplus_gemm with A(G).  Both passes read and write each row once.
 *
 * rd_split_info_t describes a built plan (rd_split_plan fills it):
 *   m, j     rows of the grid column and the split (rows 1..j in pass 1);
 *   N        C_m, the order of A(G) (rows and columns of B and R);
 *   n_rho, n_sigma  distinct row-type prefixes (rows 1..j) and suffixes
 *            (rows j+1..m) over the C_m words: the staged rows per fiber;
 *   n_pi, n_phi     C_j and C_{m-j}: the correct prefixes and suffixes;
 *   list1_entries, list2_entries  list entries of the two passes (one per
 *            admitted slot of a fiber and output group, plus padding);
 *   x_rows   rows of the intermediate X: the pairs (pi, sigma) for which
 *            some word (rho, sigma) has rho admitted by pi (the others are
 *            RD_INF and not stored);
 *   plan_bytes  device bytes of the plan;
 *   w1, w2   column-slab widths of the two passes (32, 64, 128 or 256); chosen
 *            by rd_split_plan, and a caller may set another of these values
 *            if its staged fiber fits in shared memory (else RD_ERR_ARG);
 *   slots1, slots2  rows staged per fiber at most (words of one sigma in
 *            pass 1, finite rows of X of one pi in pass 2);
 *   lmax1, lmax2    list entries of one fiber at most (staged with it);
 *   k1, k2   column slabs one CTA sweeps per fiber (1..64, default 8; a
 *            caller may change them like w1, w2);
 *            an RD_TUNE_SPLIT entry of the tuning table for (m, j) replaces
 *            the defaults of w1, k1, w2, k2 when its widths fit;
 *   chunk_cols  0 (default): both passes run over all N columns, X has
 *            x_rows x N entries; > 0 (a multiple of 128): they run chunk by
 *            chunk of that many columns and X holds one chunk (x_rows x
 *            chunk_cols), so X can stay in L2 between the two passes.
 */
typedef struct {
  int32_t m, j;
  int64_t N;
  int32_t n_rho, n_sigma, n_pi, n_phi;
  int64_t list1_entries, list2_entries;
  int64_t x_rows;
  uint64_t plan_bytes;
  int32_t w1, w2;
  int32_t slots1, slots2;
  int32_t lmax1, lmax2;
  int32_t k1, k2;
  int32_t chunk_cols;
} rd_split_info_t;

/* rd_split_default_j -- the split used by default: floor(m / 2) for m <= 10,
 * ceil(m / 2) from m = 11 on (smaller largest fibers there); 0 when m is
 * outside [2, RD_MAX_M] or a part would exceed 8 rows. */
int rd_split_default_j(int m);

/* rd_split_plan_bytes -- device bytes rd_split_plan needs for (m, j), from m
 * and j alone (host arithmetic, no device work).  RD_ERR_ARG for m outside
 * [2, RD_MAX_M], j outside [1, m-1], or a part of more than 8 rows. */
rd_status rd_split_plan_bytes(int m, int j, size_t *bytes);

/*
 * rd_split_plan -- builds the plan for (m, j) in plan_dev (caller-owned,
 * 256-byte aligned, at least rd_split_plan_bytes) on the GPU: the words
 * (rd_enumerate_states), their row types, the ranks of the row-type prefixes
 * and suffixes, the admitted lists of each pi and each phi, the fiber table
 * [sigma][rho] -> p with w(p), and the row map [pi][phi] -> q.  Fills *info.
 * Synchronous.  RD_ERR_ARG (bad m, j or pointer, or a fiber too large for
 * shared memory), RD_ERR_NOMEM (plan_bytes too small), RD_ERR_RANGE (an
 * internal count broke its bound), RD_ERR_CUDA.
 */
rd_status rd_split_plan(int m, int j, void *plan_dev, size_t plan_bytes, rd_split_info_t *info, cudaStream_t s);

/*
 * rd_split_minplus -- C = A(G) (x) B for the m of the plan, entries of B in
 * [0, RD_MAX_FINITE] or RD_INF.  B (N x N, ldb), C (N x N, ldc) and the
 * intermediate X_dev (info->x_rows x ldx int16) are caller-owned device
 * buffers, 16-byte aligned, leading dimensions multiples of 8, ldb and ldc
 * >= N, ldx >= N (or >= info->chunk_cols when that is set); X is overwritten.  Columns N..ld-1 of C are not written.  min_out (nullable,
 * device int32): set to min C, RD_INF if all entries are RD_INF.  Asynchronous
 * on s.  RD_ERR_ARG for an invalid plan description or operand.
 */
rd_status rd_split_minplus(const rd_split_info_t *info, const void *plan_dev, const int16_t *B, int64_t ldb,
                           int16_t *X_dev, int64_t ldx, int16_t *C, int64_t ldc, int32_t *min_out, cudaStream_t s);

/*
 * rd_split_check_flags -- the index checks of a checked build of this library
 * (compiled with -DRD_CHECKED; paper_2409_17658_gb300.build.build(checked=True)
 * makes librd_checked.so).  In such a build the row-split passes (the kernels of
 * rd_split_minplus and of the period searches that step with it) test every
 * index they take from plan data before using it and skip the access when the
 * test fails, OR-ing one bit per kind into a device word: 1 an input row (a word
 * of B, resp. a row of X) past the operand, 2 a staged-row number in a list past
 * the fiber's staged rows, 4 a group number or sub-list bound past the fiber's
 * groups or list, 8 an output row past X, resp. R.  *flags receives the word of
 * the current device; reset != 0 clears it.  Read it once the calls it should
 * cover have completed (synchronise their streams first).  It stands in for a
 * memory checker on GPUs where none can run.  A normal build has no checks:
 * *flags = 0 and RD_NOT_FOUND.  RD_ERR_ARG for a null flags.
 */
rd_status rd_split_check_flags(uint32_t *flags, int reset);

/*
 * rd_power_until_periodic_split -- rd_power_until_periodic (same work buffer,
 * outputs and errors) for A = A(G) of the plan's m, with the power step
 * R = A (x) P_k run by the two passes of rd_split_minplus.  A_dev (N x N,
 * lda) is read once, for the first power (it may sit in the ring slot of
 * power 0, see rd_power_slot); X_dev as in rd_split_minplus.
 * Short rings: when the only power whose hash matches the new power P_j has
 * left the ring and the ring has at least 3 slots, the search stops at j,
 * re-derives that power P_i from A(G) (rebuilt for the plan's m) in the two
 * slots that do not hold P_j -- the same products and normalisation as the
 * search -- and compares it with P_j entry by entry: equal gives the relation
 * (k, p) = (i, j - i) and RD_OK; otherwise (a hash collision) RD_ERR_NOMEM.
 * This lets m = 11 (73 GB per power) search with 3 slots.
 */
rd_status rd_power_until_periodic_split(const int16_t *A_dev, int64_t lda, const rd_split_info_t *info,
                                        const void *plan_dev, int16_t *X_dev, int64_t ldx, int kmax, void *work_dev,
                                        size_t work_bytes, int64_t *gamma_host, int32_t *k_out, int32_t *p_out,
                                        int64_t *q_out, cudaStream_t s);

/*
 * rd_power_until_periodic_multi -- up to 16 period searches advanced together
 * (for instance A(G) for m = 1..9).  Each run has its own operand A (dense, for
 * the first power), its block-sparse form (the same R for all runs), its own
 * work buffer (rd_power_work_bytes) and its own outputs, with the meaning of
 * rd_power_until_periodic_sparse; `status` receives that call's status for the
 * run.  A run may instead carry a row-split plan (split_* fields), for the step
 * of rd_power_until_periodic_split.  The runs advance in groups, each on a
 * stream of its own (forked from a private stream ordered after s, joined back
 * after each block of steps), so the groups' steps run concurrently:
 *  - all sparse-step runs form one group whose step is ONE launch of a
 *    persistent kernel (R = 1 or 2; other R use one launch per phase) walking a
 *    list of work items of every run -- product tiles, normaliser parts, a
 *    finalize item, compare parts -- in that dependency order per run, each
 *    dependency a wait bounded by time (about a second; past it the run stops
 *    with RD_ERR_TIMEOUT);
 *  - each row-split run is a group of its own, stepped by its two pass
 *    launches, then finalize and compare.
 * Stopped runs exit at kernel entry.  graph_steps > 0 captures that many steps
 * of every group into one CUDA graph and replays it until every run has
 * stopped; 0 enqueues the steps directly.  Returns RD_OK when the batch ran
 * (per-run results in runs[i].status), RD_ERR_ARG / RD_ERR_NOMEM / RD_ERR_CUDA
 * otherwise.  Synchronous.
 */
typedef struct {
  const int16_t *A;
  int64_t N;
  int64_t lda;
  const int64_t *block_start;
  const uint32_t *records;
  void *work;
  size_t work_bytes;
  int64_t *gamma_host; /* kmax + 1 entries */
  int32_t k, p;        /* outputs */
  int64_t q;
  rd_status status;
  /* Optional row-split step: with split_info non-null (a plan of
   * rd_split_plan for this run's A(G)), the run's power step is the two passes
   * of rd_split_minplus through split_plan and the intermediate split_X
   * (split_info->x_rows x split_ldx), and block_start / records may be null. */
  const rd_split_info_t *split_info;
  const void *split_plan;
  int16_t *split_X;
  int64_t split_ldx;
} rd_power_run;

rd_status rd_power_until_periodic_multi(rd_power_run *runs, int count, int R, int kmax, int graph_steps,
                                        cudaStream_t s);

/*
 * rd_power_until_periodic_multi_bounded -- rd_power_until_periodic_multi with
 * the failure handling of its one-launch step exposed, so that the timeout path
 * runs without faulting or hanging a GPU: wait_ms (1..60000) bounds every wait
 * of an item for its run's previous level (rd_power_until_periodic_multi uses
 * 1000), and stall_run (-1: none) makes that run's product level count one item
 * more than it has, as a lost item would, so its normaliser items wait until
 * the bound runs out.  That run then stops with status RD_ERR_TIMEOUT; its
 * later items do no work and wait for nothing, and every other run's search
 * and results are unaffected.  Only runs of the sparse step can be stalled (a
 * row-split stall_run is ignored).
 */
rd_status rd_power_until_periodic_multi_bounded(rd_power_run *runs, int count, int R, int kmax, int graph_steps,
                                                uint32_t wait_ms, int32_t stall_run, cudaStream_t s);

/*
 * Relation records: checkpoint and resume of the per-m results.  What the
 * period search yields for A(G) of P_m -- the first repeat A^(k+p) = q (x) A^k
 * (Lemma 2, Algorithm 2) and gamma[n] = min diag(A^n) for n <= k + p
 * (Corollary 6) -- fixes gamma_R(P_m box C_n) for every n through the solution
 * of the finite-difference equation of Prop. 7, in a few hundred bytes.  A
 * record exported by one process can be imported by another, which then answers
 * every n of that m on the host with no device work (the search costs about
 * 0.35 s and 87 GB of device memory at m = 10, 9 s and 225 GB at m = 11).
 * Records describe the transfer matrix of Sec. 4.A (rd_build_transfer), not the
 * Appendix variant.
 *   m      1..RD_MAX_M.
 *   found  1: A^(k+p) = q (x) A^k with the smallest k + p; 0: no relation with
 *          k + p <= j (then k = p = 0, q = 0).
 *   k, p   found: k >= 1, p >= 1.
 *   q      found: gamma(n + p) - gamma(n) for every n >= k.
 *   j      gamma[1..j] are recorded: j = k + p when found, else the kmax
 *          searched; 1 <= j <= RD_RELATION_MAX_J.
 * The gamma array that goes with a record has j + 1 entries; gamma[0] is not
 * used (RD_GAMMA_UNSET on export, ignored on import).
 */
#define RD_RELATION_MAX_J (1 << 20)
typedef struct {
  int32_t m;
  int32_t found;
  int32_t k, p;
  int64_t q;
  int32_t j;
  int32_t reserved; /* 0 */
} rd_relation_t;

/*
 * Query server with continuous batching (for many gamma_R(P_m box C_n) queries).
 * A worker thread on the device current at creation keeps one period-search job
 * per m that has been asked for and is not settled yet.  Each step advances all
 * admitted jobs together (rd_power_until_periodic_multi's launches); queries are
 * answered as soon as gamma(n) is known -- power n computed, or the relation
 * (k, p, q) found, after which the m is answered on the host by Prop. 7 for the
 * life of the server and its device memory is freed.  Jobs are admitted in
 * arrival order while their device footprint (A(G), block-sparse form with
 * R = 2, work buffer with 8 powers) fits hbm_budget_bytes; a job larger than the
 * whole budget answers RD_ERR_NOMEM.  At most 16 jobs run at once.  The server
 * allocates and frees its own device memory.
 */
typedef struct rd_server rd_server;
typedef struct {
  uint64_t submitted, answered, steps, jobs_admitted, jobs_completed;
  size_t bytes_in_use, bytes_peak;
} rd_server_stats_t;

/* rd_server_create -- start a server; kmax (8..4096) bounds the powers per m. */
rd_status rd_server_create(size_t hbm_budget_bytes, int kmax, rd_server **out);

/* rd_server_submit -- enqueue `count` queries (m[i] in [1, RD_MAX_M], n[i] >= 3); tickets out.  Thread-safe. */
rd_status rd_server_submit(rd_server *sv, int count, const int32_t *m, const int64_t *n, uint64_t *tickets);

/*
 * rd_server_wait -- wait (up to timeout_s seconds in total) for the given
 * tickets; on RD_OK fills gamma[i], status[i] (the query's own rd_status) and
 * latency_s[i] (submit to answer, nullable) and forgets the tickets.
 * RD_ERR_TIMEOUT when some ticket was not answered in time (none is forgotten).
 * Thread-safe.
 */
rd_status rd_server_wait(rd_server *sv, int count, const uint64_t *tickets, double timeout_s, int64_t *gamma,
                         int32_t *status, double *latency_s);

rd_status rd_server_stats(rd_server *sv, rd_server_stats_t *out);
/* rd_server_export -- the server's final record for m (rd_relation_t above): RD_OK with
 * *rel filled (gamma[0..j] too when gamma is not NULL and cap >= rel->j + 1, else
 * RD_ERR_ARG), RD_NOT_FOUND when the server holds no final record for m (never searched,
 * or its search still running), or the status its search failed with.  No CUDA call. */
rd_status rd_server_export(rd_server *sv, int m, rd_relation_t *rel, int64_t *gamma, int64_t cap);
/* rd_server_import -- warm start: installs a record (checked as by rd_gamma_R_import, else
 * RD_ERR_ARG) as the server's final record for rel->m.  Queries routed after the call are
 * answered from it on the host, with no job; a search already running for that m still
 * completes, and its own record then replaces the imported one. */
rd_status rd_server_import(rd_server *sv, const rd_relation_t *rel, const int64_t *gamma);

/* rd_server_destroy -- stop the worker, free its device memory; unanswered tickets are dropped. */
rd_status rd_server_destroy(rd_server *sv);

/*
 * rd_power_until_periodic_noalloc -- the same search as rd_power_until_periodic
 * (same arguments and results, minus the work buffer), for callers that must not
 * allocate device memory: for example code whose device memory is all owned by
 * another allocator (a framework's caching pool, where a cudaMalloc would fail or
 * fragment it), plug-ins whose host forbids device allocations, and
 * latency-critical loops that cannot afford cudaMalloc/cudaFree, which may
 * synchronise the whole device.  The paper has no counterpart; this is a
 * deployment convenience.
 *   Scratch: a static device array of RD_NOALLOC_SCRATCH_BYTES inside the
 *   library, in a module of its own.  Under CUDA's lazy module loading (the
 *   default, CUDA_MODULE_LOADING=LAZY) it is reserved on a device when this
 *   entry point is first used there; with CUDA_MODULE_LOADING=EAGER every
 *   process that loads the library reserves it on each device as the context is
 *   created, whether or not it ever calls this entry point.  Either way it is
 *   held until the process exits, and it lies outside the HBM budget that
 *   rd_server admits jobs against.  Problems that need more --
 *   rd_power_work_bytes(N, lda, kmax, 2) > RD_NOALLOC_SCRATCH_BYTES -- are
 *   rejected with RD_ERR_NOMEM before any device work; within the limit the ring
 *   holds as many powers as fit (A(G) for m <= 7: 7 powers of N = 2507).
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current.
 *   Synchronous: every call synchronises its stream and reads the search state
 *   from the host between steps, so it must never be called while its stream
 *   (or the legacy default stream) is being captured into a CUDA graph.
 *   Sharing: every call on a device uses the same array, which keeps the previous
 *   call's contents; each call re-initialises the state it reads, so no clearing
 *   is needed between calls.  Calls that overlap on the GPU (two host threads,
 *   two streams of one device) race on the array; the call synchronises its
 *   stream before returning, so calls made one after another never overlap.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define RD_NOALLOC_SCRATCH_BYTES (96u * 1024u * 1024u)
rd_status rd_power_until_periodic_noalloc(const int16_t *A_dev, int64_t N, int64_t lda, int kmax,
                                          int64_t *gamma_host, int32_t *k_out, int32_t *p_out, int64_t *q_out,
                                          cudaStream_t s);

/*
 * Tuning table and autotuners.  The launch shape of three kernels is a choice
 * that changes time, never results: the split-K factor S of rd_minplus_gemm
 * (mode RD_TUNE_GEMM_SPLITK), the slab widths and slabs per CTA of the
 * row-split passes (RD_TUNE_SPLIT) and the rows per block of the sparse step
 * (RD_TUNE_SPARSE_R).  The library keeps one process-wide table of entries
 * keyed by (mode, key, aux):
 *   RD_TUNE_GEMM_SPLITK  key = rd_tune_bucket(max(M, N)), aux =
 *                        rd_tune_bucket(K); p[0] = S in {1, 2, 4, 8},
 *                        p[1] = output tile 0 (128 x 256) or 1 (128 x 128);
 *   RD_TUNE_SPLIT        key = m, aux = j; p[0..3] = w1, k1, w2, k2 (widths
 *                        32, 64, 128 or 256; slabs per CTA 1..64);
 *   RD_TUNE_SPARSE_R     key = rd_tune_bucket(N), aux = 0; p[0] = R in
 *                        {1, 2, 4, 8};
 * ms is the time the autotuner measured for the entry (informational).
 * rd_minplus_gemm takes S and the tile from a matching entry (when S suits
 * the product: every K slice non-empty; else its built-in rule), rd_split_plan takes the
 * widths and slabs per CTA from a matching entry (when the plan's staged rows
 * fit with them; else its built-in choice).  RD_TUNE_SPARSE_R entries are
 * recorded for the caller, who passes R to the sparse calls.  The autotuners
 * time their candidates with CUDA events and record the fastest; the table is
 * read and written as a whole by rd_tune_get / rd_tune_set, so a caller can
 * keep it in a file.  Thread-safe (one mutex); host-only except the timed
 * launches of the autotuners.
 */
enum { RD_TUNE_GEMM_SPLITK = 1, RD_TUNE_SPLIT = 2, RD_TUNE_SPARSE_R = 3 };
#define RD_TUNE_MAX 256 /* entries the table holds */
typedef struct {
  int32_t mode, key, aux;
  int32_t p[4];
  float ms;
} rd_tune_entry_t;

/* rd_tune_bucket -- ceil(log2(x)) for x >= 1 (0 for x <= 1): the size class
 * the table keys use. */
int rd_tune_bucket(int64_t x);

/* rd_tune_set -- replaces the table by entries[0..count) (count 0 clears it).
 * RD_ERR_ARG (table unchanged) when count is outside [0, RD_TUNE_MAX], entries
 * is null with count > 0, an entry has an unknown mode or parameters outside
 * the ranges above, or two entries share (mode, key, aux). */
rd_status rd_tune_set(const rd_tune_entry_t *entries, int count);

/* rd_tune_get -- copies up to cap entries into entries (nullable when cap is
 * 0) and sets *count to the number the table holds. */
rd_status rd_tune_get(rd_tune_entry_t *entries, int cap, int *count);

/* rd_tune_lookup -- the entry for (mode, key, aux) into *out; RD_NOT_FOUND
 * when there is none. */
rd_status rd_tune_lookup(int mode, int key, int aux, rd_tune_entry_t *out);

/*
 * rd_tune_gemm -- autotuner for the output tile and split-K factor of
 * rd_minplus_gemm on an M x N x K product (operands as in rd_minplus_gemm,
 * M >= 2; C is overwritten): times each tile (128 x 256; 128 x 128 for
 * products of at most four waves of its CTAs) with each S in {1, 2, 4, 8}
 * that suits the product and would not exceed four waves of CTAs (one
 * warm-up, then reps >= 1 timed products), records the fastest in the table
 * (replacing an entry with the same key) and returns it in *best (nullable).
 * Synchronous.
 */
rd_status rd_tune_gemm(const int16_t *A, int64_t lda, const int16_t *B, int64_t ldb, int16_t *C, int64_t ldc,
                       int64_t M, int64_t N, int64_t K, int reps, rd_tune_entry_t *best, cudaStream_t s);

/*
 * rd_tune_split -- autotuner for the launch shape of the row-split passes of
 * a built plan (arguments as in rd_split_minplus; X and C are overwritten):
 * times rd_split_minplus over the widths {32, 64, 128, 256} that fit and slabs per
 * CTA {1, 2, 4, 8, 16, 32}, first for pass 1 with pass 2 as in *info, then
 * for pass 2 with pass 1 at its best (one warm-up and reps >= 1 timed
 * products per candidate).  Writes the best w1, k1, w2, k2 into *info,
 * records them in the table under (m, j) and returns the entry in *best
 * (nullable).  Synchronous.
 */
rd_status rd_tune_split(rd_split_info_t *info, const void *plan_dev, const int16_t *B, int64_t ldb, int16_t *X_dev,
                        int64_t ldx, int16_t *C, int64_t ldc, int reps, rd_tune_entry_t *best, cudaStream_t s);

/*
 * rd_measure_addmin_peak -- the roofline denominator of the dense (min,+)
 * product: the add-mins per SM clock and per second that the DPX unit retires
 * on the current device.  The paper has no counterpart (its kernel ran on the
 * scalar ALU of a Kepler GPU); the product's throughput is reported against
 * this figure.  One full wave of CTAs (every SM at its resident limit) runs 16
 * independent chains per thread of __viaddmin_s16x2 -- min(a + b, c) on both
 * int16 halves of a word, 2 add-mins per instruction -- for 8 x trips steps per
 * chain, register operands only, after a short warm-up launch.  *out gets:
 *   addmin_per_clk_per_sm  add-mins per SM cycle, from each CTA's clock64()
 *                          span (the slowest CTA counts), so it does not depend
 *                          on the clock the GPU ran at;
 *   addmin_per_s           add-mins per second of CUDA-event time;
 *   sm_mhz                 the SM clock that implies (cycles / event time);
 *   ms, sm_count, ctas_per_sm  as timed and launched;
 *   lanes_per_clk_per_sm   the nominal DPX issue width, 64 s16x2 lanes per SM
 *                          and clock, so the nominal peak is
 *                          sm_count x 64 x 2 x clock.
 * work_dev: device scratch (16-byte aligned, >= RD_PEAK_WORK_BYTES) for the
 * per-CTA cycle counts.  trips in [1, 2^30]; 8192 takes about 17 ms on a
 * GB300.  RD_ERR_ARG for bad arguments, RD_ERR_NOMEM for a short work buffer.
 * Synchronous.
 */
#define RD_PEAK_WORK_BYTES 65536u
typedef struct {
  double addmin_per_clk_per_sm;
  double addmin_per_s;
  double sm_mhz;
  double ms;
  int32_t sm_count;
  int32_t ctas_per_sm;
  int32_t lanes_per_clk_per_sm;
} rd_addmin_peak_t;
rd_status rd_measure_addmin_peak(void *work_dev, size_t work_bytes, int64_t trips, rd_addmin_peak_t *out,
                                 cudaStream_t s);

/*
 * rd_gamma_R -- gamma_R(P_m box C_n) for m in [1, RD_MAX_M], n >= 3 (C_n needs
 * n >= 3).  The first call for a given m builds A(G) and runs the period
 * search: in one CTA (rd_power_until_periodic) when C_m <= 128 (m <= 4), else
 * by rd_power_until_periodic_split, on the current device, in device memory this
 * call allocates and frees (about 11 powers of C_m x C_m int16: 10 GB at m = 9,
 * 87 GB at m = 10; RD_ERR_NOMEM when that does not fit); the result (gamma for n < k + p, and (k, p, q)) is
 * cached per m for the life of the process, and later calls evaluate the
 * solution of the finite-difference equation of Prop. 7 on the host:
 * gamma(n) = gamma(k + (n - k) mod p) + q floor((n - k) / p) for n >= k.
 * Thread-safe.  Synchronous.
 */
rd_status rd_gamma_R(int m, int64_t n, int64_t *out);

/* rd_gamma_R_clear -- forgets every cached m, so the next rd_gamma_R(m, .) runs its period search again
 * (a cold start, e.g. for timing).  Thread-safe; waits for a search in progress. */
rd_status rd_gamma_R_clear(void);

/*
 * rd_gamma_R_export -- the record rd_gamma_R holds for m, running the period
 * search first when m is not cached (as rd_gamma_R does; same devices, memory
 * and errors).  *rel is filled on RD_OK; gamma (host, may be NULL to learn
 * rel->j first) receives gamma[0..j] and needs cap >= rel->j + 1, else
 * RD_ERR_ARG (with *rel filled).  Thread-safe.
 */
rd_status rd_gamma_R_export(int m, rd_relation_t *rel, int64_t *gamma, int64_t cap);

/*
 * rd_gamma_R_import -- installs a record (for example one saved by an earlier
 * process) as rd_gamma_R's cache entry for rel->m, replacing any entry; later
 * rd_gamma_R(rel->m, n) calls answer from it with no device work.  No CUDA call.
 * The record is checked against what every transfer-matrix record satisfies,
 * else RD_ERR_ARG and the cache is unchanged:
 *   the fields are in the ranges above;
 *   0 <= gamma[n] <= 2 m n for n = 1..j (labels are non-negative, and the word
 *   of m letters a, which follows itself, gives a closed walk of label 2 m n);
 *   found: gamma[k + p] = gamma[k] + q (min diag(q (x) A^k) = q + min diag A^k).
 * It cannot tell a wrong record that passes these checks: the caller vouches
 * for the record's origin.  Thread-safe.
 */
rd_status rd_gamma_R_import(const rd_relation_t *rel, const int64_t *gamma);

#ifdef __cplusplus
}
#endif
#endif /* RD_H */
