/*
 * rd_oracle.c -- plain CPU oracle for the Roman-domination transfer-matrix method
 * of "Powers of large matrices on GPU platforms to compute the Roman domination
 * number of cylindrical graphs" (arXiv 2409.17658).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file.  Only the test suite, the smoke check of the build
 * entry point and the CPU-baseline leg of the benchmark use it.  It shares no
 * code, header, table or constant generator with the CUDA library: the one
 * interface constant it repeats (the int16 encoding of infinity used by the
 * library's operands, 0x3FFF) is restated below from the interface contract.
 *
 * Everything is computed the slow, obvious way, in int64, with an explicit
 * infinity, and WITHOUT the min-normalisation the GPU path uses, so the GPU's
 * offset bookkeeping is checked independently.  Each function cites the
 * passage of the paper it follows.
 *
 * Letter encoding (a reading: the paper fixes no order of states):
 *   a = 0 (f = 2), b = 1 (f = 1), c = 2 (f = 0, dominated), d = 3 (f = 0, not
 *   dominated yet); Sec. 4.A, the labelling list.  A word p_1..p_m (row 1 at the
 *   top) is stored as code = sum_i letter(p_i) * 4^(m-i), i.e. p_1 in the most
 *   significant 2 bits, so increasing codes are lexicographic order a<b<c<d.
 *
 * Parity pins for each function live in tests/test_oracle_pins.py; the only
 * function here without an independent pin is noted as such where it appears.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define RDO_INF ((int64_t)0x3FFFFFFFFFFFFFFFLL) /* oracle's own infinity */
#define RDO_I16_INF 0x3FFF                        /* interface encoding of infinity in int16 operands */
#define LA 0
#define LB 1
#define LC 2
#define LD 3

int rdo_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* letter of row i (1-based, i = 1..m) of a word code */
static int letter(int m, uint32_t code, int i) { return (int)((code >> (2 * (m - i))) & 3u); }

/* ---- Definition 4 (Sec. 4.A): a correct word has no factor ad, da, ab, ba, bb ---- */
static int is_correct_word(int m, uint32_t code) {
  for (int i = 1; i < m; ++i) {
    int x = letter(m, code, i), y = letter(m, code, i + 1);
    if (x == LA && y == LD) return 0;
    if (x == LD && y == LA) return 0;
    if (x == LA && y == LB) return 0;
    if (x == LB && y == LA) return 0;
    if (x == LB && y == LB) return 0;
  }
  return 1;
}

/* Arc label of Sec. 4.A: l(q,p) = 2 p(a) + p(b), the weight of the destination word. */
static int32_t word_weight(int m, uint32_t code) {
  int32_t w = 0;
  for (int i = 1; i <= m; ++i) {
    int x = letter(m, code, i);
    if (x == LA) w += 2;
    if (x == LB) w += 1;
  }
  return w;
}

/* Number of correct words of length m (Table 1 column C_m), by direct enumeration of all 4^m words. */
int64_t rdo_num_words(int m) {
  if (m < 1 || m > 15) return -1;
  int64_t count = 0;
  for (uint64_t code = 0; code < ((uint64_t)1 << (2 * m)); ++code)
    if (is_correct_word(m, (uint32_t)code)) ++count;
  return count;
}

/* All correct words in increasing code order with their weights; returns the count or -1. */
int64_t rdo_words(int m, uint32_t *code_out, int32_t *weight_out, int64_t cap) {
  if (m < 1 || m > 15) return -1;
  int64_t n = 0;
  for (uint64_t code = 0; code < ((uint64_t)1 << (2 * m)); ++code) {
    if (!is_correct_word(m, (uint32_t)code)) continue;
    if (n >= cap) return -1;
    code_out[n] = (uint32_t)code;
    weight_out[n] = word_weight(m, (uint32_t)code);
    ++n;
  }
  return n;
}

/*
 * "p can follow q" (Sec. 4.A, the three lists of conditions for the first row,
 * the intermediate rows 2..m-1 and the last row).  Row i of p is checked against
 * row i of q.  "p_i = c and a vertical neighbour is a" uses p_{i-1} and/or
 * p_{i+1} when they exist: the first row only has p_2, the last row only
 * p_{m-1}.  Readings (the paper is garbled or silent):
 *   - the intermediate-row cases q_i = b and q_i = c print "or p_1 = d"; we read
 *     p_i = d, the same letter as the first- and last-row lists;
 *   - m = 1 is not covered (the rules mention p_2); a one-row column has no
 *     vertical neighbour, so "p_i = c and neighbour a" is never true.
 */
static int has_vertical_a(int m, uint32_t p, int i) {
  if (i > 1 && letter(m, p, i - 1) == LA) return 1;
  if (i < m && letter(m, p, i + 1) == LA) return 1;
  return 0;
}

int rdo_follows(int m, uint32_t q, uint32_t p) {
  for (int i = 1; i <= m; ++i) {
    int qi = letter(m, q, i), pi = letter(m, p, i);
    int ok;
    switch (qi) {
      case LA: ok = (pi == LA || pi == LC); break;
      case LB: ok = (pi == LD) || (pi == LC && has_vertical_a(m, p, i)); break;
      case LC: ok = (pi == LA || pi == LB || pi == LD) || (pi == LC && has_vertical_a(m, p, i)); break;
      default: ok = (pi == LA); break; /* q_i = d: the vertex must be dominated from the next column */
    }
    if (!ok) return 0;
  }
  return 1;
}

/*
 * Matrix A(G) of Corollary 6: A[q][p] = l(q,p) if p can follow q, else infinity.
 * Rows and columns follow the word order of rdo_words.  A is N x N row-major int64.
 */
int rdo_transfer(int m, int64_t *A, int64_t N) {
  int64_t n = rdo_num_words(m);
  if (n < 0 || n != N) return 1;
  uint32_t *code = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
  int32_t *wt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!code || !wt) { free(code); free(wt); return 2; }
  rdo_words(m, code, wt, N);
  for (int64_t q = 0; q < N; ++q)
    for (int64_t p = 0; p < N; ++p)
      A[q * N + p] = rdo_follows(m, code[q], code[p]) ? (int64_t)wt[p] : RDO_INF;
  free(code);
  free(wt);
  return 0;
}

/* Textbook (min,+) product of Sec. 3: Z[i][j] = min_t X[i][t] + Y[t][j]; an infinite term is infinite. */
void rdo_minplus(const int64_t *X, const int64_t *Y, int64_t *Z, int64_t rows, int64_t inner, int64_t cols) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t j = 0; j < cols; ++j) {
      int64_t best = RDO_INF;
      for (int64_t t = 0; t < inner; ++t) {
        int64_t x = X[i * inner + t], y = Y[t * cols + j];
        if (x == RDO_INF || y == RDO_INF) continue;
        if (x + y < best) best = x + y;
      }
      Z[i * cols + j] = best;
    }
}

/*
 * The same product on the library's int16 operand encoding: entries equal to
 * 0x3FFF are infinity, all others are finite.  Leading dimensions in elements.
 * The result is written back in the same encoding (infinity -> 0x3FFF), as
 * int32 so that a finite result is never confused with the sentinel.
 */
void rdo_minplus_i16(const int16_t *X, int64_t ldx, const int16_t *Y, int64_t ldy, int32_t *Z, int64_t ldz,
                     int64_t rows, int64_t inner, int64_t cols) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t j = 0; j < cols; ++j) {
      int64_t best = RDO_INF;
      for (int64_t t = 0; t < inner; ++t) {
        int64_t x = X[i * ldx + t], y = Y[t * ldy + j];
        if (x == RDO_I16_INF || y == RDO_I16_INF) continue;
        if (x + y < best) best = x + y;
      }
      Z[i * ldz + j] = (best == RDO_INF) ? RDO_I16_INF : (int32_t)best;
    }
}

/* Selected entries (ri[e], cj[e]) of the int16-encoded product, one O(inner) minimum each. */
void rdo_minplus_i16_entries(const int16_t *X, int64_t ldx, const int16_t *Y, int64_t ldy, int64_t inner,
                             const int64_t *ri, const int64_t *cj, int64_t count, int32_t *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t e = 0; e < count; ++e) {
    int64_t best = RDO_INF;
    for (int64_t t = 0; t < inner; ++t) {
      int64_t x = X[ri[e] * ldx + t], y = Y[t * ldy + cj[e]];
      if (x == RDO_I16_INF || y == RDO_I16_INF) continue;
      if (x + y < best) best = x + y;
    }
    out[e] = (best == RDO_INF) ? RDO_I16_INF : (int32_t)best;
  }
}

/*
 * One power step Z = X (x) A where A is given by its arcs (Theorem 1: extending
 * every walk by one arc of G).  Terms whose A entry is infinite can never be the
 * minimum unless every term is infinite, so iterating over the finite entries of
 * A only gives exactly the textbook product.  Arc lists: for each row t of A,
 * arcs arc_col[arc_ptr[t] .. arc_ptr[t+1]) with labels arc_w[...].
 */
static void power_step(const int64_t *X, int64_t N, const int64_t *arc_ptr, const int64_t *arc_col,
                       const int64_t *arc_w, int64_t *Z) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; ++i) {
    int64_t *zi = Z + i * N;
    for (int64_t j = 0; j < N; ++j) zi[j] = RDO_INF;
    for (int64_t t = 0; t < N; ++t) {
      int64_t x = X[i * N + t];
      if (x == RDO_INF) continue;
      for (int64_t e = arc_ptr[t]; e < arc_ptr[t + 1]; ++e) {
        int64_t v = x + arc_w[e];
        if (v < zi[arc_col[e]]) zi[arc_col[e]] = v;
      }
    }
  }
}

static int build_arcs(const int64_t *A, int64_t N, int64_t **ptr, int64_t **col, int64_t **w) {
  int64_t nnz = 0;
  for (int64_t i = 0; i < N * N; ++i) nnz += (A[i] != RDO_INF);
  *ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
  *col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
  *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
  if (!*ptr || !*col || !*w) return 2;
  int64_t e = 0;
  for (int64_t t = 0; t < N; ++t) {
    (*ptr)[t] = e;
    for (int64_t j = 0; j < N; ++j)
      if (A[t * N + j] != RDO_INF) { (*col)[e] = j; (*w)[e] = A[t * N + j]; ++e; }
  }
  (*ptr)[N] = e;
  return 0;
}

/* Z = X (x) A for a dense A, through its arc lists (the product used when powering). */
int rdo_power_step(const int64_t *X, const int64_t *A, int64_t N, int64_t *Z) {
  int64_t *ptr = 0, *col = 0, *w = 0;
  int rc = build_arcs(A, N, &ptr, &col, &w);
  if (rc == 0) power_step(X, N, ptr, col, w, Z);
  free(ptr); free(col); free(w);
  return rc;
}

/* Is Y = beta (x) X entrywise for some finite beta (infinity matching infinity)?  Lemma 2, Prop. 7. */
static int same_up_to_offset(const int64_t *X, const int64_t *Y, int64_t n2, int64_t *beta) {
  int have = 0;
  int64_t b = 0;
  for (int64_t e = 0; e < n2; ++e) {
    int xi = (X[e] == RDO_INF), yi = (Y[e] == RDO_INF);
    if (xi != yi) return 0;
    if (xi) continue;
    if (!have) { b = Y[e] - X[e]; have = 1; }
    else if (Y[e] - X[e] != b) return 0;
  }
  *beta = have ? b : 0;
  return 1;
}

static int64_t diag_min(const int64_t *X, int64_t N) {
  int64_t best = RDO_INF;
  for (int64_t p = 0; p < N; ++p)
    if (X[p * N + p] < best) best = X[p * N + p];
  return best;
}

/*
 * Algorithm 2 with the first-repeat stopping rule: compute A^1, A^2, ... (raw,
 * never normalised) and stop at the smallest j for which some i < j has
 * A^j = q (x) A^i.  Reports (k, p, q) = (i, j - i, q), and gamma[k'] =
 * min_p (A^k')_pp for k' = 1..j (Corollary 6; gamma_R needs k' >= 3).  gamma
 * has room for kmax + 1 entries (index 0 unused).  Returns 0 when a repeat was
 * found, 5 when none was found up to kmax (gamma[1..kmax] still valid), another
 * value on bad arguments.  Keeps all powers, so memory is kmax * N^2 * 8 bytes.
 * A is given as N x N int64 with RDO_INF; pass m >= 1 to build it here, or
 * m = 0 and a caller matrix in A_in.
 */
int rdo_power_until_periodic(int m, const int64_t *A_in, int64_t N_in, int kmax, int64_t *gamma, int32_t *k_out,
                             int32_t *p_out, int64_t *q_out, int32_t *j_out) {
  if (kmax < 1) return 1;
  int64_t N = (m >= 1) ? rdo_num_words(m) : N_in;
  if (N <= 0) return 1;
  size_t n2 = (size_t)N * (size_t)N;
  int64_t **pw = (int64_t **)calloc((size_t)kmax + 1, sizeof(int64_t *));
  if (!pw) return 2;
  pw[1] = (int64_t *)malloc(sizeof(int64_t) * n2);
  if (!pw[1]) { free(pw); return 2; }
  if (m >= 1) rdo_transfer(m, pw[1], N);
  else memcpy(pw[1], A_in, sizeof(int64_t) * n2);
  int64_t *ptr = 0, *col = 0, *w = 0;
  int rc = build_arcs(pw[1], N, &ptr, &col, &w);
  if (rc == 0) {
    rc = 5;
    gamma[1] = diag_min(pw[1], N);
    *j_out = 1;
    for (int j = 2; j <= kmax; ++j) {
      pw[j] = (int64_t *)malloc(sizeof(int64_t) * n2);
      if (!pw[j]) { rc = 2; break; }
      power_step(pw[j - 1], N, ptr, col, w, pw[j]);
      gamma[j] = diag_min(pw[j], N);
      *j_out = j;
      int found = 0;
      for (int i = 1; i < j && !found; ++i) {
        int64_t beta;
        if (same_up_to_offset(pw[i], pw[j], (int64_t)n2, &beta)) {
          *k_out = i; *p_out = j - i; *q_out = beta; found = 1;
        }
      }
      if (found) { rc = 0; break; }
    }
  }
  for (int k = 0; k <= kmax; ++k) free(pw[k]);
  free(pw); free(ptr); free(col); free(w);
  return rc;
}

/*
 * Arc lists of A(G) straight from the follow rules (Cor. 6), without the dense
 * matrix: arcs q -> p with label wt[p], p in increasing order.
 */
static int build_arcs_from_rules(int m, int64_t N, const uint32_t *code, const int32_t *wt, int64_t **ptr,
                                 int64_t **col, int64_t **w) {
  *ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
  if (!*ptr) return 2;
  int64_t *deg = *ptr + 1;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < N; ++q) {
    int64_t d = 0;
    for (int64_t p = 0; p < N; ++p) d += rdo_follows(m, code[q], code[p]);
    deg[q] = d;
  }
  (*ptr)[0] = 0;
  for (int64_t q = 0; q < N; ++q) (*ptr)[q + 1] += (*ptr)[q];
  const int64_t nnz = (*ptr)[N];
  *col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
  *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz ? nnz : 1));
  if (!*col || !*w) return 2;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < N; ++q) {
    int64_t e = (*ptr)[q];
    for (int64_t p = 0; p < N; ++p)
      if (rdo_follows(m, code[q], code[p])) {
        (*col)[e] = p;
        (*w)[e] = wt[p];
        ++e;
      }
  }
  return 0;
}

/*
 * Selected rows of the raw powers: out[(k-1)*nrows*N + r*N + j] = (A^k)[rows[r]][j]
 * for k = 1..kmax, by repeated vector-matrix products e_i (x) A (x) A ...
 * (Theorem 1 applied to walks starting at one word).  Infinity is RDO_INF.
 */
int rdo_power_rows(int m, const int64_t *rows, int nrows, int kmax, int64_t *out) {
  int64_t N = rdo_num_words(m);
  if (N <= 0 || kmax < 1) return 1;
  uint32_t *code = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
  int32_t *wt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!code || !wt) { free(code); free(wt); return 2; }
  rdo_words(m, code, wt, N);
  int64_t *ptr = 0, *col = 0, *w = 0;
  if (build_arcs_from_rules(m, N, code, wt, &ptr, &col, &w)) { free(code); free(wt); free(ptr); free(col); free(w); return 2; }
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < nrows; ++r) {
    int64_t *cur = out + (size_t)r * N; /* k = 1: row rows[r] of A */
    for (int64_t j = 0; j < N; ++j) cur[j] = RDO_INF;
    for (int64_t e = ptr[rows[r]]; e < ptr[rows[r] + 1]; ++e) cur[col[e]] = w[e];
    for (int k = 2; k <= kmax; ++k) {
      int64_t *prev = out + ((size_t)(k - 2) * nrows + r) * N;
      int64_t *nxt = out + ((size_t)(k - 1) * nrows + r) * N;
      for (int64_t j = 0; j < N; ++j) nxt[j] = RDO_INF;
      for (int64_t t = 0; t < N; ++t) {
        if (prev[t] == RDO_INF) continue;
        for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) {
          int64_t v = prev[t] + w[e];
          if (v < nxt[col[e]]) nxt[col[e]] = v;
        }
      }
    }
  }
  free(code); free(wt); free(ptr); free(col); free(w);
  return 0;
}

/*
 * Algorithm 2 with the first-repeat rule (Lemma 2, Prop. 7), one start word at a
 * time, so that no power is ever held whole (m = 9 has N = 21909; one dense power
 * in int64 is 3.8 GB and the search needs 27 of them).
 *
 * Row p of A^k is e_p (x) A^k: by Theorem 1 its entry t is the least label of a
 * k-arc walk from word p to word t.  For each p the rows k = 1..kmax are built by
 * extending every walk by one arc (arcs from the Sec. 4.A rules, label = weight of
 * the destination word).  Then, for that row alone:
 *   - gamma[k] = min over p of (A^k)_pp (Corollary 6) takes the diagonal entry;
 *   - for every pair i < j <= kmax, "row p of A^j = beta + row p of A^i" is tested
 *     (same infinite entries, one constant difference on the finite ones).
 * A^j = beta (x) A^i holds for the matrix iff it holds for every row with one
 * common beta, so each pair keeps one flag and the beta of the first row that has
 * a finite entry.  The answer is the smallest j with a surviving pair (i, j),
 * reported as (k, p, q) = (i, j - i, beta) -- the same rule and the same results
 * as rdo_power_until_periodic.  gamma[1..kmax] are all filled; j_out is the j of
 * the repeat, or kmax when none was found (return 5).  Memory: kmax * N int64 per
 * thread.
 */
int rdo_power_until_periodic_rows(int m, int kmax, int64_t *gamma, int32_t *k_out, int32_t *p_out, int64_t *q_out,
                                  int32_t *j_out) {
  int64_t N = rdo_num_words(m);
  if (N <= 0 || kmax < 2 || kmax > 200) return 1;
  uint32_t *code = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
  int32_t *wt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!code || !wt) { free(code); free(wt); return 2; }
  rdo_words(m, code, wt, N);
  int64_t *ptr = 0, *col = 0, *w = 0;
  if (build_arcs_from_rules(m, N, code, wt, &ptr, &col, &w)) {
    free(code); free(wt); free(ptr); free(col); free(w);
    return 2;
  }
  /* pair (i, j), 1 <= i < j <= kmax, is slot (j-1)(j-2)/2 + (i-1) */
  const int npairs = kmax * (kmax - 1) / 2;
  int64_t *gmin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(kmax + 1));
  int *alive = (int *)malloc(sizeof(int) * (size_t)npairs);
  int *have = (int *)malloc(sizeof(int) * (size_t)npairs);
  int64_t *beta = (int64_t *)malloc(sizeof(int64_t) * (size_t)npairs);
  int rc = 0;
  if (!gmin || !alive || !have || !beta) rc = 2;
  if (rc == 0) {
    for (int k = 0; k <= kmax; ++k) gmin[k] = RDO_INF;
    for (int s = 0; s < npairs; ++s) { alive[s] = 1; have[s] = 0; beta[s] = 0; }
#pragma omp parallel
    {
      int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)kmax * (size_t)N); /* row of A^k at (k-1)*N */
      int64_t *lmin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(kmax + 1));
      int *lalive = (int *)malloc(sizeof(int) * (size_t)npairs);
      int *lhave = (int *)malloc(sizeof(int) * (size_t)npairs);
      int64_t *lbeta = (int64_t *)malloc(sizeof(int64_t) * (size_t)npairs);
      int ok = rows && lmin && lalive && lhave && lbeta;
      if (ok) {
        for (int k = 0; k <= kmax; ++k) lmin[k] = RDO_INF;
        for (int s = 0; s < npairs; ++s) { lalive[s] = 1; lhave[s] = 0; lbeta[s] = 0; }
      }
#pragma omp for schedule(dynamic, 8)
      for (int64_t p = 0; p < N; ++p) {
        if (!ok) continue;
        int64_t *cur = rows; /* k = 1: row p of A */
        for (int64_t t = 0; t < N; ++t) cur[t] = RDO_INF;
        for (int64_t e = ptr[p]; e < ptr[p + 1]; ++e) cur[col[e]] = w[e];
        for (int k = 2; k <= kmax; ++k) {
          const int64_t *prev = rows + (size_t)(k - 2) * N;
          int64_t *nxt = rows + (size_t)(k - 1) * N;
          for (int64_t t = 0; t < N; ++t) nxt[t] = RDO_INF;
          for (int64_t t = 0; t < N; ++t) {
            if (prev[t] == RDO_INF) continue;
            for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) {
              int64_t v = prev[t] + w[e];
              if (v < nxt[col[e]]) nxt[col[e]] = v;
            }
          }
        }
        for (int k = 1; k <= kmax; ++k) {
          int64_t d = rows[(size_t)(k - 1) * N + p];
          if (d < lmin[k]) lmin[k] = d;
        }
        for (int j = 2; j <= kmax; ++j)
          for (int i = 1; i < j; ++i) {
            const int s = (j - 1) * (j - 2) / 2 + (i - 1);
            if (!lalive[s]) continue;
            int64_t b;
            if (!same_up_to_offset(rows + (size_t)(i - 1) * N, rows + (size_t)(j - 1) * N, N, &b)) {
              lalive[s] = 0;
              continue;
            }
            int row_has_finite = 0;
            for (int64_t t = 0; t < N && !row_has_finite; ++t) row_has_finite = (rows[(size_t)(i - 1) * N + t] != RDO_INF);
            if (!row_has_finite) continue; /* an all-infinite row fixes no beta */
            if (!lhave[s]) { lhave[s] = 1; lbeta[s] = b; }
            else if (lbeta[s] != b) lalive[s] = 0;
          }
      }
#pragma omp critical
      {
        if (!ok) rc = 2;
        else {
          for (int k = 1; k <= kmax; ++k)
            if (lmin[k] < gmin[k]) gmin[k] = lmin[k];
          for (int s = 0; s < npairs; ++s) {
            if (!lalive[s]) { alive[s] = 0; continue; }
            if (!lhave[s]) continue;
            if (!have[s]) { have[s] = 1; beta[s] = lbeta[s]; }
            else if (beta[s] != lbeta[s]) alive[s] = 0;
          }
        }
      }
      free(rows); free(lmin); free(lalive); free(lhave); free(lbeta);
    }
  }
  if (rc == 0) {
    rc = 5;
    for (int k = 1; k <= kmax; ++k) gamma[k] = gmin[k];
    *j_out = kmax;
    for (int j = 2; j <= kmax && rc == 5; ++j)
      for (int i = 1; i < j; ++i) {
        const int s = (j - 1) * (j - 2) / 2 + (i - 1);
        if (alive[s]) {
          *k_out = i; *p_out = j - i; *q_out = have[s] ? beta[s] : 0; *j_out = j;
          rc = 0;
          break;
        }
      }
  }
  free(code); free(wt); free(ptr); free(col); free(w);
  free(gmin); free(alive); free(have); free(beta);
  return rc;
}

/*
 * Brute force from the definition (Sec. 1): gamma_R(G) is the least weight
 * sum f(v) over f: V -> {0,1,2} such that every v with f(v) = 0 has a neighbour w
 * with f(w) = 2.  G = P_m box C_n: vertex (r, c), r = 0..m-1 along the path, c =
 * 0..n-1 around the cycle; neighbours (r +- 1, c) when in range and (r, c +- 1 mod n).
 * Exhaustive depth-first search over all 3^(mn) assignments in vertex order
 * v = c*m + r.  A branch is cut only when (i) its weight already reaches the
 * best found, or (ii) some vertex and its whole neighbourhood are assigned and
 * the vertex is 0 with no neighbour 2 -- both cuts discard only assignments that
 * cannot be better RDFs.  Every complete assignment is re-checked in full.
 */
typedef struct {
  int m, n, V;
  int nb[64][4], deg[64];
  int last_needed[64]; /* vertex index after which v's closed neighbourhood is fully assigned */
  int f[64];
  int64_t best;
} bf_state;

static int bf_ok(const bf_state *s, int v) {
  if (s->f[v] != 0) return 1;
  for (int e = 0; e < s->deg[v]; ++e)
    if (s->f[s->nb[v][e]] == 2) return 1;
  return 0;
}

static void bf_rec(bf_state *s, int v, int64_t w) {
  if (w >= s->best) return;
  if (v == s->V) {
    for (int u = 0; u < s->V; ++u)
      if (!bf_ok(s, u)) return;
    s->best = w;
    return;
  }
  for (int val = 0; val <= 2; ++val) {
    s->f[v] = val;
    int fine = 1;
    for (int u = 0; u < s->V && fine; ++u)
      if (s->last_needed[u] == v && !bf_ok(s, u)) fine = 0;
    if (fine) bf_rec(s, v + 1, w + val);
  }
  s->f[v] = -1;
}

int64_t rdo_brute_force(int m, int n) {
  if (m < 1 || n < 3 || m * n > 64) return -1;
  bf_state *s = (bf_state *)calloc(1, sizeof(bf_state));
  if (!s) return -1;
  s->m = m; s->n = n; s->V = m * n;
  for (int c = 0; c < n; ++c)
    for (int r = 0; r < m; ++r) {
      int v = c * m + r, d = 0;
      if (r > 0) s->nb[v][d++] = c * m + (r - 1);
      if (r < m - 1) s->nb[v][d++] = c * m + (r + 1);
      s->nb[v][d++] = ((c + 1) % n) * m + r;
      s->nb[v][d++] = ((c + n - 1) % n) * m + r;
      s->deg[v] = d;
    }
  for (int v = 0; v < s->V; ++v) {
    int last = v;
    for (int e = 0; e < s->deg[v]; ++e)
      if (s->nb[v][e] > last) last = s->nb[v][e];
    s->last_needed[v] = last;
    s->f[v] = -1;
  }
  s->best = 2 * (int64_t)s->V + 1; /* f = 1 everywhere is an RDF of weight V */
  bf_rec(s, 0, 0);
  int64_t r = s->best;
  free(s);
  return r;
}

/*
 * Second exact method, sharing nothing with the column words: dynamic
 * programming along the PATH direction.  Row r (r = 1..m) is one copy of C_n
 * with an assignment g in {0,1,2}^n.  After row r is placed, the state is
 * (g_r, U_r) where U_r is the set of 0-vertices of row r that are dominated
 * neither by row r - 1 nor inside row r (cycle neighbours); they must be
 * dominated by a 2 in the same column of row r + 1.  Virtual rows 0 and m+1
 * carry no 2s, so U_m must be empty.
 */
int64_t rdo_row_dp(int m, int n) {
  if (m < 1 || n < 3 || n > 9) return -1;
  int64_t G = 1;
  for (int i = 0; i < n; ++i) G *= 3;
  int64_t S = G << n; /* state index: g * 2^n + U */
  int *wt = (int *)malloc(sizeof(int) * (size_t)G);
  uint32_t *two = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)G);
  uint32_t *open = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)G); /* zeros with no 2 among their cycle neighbours */
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
  int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
  if (!wt || !two || !open || !cur || !nxt) { free(wt); free(two); free(open); free(cur); free(nxt); return -2; }
  for (int64_t g = 0; g < G; ++g) {
    int val[16];
    int64_t x = g;
    int w = 0;
    uint32_t tm = 0;
    for (int c = 0; c < n; ++c) { val[c] = (int)(x % 3); x /= 3; w += val[c]; if (val[c] == 2) tm |= 1u << c; }
    uint32_t op = 0;
    for (int c = 0; c < n; ++c)
      if (val[c] == 0 && val[(c + 1) % n] != 2 && val[(c + n - 1) % n] != 2) op |= 1u << c;
    wt[g] = w; two[g] = tm; open[g] = op;
  }
  for (int64_t s = 0; s < S; ++s) cur[s] = RDO_INF;
  for (int64_t g = 0; g < G; ++g) cur[(g << n) | open[g]] = wt[g]; /* row 1: nothing above */
  for (int r = 2; r <= m; ++r) {
    for (int64_t s = 0; s < S; ++s) nxt[s] = RDO_INF;
    for (int64_t s = 0; s < S; ++s) {
      if (cur[s] == RDO_INF) continue;
      int64_t g = s >> n;
      uint32_t U = (uint32_t)(s & ((1 << n) - 1));
      for (int64_t h = 0; h < G; ++h) {
        if ((U & ~two[h]) != 0) continue; /* an undominated 0 above needs a 2 below it */
        uint32_t Uh = open[h] & ~two[g];  /* zeros of row r not covered by row r-1 or their own row */
        int64_t v = cur[s] + wt[h];
        int64_t idx = (h << n) | Uh;
        if (v < nxt[idx]) nxt[idx] = v;
      }
    }
    int64_t *t = cur; cur = nxt; nxt = t;
  }
  int64_t best = RDO_INF;
  for (int64_t g = 0; g < G; ++g)
    if (cur[g << n] < best) best = cur[g << n]; /* U_m empty */
  free(wt); free(two); free(open); free(cur); free(nxt);
  return best;
}

/*
 * Algorithm 1 for every n = 1..nmax: gamma[n] = min_p (A^n)_pp (Corollary 6),
 * powering straight through with no period detection.  Keeps two powers only.
 */
int rdo_gamma_direct(int m, int nmax, int64_t *gamma) {
  int64_t N = rdo_num_words(m);
  if (N <= 0 || nmax < 1) return 1;
  size_t n2 = (size_t)N * (size_t)N;
  int64_t *A = (int64_t *)malloc(sizeof(int64_t) * n2);
  int64_t *X = (int64_t *)malloc(sizeof(int64_t) * n2);
  int64_t *Z = (int64_t *)malloc(sizeof(int64_t) * n2);
  int64_t *ptr = 0, *col = 0, *w = 0;
  if (!A || !X || !Z) { free(A); free(X); free(Z); return 2; }
  rdo_transfer(m, A, N);
  if (build_arcs(A, N, &ptr, &col, &w)) { free(A); free(X); free(Z); return 2; }
  memcpy(X, A, sizeof(int64_t) * n2);
  gamma[1] = diag_min(X, N);
  for (int n = 2; n <= nmax; ++n) {
    power_step(X, N, ptr, col, w, Z);
    int64_t *t = X; X = Z; Z = t;
    gamma[n] = diag_min(X, N);
  }
  free(A); free(X); free(Z); free(ptr); free(col); free(w);
  return 0;
}

/* Rows rows[r] of A(G) (Corollary 6), out[r*N + p], for sizes where the full matrix is too large. */
int rdo_transfer_rows(int m, const int64_t *rows, int nrows, int64_t *out) {
  int64_t N = rdo_num_words(m);
  if (N <= 0) return 1;
  uint32_t *code = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
  int32_t *wt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!code || !wt) { free(code); free(wt); return 2; }
  rdo_words(m, code, wt, N);
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < nrows; ++r)
    for (int64_t p = 0; p < N; ++p)
      out[(int64_t)r * N + p] = rdo_follows(m, code[rows[r]], code[p]) ? (int64_t)wt[p] : RDO_INF;
  free(code);
  free(wt);
  return 0;
}

/* ======================================================================
 * Appendix variant: almost Roman dominating functions on the top m rows of a
 * tall cylinder (the paper uses m = 4).  Vertices of the last row need not be
 * dominated, and the arc label counts the loss 5 g - 2 |D(g)|.
 * ====================================================================== */

/*
 * "p can follow q" for the variant (Appendix, conditions for a word to follow
 * another): rows 1..m-1 as in Sec. 4.A; in the last row, q_m = d no longer
 * forces p_m = a and behaves like q_m = c.  Readings of two typos: the
 * forbidden factors are ad, da, ab, ba, bb as in Definition 4 (the appendix
 * prints "ac, ca"), and the last-row case q_m = b reads "or p_m = d" (printed
 * "p_3 = d").
 */
int rdo_follows_loss(int m, uint32_t q, uint32_t p) {
  for (int i = 1; i <= m; ++i) {
    int qi = letter(m, q, i), pi = letter(m, p, i);
    if (i == m && qi == LD) qi = LC; /* the last row needs no domination */
    int ok;
    switch (qi) {
      case LA: ok = (pi == LA || pi == LC); break;
      case LB: ok = (pi == LD) || (pi == LC && has_vertical_a(m, p, i)); break;
      case LC: ok = (pi == LA || pi == LB || pi == LD) || (pi == LC && has_vertical_a(m, p, i)); break;
      default: ok = (pi == LA); break;
    }
    if (!ok) return 0;
  }
  return 1;
}

/* Algorithm 3: nd(q,p), the vertices newly dominated by column p after column q. */
int rdo_nd(int m, uint32_t q, uint32_t p) {
  int nd = 0;
  for (int i = 1; i <= m; ++i) {
    const int qi = letter(m, q, i), pi = letter(m, p, i);
    if (qi == LA && pi == LA) nd += 1;
    else if (qi == LB && pi == LC) nd += 1;
    else if (qi == LC && pi == LA) nd += 2;
    else if ((qi == LC || qi == LD) && (pi == LB || pi == LC)) nd += 1;
    else if (qi == LD && pi == LA) nd += 3;
  }
  if (letter(m, p, m) == LA) nd += 1; /* the vertex below the strip */
  return nd;
}

/* The variant's matrix: A[q][p] = 10 p(a) + 5 p(b) - 2 nd(q,p) on arcs, else infinity (raw, may be negative). */
int rdo_transfer_loss(int m, int64_t *A, int64_t N) {
  int64_t n = rdo_num_words(m);
  if (n < 0 || n != N) return 1;
  uint32_t *code = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
  int32_t *wt = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!code || !wt) { free(code); free(wt); return 2; }
  rdo_words(m, code, wt, N);
  for (int64_t q = 0; q < N; ++q)
    for (int64_t p = 0; p < N; ++p) {
      if (!rdo_follows_loss(m, code[q], code[p])) { A[q * N + p] = RDO_INF; continue; }
      int na = 0, nb = 0;
      for (int i = 1; i <= m; ++i) {
        na += letter(m, code[p], i) == LA;
        nb += letter(m, code[p], i) == LB;
      }
      A[q * N + p] = 10 * na + 5 * nb - 2 * rdo_nd(m, code[q], code[p]);
    }
  free(code);
  free(wt);
  return 0;
}

/*
 * Exhaustive 2 L_a(n) from the definition (Appendix): the least 5 g(P_m box C_n)
 * - 2 |D(g)| over g: V -> {0,1,2} such that every 0-vertex outside the last row
 * has a neighbour valued 2; D(g) = R_1 with N[R_2], neighbourhoods taken in the
 * taller cylinder, so a 2 in the last row also dominates the vertex below it.
 * All 3^(mn) assignments are visited (mn <= 20).
 */
int64_t rdo_brute_force_loss(int m, int n) {
  if (m < 2 || n < 3 || m * n > 20) return INT64_MIN;
  const int V = m * n;
  int f[20];
  for (int v = 0; v < V; ++v) f[v] = 0;
  int64_t best = INT64_MAX;
  for (;;) {
    int ok = 1;
    int64_t w = 0, dom = 0;
    for (int c = 0; c < n && ok; ++c)
      for (int r = 0; r < m; ++r) {
        const int v = c * m + r;
        w += f[v];
        int has2 = (f[v] == 2);
        if (r > 0 && f[v - 1] == 2) has2 = 1;
        if (r < m - 1 && f[v + 1] == 2) has2 = 1;
        if (f[((c + 1) % n) * m + r] == 2) has2 = 1;
        if (f[((c + n - 1) % n) * m + r] == 2) has2 = 1;
        const int dominated = (f[v] >= 1) || has2;
        if (!dominated && r < m - 1) { ok = 0; break; }
        dom += dominated;
        if (r == m - 1 && f[v] == 2) dom += 1; /* the vertex below, outside the strip */
      }
    if (ok && 5 * w - 2 * dom < best) best = 5 * w - 2 * dom;
    int v = 0;
    while (v < V && f[v] == 2) f[v++] = 0;
    if (v == V) break;
    ++f[v];
  }
  return best;
}
