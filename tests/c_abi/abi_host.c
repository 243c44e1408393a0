/* A plain C (C11) caller of the library's C ABI (include/rd.h), host-side entry points only: it must compile as
 * C, link against librd.so and run without a GPU.  Prints one line per check; exits non-zero on a failure.
 * Arguments: the first repeat of A(G) for m = 1 as the oracle finds it -- k p q j gamma(1) .. gamma(j). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "rd.h"

static int fails = 0;

static void check(int ok, const char *what) {
  printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) fails++;
}

int main(int argc, char **argv) {
  if (argc < 5) return 2;
  const int j = atoi(argv[4]);
  if (j < 1 || j > 64 || argc != 5 + j) return 2;
  int64_t n = 0;
  check(rd_state_count(9, &n) == RD_OK && n == 21909, "rd_state_count(9) = 21909 (Table 1)");
  check(rd_state_count(0, &n) == RD_ERR_ARG, "rd_state_count(0) rejected");
  int64_t ld = 0;
  check(rd_padded_dim(21909, &ld) == RD_OK && ld == 21912, "rd_padded_dim(21909) = 21912");

  /* m = 1, whose gamma_R(C_n) = ceil(2n/3): the oracle's record installed through the C ABI */
  rd_relation_t rel = {1, 1, atoi(argv[1]), atoi(argv[2]), atoll(argv[3]), j, 0};
  int64_t gamma[65];
  gamma[0] = RD_GAMMA_UNSET;
  for (int i = 1; i <= j; ++i) gamma[i] = atoll(argv[4 + i]);
  int ok_import = rd_gamma_R_import(&rel, gamma) == RD_OK;
  check(ok_import, "rd_gamma_R_import of a consistent m = 1 record");
  int64_t g = 0;
  int all = ok_import;
  for (int64_t k = 3; k <= 3000 && all; ++k) all = rd_gamma_R(1, k, &g) == RD_OK && g == (2 * k + 2) / 3;
  check(all, "rd_gamma_R(1, n) = ceil(2n/3) for n = 3..3000 from the record");
  rd_relation_t back;
  int64_t gb[65];
  int same = rd_gamma_R_export(1, &back, gb, 65) == RD_OK && back.found == 1 && back.k == rel.k &&
             back.p == rel.p && back.q == rel.q && back.j == j;
  for (int i = 1; i <= j && same; ++i) same = gb[i] == gamma[i];
  check(same, "rd_gamma_R_export returns the record");
  check(rd_gamma_R_export(1, &back, gb, j) == RD_ERR_ARG, "a gamma buffer one entry short is rejected");
  rel.q += 1; /* gamma[k + p] != gamma[k] + q */
  check(rd_gamma_R_import(&rel, gamma) == RD_ERR_ARG, "an inconsistent record is rejected");
  check(rd_gamma_R_clear() == RD_OK, "rd_gamma_R_clear");

  uint32_t flags = 1;
  check(rd_split_check_flags(&flags, 0) == RD_NOT_FOUND && flags == 0, "no index checks in the normal build");
  check(rd_sparse_record_words(2) == 4 && rd_sparse_record_words(3) == 0, "rd_sparse_record_words");
  check(rd_tune_bucket(1024) == 10, "rd_tune_bucket(1024) = 10");
  return fails != 0;
}
