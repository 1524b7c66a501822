/* A plain C consumer of the C ABI (compiled and run by tests/test_abi_c.py on the CPU): it
 * includes only include/fpdqt.h, links libfpdqt.so and calls the host-only planners and the
 * error API, printing one line per query for the test to compare with the Python binding. */
#include <stdio.h>

#include "fpdqt.h"

int main(void) {
  static const uint32_t primes[] = {2, 3, 7, 31, 251};
  static const uint32_t degs[][2] = {{2, 2}, {1, 6}, {31, 32}, {511, 511}, {1023, 1023}};
  for (unsigned i = 0; i < sizeof primes / sizeof primes[0]; ++i) {
    for (unsigned j = 0; j < sizeof degs / sizeof degs[0]; ++j) {
      for (int algo = FP_ALGO_AUTO; algo <= FP_ALGO_KARATSUBA; ++algo) {
        fp_polymul_plan_t pl;
        const fp_status s = fp_polymul_plan(primes[i], degs[j][0], degs[j][1], algo, &pl);
        if (s == FP_OK)
          printf("plan %u %u %u %d ok %u %u %u %u %u %u %u %u\n", primes[i], degs[j][0], degs[j][1], algo,
                 pl.kernel, pl.word, pl.blk_a, pl.blk_b, pl.b, pl.ndig, pl.L, pl.m);
        else
          printf("plan %u %u %u %d err %d\n", primes[i], degs[j][0], degs[j][1], algo, (int)s);
      }
    }
    fp_dqt_params prm;
    if (fp_dqt_choose(primes[i], 3, 1000, FP_WORD_U64, &prm) == FP_OK)
      printf("dqt %u ok %u %u\n", primes[i], prm.b, prm.ndig);
    uint32_t b = 0, e = 0, chunk = 0;
    if (fp_mm_choose(primes[i], 4096, FP_MM_RIGHT_F64, &b, &e, &chunk) == FP_OK)
      printf("mm %u ok %u %u %u\n", primes[i], b, e, chunk);
  }
  /* an invalid call returns a status and leaves a message; nothing is thrown */
  fp_polymul_plan_t pl;
  const fp_status bad = fp_polymul_plan(4, 2, 2, FP_ALGO_AUTO, &pl);
  const char* msg = fp_last_error();
  printf("bad %d %s\n", (int)bad, msg && msg[0] ? "message" : "none");
  return 0;
}
