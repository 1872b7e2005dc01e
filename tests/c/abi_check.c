/* A plain C99 client of the C ABI: it includes include/bdu.h, links against
 * libbdu.so and exercises the calls that need no GPU (version, defaults and
 * the argument checks of the create functions, which fail before any device
 * work).  Exit status 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "bdu.h"

#define CHECK(cond)                                              \
  do {                                                           \
    if (!(cond)) {                                               \
      fprintf(stderr, "check failed line %d: %s\n", __LINE__, #cond); \
      return 1;                                                  \
    }                                                            \
  } while (0)

int main(void) {
  bdu_options o;
  bdu_handle h = (bdu_handle)1;
  bdu_thin_handle t = (bdu_thin_handle)1;
  double Q[16] = {0}, P[16] = {0}, d[4] = {1, 1, 1, 1}, e[3] = {0, 0, 0};

  CHECK(bdu_version() >= 100);
  bdu_default_options(&o);
  CHECK(o.precision == BDU_FP64 && o.nb == 0 && o.graphs == 1 && o.reorth_every == -1);

  /* m < 1: rejected before any device work, *h cleared, message set */
  CHECK(bdu_create(&h, 0, 4, Q, d, e, P, &o) == BDU_EINVAL && h == NULL);
  CHECK(strstr(bdu_last_error(NULL), "m, n >= 1") != NULL);
  /* NULL inputs */
  CHECK(bdu_create(&h, 4, 4, NULL, d, e, P, NULL) == BDU_EINVAL);
  /* rank-k tracking: k must be below min(m, n) */
  CHECK(bdu_thin_create(&t, 4, 4, 4, Q, d, e, P, &o) == BDU_EINVAL && t == NULL);
  CHECK(strstr(bdu_thin_last_error(NULL), "min(m, n)") != NULL);
  /* NULL handles */
  CHECK(bdu_update(NULL, NULL, NULL, 1) == BDU_EINVAL);
  CHECK(bdu_thin_update(NULL, NULL, NULL, NULL, NULL) == BDU_EINVAL);
  bdu_destroy(NULL);
  bdu_thin_destroy(NULL);
  printf("abi_check ok\n");
  return 0;
}
