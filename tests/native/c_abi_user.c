/* A plain C99 user of the C ABI (no Python, no C++): the header compiles as
 * C with every warning an error, and the host-side entry points answer
 * without a GPU (sizes, argument errors, knobs, messages). */
#include <stdio.h>
#include <string.h>

#include "jsvd.h"

int main(void)
{
  size_t bytes = 0, hbytes = 0;
  jsvd_opts o;
  jsvd_evd2_streams s;
  int rc;
  printf("version %d\n", jsvd_version());
  rc = jsvd_svd_workspace_size(JSVD_COMPLEX, NULL, 4096, 2048, &bytes);
  printf("svd_ws %d %lu\n", rc, (unsigned long)bytes);
  printf("svd_ws_bad_n %d\n", jsvd_svd_workspace_size(JSVD_REAL, NULL, 4, 8, &bytes));
  memset(&o, 0, sizeof o);
  o.permute = 2;
  printf("svd_ws_bad_opts %d\n", jsvd_svd_workspace_size(JSVD_REAL, &o, 8, 4, &bytes));
  rc = jsvd_evd2x2_host_workspace_size(&hbytes);
  printf("host_ws %d %lu\n", rc, (unsigned long)hbytes);
  memset(&s, 0, sizeof s);
  printf("evd_missing_stream %d\n", jsvd_evd2x2_batched(JSVD_REAL, &s, 10, NULL));
  printf("evd_empty %d\n", jsvd_evd2x2_batched(JSVD_REAL, &s, 0, NULL));
  printf("tune_bad %d\n", jsvd_tune_set(JSVD_TUNE_SVD_STEP, 6, 0));
  printf("tune_ok %d\n", jsvd_tune_set(JSVD_TUNE_SVD_STEP, 0, 0));
  printf("message %s\n", jsvd_strerror(JSVD_E_WORKSPACE));
  return 0;
}
