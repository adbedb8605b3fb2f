/* A plain C client of the ncpadj C-ABI (no C++, no Python), used by the CPU tests to show the
 * header and the library work from C.  It calls only entry points that need no device: the
 * version, status names, default options, argument checks that fail before any device work,
 * and ncpadj_ctx_create on a device that does not exist.  Prints one line per check. */
#include <stdio.h>
#include <string.h>

#include "ncpadj.h"

int main(void) {
  int bad = 0;
  const char* v = ncpadj_version();
  printf("version %s\n", v);
  if (!v || !strstr(v, "sm_103a")) bad = 1;
  if (strcmp(ncpadj_status_string(NCPADJ_OK), "OK") != 0) bad = 1;
  if (strcmp(ncpadj_status_string(NCPADJ_ERR_INVALID_ARG), "INVALID_ARG") != 0) bad = 1;
  ncpadj_options o;
  memset(&o, 0xff, sizeof o);
  ncpadj_options_default(&o);
  printf("options eps=%g rtol=%g max_iters=%d restart=%d precision=%d precond=%d\n", o.eps, o.rtol,
         (int)o.max_iters, (int)o.gmres_restart, (int)o.precision, (int)o.precond);
  if (o.eps != 1e-4 || o.rtol != 1e-8 || o.gmres_restart != 64 || o.precision != NCPADJ_FP64 ||
      o.precond != NCPADJ_PRECOND_WOODBURY || o.cap_block != 0)
    bad = 1;
  /* rejected before any device work */
  ncpadj_status s = ncpadj_adjoint_step(NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
  printf("adjoint_step(NULL...) -> %s: %s\n", ncpadj_status_string(s), ncpadj_last_error());
  if (s == NCPADJ_OK || ncpadj_last_error()[0] == 0) bad = 1;
  ncpadj_scene_info info;
  if (ncpadj_scene_get_info(NULL, &info) != NCPADJ_ERR_INVALID_ARG) bad = 1;
  ncpadj_ctx ctx = NULL;
  s = ncpadj_ctx_create(1000000, &ctx);
  printf("ctx_create(1000000) -> %s\n", ncpadj_status_string(s));
  if (s == NCPADJ_OK || ctx != NULL) bad = 1;
  ncpadj_ctx_destroy(NULL);
  ncpadj_scene_destroy(NULL);
  printf(bad ? "FAIL\n" : "PASS\n");
  return bad;
}
