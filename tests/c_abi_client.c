/* A plain C99 client of libdgcns: only include/dgcns.h and the shared library, no CUDA headers,
 * no C++, no Python.  It checks the host-side contract of dg_cns_create (argument validation,
 * error codes, the message of a failed create, *out left NULL) and the NULL-context calls, then
 * creates a valid Taylor--Green context of 2^3 cells, k = 3.  On a machine with a GPU that context
 * is created and destroyed; without one the create must fail with DGCNS_ERR_CUDA.  Prints one
 * "name code" line per check and exits 0 when every expectation holds. */
#include <stdio.h>
#include <string.h>

#include "dgcns.h"

static int failures = 0;

static void expect(const char* name, int got, int want) {
  printf("%s %d\n", name, got);
  if (got != want) {
    fprintf(stderr, "%s: got %d, want %d (%s)\n", name, got, want, dg_cns_last_error(NULL));
    ++failures;
  }
}

static void tgv_setup(dgcns_mesh* m, dgcns_params* p) {
  const double pi = 3.14159265358979323846;
  memset(m, 0, sizeof(*m));
  memset(p, 0, sizeof(*p));
  for (int d = 0; d < 3; ++d) {
    m->n[d] = 2;
    m->lo[d] = -pi;
    m->hi[d] = pi;
    m->periodic[d] = 1;
  }
  m->mapping = DGCNS_MAP_AFFINE;
  p->k = 3;
  p->nq_conv = 5;
  p->nq_visc = 4;
  p->gamma = 1.4;
  p->Pr = 0.71;
  p->Re = 1600.0;
  p->Ma = 0.1;
  p->R = 287.0;
  p->rho0 = 1.0;
  p->U0 = 1.0;
  p->L = 1.0;
  p->precision = DGCNS_FP64;
  p->kernel = DGCNS_KERNEL_FACES;
  p->geometry = DGCNS_GEO_STORED;
}

int main(int argc, char** argv) {
  const int have_gpu = argc > 1 && strcmp(argv[1], "gpu") == 0;
  dgcns_mesh m;
  dgcns_params p;
  dgcns_ctx* ctx = (dgcns_ctx*)&m; /* any non-NULL value: a failed create must reset it */

  tgv_setup(&m, &p);
  p.k = 0;
  expect("create_k0", dg_cns_create(&m, &p, NULL, &ctx), DGCNS_ERR_UNSUPPORTED);
  if (ctx != NULL) ++failures;

  tgv_setup(&m, &p);
  p.nq_visc = 3;
  expect("create_nq_below_k_plus_1", dg_cns_create(&m, &p, NULL, &ctx), DGCNS_ERR_INVALID_ARG);

  tgv_setup(&m, &p);
  m.n[0] = 2048;
  m.n[1] = 1024;
  m.n[2] = 1024;
  expect("create_too_many_cells", dg_cns_create(&m, &p, NULL, &ctx), DGCNS_ERR_INVALID_ARG);
  if (strstr(dg_cns_last_error(NULL), "too many cells") == NULL) ++failures;

  tgv_setup(&m, &p);
  p.nq_conv = 9;
  p.nq_visc = 9;
  expect("create_not_instantiated", dg_cns_create(&m, &p, NULL, &ctx), DGCNS_ERR_UNSUPPORTED);

  /* host-only face table of a rotated-frame mesh: neighbours are cell indices, frames lie in [0, 48),
     orientation codes in 9 bits; a wall is refused */
  {
    dgcns_mesh r;
    int table[8 * 12], frames[8];
    memset(&r, 0, sizeof r);
    for (int d = 0; d < 3; ++d) {
      r.n[d] = 2;
      r.hi[d] = 1.0;
      r.periodic[d] = 1;
    }
    r.mapping = DGCNS_MAP_ROTATED;
    r.map_param = 1806.0;
    expect("face_table", dg_cns_face_table(&r, table, frames), DGCNS_OK);
    for (int i = 0; i < 8; ++i)
      if (frames[i] < 0 || frames[i] > 47) ++failures;
    for (int i = 0; i < 8 * 6; ++i)
      if (table[2 * i] < 0 || table[2 * i] > 7 || table[2 * i + 1] < 0 || table[2 * i + 1] > 511) ++failures;
    r.periodic[2] = 0;
    expect("face_table_wall", dg_cns_face_table(&r, table, frames), DGCNS_ERR_INVALID_ARG);
  }

  expect("create_null_out", dg_cns_create(&m, &p, NULL, NULL), DGCNS_ERR_INVALID_ARG);
  expect("destroy_null", dg_cns_destroy(NULL), DGCNS_ERR_INVALID_ARG);
  expect("apply_null", dg_cns_apply(NULL, NULL, NULL, DGCNS_OP_L), DGCNS_ERR_INVALID_ARG);
  expect("status_null", dg_cns_status(NULL), DGCNS_ERR_INVALID_ARG);

  tgv_setup(&m, &p);
  const int rc = dg_cns_create(&m, &p, NULL, &ctx);
  if (have_gpu) {
    expect("create_valid", rc, DGCNS_OK);
    if (rc == DGCNS_OK) {
      int64_t nc = 0, nn = 0, nd = 0;
      expect("sizes", dg_cns_sizes(ctx, &nc, &nn, &nd), DGCNS_OK);
      if (nc != 8 || nn != 8 * 64 || nd != 5 * 8 * 64) ++failures;
      expect("destroy", dg_cns_destroy(ctx), DGCNS_OK);
    }
  } else {
    expect("create_valid_without_gpu", rc, DGCNS_ERR_CUDA);
    if (ctx != NULL) ++failures;
  }
  printf("failures %d\n", failures);
  return failures == 0 ? 0 : 1;
}
