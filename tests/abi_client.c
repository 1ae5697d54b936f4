/* A plain C99 client of the C ABI (include/imdp.h), built and run by
 * tests/test_abi.py: the header must compile as strict C and the host-only
 * calls must work through it without a GPU. Reads the bmdp-tool fixture of the
 * Sec. 3.1 model, writes it back and reads the copy, and compares the arrays. */
#include <stdio.h>
#include <string.h>

#include "imdp.h"

static int same(const imdp_file* a, const imdp_file* b) {
  if (a->n_states != b->n_states || a->n_cols != b->n_cols || a->nnz != b->nnz) return 0;
  if (memcmp(a->stateptr, b->stateptr, sizeof(int32_t) * (size_t)(a->n_states + 1)) != 0) return 0;
  if (memcmp(a->colptr, b->colptr, sizeof(int32_t) * (size_t)(a->n_cols + 1)) != 0) return 0;
  if (memcmp(a->rowval, b->rowval, sizeof(int32_t) * (size_t)a->nnz) != 0) return 0;
  if (memcmp(a->lower, b->lower, sizeof(double) * (size_t)a->nnz) != 0) return 0;
  return memcmp(a->upper, b->upper, sizeof(double) * (size_t)a->nnz) == 0;
}

int main(int argc, char** argv) {
  imdp_file* f = NULL;
  imdp_file* g = NULL;
  imdp_status st;
  if (argc != 3) return 2;
  printf("version %s\n", imdp_version());
  printf("status %s\n", imdp_status_string(IMDP_EINFEASIBLE));
  st = imdp_read_bmdp_tool(argv[1], &f);
  if (st != IMDP_OK) {
    printf("read failed: %s\n", imdp_last_error());
    return 1;
  }
  printf("model %d states %d columns %lld transitions, terminal %d\n", f->n_states, f->n_cols, (long long)f->nnz,
         f->spec.n_reach == 1 ? f->spec.reach[0] : -1);
  st = imdp_write_bmdp_tool(argv[2], f->n_states, f->n_cols, f->stateptr, f->colptr, f->rowval, f->lower, f->upper,
                            f->spec.reach, f->spec.n_reach);
  if (st == IMDP_OK) st = imdp_read_bmdp_tool(argv[2], &g);
  printf("round trip %s\n", st == IMDP_OK && same(f, g) ? "same" : "different");
  {
    imdp_file* h = NULL;
    st = imdp_read_bmdp_tool("/nonexistent/file.bmdp", &h);
    printf("missing file: %s%s\n", imdp_status_string(st), h == NULL ? "" : " (output set)");
  }
  imdp_file_free(f);
  imdp_file_free(g);
  imdp_file_free(NULL);
  return 0;
}
