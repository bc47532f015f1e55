/*
 * A plain C consumer of the h2sp C ABI (include/h2sp.h), with no CUDA call:
 * the host analysis of a hand-built H^2 structure (Definition 4.9) and the
 * integer exports.  Two leaves of four points under one root; the leaves are
 * an admissible pair (rank 2 bases), each leaf is close only to itself.
 * Expected S (§3): the non-basis parts of the two leaves (2 rows each), then
 * the top node (the root, 2 + 2 basis rows); blocks: each leaf with itself
 * and with the top node (a row and a column panel), the top with itself.
 * Prints "ok" and exits 0 when every check holds.
 */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "h2sp.h"

#define CHECK(c)                                                     \
  do {                                                               \
    if (!(c)) {                                                      \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c); \
      return 1;                                                      \
    }                                                                \
  } while (0)

int main(void) {
  const int32_t level_ptr[3] = {0, 1, 3};
  const int32_t parent[3] = {-1, 0, 0};
  const int64_t begin[3] = {0, 0, 4}, size[3] = {8, 4, 4};
  const int32_t rank[3] = {0, 2, 2};
  const int64_t far_ptr[4] = {0, 0, 1, 2};
  const int32_t far_col[2] = {2, 1};
  const int64_t near_ptr[3] = {0, 1, 2};
  const int32_t near_col[2] = {1, 2};
  const int64_t leaf_basis_off[2] = {0, 8}, transfer_off[3] = {0, 0, 0}, coupling_off[2] = {0, 4};
  const int64_t near_off[2] = {0, 16};
  h2sp_h2_desc d;
  memset(&d, 0, sizeof d);
  d.n = 8;
  d.depth = 1;
  d.level_ptr = level_ptr;
  d.parent = parent;
  d.begin = begin;
  d.size = size;
  d.rank = rank;
  d.far_ptr = far_ptr;
  d.far_col = far_col;
  d.near_ptr = near_ptr;
  d.near_col = near_col;
  d.leaf_basis_off = leaf_basis_off;
  d.transfer_off = transfer_off;
  d.coupling_off = coupling_off;
  d.near_off = near_off;

  h2sp_handle *h = NULL;
  CHECK(h2sp_analyze(NULL, &h) == H2SP_EINVAL);
  CHECK(h2sp_analyze(&d, &h) == H2SP_OK && h != NULL);

  h2sp_stats st;
  CHECK(h2sp_query(h, &st) == H2SP_OK);
  CHECK(st.n == 8 && st.depth == 1 && st.lstop == 1 && st.nnodes == 3 && st.nsys == 1);
  CHECK(st.nnzb == 7 && st.nnz == 2 * 2 + 2 * 2 + 2 * (2 * 4) * 2 + 4 * 4);
  CHECK(st.factor_prec == -1 && st.sparsify_prec == -1);

  int64_t node_size[3], brow_ptr[4], val_off[7];
  int32_t bcol[7];
  CHECK(h2sp_export_S(h, node_size, brow_ptr, bcol, val_off, NULL, NULL) == H2SP_OK);
  CHECK(node_size[0] == 2 && node_size[1] == 2 && node_size[2] == 4);
  CHECK(brow_ptr[0] == 0 && brow_ptr[1] == 2 && brow_ptr[2] == 4 && brow_ptr[3] == 7);
  CHECK(bcol[0] == 0 && bcol[1] == 2 && bcol[2] == 1 && bcol[3] == 2);
  CHECK(bcol[4] == 0 && bcol[5] == 1 && bcol[6] == 2);

  /* calls that need device buffers or factors are refused on an analysis handle */
  double ld = 0.0;
  CHECK(h2sp_factor(h, H2SP_FP64, NULL) == H2SP_ESTATE);
  CHECK(h2sp_logdet(h, &ld, NULL, NULL) == H2SP_ESTATE);
  CHECK(h2sp_refactor(h, NULL) == H2SP_ESTATE);
  CHECK(strlen(h2sp_status_string(H2SP_ESTATE)) > 0);
  h2sp_destroy(h);
  h2sp_destroy(NULL);
  printf("ok\n");
  return 0;
}
