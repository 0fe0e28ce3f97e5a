/* A plain C99 program against include/hytet.h: it builds the unit cube as
 * 6 Kuhn tetrahedra through the C ABI, prints its primitive counts, the
 * index function t_w at a few points, the P2 quadrature rule's weight sum
 * and the plane-tile count of level 5.  Every call here is host code, so it
 * runs without a GPU.  Exit status 0 when every call succeeded. */
#include <stdio.h>

#include "hytet.h"

static int check(int status, const char* what) {
  if (status != HG_OK) fprintf(stderr, "%s failed (%d): %s\n", what, status, hg_last_error());
  return status != HG_OK;
}

int main(void) {
  double xyz[8 * 3];
  int64_t cells[6 * 4];
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int v, c, q, fails = 0;
  for (v = 0; v < 8; ++v) {            /* vertex id = x + 2y + 4z */
    xyz[3 * v + 0] = v & 1;
    xyz[3 * v + 1] = (v >> 1) & 1;
    xyz[3 * v + 2] = (v >> 2) & 1;
  }
  for (c = 0; c < 6; ++c) {            /* Kuhn path 0 -> e_s1 -> e_s1 + e_s2 -> (1,1,1) */
    int id = 0;
    cells[4 * c] = 0;
    for (q = 0; q < 3; ++q) {
      id |= 1 << perms[c][q];
      cells[4 * c + q + 1] = id;
    }
  }
  hg_mesh* mesh = NULL;
  fails += check(hg_mesh_create(xyz, 8, cells, 6, &mesh), "hg_mesh_create");
  if (!mesh) return 1;
  int64_t counts[6];
  fails += check(hg_mesh_counts(mesh, counts), "hg_mesh_counts");
  printf("counts %lld %lld %lld %lld %lld %lld\n", (long long)counts[0], (long long)counts[1],
         (long long)counts[2], (long long)counts[3], (long long)counts[4], (long long)counts[5]);
  hg_mesh_destroy(mesh);
  int64_t t;
  fails += check(hg_index_tw(3, 0, 2, 0, &t), "hg_index_tw");
  printf("tw3 020 %lld\n", (long long)t);
  fails += check(hg_index_tw(3, 0, 0, 2, &t), "hg_index_tw");
  printf("tw3 002 %lld\n", (long long)t);
  printf("tw3 bad %d\n", hg_index_tw(3, 1, 1, 1, &t));
  double bary[14 * 4], w[14], sum = 0.0;
  int np = 0;
  fails += check(hg_quadrature_rule(bary, w, &np), "hg_quadrature_rule");
  for (q = 0; q < np; ++q) sum += w[q];
  printf("quadrature %d %.15f\n", np, sum);
  int ntiles = 0;
  fails += check(hg_plane_tiles(5, NULL, &ntiles), "hg_plane_tiles");
  printf("tiles5 %d\n", ntiles);
  return fails ? 1 : 0;
}
