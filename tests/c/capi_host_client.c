/* A plain C99 client of the library's host-side calls: grid, mesh, CSR,
 * permutation and EqualRegions partition with one-ring halos (Sec. 4.2,
 * 4.3, 4.4).  It needs no GPU.  Built and run by tests/test_capi_c.py; it
 * prints one line per check and returns the number of failed checks.
 *
 *   usage: capi_host_client N nparts
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "nabla_b300.h"

static int failures = 0;

static void check(int ok, const char *what) {
  printf("%s %s\n", ok ? "ok  " : "FAIL", what);
  if (!ok) ++failures;
}

int main(int argc, char **argv) {
  const int N = argc > 1 ? atoi(argv[1]) : 32;
  const int nparts = argc > 2 ? atoi(argv[2]) : 4;
  printf("version %s\n", nb_version());

  /* a bad Gaussian number is rejected with a message */
  nb_grid *bad = NULL;
  check(nb_grid_create_octahedral(0, &bad) == NB_EINVAL && bad == NULL, "O0 rejected with NB_EINVAL");
  check(strlen(nb_last_error()) > 0, "nb_last_error set");

  nb_grid *grid = NULL;
  check(nb_grid_create_octahedral(N, &grid) == NB_OK, "grid created");
  int64_t V = 0;
  nb_grid_size(grid, &V);
  check(V == 4LL * N * N + 36LL * N, "V = 4N^2 + 36N");

  int32_t *pl = (int32_t *)malloc(sizeof(int32_t) * 2 * N);
  nb_grid_pl(grid, pl);
  int rows_ok = 1;
  for (int j = 0; j < 2 * N; ++j) {
    const int d = j < N ? j : 2 * N - 1 - j;
    rows_ok &= pl[j] == 20 + 4 * d;
  }
  check(rows_ok, "row lengths 20 + 4j from either pole");

  nb_mesh *mesh = NULL;
  check(nb_mesh_create(grid, 1, &mesh) == NB_OK, "mesh created (Hilbert order)");
  int64_t nv = 0, ne = 0, nt = 0;
  nb_mesh_sizes(mesh, &nv, &ne, &nt);
  check(nv == V && ne == 3 * V - 6 && nt == 2 * V - 4, "Euler: E = 3V - 6, F = 2V - 4");

  int64_t *row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V + 1));
  int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne));
  nb_mesh_csr(mesh, row_ptr, nbr);
  int32_t *mate = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  check(nb_mesh_node_pairs(mesh, mate) == NB_OK, "node pairs queried");
  int csr_ok = row_ptr[0] == 0 && row_ptr[V] == 2 * ne;
  int64_t npaired = 0;
  for (int64_t i = 0; i < V && csr_ok; ++i) {
    const int64_t p0 = row_ptr[i];
    /* a paired row: shared A < B, the partner, then the other three ascending */
    const int paired = mate[i] >= 0;
    npaired += paired;
    if (paired) csr_ok &= row_ptr[i + 1] - p0 == 6 && nbr[p0 + 2] == mate[i] && mate[mate[i]] == i;
    for (int64_t p = p0; p < row_ptr[i + 1]; ++p) {
      csr_ok &= nbr[p] >= 0 && nbr[p] < V && nbr[p] != i;
      if (p > p0 && !(paired && (p == p0 + 2 || p == p0 + 3))) csr_ok &= nbr[p] > nbr[p - 1];
    }
  }
  check(csr_ok, "CSR: neighbours in range, ascending (paired rows: shared pair, partner, rest), no self loops");
  check(npaired > V / 2, "most nodes are paired");
  free(mate);

  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  char *seen = (char *)calloc((size_t)V, 1);
  nb_mesh_permutation(mesh, perm);
  int perm_ok = 1;
  for (int64_t i = 0; i < V; ++i) {
    perm_ok &= perm[i] >= 0 && perm[i] < V && !seen[perm[i]];
    if (perm[i] >= 0 && perm[i] < V) seen[perm[i]] = 1;
  }
  check(perm_ok, "permutation new -> old is a bijection");

  /* EqualRegions: every part V / nparts points (+-1); in mesh order for halos */
  int32_t *part = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  int32_t nzones = 0;
  check(nb_partition_equal_regions(grid, nparts, part, NULL, &nzones) == NB_OK, "EqualRegions partition");
  int64_t *count = (int64_t *)calloc((size_t)nparts, sizeof(int64_t));
  for (int64_t i = 0; i < V; ++i) count[part[i]]++;
  int bal = 1;
  for (int p = 0; p < nparts; ++p) bal &= count[p] >= V / nparts && count[p] <= V / nparts + 1;
  check(bal, "parts hold V / nparts points (+-1)");

  int32_t *mpart = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
  for (int64_t i = 0; i < V; ++i) mpart[i] = part[perm[i]];
  int64_t total_owned = 0, nowned = 0, nhalo = 0;
  int halo_ok = 1;
  for (int p = 0; p < nparts; ++p) {
    nb_partition_halo(mesh, mpart, p, &nowned, NULL, &nhalo, NULL);
    int32_t *owned = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nowned > 0 ? nowned : 1));
    int32_t *halo = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nhalo > 0 ? nhalo : 1));
    nb_partition_halo(mesh, mpart, p, &nowned, owned, &nhalo, halo);
    total_owned += nowned;
    /* every halo node is owned elsewhere and neighbours an owned node */
    for (int64_t h = 0; h < nhalo; ++h) {
      const int32_t j = halo[h];
      int touches = 0;
      for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) touches |= mpart[nbr[q]] == p;
      halo_ok &= mpart[j] != p && touches;
    }
    /* every off-part neighbour of an owned node is in the halo */
    for (int64_t o = 0; o < nowned; ++o)
      for (int64_t q = row_ptr[owned[o]]; q < row_ptr[owned[o] + 1]; ++q) {
        const int32_t j = nbr[q];
        if (mpart[j] == p) continue;
        int64_t lo = 0, hi = nhalo;
        while (lo < hi) {
          const int64_t mid = (lo + hi) / 2;
          if (halo[mid] < j) lo = mid + 1;
          else hi = mid;
        }
        halo_ok &= lo < nhalo && halo[lo] == j;
      }
    free(owned);
    free(halo);
  }
  check(total_owned == V, "owned nodes cover the mesh once");
  check(halo_ok, "halos are exactly the one-ring of the owned nodes");

  nb_mesh_release(mesh);
  nb_grid_release(grid);
  free(pl);
  free(row_ptr);
  free(nbr);
  free(perm);
  free(seen);
  free(part);
  free(count);
  free(mpart);
  printf("failures %d\n", failures);
  return failures;
}
