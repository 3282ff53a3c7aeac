// Element partitions and halo lists of a sharded condensed operator (host only).
//
// Not in the paper.  The condensation (Sec. 2.2, eqs. StaticCondBlock, SC_step1, SC_step2)
// is local to each element, so a run over several GPUs would give each rank whole elements:
// assembly, interior inverses, Schur blocks and back-substitution need no exchange.  The
// implicit operator S x_b = A_bb x_b - A_bi A_ii^-1 A_ib x_b needs two per application:
//   * before the interior pass, the boundary values x_b of every element that couples to an
//     owned element's rows: its 6 face neighbours (the interior and boundary rows see the
//     neighbour's face values through the fluxes and the lifted gradient) and its 12 edge
//     neighbours (BR1: the lifted gradient at a face node reaches across the adjacent face);
//   * before the boundary pass, the interior values u = A_ii^-1 (A_ib x_b) of its face
//     neighbours (a boundary row sees the neighbour's interior nodes on the line normal to
//     the shared face through the viscous flux).
// This build runs on one GPU (replicas); the lists are the layout of a sharded run and are
// tested with CPU ranks.
#include <algorithm>
#include <vector>

#include "sc_internal.cuh"

namespace {

inline int wrap(int i, int n) { return ((i % n) + n) % n; }

// The 6 face (f = 1) or 12 edge (f = 2) neighbours of element (x, y, z) on the periodic n^3 mesh.
void neighbours(int n, int e, int kind, std::vector<int>& out) {
  const int x = e % n, y = (e / n) % n, z = e / (n * n);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz != kind) continue;
        out.push_back(wrap(x + dx, n) + n * (wrap(y + dy, n) + n * wrap(z + dz, n)));
      }
}

}  // namespace

extern "C" {

sc_status sc_partition_slabs(int n, int nparts, int* part) {
  if (!part || n < 1 || n > 32 || nparts < 1 || nparts > n) return SC_ERR_ARG;
  for (int e = 0; e < n * n * n; ++e) part[e] = (int)((long long)(e / (n * n)) * nparts / n);
  return SC_OK;
}

sc_status sc_partition_halo(int n, const int* part, int rank, int* counts, int* owned, int* halo_b, int* halo_u) {
  if (!part || !counts || !owned || !halo_b || !halo_u || n < 1 || n > 32 || rank < 0) return SC_ERR_ARG;
  const int K = n * n * n;
  std::vector<char> is_owned(K, 0), in_b(K, 0), in_u(K, 0);
  int no = 0;
  for (int e = 0; e < K; ++e)
    if (part[e] == rank) { is_owned[e] = 1; owned[no++] = e; }
  std::vector<int> nb;
  for (int i = 0; i < no; ++i) {
    nb.clear();
    neighbours(n, owned[i], 1, nb);
    for (int m : nb)
      if (!is_owned[m]) in_b[m] = in_u[m] = 1;
    nb.clear();
    neighbours(n, owned[i], 2, nb);
    for (int m : nb)
      if (!is_owned[m]) in_b[m] = 1;
  }
  int hb = 0, hu = 0;
  for (int e = 0; e < K; ++e) {
    if (in_b[e]) halo_b[hb++] = e;
    if (in_u[e]) halo_u[hu++] = e;
  }
  counts[0] = no;
  counts[1] = hb;
  counts[2] = hu;
  return SC_OK;
}

}  // extern "C"
