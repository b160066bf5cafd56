// Element-tile domain decomposition of one grid (the sharding of the Schur
// system over devices, host side).
//
// The mx x my elements are split into px x py contiguous tiles; rank
// ty * px + tx owns element columns [ix0, ix1) and rows [iy0, iy1), with
// ix0 = tx mx / px (integer division), so tile sizes differ by at most one.
// A rank owns the interface slots of its own elements.  Every per-step
// exchange of Algorithm 3 (Sec. 2) across a cut goes through the two slot
// lists of each side of the tile:
//   own[k]    : this rank's slot (e, F, t) on the cut face F of its boundary
//               element e,
//   facing[k] : the peer's slot (nbr(e, F), opp F, t) across it,
// ordered along the cut (element row or column ascending, then t), so that a
// rank's facing list towards a peer is the peer's own list towards it.  The
// Schur apply in push form sends the products T_e v_e destined for `facing`;
// a block-Jacobi block of a black element on the cut reads the peer's values
// at `facing` and sends its results back to them; Z^T v adds the two sides'
// partial sums of each cut interface (an all-reduce of the d-vector, after
// which every rank runs the same coarse solve); the Gram-Schmidt dot
// products are all-reduced.
#include <cstring>

#include "smpm_internal.h"

namespace smpm {

namespace {

void tile_of(const Geometry& g, int px, int py, int rank, smpm_tile* t) {
  const int tx = rank % px, ty = rank / px;
  std::memset(t, 0, sizeof(*t));
  t->px = px;
  t->py = py;
  t->rank = rank;
  t->ix0 = static_cast<int>(static_cast<long long>(tx) * g.mx / px);
  t->ix1 = static_cast<int>(static_cast<long long>(tx + 1) * g.mx / px);
  t->iy0 = static_cast<int>(static_cast<long long>(ty) * g.my / py);
  t->iy1 = static_cast<int>(static_cast<long long>(ty + 1) * g.my / py);
  t->nel_owned = static_cast<long long>(t->ix1 - t->ix0) * (t->iy1 - t->iy0);
  const int peer[4] = {tx > 0 ? rank - 1 : -1, tx < px - 1 ? rank + 1 : -1, ty > 0 ? rank - px : -1,
                       ty < py - 1 ? rank + px : -1};
  t->npeers = 0;
  for (int s = 0; s < 4; ++s) {
    t->peers[s] = peer[s];
    const long long along = s < 2 ? (t->iy1 - t->iy0) : (t->ix1 - t->ix0);
    t->halo[s] = peer[s] >= 0 ? along * g.n : 0;
    if (peer[s] >= 0) ++t->npeers;
  }
}

}  // namespace

int partition_tile(const Geometry& g, int px, int py, int rank, smpm_tile* t) {
  if (px < 1 || py < 1 || px > g.mx || py > g.my || rank < 0 || rank >= px * py) return SMPM_EINVAL;
  tile_of(g, px, py, rank, t);
  return SMPM_OK;
}

int partition_halo(const Geometry& g, int px, int py, int rank, int side, long long* own, long long* facing) {
  smpm_tile t;
  const int st = partition_tile(g, px, py, rank, &t);
  if (st != SMPM_OK) return st;
  if (side < 0 || side > 3 || t.peers[side] < 0) return SMPM_EINVAL;
  const int n = g.n, M = g.M, F = side;  // side W/E/S/N is the cut face of the boundary elements
  long long k = 0;
  if (F < 2) {
    const int ix = F == FACE_W ? t.ix0 : t.ix1 - 1;
    for (int iy = t.iy0; iy < t.iy1; ++iy) {
      const int e = iy * g.mx + ix, e2 = g.neighbour(e, F);
      for (int s = 0; s < n; ++s, ++k) {
        if (own) own[k] = static_cast<long long>(e) * M + F * n + s;
        if (facing) facing[k] = static_cast<long long>(e2) * M + opposite(F) * n + s;
      }
    }
  } else {
    const int iy = F == FACE_S ? t.iy0 : t.iy1 - 1;
    for (int ix = t.ix0; ix < t.ix1; ++ix) {
      const int e = iy * g.mx + ix, e2 = g.neighbour(e, F);
      for (int s = 0; s < n; ++s, ++k) {
        if (own) own[k] = static_cast<long long>(e) * M + F * n + s;
        if (facing) facing[k] = static_cast<long long>(e2) * M + opposite(F) * n + s;
      }
    }
  }
  return SMPM_OK;
}

}  // namespace smpm
