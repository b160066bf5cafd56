// Internal declarations shared by the host factor step and the CUDA solve.
#pragma once
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/smpm.h"

namespace smpm {

enum { FACE_W = 0, FACE_E = 1, FACE_S = 2, FACE_N = 3 };
constexpr int kMaxN = 32;         // GLL points per direction
constexpr int kMaxRestart = 200;  // GMRES restart length

inline int opposite(int F) { return F ^ 1; }

// Geometry and indexing of one grid (Sec. 1.2).  Element e = iy*mx + ix;
// slot (e, F, t) at e*M + F*n + t with M = 4n; interfaces numbered row by
// row: in element row iy, the mx-1 vertical interfaces (ix | ix+1) at
// iy*(2mx-1) + ix, then the mx horizontal ones (row iy | iy+1) at
// iy*(2mx-1) + mx-1 + ix.  A graded grid has column edges xe (mx+1) and row
// edges ye (my+1): element (ix, iy) covers [xe[ix], xe[ix+1]] x
// [ye[iy], ye[iy+1]]; a uniform grid covers [0,Lx]x[0,Ly] with spacing hx, hy.
struct Geometry {
  int mx = 0, my = 0, n = 0, M = 0;
  double Lx = 1, Ly = 1, hx = 1, hy = 1;
  long long nel = 0, nn = 0, r = 0, kp = 0, d = 0, k = 0;
  bool graded = false;
  std::vector<double> xe, ye;

  double col_h(int ix) const { return graded ? xe[ix + 1] - xe[ix] : hx; }
  double row_h(int iy) const { return graded ? ye[iy + 1] - ye[iy] : hy; }
  double col_x0(int ix) const { return graded ? xe[ix] : ix * hx; }
  double row_y0(int iy) const { return graded ? ye[iy] : iy * hy; }
  double hx_of(int e) const { return col_h(e % mx); }
  double hy_of(int e) const { return row_h(e / mx); }
  // element size across face F: h_x for W/E faces, h_y for S/N faces
  double hperp(int e, int F) const { return F < 2 ? hx_of(e) : hy_of(e); }

  int neighbour(int e, int F) const {
    int ix = e % mx, iy = e / mx;
    switch (F) {
      case FACE_W: return ix > 0 ? e - 1 : -1;
      case FACE_E: return ix < mx - 1 ? e + 1 : -1;
      case FACE_S: return iy > 0 ? e - mx : -1;
      default: return iy < my - 1 ? e + mx : -1;
    }
  }
  int iface(int e, int F) const {
    int ix = e % mx, iy = e / mx, row = 2 * mx - 1;
    switch (F) {
      case FACE_W: return ix > 0 ? iy * row + ix - 1 : -1;
      case FACE_E: return ix < mx - 1 ? iy * row + ix : -1;
      case FACE_S: return iy > 0 ? (iy - 1) * row + mx - 1 + ix : -1;
      default: return iy < my - 1 ? iy * row + mx - 1 + ix : -1;
    }
  }
  int mask(int e) const {
    int m = 0;
    for (int F = 0; F < 4; ++F)
      if (neighbour(e, F) >= 0) m |= 1 << F;
    return m;
  }
  bool black(int e) const { return ((e % mx) + (e / mx)) % 2 == 0; }
  // (a, b) of face node t of face F
  void face_node(int F, int t, int* a, int* b) const {
    switch (F) {
      case FACE_W: *a = 0; *b = t; break;
      case FACE_E: *a = n - 1; *b = t; break;
      case FACE_S: *a = t; *b = 0; break;
      default: *a = t; *b = n - 1; break;
    }
  }
};

// Everything the factor step produces, in host memory (FP64).
struct Factors {
  // face data per element column (W/E faces) and row (S/N faces), three
  // values each: penalty tau, Robin identity weight p, derivative scale 2/h
  std::vector<double> colg, rowg;
  std::vector<double> x1d, w1d, D;                  // GLL nodes, weights, D (n*n)
  // fast diagonalisation of the 1-D operators K_x (uniform grids: 4 classes
  // by the W/E face types; graded: one per column) and K_y (by S/N types, or
  // one per row): per entry V (n*n), Vinv (n*n), lam (n)
  std::vector<double> fdx, fdy;
  std::vector<double> T;     // nel * M*M : T_e[(F,t),(G,s)] row-major
  std::vector<int> tcls;     // nel : class of T_e (elements of one class hold identical T_e)
  std::vector<double> Rs;    // nel * M*4 : row sums of T_e per input face
  std::vector<int> black, white;
  std::vector<double> G;     // nblack * M*M : (I - X Y)^-1
  std::vector<double> X;     // nblack * 4*n*n : X_F blocks
  std::vector<double> C;     // d*d coarse matrix
  std::vector<double> H;     // d*d regularised coarse inverse
  std::vector<double> c0;    // d : right null vector of C
  std::vector<double> uL, uS, uC, what;  // r, kp, d, r
  std::vector<double> B1;    // kp : B 1 (right null vector of S)
  // deflation weights, 4 per element (0 on boundary faces): z_j takes the
  // value zw[4e + F] on the n slots of face F of e, with zw = B1 / beta_j and
  // beta_j the mean of B1 over interface j's two sides (all 1 on a uniform
  // grid, where z_j is the indicator of Sec. 2); zwa: the adjoint system's
  // weights, zwa[4e + F] = zw[4 nbr(e,F) + opp F]
  std::vector<double> zw, zwa;
  bool operator_only = false;  // only T_e and its row sums (SMPM_FLAG_OPERATOR_ONLY)
  int null_iterations = 0;   // GMRES steps of the u_S bordered solve
  double null_relres = 0;
  // Transposed system for the adjoint solve (built with SMPM_FLAG_ADJOINT).
  // With Phi the involution that swaps the two slots facing each other across
  // an interface, Phi S^T Phi is again "I + push form" with T~_e = T_e^T, the
  // same checkerboard blocks and the same Z, coarse matrix C^T, left null
  // vector Phi B1 = B1 and coarse null vectors swapped (left c0, right u_C).
  bool has_adjoint = false;
  std::vector<double> Ta;          // nel * M*M : T_e^T, row-major
  std::vector<double> Rsa, Ga, Xa; // as Rs, G, X for T~
  std::vector<double> Ha;          // d*d : (I - u_C u_C^T) K^-T (I - c0^ c0^T)
  std::vector<double> uSa;         // kp : B1 / |B1|
  std::vector<double> fdxT, fdyT;  // fast diagonalisation of K^T: (Vinv^T, V^T, lam)
};

// Host factor step (smpm_factor_host.cpp).
int factor_host(const Geometry& g, const smpm_opts& o, Factors* f, std::string* err);
// Fast-diagonalisation entry of element e in x and y: the face-type class
// on a uniform grid, the column / row on a graded one.
inline int xclass(const Geometry& g, int e) {
  int ix = e % g.mx;
  return g.graded ? ix : ((ix > 0 ? 1 : 0) | (ix < g.mx - 1 ? 2 : 0));
}
inline int yclass(const Geometry& g, int e) {
  int iy = e / g.mx;
  return g.graded ? iy : ((iy > 0 ? 1 : 0) | (iy < g.my - 1 ? 2 : 0));
}
// Element-tile partition (smpm_partition.cpp).
int partition_tile(const Geometry& g, int px, int py, int rank, smpm_tile* t);
int partition_halo(const Geometry& g, int px, int py, int rank, int side, long long* own, long long* facing);
// GLL nodes and weights, differentiation matrix (host).
void gll(int n, std::vector<double>* x, std::vector<double>* w);
void diff_matrix(const std::vector<double>& x, std::vector<double>* D);

}  // namespace smpm
