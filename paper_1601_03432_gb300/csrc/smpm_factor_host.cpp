// Host factor step of the deflated Schur-complement method (FP64).
//
// Builds, from the definitions of Sec. 1.2 - 2 of Joshi & Diamessis:
//   * GLL nodes/weights (Golub-Welsch on the Jacobi matrix of P_N', Newton
//     polish) and the differentiation matrix (barycentric form), Sec. 1.2;
//   * the element operator A_e of Sec. 1.3, which on an axis-aligned
//     rectangle is exactly the Kronecker sum I (x) K_x + K_y (x) I of two 1-D
//     operators, inverted by fast diagonalisation (K = V diag(lam) V^-1 from
//     the symmetric eigenproblem of W^1/2 K W^-1/2, W the GLL weights);
//   * T_e = B_e A_e^-1 E_e (4n x 4n): the map from element e's own interface
//     slots to the neighbours' slots facing e, i.e. the element's share of
//     S = I + B A^-1 E (Eq. schur_complement_system);
//   * the block-Jacobi blocks of Sec. 2 / Fig. 2 in reduced form: for a black
//     element, M_b = [[I, X], [Y, I]] over (own slots, facing slots) with
//     Y = T_e and X the four n x n blocks of the neighbours' T facing e, and
//     M_b^-1 is applied through G = (I - X Y)^-1;
//   * C = Z^T S Z, its right null vector c0 (Z c0 = B 1), its left null
//     vector u_C and the regularised inverse H (C y = r - u_C u_C^T r,
//     c0^T y = 0) from one dense LU of the bordered matrix [[C, c0], [c0^T, 0]];
//   * u_S, the unit left null vector of S, from the bordered system
//     [[S^T, a], [a^T, 0]] [y; eta] = [0; 1], a = B1/||B1||, by
//     right-preconditioned GMRES with iterative refinement,
//     and u_L = -A^-T B^T u_S normalised (u_L^T L = -u_S^T S B = 0), Sec. 1.4.
//
// Graded grids (column widths and row heights of their own): tau_F, p_F and
// the derivative scale of every face come from the element that owns the face,
// so T_e depends on e's size and on its neighbours' facing faces.  B 1 then
// differs between the two sides of an interface, and the deflation vectors
// z_j are its restrictions to interface j (scaled by the mean of the two
// sides) instead of 0/1 indicators; on a uniform grid both are the same.  C =
// Z^T S Z stays singular with right null vector c0 = the per-interface means.
// Identical element matrices (same face types and sizes) are computed once
// and copied: the stored factors are per element.
#include <unistd.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "smpm_internal.h"

namespace smpm {
namespace {

// ---------------------------------------------------------------- dense LA
// Cyclic Jacobi eigen-solver for a symmetric n x n matrix (row-major).
// On return lam holds the eigenvalues and V (row-major) the eigenvectors as
// columns.
void sym_eig(int n, std::vector<double> A, std::vector<double>* lam, std::vector<double>* V) {
  V->assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) (*V)[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- J^T A J
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = (*V)[k * n + p], vkq = (*V)[k * n + q];
          (*V)[k * n + p] = c * vkp - s * vkq;
          (*V)[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  lam->resize(n);
  for (int i = 0; i < n; ++i) (*lam)[i] = A[i * n + i];
}

// LU with partial pivoting (row-major, in place).
struct DenseLU {
  int n = 0;
  std::vector<double> a;
  std::vector<int> piv;
  bool ok = false;
};

// Factors the matrix held in A (moved in: no second copy of it is made).
DenseLU lu_factor_move(std::vector<double>&& A, int n) {
  DenseLU f;
  f.n = n;
  f.a = std::move(A);
  f.piv.resize(n);
  double* a = f.a.data();
  f.ok = true;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(a[static_cast<size_t>(k) * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(a[static_cast<size_t>(i) * n + k]);
      if (v > best) { best = v; p = i; }
    }
    f.piv[k] = p;
    if (best == 0.0) { f.ok = false; continue; }
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[static_cast<size_t>(k) * n + j], a[static_cast<size_t>(p) * n + j]);
    double inv = 1.0 / a[static_cast<size_t>(k) * n + k];
    double* rk = a + static_cast<size_t>(k) * n;
#pragma omp parallel for schedule(static) if (n - k > 256)
    for (int i = k + 1; i < n; ++i) {
      double* ri = a + static_cast<size_t>(i) * n;
      double l = ri[k] * inv;
      ri[k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) ri[j] -= l * rk[j];
    }
  }
  return f;
}

void lu_solve(const DenseLU& f, double* b) {
  const int n = f.n;
  const double* a = f.a.data();
  for (int k = 0; k < n; ++k)
    if (f.piv[k] != k) std::swap(b[k], b[f.piv[k]]);
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    const double* ri = a + static_cast<size_t>(i) * n;
    for (int j = 0; j < i; ++j) s -= ri[j] * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    const double* ri = a + static_cast<size_t>(i) * n;
    for (int j = i + 1; j < n; ++j) s -= ri[j] * b[j];
    b[i] = s / ri[i];
  }
}

// Solve A X = B for nrhs right-hand sides at once: B row-major n x nrhs.
// Row operations on whole rows of B (contiguous, vectorisable) stream the
// factors once per call instead of once per right-hand side.
void lu_solve_multi(const DenseLU& f, double* B, int nrhs) {
  const int n = f.n;
  const double* a = f.a.data();
  for (int k = 0; k < n; ++k)
    if (f.piv[k] != k)
      for (int c = 0; c < nrhs; ++c)
        std::swap(B[static_cast<size_t>(k) * nrhs + c], B[static_cast<size_t>(f.piv[k]) * nrhs + c]);
  for (int i = 0; i < n; ++i) {
    double* bi = B + static_cast<size_t>(i) * nrhs;
    const double* ri = a + static_cast<size_t>(i) * n;
    for (int j = 0; j < i; ++j) {
      const double l = ri[j];
      if (l == 0.0) continue;
      const double* bj = B + static_cast<size_t>(j) * nrhs;
      for (int c = 0; c < nrhs; ++c) bi[c] -= l * bj[c];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double* bi = B + static_cast<size_t>(i) * nrhs;
    const double* ri = a + static_cast<size_t>(i) * n;
    for (int j = i + 1; j < n; ++j) {
      const double u = ri[j];
      if (u == 0.0) continue;
      const double* bj = B + static_cast<size_t>(j) * nrhs;
      for (int c = 0; c < nrhs; ++c) bi[c] -= u * bj[c];
    }
    const double inv = 1.0 / ri[i];
    for (int c = 0; c < nrhs; ++c) bi[c] *= inv;
  }
}

// Solve A^T x = b with the factors of A.
void lu_solve_T(const DenseLU& f, double* b) {
  const int n = f.n;
  const double* a = f.a.data();
  for (int j = 0; j < n; ++j) {  // U^T z = b
    double s = b[j];
    for (int i = 0; i < j; ++i) s -= a[static_cast<size_t>(i) * n + j] * b[i];
    b[j] = s / a[static_cast<size_t>(j) * n + j];
  }
  for (int j = n - 1; j >= 0; --j) {  // L^T w = z
    double s = b[j];
    for (int i = j + 1; i < n; ++i) s -= a[static_cast<size_t>(i) * n + j] * b[i];
    b[j] = s;
  }
  for (int k = n - 1; k >= 0; --k)
    if (f.piv[k] != k) std::swap(b[k], b[f.piv[k]]);
}

// -------------------------------------------------------------- Legendre
void legendre(int N, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1;
  *dp = d1;
}

// 1-D operator K (n x n, row-major) of one direction: s^2 D^2 plus the face
// rows of Eq. smpm_poisson: on the low face (outward normal -1) the row gets
// tau (p * chi_lo * e_0 - s D[0,:]), on the high face tau (p * chi_hi *
// e_{n-1} + s D[n-1,:]); chi = 1 for an interface face, 0 on the boundary.
void build_K(const Geometry& g, const std::vector<double>& D, double s, double tau, double p, bool chi_lo,
             bool chi_hi, std::vector<double>* K) {
  const int n = g.n;
  K->assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0;
      for (int c = 0; c < n; ++c) acc += D[i * n + c] * D[c * n + j];
      (*K)[i * n + j] = s * s * acc;
    }
  for (int j = 0; j < n; ++j) {
    (*K)[j] += tau * (-s * D[j]);
    (*K)[(n - 1) * n + j] += tau * (s * D[(n - 1) * n + j]);
  }
  if (chi_lo) (*K)[0] += tau * p;
  if (chi_hi) (*K)[(n - 1) * n + n - 1] += tau * p;
}

// Fast-diagonalisation factors of K: out = [V (n*n) | Vinv (n*n) | lam (n)].
void fast_diag(int n, const std::vector<double>& w, const std::vector<double>& K, double* out) {
  std::vector<double> Ks(static_cast<size_t>(n) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = std::sqrt(w[i]) * K[i * n + j] / std::sqrt(w[j]);
      double b = std::sqrt(w[j]) * K[j * n + i] / std::sqrt(w[i]);
      Ks[i * n + j] = 0.5 * (a + b);
    }
  std::vector<double> lam, Q;
  sym_eig(n, Ks, &lam, &Q);
  double* V = out;
  double* Vi = out + n * n;
  double* L = out + 2 * n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      V[i * n + j] = Q[i * n + j] / std::sqrt(w[i]);
      Vi[i * n + j] = Q[j * n + i] * std::sqrt(w[j]);
    }
  for (int i = 0; i < n; ++i) L[i] = lam[i];
}

// U = A_e^-1 B for one element (B, U: n x n with U[b][a]), by fast
// diagonalisation: U = Vy ((Vy^-1 B Vx^-T) ./ (lx_i + ly_j)) Vx^T.
void elem_solve(int n, const double* fx, const double* fy, const double* B, double* U) {
  const double *Vx = fx, *Vxi = fx + n * n, *lx = fx + 2 * n * n;
  const double *Vy = fy, *Vyi = fy + n * n, *ly = fy + 2 * n * n;
  std::vector<double> t1(n * n), t2(n * n);
  for (int j = 0; j < n; ++j)  // t1 = Vyi B
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int b = 0; b < n; ++b) s += Vyi[j * n + b] * B[b * n + a];
      t1[j * n + a] = s;
    }
  for (int j = 0; j < n; ++j)  // t2 = t1 Vxi^T ./ (lx + ly)
    for (int i = 0; i < n; ++i) {
      double s = 0;
      for (int a = 0; a < n; ++a) s += t1[j * n + a] * Vxi[i * n + a];
      t2[j * n + i] = s / (lx[i] + ly[j]);
    }
  for (int j = 0; j < n; ++j)  // t1 = t2 Vx^T
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int i = 0; i < n; ++i) s += t2[j * n + i] * Vx[a * n + i];
      t1[j * n + a] = s;
    }
  for (int b = 0; b < n; ++b)  // U = Vy t1
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int j = 0; j < n; ++j) s += Vy[b * n + j] * t1[j * n + a];
      U[b * n + a] = s;
    }
}

// U = A_e^-T B: U = Vyi^T ((Vy^T B Vx) ./ (lx_i + ly_j)) Vxi.
void elem_solve_T(int n, const double* fx, const double* fy, const double* B, double* U) {
  const double *Vx = fx, *Vxi = fx + n * n, *lx = fx + 2 * n * n;
  const double *Vy = fy, *Vyi = fy + n * n, *ly = fy + 2 * n * n;
  std::vector<double> t1(n * n), t2(n * n);
  for (int j = 0; j < n; ++j)
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int b = 0; b < n; ++b) s += Vy[b * n + j] * B[b * n + a];
      t1[j * n + a] = s;
    }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double s = 0;
      for (int a = 0; a < n; ++a) s += t1[j * n + a] * Vx[a * n + i];
      t2[j * n + i] = s / (lx[i] + ly[j]);
    }
  for (int j = 0; j < n; ++j)
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int i = 0; i < n; ++i) s += t2[j * n + i] * Vxi[i * n + a];
      t1[j * n + a] = s;
    }
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      double s = 0;
      for (int j = 0; j < n; ++j) s += Vyi[j * n + b] * t1[j * n + a];
      U[b * n + a] = s;
    }
}

// n_F . grad U at face node t of face F of one element (U[b][a]); sc = 2/h
// of the element along the face normal.
double normal_derivative(const Geometry& g, const std::vector<double>& D, const double* U, int F, int t, double sc) {
  const int n = g.n;
  double acc = 0;
  switch (F) {
    case FACE_W: for (int c = 0; c < n; ++c) acc += D[c] * U[t * n + c]; return -sc * acc;
    case FACE_E: for (int c = 0; c < n; ++c) acc += D[(n - 1) * n + c] * U[t * n + c]; return sc * acc;
    case FACE_S: for (int c = 0; c < n; ++c) acc += D[c] * U[c * n + t]; return -sc * acc;
    default: for (int c = 0; c < n; ++c) acc += D[(n - 1) * n + c] * U[c * n + t]; return sc * acc;
  }
}

struct Ctx {
  const Geometry& g;
  Factors* f;
  // [tau, p, 2/h] of face F of element e (from e's column for W/E, row for S/N)
  const double* face(int e, int F) const {
    return F < 2 ? f->colg.data() + 3 * (e % g.mx) : f->rowg.data() + 3 * (e / g.mx);
  }
  const double* fx(int e) const { return f->fdx.data() + static_cast<size_t>(xclass(g, e)) * (2 * g.n * g.n + g.n); }
  const double* fy(int e) const { return f->fdy.data() + static_cast<size_t>(yclass(g, e)) * (2 * g.n * g.n + g.n); }
};

// T_e for element e (M x M, row (F,t) = the flux into the neighbour across F,
// column (G,s) = e's own slot).  Row (F,t) equals the B row of slot
// (e' = nbr(e,F), opp F, t): -tau' (p' w - n_F.grad w) at e's face node (F,t),
// with tau', p' those of e''s face opp F, the gradient taken with e's own
// size, and w = A_e^-1 E_e (unit value at the face node of slot (G,s)).
void element_T(const Ctx& c, int e, double* T) {
  const Geometry& g = c.g;
  const int n = g.n, M = g.M;
  std::fill(T, T + M * M, 0.0);
  std::vector<double> B(n * n), U(n * n);
  for (int G = 0; G < 4; ++G) {
    if (g.neighbour(e, G) < 0) continue;
    for (int s = 0; s < n; ++s) {
      std::fill(B.begin(), B.end(), 0.0);
      int a, b;
      g.face_node(G, s, &a, &b);
      B[b * n + a] = 1.0;
      elem_solve(n, c.fx(e), c.fy(e), B.data(), U.data());
      for (int F = 0; F < 4; ++F) {
        const int e2 = g.neighbour(e, F);
        if (e2 < 0) continue;
        const double* fn = c.face(e2, opposite(F));
        const double se = c.face(e, F)[2];
        for (int t = 0; t < n; ++t) {
          int aa, bb;
          g.face_node(F, t, &aa, &bb);
          double val = fn[1] * U[bb * n + aa] - normal_derivative(g, c.f->D, U.data(), F, t, se);
          T[(F * n + t) * M + G * n + s] = -fn[0] * val;
        }
      }
    }
  }
}

// ----------------------------------------------------- slot operators (host)
// Class representatives.  Elements of one T class (same face types and, on a
// graded grid, the same own and facing sizes) hold identical T_e, and black
// blocks with the same key (own T class, then the four neighbours' classes)
// identical G_b and X_b: the factor step computes T_e and G_b once per class
// and copies them, and gathers X_b from the neighbours' identical T.  The
// host operators below read the representative's copy, which gives the same
// arithmetic from a cache-resident working set.
struct ClassReps {
  std::vector<long long> t;  // per element: element whose T_e it reads
  std::vector<long long> b;  // per black block: block whose G_b, X_b it reads
};

using BlockKey = std::array<int, 5>;
BlockKey block_key(const Geometry& g, const std::vector<int>& tcls, int e) {
  BlockKey k{tcls[e], -1, -1, -1, -1};
  for (int F = 0; F < 4; ++F) {
    const int e2 = g.neighbour(e, F);
    k[F + 1] = e2 >= 0 ? tcls[e2] : -1;
  }
  return k;
}

ClassReps class_reps(const Geometry& g, const std::vector<int>& black, const std::vector<int>& tcls) {
  ClassReps c;
  c.t.resize(g.nel);
  std::map<int, long long> first_t;
  for (long long e = 0; e < g.nel; ++e) c.t[e] = first_t.emplace(tcls[e], e).first->second;
  c.b.resize(black.size());
  std::map<BlockKey, long long> first_b;
  for (size_t ib = 0; ib < black.size(); ++ib)
    c.b[ib] = first_b.emplace(block_key(g, tcls, black[ib]), static_cast<long long>(ib)).first->second;
  return c;
}

// out = S^T y on padded slot vectors: out_e = y_e + T_e^T yhat_e, yhat_e the
// neighbours' slots facing e (T_e read row by row).
void apply_ST(const Geometry& g, const Factors& f, const ClassReps& cr, const double* y, double* out) {
  const int n = g.n, M = g.M;
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < g.nel; ++e) {
    double yh[4 * kMaxN], acc[4 * kMaxN];
    for (int F = 0; F < 4; ++F) {
      int e2 = g.neighbour(static_cast<int>(e), F);
      for (int t = 0; t < n; ++t) yh[F * n + t] = e2 >= 0 ? y[e2 * M + opposite(F) * n + t] : 0.0;
    }
    const double* T = f.T.data() + static_cast<size_t>(cr.t[e]) * M * M;
    for (int col = 0; col < M; ++col) acc[col] = y[e * M + col];
    for (int row = 0; row < M; ++row) {
      const double yr = yh[row];
      const double* Tr = T + static_cast<size_t>(row) * M;
      for (int col = 0; col < M; ++col) acc[col] += Tr[col] * yr;
    }
    for (int col = 0; col < M; ++col) out[e * M + col] = acc[col];
  }
}

// out = M^-T y, block by block: with M_b = [[I, X], [Y, I]],
// M_b^T [a; b] = [p; q] gives a = G^T (p - Y^T q), b = q - X^T a.
void apply_MinvT(const Geometry& g, const Factors& f, const ClassReps& cr, const double* y, double* out) {
  const int n = g.n, M = g.M;
  const long long nb = static_cast<long long>(f.black.size());
#pragma omp parallel for schedule(static)
  for (long long ib = 0; ib < nb; ++ib) {
    int e = f.black[ib];
    double p[4 * kMaxN], q[4 * kMaxN], r1[4 * kMaxN], a[4 * kMaxN];
    int nb4[4];
    for (int F = 0; F < 4; ++F) {
      nb4[F] = g.neighbour(e, F);
      for (int t = 0; t < n; ++t) {
        p[F * n + t] = y[e * M + F * n + t];
        q[F * n + t] = nb4[F] >= 0 ? y[nb4[F] * M + opposite(F) * n + t] : 0.0;
      }
    }
    const double* T = f.T.data() + static_cast<size_t>(cr.t[e]) * M * M;
    const double* Gm = f.G.data() + static_cast<size_t>(cr.b[ib]) * M * M;
    const double* X = f.X.data() + static_cast<size_t>(cr.b[ib]) * 4 * n * n;
    for (int c2 = 0; c2 < M; ++c2) r1[c2] = p[c2];
    for (int row = 0; row < M; ++row) {  // r1 = p - T^T q, rows of T in order
      const double qr = q[row];
      const double* Tr = T + static_cast<size_t>(row) * M;
      for (int c2 = 0; c2 < M; ++c2) r1[c2] -= Tr[c2] * qr;
    }
    for (int c2 = 0; c2 < M; ++c2) a[c2] = 0.0;
    for (int row = 0; row < M; ++row) {  // a = G^T r1
      const double rr = r1[row];
      const double* Gr = Gm + static_cast<size_t>(row) * M;
      for (int c2 = 0; c2 < M; ++c2) a[c2] += Gr[c2] * rr;
    }
    for (int F = 0; F < 4; ++F) {
      for (int t = 0; t < n; ++t) {
        double s = 0;
        for (int s2 = 0; s2 < n; ++s2) s += X[(F * n + s2) * n + t] * a[F * n + s2];
        out[e * M + F * n + t] = a[F * n + t];
        if (nb4[F] >= 0) out[nb4[F] * M + opposite(F) * n + t] = q[F * n + t] - s;
      }
    }
  }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// Restarted right-preconditioned GMRES (CGS2) on the bordered transposed
// system for u_S, with the unit border vector a = B1 / ||B1||.  Unknown
// z = [y (kp); eta]; operator K P z = [S^T (M^-T y) + a eta; a^T (M^-T y)].
// The true residual is recomputed at every restart and the solve repeats
// (iterative refinement, three digits per cycle) until the residual is
// below 1e-14 or stops decreasing.  Below 1e-12 a cycle takes at most 40
// steps: there the null vector itself no longer improves (||S^T u_S|| is set
// by the operator's round-off), and short cycles recompute the true residual
// more often than long stagnating ones.
int left_null_S(const Geometry& g, Factors* f, std::string* err) {
  const size_t kp = static_cast<size_t>(g.kp), N = kp + 1;
  std::vector<double> a(f->B1);
  double an = std::sqrt(dot(a, a));
  for (auto& v : a) v /= an;
  std::vector<double> tmp(kp), tmp2(kp);
  const ClassReps cr = class_reps(g, f->black, f->tcls);
  auto op = [&](const std::vector<double>& z, std::vector<double>& out) {
    apply_MinvT(g, *f, cr, z.data(), tmp.data());
    apply_ST(g, *f, cr, tmp.data(), tmp2.data());
    double eta = z[kp], s = 0;
    for (size_t i = 0; i < kp; ++i) {
      out[i] = tmp2[i] + a[i] * eta;
      s += a[i] * tmp[i];
    }
    out[kp] = s;
  };
  const int m = 300, m_tail = 40, maxit = 4000;
  std::vector<double> x(N, 0.0), r(N, 0.0), w(N);
  r[kp] = 1.0;  // b = [0; 1], x0 = 0
  std::vector<std::vector<double>> V;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1);
  int total = 0;
  double beta = 1.0, best = 1e300;
  while (total < maxit) {
    beta = std::sqrt(dot(r, r));
    if (beta <= 1e-14 || beta >= 0.5 * best) break;  // accurate enough, or no progress
    best = beta;
    const double tol = 1e-3 * beta;                   // each cycle gains three digits
    V.assign(1, r);
    for (auto& v : V[0]) v /= beta;
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    const int mcyc = beta < 1e-12 ? m_tail : m;
    int j = 0;
    for (; j < mcyc && total < maxit; ++j) {
      op(V[j], w);
      // classical Gram-Schmidt, twice: h1 = V^T w; w -= V h1 and, in the
      // same pass over each block, h2 = V^T w; then w -= V h2.  Blocks of
      // entries in which each basis vector is read contiguously; every
      // thread sums its blocks in order, then the threads' sums are added.
      {
        constexpr long long kBlk = 2048;
        const long long nblk = (static_cast<long long>(N) + kBlk - 1) / kBlk;
        std::vector<double> h1(j + 1, 0.0), h2(j + 1, 0.0);
        auto dots = [&](long long q0, long long q1, std::vector<double>& hp) {
          for (int i = 0; i <= j; ++i) {  // four partial sums: independent add chains
            const double* Vi = V[i].data();
            double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            long long q = q0;
            for (; q + 4 <= q1; q += 4) {
              a0 += Vi[q] * w[q];
              a1 += Vi[q + 1] * w[q + 1];
              a2 += Vi[q + 2] * w[q + 2];
              a3 += Vi[q + 3] * w[q + 3];
            }
            for (; q < q1; ++q) a0 += Vi[q] * w[q];
            hp[i] += (a0 + a1) + (a2 + a3);
          }
        };
        auto subtract = [&](long long q0, long long q1, const std::vector<double>& hv) {
          for (int i = 0; i <= j; ++i) {
            const double* Vi = V[i].data();
            const double hi = hv[i];
            for (long long q = q0; q < q1; ++q) w[q] -= hi * Vi[q];
          }
        };
        for (int pass = 0; pass < 2; ++pass) {  // pass 0: h1; pass 1: subtract h1, h2
          std::vector<double>& hout = pass ? h2 : h1;
#pragma omp parallel
          {
            std::vector<double> hp(j + 1, 0.0);
#pragma omp for schedule(static) nowait
            for (long long b = 0; b < nblk; ++b) {
              const long long q0 = b * kBlk, q1 = std::min<long long>(q0 + kBlk, static_cast<long long>(N));
              if (pass) subtract(q0, q1, h1);
              dots(q0, q1, hp);
            }
#pragma omp critical
            for (int i = 0; i <= j; ++i) hout[i] += hp[i];
          }
        }
#pragma omp parallel for schedule(static)
        for (long long b = 0; b < nblk; ++b)
          subtract(b * kBlk, std::min<long long>((b + 1) * kBlk, static_cast<long long>(N)), h2);
        for (int i = 0; i <= j; ++i) H[i * m + j] = h1[i] + h2[i];
      }
      double hn = std::sqrt(dot(w, w));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      double den = std::hypot(H[j * m + j], hn);
      cs[j] = H[j * m + j] / den;
      sn[j] = hn / den;
      H[j * m + j] = den;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++total;
      if (std::fabs(gv[j + 1]) <= tol || hn == 0.0) { ++j; break; }
      V.push_back(w);
      for (auto& v : V.back()) v /= hn;
    }
    std::vector<double> yv(j);
    for (int i = j - 1; i >= 0; --i) {
      double s = gv[i];
      for (int k2 = i + 1; k2 < j; ++k2) s -= H[i * m + k2] * yv[k2];
      yv[i] = s / H[i * m + i];
    }
    for (int i = 0; i < j; ++i)
      for (size_t q = 0; q < N; ++q) x[q] += yv[i] * V[i][q];
    op(x, w);
    for (size_t q = 0; q < N; ++q) r[q] = (q == kp ? 1.0 : 0.0) - w[q];
  }
  f->null_iterations = total;
  f->null_relres = std::sqrt(dot(r, r));
  if (!(f->null_relres <= 1e-12)) {
    *err = "u_S bordered solve did not converge (residual " + std::to_string(f->null_relres) + ")";
    return SMPM_ENOTCONV;
  }
  std::vector<double> y(kp);
  apply_MinvT(g, *f, cr, x.data(), y.data());
  double nrm = std::sqrt(dot(y, y));
  size_t imax = 0;
  for (size_t i = 0; i < kp; ++i)
    if (std::fabs(y[i]) > std::fabs(y[imax])) imax = i;
  double sg = y[imax] >= 0 ? 1.0 : -1.0;
  f->uS.resize(kp);
  for (size_t i = 0; i < kp; ++i) f->uS[i] = sg * y[i] / nrm;
  return SMPM_OK;
}

// Weighted row sums of T_e over each input face:
// Rs[row * 4 + G] = zw[4e + G] sum_q T_e[row, G n + q] (the pushed part of S Z,
// one column per face of e).
void row_sums(const Geometry& g, const std::vector<double>& T, const std::vector<double>& zw,
              std::vector<double>* Rs) {
  const int n = g.n, M = g.M;
  Rs->assign(static_cast<size_t>(g.nel) * M * 4, 0.0);
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < g.nel; ++e) {
    const double* Te = T.data() + static_cast<size_t>(e) * M * M;
    double* R = Rs->data() + static_cast<size_t>(e) * M * 4;
    for (int row = 0; row < M; ++row)
      for (int G = 0; G < 4; ++G) {
        double acc = 0;
        for (int q = 0; q < n; ++q) acc += Te[row * M + G * n + q];
        R[row * 4 + G] = zw[4 * e + G] * acc;
      }
  }
}

// Block-Jacobi factors of the checkerboard blocks of I + (push form of T)
// (Sec. 2, Fig. 2): per black element the X_F blocks (the neighbours' T rows
// facing e, restricted to their slots facing e) and G = (I - X Y)^-1 with
// Y = T_e; identical blocks (same own and neighbour T classes) share one
// inversion.
int block_factors(const Geometry& g, const std::vector<int>& black, const std::vector<double>& T,
                  const std::vector<int>& tcls, std::vector<double>* Gout, std::vector<double>* Xout,
                  std::string* err) {
  const int n = g.n, M = g.M;
  const size_t nb = black.size();
  Gout->assign(nb * M * M, 0.0);
  Xout->assign(nb * 4 * n * n, 0.0);
#pragma omp parallel for schedule(static)
  for (long long ib = 0; ib < static_cast<long long>(nb); ++ib) {
    const int e = black[ib];
    double* X = Xout->data() + ib * 4 * n * n;
    for (int F = 0; F < 4; ++F) {
      int e2 = g.neighbour(e, F);
      if (e2 < 0) continue;
      const double* T2 = T.data() + static_cast<size_t>(e2) * M * M;
      int Fo = opposite(F);
      for (int t = 0; t < n; ++t)
        for (int q = 0; q < n; ++q) X[(F * n + t) * n + q] = T2[(Fo * n + t) * M + Fo * n + q];
    }
  }
  // one representative block per key, inverted in parallel, then copied
  std::map<BlockKey, int> first;
  std::vector<int> rep(nb), reps;
  for (size_t ib = 0; ib < nb; ++ib) {
    auto it = first.emplace(block_key(g, tcls, black[ib]), static_cast<int>(reps.size()));
    if (it.second) reps.push_back(static_cast<int>(ib));
    rep[ib] = it.first->second;
  }
  std::vector<std::vector<double>> ginv(reps.size());
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (long long ir = 0; ir < static_cast<long long>(reps.size()); ++ir) {
    const int ib = reps[ir], e = black[ib];
    const double* X = Xout->data() + static_cast<size_t>(ib) * 4 * n * n;
    {
      const double* Y = T.data() + static_cast<size_t>(e) * M * M;
      std::vector<double> A(static_cast<size_t>(M) * M, 0.0);
      for (int F = 0; F < 4; ++F)
        for (int t = 0; t < n; ++t)
          for (int col = 0; col < M; ++col) {
            double acc = 0;
            for (int q = 0; q < n; ++q) acc += X[(F * n + t) * n + q] * Y[(F * n + q) * M + col];
            A[(F * n + t) * M + col] = (F * n + t == col ? 1.0 : 0.0) - acc;
          }
      DenseLU lu = lu_factor_move(std::move(A), M);
      if (!lu.ok) { bad += 1; continue; }
      std::vector<double> Gi(static_cast<size_t>(M) * M), col(M);
      for (int j = 0; j < M; ++j) {
        std::fill(col.begin(), col.end(), 0.0);
        col[j] = 1.0;
        lu_solve(lu, col.data());
        for (int i = 0; i < M; ++i) Gi[i * M + j] = col[i];
      }
      ginv[ir] = std::move(Gi);
    }
  }
  if (bad) { *err = "singular block-Jacobi block"; return SMPM_EINVAL; }
#pragma omp parallel for schedule(static)
  for (long long ib = 0; ib < static_cast<long long>(nb); ++ib)
    std::memcpy(Gout->data() + ib * M * M, ginv[rep[ib]].data(), sizeof(double) * M * M);
  return SMPM_OK;
}

// Transposed fast diagonalisation: K = V diag(lam) Vinv gives
// K^T = Vinv^T diag(lam) V^T, stored in the same (V, Vinv, lam) layout.
void transpose_fd(int n, const std::vector<double>& fd, std::vector<double>* out) {
  const size_t fds = 2 * (size_t)n * n + n;
  out->assign(fd.size(), 0.0);
  for (size_t cls = 0; cls * fds < fd.size(); ++cls) {
    const double* V = fd.data() + cls * fds;
    const double* Vi = V + n * n;
    double* W = out->data() + cls * fds;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        W[i * n + j] = Vi[j * n + i];
        W[n * n + i * n + j] = V[j * n + i];
      }
    for (int i = 0; i < n; ++i) W[2 * n * n + i] = V[2 * n * n + i];
  }
}

}  // namespace

// -------------------------------------------------------------- public
void gll(int n, std::vector<double>* x, std::vector<double>* w) {
  const int N = n - 1;
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  (*x)[0] = -1.0;
  (*x)[n - 1] = 1.0;
  const int m = N - 1;  // interior nodes: zeros of P_N' ~ Gegenbauer C^(3/2)_{N-1}
  if (m > 0) {
    std::vector<double> J(static_cast<size_t>(m) * m, 0.0), lam, V;
    for (int k = 1; k < m; ++k) {
      double b = std::sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
      J[(k - 1) * m + k] = b;
      J[k * m + k - 1] = b;
    }
    sym_eig(m, J, &lam, &V);
    std::sort(lam.begin(), lam.end());
    for (int i = 0; i < m; ++i) {
      double xi = lam[i];
      for (int it = 0; it < 8; ++it) {  // Newton on P_N'
        double p, dp;
        legendre(N, xi, &p, &dp);
        double ddp = (2.0 * xi * dp - N * (N + 1.0) * p) / (1.0 - xi * xi);
        double step = dp / ddp;
        xi -= step;
        if (std::fabs(step) < 1e-17) break;
      }
      (*x)[i + 1] = xi;
    }
  }
  for (int i = 0; i < n; ++i) {
    double p, dp;
    legendre(N, (*x)[i], &p, &dp);
    (*w)[i] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

void diff_matrix(const std::vector<double>& x, std::vector<double>* D) {
  const int n = static_cast<int>(x.size());
  std::vector<double> lam(n, 1.0);  // barycentric weights
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (x[j] - x[k]);
  D->assign(static_cast<size_t>(n) * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0;
    for (int j = 0; j < n; ++j)
      if (j != i) {
        double v = (lam[j] / lam[i]) / (x[i] - x[j]);
        (*D)[i * n + j] = v;
        diag -= v;
      }
    (*D)[i * n + i] = diag;
  }
}

// The coarse solve is dense (Sec. 2): C, the LU of the bordered K (factored
// in place) and the leading block of K^-1, which becomes H = C^+ in place,
// hold 3 (d+1)^2 doubles on the host at once; with the adjoint, H and the
// adjoint's Ha are separate arrays (5 (d+1)^2).  Refused before any work
// when that exceeds the machine's physical memory.
static int coarse_memory_check(const Geometry& g, bool adjoint, std::string* err) {
  const double dd = static_cast<double>(g.d + 1);
  const double need = (adjoint ? 5.0 : 3.0) * dd * dd * sizeof(double);
  const long pages = sysconf(_SC_PHYS_PAGES), page = sysconf(_SC_PAGE_SIZE);
  const double have = static_cast<double>(pages) * static_cast<double>(page);
  if (pages <= 0 || page <= 0 || need <= have) return SMPM_OK;
  char msg[200];
  std::snprintf(msg, sizeof msg,
                "the dense coarse matrices (d = %lld interfaces) need %.3g GB of host memory, more than this "
                "machine has (%.3g GB)", g.d, need * 1e-9, have * 1e-9);
  *err = msg;
  return SMPM_ENOMEM;
}

static int factor_host_body(const Geometry& g, const smpm_opts& o, Factors* f, std::string* err) {
  const bool op_only = (o.flags & SMPM_FLAG_OPERATOR_ONLY) != 0;
  if (!op_only) {
    const int st = coarse_memory_check(g, (o.flags & SMPM_FLAG_ADJOINT) != 0, err);
    if (st != SMPM_OK) return st;
  }
  const int n = g.n, M = g.M;
  const double nn1 = n * (n - 1.0);
  // per column (W/E faces) and row (S/N faces): tau = -alpha n(n-1)/h, the
  // identity weight of the Robin flux R = p I + n.grad (scaled by the
  // element's own length, or 1 under the literal reading R = I + n.grad) and
  // the derivative scale 2/h
  const bool literal = (o.flags & SMPM_FLAG_ROBIN_LITERAL) != 0;
  auto face_data = [&](double h, double* out) {
    out[0] = -o.tau_scale * nn1 / h;
    out[1] = literal ? 1.0 : o.robin_scale * nn1 / h;
    out[2] = 2.0 / h;
  };
  f->colg.assign(3 * static_cast<size_t>(g.mx), 0.0);
  f->rowg.assign(3 * static_cast<size_t>(g.my), 0.0);
  for (int ix = 0; ix < g.mx; ++ix) face_data(g.col_h(ix), f->colg.data() + 3 * ix);
  for (int iy = 0; iy < g.my; ++iy) face_data(g.row_h(iy), f->rowg.data() + 3 * iy);
  gll(n, &f->x1d, &f->w1d);
  diff_matrix(f->x1d, &f->D);

  // 1-D operators and their fast diagonalisation: 4 classes per direction
  // (face types) on a uniform grid, one per column / row on a graded one
  const int fds = 2 * n * n + n;
  const int nfx = g.graded ? g.mx : 4, nfy = g.graded ? g.my : 4;
  f->fdx.assign(static_cast<size_t>(nfx) * fds, 0.0);
  f->fdy.assign(static_cast<size_t>(nfy) * fds, 0.0);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < nfx + nfy; ++i) {
    std::vector<double> K;
    const bool xdir = i < nfx;
    const int c = xdir ? i : i - nfx, m = xdir ? g.mx : g.my;
    // face types of the entry: bit 0 = low-side interface, bit 1 = high side
    const int cls = g.graded ? ((c > 0 ? 1 : 0) | (c < m - 1 ? 2 : 0)) : c;
    const double* fd = (xdir ? f->colg.data() : f->rowg.data()) + 3 * (g.graded ? c : 0);
    build_K(g, f->D, fd[2], fd[0], fd[1], cls & 1, cls & 2, &K);
    fast_diag(n, f->w1d, K, (xdir ? f->fdx.data() : f->fdy.data()) + static_cast<size_t>(c) * fds);
  }
  // the element operator I (x) K_x + K_y (x) I is singular only for the
  // element without interfaces (mx = my = 1)
  for (int cx = 0; cx < nfx; ++cx)
    for (int cy = 0; cy < nfy; ++cy) {
      const int clsx = g.graded ? ((cx > 0 ? 1 : 0) | (cx < g.mx - 1 ? 2 : 0)) : cx;
      const int clsy = g.graded ? ((cy > 0 ? 1 : 0) | (cy < g.my - 1 ? 2 : 0)) : cy;
      if ((clsx | clsy) == 0) continue;
      const double* lx = f->fdx.data() + static_cast<size_t>(cx) * fds + 2 * n * n;
      const double* ly = f->fdy.data() + static_cast<size_t>(cy) * fds + 2 * n * n;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          if (!(std::fabs(lx[i] + ly[j]) > 0)) { *err = "singular element operator"; return SMPM_EINVAL; }
    }
  Ctx c{g, f};

  // T_e, computed once per class: elements with the same face types, the same
  // size and the same facing sizes of their neighbours hold identical T_e
  f->T.assign(static_cast<size_t>(g.nel) * M * M, 0.0);
  f->tcls.assign(g.nel, 0);
  std::vector<int> trep;
  {
    std::map<std::vector<double>, int> tkeys;
    for (long long e = 0; e < g.nel; ++e) {
      const int ei = static_cast<int>(e);
      std::vector<double> key{static_cast<double>(g.mask(ei)), g.hx_of(ei), g.hy_of(ei)};
      for (int F = 0; F < 4; ++F) {
        const int e2 = g.neighbour(ei, F);
        key.push_back(e2 >= 0 ? g.hperp(e2, opposite(F)) : 0.0);
      }
      auto it = tkeys.emplace(std::move(key), static_cast<int>(trep.size()));
      if (it.second) trep.push_back(ei);
      f->tcls[e] = it.first->second;
    }
  }
  std::vector<std::vector<double>> tcache(trep.size());
#pragma omp parallel for schedule(dynamic, 1)
  for (long long i = 0; i < static_cast<long long>(trep.size()); ++i) {
    tcache[i].assign(static_cast<size_t>(M) * M, 0.0);
    element_T(c, trep[i], tcache[i].data());
  }
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < g.nel; ++e)
    std::memcpy(f->T.data() + static_cast<size_t>(e) * M * M, tcache[f->tcls[e]].data(), sizeof(double) * M * M);

  // B 1 (slot (e, F, t): -tau p of e's face F), the per-interface means c0 of
  // its two sides, and the deflation weights zw = B1 / c0 (Sec. 2's z_j on a
  // uniform grid, where both sides agree and every weight is 1)
  auto tau_p = [&](int e, int F) { const double* fc = c.face(e, F); return -fc[0] * fc[1]; };
  const int d = static_cast<int>(g.d);
  f->B1.assign(g.kp, 0.0);
  f->c0.assign(d, 0.0);
  f->zw.assign(4 * static_cast<size_t>(g.nel), 0.0);
  f->zwa.assign(4 * static_cast<size_t>(g.nel), 0.0);
  for (long long e = 0; e < g.nel; ++e)
    for (int F = 0; F < 4; ++F) {
      const int ei = static_cast<int>(e), e2 = g.neighbour(ei, F);
      if (e2 < 0) continue;
      const double here = tau_p(ei, F), there = tau_p(e2, opposite(F));
      const double beta = 0.5 * (here + there);
      f->c0[g.iface(ei, F)] = beta;
      f->zw[4 * e + F] = here / beta;
      f->zwa[4 * e + F] = there / beta;
      for (int t = 0; t < n; ++t) f->B1[e * M + F * n + t] = here;
    }
  row_sums(g, f->T, f->zw, &f->Rs);
  if (op_only) {  // the element factors of S only
    f->operator_only = true;
    return SMPM_OK;
  }

  // checkerboard blocks
  f->black.clear();
  f->white.clear();
  for (long long e = 0; e < g.nel; ++e) (g.black(static_cast<int>(e)) ? f->black : f->white).push_back(static_cast<int>(e));
  {
    int st = block_factors(g, f->black, f->T, f->tcls, &f->G, &f->X, err);
    if (st != SMPM_OK) return st;
  }

  // the coarse matrix C = Z^T S Z: the identity part sum_slots w^2 = n (w^2 of
  // both sides) on the diagonal (2n on a uniform grid); row (Fp, t) of T_e
  // feeds the slot (nbr, opp Fp, t) of interface i, weighted by its zw
  f->C.assign(static_cast<size_t>(d) * d, 0.0);
  for (long long e = 0; e < g.nel; ++e)
    for (int F = 0; F < 4; ++F) {
      const int j = g.iface(static_cast<int>(e), F);
      if (j >= 0) f->C[static_cast<size_t>(j) * d + j] += n * f->zw[4 * e + F] * f->zw[4 * e + F];
    }
  for (long long e = 0; e < g.nel; ++e) {
    const double* R = f->Rs.data() + static_cast<size_t>(e) * M * 4;
    for (int Fp = 0; Fp < 4; ++Fp) {
      int i = g.iface(static_cast<int>(e), Fp);
      if (i < 0) continue;
      const double wout = f->zwa[4 * e + Fp];  // weight of the slot (nbr, opp Fp, t)
      for (int F = 0; F < 4; ++F) {
        int j = g.iface(static_cast<int>(e), F);
        if (j < 0) continue;
        double s = 0;
        for (int t = 0; t < n; ++t) s += R[(Fp * n + t) * 4 + F];
        f->C[static_cast<size_t>(i) * d + j] += wout * s;
      }
    }
  }
  // bordered K = [[C, c0^], [c0^T, 0]] with the unit c0^ = c0 / |c0|: u_C from
  // K^T [y; eta] = [0; 1], H from K^-1.  The border's length does not change
  // the leading block of K^-1 (the constraint c0^T y = 0 is the same), but
  // c0 itself (-tau p per interface, ~1e7 on fine grids) against entries of C
  // of order n would make K badly scaled and its inverse inaccurate by orders
  // of magnitude on elongated grids.
  std::vector<double> Kinv;  // leading d x d block of K^-1 (kept for the adjoint)
  {
    const int d1 = d + 1;
    double c0n = 0;
    for (int i = 0; i < d; ++i) c0n += f->c0[i] * f->c0[i];
    c0n = std::sqrt(c0n);
    std::vector<double> K1(static_cast<size_t>(d1) * d1, 0.0);
    for (int i = 0; i < d; ++i) {
      for (int j = 0; j < d; ++j) K1[static_cast<size_t>(i) * d1 + j] = f->C[static_cast<size_t>(i) * d + j];
      K1[static_cast<size_t>(i) * d1 + d] = f->c0[i] / c0n;
      K1[static_cast<size_t>(d) * d1 + i] = f->c0[i] / c0n;
    }
    DenseLU lu = lu_factor_move(std::move(K1), d1);
    if (!lu.ok) { *err = "singular bordered coarse matrix"; return SMPM_EINVAL; }
    std::vector<double> y(d1, 0.0);
    y[d] = 1.0;
    lu_solve_T(lu, y.data());
    double nrm = 0;
    int imax = 0;
    for (int i = 0; i < d; ++i) {
      nrm += y[i] * y[i];
      if (std::fabs(y[i]) > std::fabs(y[imax])) imax = i;
    }
    nrm = std::sqrt(nrm) * (y[imax] >= 0 ? 1.0 : -1.0);
    f->uC.resize(d);
    for (int i = 0; i < d; ++i) f->uC[i] = y[i] / nrm;
    Kinv.assign(static_cast<size_t>(d) * d, 0.0);
    constexpr int kCols = 64;  // right-hand sides per block solve
    const int nblk = (d + kCols - 1) / kCols;
#pragma omp parallel for schedule(dynamic, 1)
    for (int bk = 0; bk < nblk; ++bk) {
      const int j0 = bk * kCols, nc = std::min(kCols, d - j0);
      std::vector<double> Bm(static_cast<size_t>(d1) * nc, 0.0);
      for (int c = 0; c < nc; ++c) Bm[static_cast<size_t>(j0 + c) * nc + c] = 1.0;
      lu_solve_multi(lu, Bm.data(), nc);
      for (int i = 0; i < d; ++i)
        for (int c = 0; c < nc; ++c) Kinv[static_cast<size_t>(i) * d + j0 + c] = Bm[static_cast<size_t>(i) * nc + c];
    }
    // H = Kinv (I - u_C u_C^T); in place unless the adjoint needs Kinv
    const bool keep = (o.flags & SMPM_FLAG_ADJOINT) != 0;
    lu = DenseLU();
    if (keep) f->H.assign(static_cast<size_t>(d) * d, 0.0);
    double* Hd = keep ? f->H.data() : Kinv.data();
#pragma omp parallel for schedule(static)
    for (int i = 0; i < d; ++i) {
      double s = 0;
      for (int j = 0; j < d; ++j) s += Kinv[static_cast<size_t>(i) * d + j] * f->uC[j];
      for (int j = 0; j < d; ++j) Hd[static_cast<size_t>(i) * d + j] = Kinv[static_cast<size_t>(i) * d + j] - s * f->uC[j];
    }
    if (!keep) f->H = std::move(Kinv);
  }

  // null vectors of S and L
  int st = left_null_S(g, f, err);
  if (st != SMPM_OK) return st;
  f->uL.assign(g.r, 0.0);
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < g.nel; ++e) {
    // (B^T u_S)_e = sum over interface faces G of e, t:
    //   -tau_G (p_G e_q(G,t) - n_G.grad|_(G,t))^T u_S(nbr(e,G), opp G, t)
    std::vector<double> bt(n * n, 0.0), U(n * n);
    for (int G = 0; G < 4; ++G) {
      int e2 = g.neighbour(static_cast<int>(e), G);
      if (e2 < 0) continue;
      // the slot (e2, opp G, t) is written with e2's tau, p and e's own gradient
      const double* fn = c.face(e2, opposite(G));
      const double tg = fn[0], pg = fn[1], sc = c.face(static_cast<int>(e), G)[2];
      for (int t = 0; t < n; ++t) {
        double v = -tg * f->uS[e2 * M + opposite(G) * n + t];
        int a, b;
        g.face_node(G, t, &a, &b);
        bt[b * n + a] += pg * v;
        for (int q = 0; q < n; ++q) {  // minus the transposed normal-derivative row
          switch (G) {
            case FACE_W: bt[t * n + q] -= -sc * f->D[q] * v; break;
            case FACE_E: bt[t * n + q] -= sc * f->D[(n - 1) * n + q] * v; break;
            case FACE_S: bt[q * n + t] -= -sc * f->D[q] * v; break;
            default: bt[q * n + t] -= sc * f->D[(n - 1) * n + q] * v; break;
          }
        }
      }
    }
    elem_solve_T(n, c.fx(static_cast<int>(e)), c.fy(static_cast<int>(e)), bt.data(), U.data());
    for (int q = 0; q < n * n; ++q) f->uL[e * n * n + q] = -U[q];
  }
  {
    double nrm = 0;
    size_t imax = 0;
    for (size_t i = 0; i < f->uL.size(); ++i) {
      nrm += f->uL[i] * f->uL[i];
      if (std::fabs(f->uL[i]) > std::fabs(f->uL[imax])) imax = i;
    }
    nrm = std::sqrt(nrm) * (f->uL[imax] >= 0 ? 1.0 : -1.0);
    for (auto& v : f->uL) v /= nrm;
  }
  // normalised GLL mass for the zero-mean step
  f->what.assign(g.r, 0.0);
  double tot = 0;
  for (long long e = 0; e < g.nel; ++e)
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        double w = f->w1d[a] * f->w1d[b] * g.hx_of(static_cast<int>(e)) * g.hy_of(static_cast<int>(e)) / 4.0;
        f->what[e * n * n + b * n + a] = w;
        tot += w;
      }
  for (auto& v : f->what) v /= tot;

  if (o.flags & SMPM_FLAG_ADJOINT) {
    // transposed system: T~_e = T_e^T in the same push form (the slot swap
    // Phi maps S^T to I + push(T^T)); blocks, row sums and fast
    // diagonalisation follow from it, the coarse matrix is C^T
    f->Ta.resize(f->T.size());
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < g.nel; ++e) {
      const double* Te = f->T.data() + static_cast<size_t>(e) * M * M;
      double* Ae = f->Ta.data() + static_cast<size_t>(e) * M * M;
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) Ae[i * M + j] = Te[j * M + i];
    }
    row_sums(g, f->Ta, f->zwa, &f->Rsa);
    int sta = block_factors(g, f->black, f->Ta, f->tcls, &f->Ga, &f->Xa, err);
    if (sta != SMPM_OK) return sta;
    transpose_fd(n, f->fdx, &f->fdxT);
    transpose_fd(n, f->fdy, &f->fdyT);
    // C^T is singular with left null vector c0 and right null vector u_C;
    // (K^T)^-1 = (K^-1)^T solves the bordered [[C^T, c0], [c0^T, 0]], so
    //   Ha = (I - u_C u_C^T) Kinv^T (I - c0^ c0^T)
    // maps r to the y with C^T y = r - c0^ (c0^T r) and u_C^T y = 0
    // (the reading with the null vectors' roles swapped)
    std::vector<double> ch(d), v(d, 0.0), w(d, 0.0);
    double cn = 0;
    for (int i = 0; i < d; ++i) cn += f->c0[i] * f->c0[i];
    cn = std::sqrt(cn);
    for (int i = 0; i < d; ++i) ch[i] = f->c0[i] / cn;
    // v_i = sum_k Kinv[k][i] ch_k ; w_j = sum_k u_k Kinv[j][k] - (u . v) ch_j
    for (int k = 0; k < d; ++k) {
      const double* row = Kinv.data() + static_cast<size_t>(k) * d;
      for (int i = 0; i < d; ++i) v[i] += row[i] * ch[k];
    }
    double uv = 0;
    for (int k = 0; k < d; ++k) uv += f->uC[k] * v[k];
#pragma omp parallel for schedule(static)
    for (int j = 0; j < d; ++j) {
      const double* row = Kinv.data() + static_cast<size_t>(j) * d;
      double acc = 0;
      for (int k = 0; k < d; ++k) acc += f->uC[k] * row[k];
      w[j] = acc - uv * ch[j];
    }
    f->Ha.assign(static_cast<size_t>(d) * d, 0.0);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        f->Ha[static_cast<size_t>(i) * d + j] =
            Kinv[static_cast<size_t>(j) * d + i] - v[i] * ch[j] - f->uC[i] * w[j];
    // left null vector of the permuted S^T: Phi B1 (Phi swaps the two slots
    // facing each other across an interface; Phi B1 = B1 where B1 is constant
    // on each interface), normalised
    double bn = 0;
    for (double b : f->B1) bn += b * b;
    bn = std::sqrt(bn);
    f->uSa.assign(g.kp, 0.0);
    for (long long e = 0; e < g.nel; ++e)
      for (int F = 0; F < 4; ++F) {
        const int e2 = g.neighbour(static_cast<int>(e), F);
        if (e2 < 0) continue;
        for (int t = 0; t < n; ++t)
          f->uSa[e * M + F * n + t] = f->B1[static_cast<size_t>(e2) * M + opposite(F) * n + t] / bn;
      }
    f->has_adjoint = true;
  }
  return SMPM_OK;
}

// The factor step throws nothing: it runs inside OpenMP regions (one grid
// per thread in smpm_factor_many) and behind the C ABI.  A failed host
// allocation -- e.g. the dense d x d coarse matrix of a very large grid --
// or a container asked for more than it can hold becomes ENOMEM.
int factor_host(const Geometry& g, const smpm_opts& o, Factors* f, std::string* err) {
  try {
    return factor_host_body(g, o, f, err);
  } catch (const std::bad_alloc&) {
    *err = "host allocation failed in the factor step";
  } catch (const std::exception& e) {
    *err = std::string("factor step: ") + e.what();
  }
  *f = Factors();
  return SMPM_ENOMEM;
}

}  // namespace smpm
