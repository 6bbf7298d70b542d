// Host-side construction of the 1-D reference tables and grids (setup time).
#pragma once
#include <cmath>
#include <cstring>
#include "common.cuh"

namespace biot {

template <typename T>
struct TabT {
  T q2[3][4][4][5];
  T bv[3][3][2];
  T bd[3][3][2];
  T mq[3][3][3];
  T wg[3];
  // scale of the integer-tap reference rows per direction and operator: mass h/30,
  // stiffness 1/(3h), G and G^T 1/6 (the elasticity kernels' constant-tap form)
  T opscale[3][4];
};

// 1-D Q2 shape functions on [0,1] with nodes {0, 1/2, 1}
inline long double q2v(int a, long double s) {
  if (a == 0) return 2.0L * (s - 0.5L) * (s - 1.0L);
  if (a == 1) return 4.0L * s * (1.0L - s);
  return 2.0L * s * (s - 0.5L);
}
inline long double q2d(int a, long double s) {
  if (a == 0) return 4.0L * s - 3.0L;
  if (a == 1) return 4.0L - 8.0L * s;
  return 4.0L * s - 1.0L;
}

// Build the tables of one grid.  Local 1-D matrices on the reference interval
// (exact rationals):  mass  [[4,2,-1],[2,16,2],[-1,2,4]]/30,
// stiffness [[7,-8,1],[-8,16,-8],[1,-8,7]]/3, and G_ab = int phi_b' phi_a =
// [[-1/2,2/3,-1/6],[-2/3,0,2/3],[1/6,-2/3,1/2]].  Global rows add the
// contributions of the cell(s) sharing a node; with zero padding outside the
// domain a boundary vertex row keeps only its own cell's centre entry.
inline void build_tables(const Grid& g, TabT<double>& t) {
  std::memset(&t, 0, sizeof(t));
  const long double Ml[3][3] = {{4, 2, -1}, {2, 16, 2}, {-1, 2, 4}};
  const long double Kl[3][3] = {{7, -8, 1}, {-8, 16, -8}, {1, -8, 7}};
  const long double Gl[3][3] = {{-0.5L, 2.0L / 3, -1.0L / 6}, {-2.0L / 3, 0, 2.0L / 3}, {1.0L / 6, -2.0L / 3, 0.5L}};
  const long double gs[2] = {0.5L - std::sqrt(3.0L) / 6.0L, 0.5L + std::sqrt(3.0L) / 6.0L};
  for (int d = 0; d < 3; ++d) {
    long double h = (d < g.dim) ? (long double)g.h[d] : 1.0L;
    long double loc[4][3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        loc[0][a][b] = Ml[a][b] * h / 30.0L;
        loc[1][a][b] = Kl[a][b] / (3.0L * h);
        loc[2][a][b] = Gl[a][b];
        loc[3][a][b] = Gl[b][a];
      }
    for (int op = 0; op < 4; ++op) {
      // interior vertex row 2m: left cell local row 2 (cols 2m-2..2m), right cell local row 0 (cols 2m..2m+2)
      long double iv[5] = {loc[op][2][0], loc[op][2][1], loc[op][2][2] + loc[op][0][0], loc[op][0][1], loc[op][0][2]};
      long double md[5] = {0, loc[op][1][0], loc[op][1][1], loc[op][1][2], 0};
      for (int k = 0; k < 5; ++k) {
        t.q2[d][op][0][k] = (double)iv[k];
        t.q2[d][op][1][k] = (double)md[k];
        t.q2[d][op][2][k] = (double)iv[k];
        t.q2[d][op][3][k] = (double)iv[k];
      }
      t.q2[d][op][2][2] = (double)loc[op][0][0];  // lower boundary: right cell only
      t.q2[d][op][3][2] = (double)loc[op][2][2];  // upper boundary: left cell only
    }
    for (int a = 0; a < 3; ++a)
      for (int q = 0; q < 2; ++q) {
        t.bv[d][a][q] = (double)(0.5L * q2v(a, gs[q]) * h);
        t.bd[d][a][q] = (double)(0.5L * q2d(a, gs[q]));
      }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) t.mq[d][a][b] = (double)(Ml[a][b] * h / 30.0L);
    t.wg[d] = (double)(0.5L * h);
    t.opscale[d][0] = (double)(h / 30.0L);
    t.opscale[d][1] = (double)(1.0L / (3.0L * h));
    t.opscale[d][2] = (double)(1.0L / 6.0L);
    t.opscale[d][3] = (double)(1.0L / 6.0L);
  }
}

template <typename T>
inline TabT<T> cast_tables(const TabT<double>& s) {
  TabT<T> t;
  const double* a = reinterpret_cast<const double*>(&s);
  T* b = reinterpret_cast<T*>(&t);
  for (size_t i = 0; i < sizeof(TabT<double>) / sizeof(double); ++i) b[i] = (T)a[i];
  return t;
}

inline Grid make_grid(int dim, const int* n, const double* lo, const double* hi, const int* ubc, const int* fbc) {
  Grid g;
  std::memset(&g, 0, sizeof(g));
  g.dim = dim;
  for (int d = 0; d < 3; ++d) {
    if (d < dim) {
      g.n[d] = n[d];
      g.nu[d] = 2 * n[d] + 1;
      g.ng[d] = 2 * n[d];
      g.h[d] = (hi[d] - lo[d]) / n[d];
    } else {
      g.n[d] = 1;
      g.nu[d] = 1;
      g.ng[d] = 1;
      g.h[d] = 1.0;
    }
  }
  for (int f = 0; f < 6; ++f) {
    g.ubc[f] = (f < 2 * dim) ? ubc[f] : U_NATURAL;
    g.fbc[f] = (f < 2 * dim) ? fbc[f] : F_NATURAL;
  }
  g.nnode = (int64_t)g.nu[0] * g.nu[1] * g.nu[2];
  g.Nu = dim * g.nnode;
  int64_t off = g.Nu;
  for (int c = 0; c < 3; ++c) {
    if (c < dim) {
      int64_t m = 1;
      for (int d = 0; d < dim; ++d) m *= (d == c) ? g.nu[d] : g.ng[d];
      g.nq[c] = m;
    } else {
      g.nq[c] = 0;
    }
    g.offq[c] = off;
    off += g.nq[c];
  }
  g.offp = off;
  g.Np = (int64_t)g.ng[0] * g.ng[1] * g.ng[2];
  g.N = off + g.Np;
  g.ncells = (int64_t)g.n[0] * g.n[1] * g.n[2];
  g.nb = 1;
  return g;
}

// coarsened grid (all directions halved), same box and boundary codes
inline Grid coarsen(const Grid& f) {
  int n[3];
  double lo[3] = {0, 0, 0}, hi[3];
  for (int d = 0; d < 3; ++d) {
    n[d] = f.n[d] / 2;
    hi[d] = f.h[d] * f.n[d];
  }
  return make_grid(f.dim, n, lo, hi, f.ubc, f.fbc);
}

}  // namespace biot
