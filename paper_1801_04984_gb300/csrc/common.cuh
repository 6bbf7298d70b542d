// Shared device-side definitions of the GB300 space-time Biot library.
//
// Discretisation (paper §Discretisation in Space / in Time): continuous Q2
// displacement, RT1 flux, DGQ1 pressure on a Cartesian mesh; dG(r) in time with
// a right-Radau Lagrange basis.  On a uniform Cartesian mesh with constant
// Lamé coefficients every spatial block factors into 1-D matrices: the global
// elasticity matrix is a sum of Kronecker products of banded 1-D Q2 matrices
// (mass M, stiffness K, derivative coupling G and its transpose), and E, B, Mp
// are Kronecker products of 1-D maps between the Q2 node grid and the Gauss
// point grid.  Only the flux mass carries a per-cell factor eta / K_c.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace biot {

constexpr int MAXR = 3;  // r <= 2 -> at most 3 temporal DoFs

enum { U_NATURAL = 0, U_DIRICHLET = 1, U_ROLLER = 2 };
enum { F_NATURAL = 0, F_NOFLOW = 1 };

// One mesh level: sizes, spacings, boundary codes and block offsets of one
// temporal level of a slab vector [u_0..u_{d-1} | q_0..q_{d-1} | p].
struct Grid {
  int dim;
  int n[3];    // cells per direction (n[2] = 1 in 2-D)
  int nu[3];   // Q2 nodes per direction, 2n+1 (1 in unused directions)
  int ng[3];   // Gauss points per direction, 2n (1 in unused directions)
  double h[3];
  int ubc[6], fbc[6];
  int64_t nnode;   // Q2 nodes per component
  int64_t Nu;      // dim * nnode
  int64_t nq[3];   // flux DoFs per component
  int64_t offq[3]; // offset of q_c inside a temporal level
  int64_t Np;      // pressure DoFs
  int64_t offp;
  int64_t N;       // DoFs per temporal level
  int64_t ncells;
  int nb;          // independent instances batched on this grid (1: a single problem).  Batched
                   // vectors are level-major: column (k, b) of a slab vector starts at
                   // (k * nb + b) * N; per-instance coefficient arrays are instance-major.
};

// Coordinates (i0, i1, i2) of the lexicographic index t (first coordinate fastest) on an
// n0 x n1 x * grid.  One temporal level of one instance has fewer than 2^31 entries
// (checked at set-up), so the division runs in 32-bit arithmetic.
__host__ __device__ __forceinline__ void unlex3(int64_t t, int n0, int n1, int& i0, int& i1, int& i2) {
  const unsigned u = (unsigned)t, q = u / (unsigned)n0;
  i0 = (int)(u - q * (unsigned)n0);
  i1 = (int)(q % (unsigned)n1);
  i2 = (int)(q / (unsigned)n1);
}

// 1-D operator taps.  Row types of a Q2 node row: 0 interior vertex, 1 mid
// node, 2 lower boundary vertex, 3 upper boundary vertex.  Taps are offsets
// -2..+2 in node index; out-of-range input nodes are zero-padded, so boundary
// rows differ from interior vertex rows only in the centre tap.
struct Tables1D {
  // [op][rowtype][tap], op: 0 M, 1 K, 2 G (test undifferentiated, trial
  // differentiated), 3 G^T
  double q2[3][4][4][5];   // per direction
  // Gauss <-> node maps, per direction: node row type a in {vertex-left-cell
  // part, mid, vertex-right-cell part} ...  stored as local cell matrices:
  // bv[a][g] = int phi_a psi_g dx (h-scaled), bd[a][g] = int phi_a' psi_g dx
  double bv[3][3][2];
  double bd[3][3][2];
  double mq[3][3][3];      // local 1-D Q2 mass along each direction (h-scaled)
  double wg[3];            // Gauss weight * h per direction (= h/2)
};

__host__ __device__ inline int rowtype(int i, int nnodes) {
  if (i & 1) return 1;
  if (i == 0) return 2;
  if (i == nnodes - 1) return 3;
  return 0;
}

// 1 if Q2 node (comp c, index ix, iy, iz) is free, 0 if essentially constrained.
__host__ __device__ inline int u_free(const Grid& g, int c, int ix, int iy, int iz) {
  int idx[3] = {ix, iy, iz};
  for (int d = 0; d < g.dim; ++d) {
    int lo = (idx[d] == 0), hi = (idx[d] == g.nu[d] - 1);
    if (lo) {
      int b = g.ubc[2 * d];
      if (b == U_DIRICHLET || (b == U_ROLLER && c == d)) return 0;
    }
    if (hi) {
      int b = g.ubc[2 * d + 1];
      if (b == U_DIRICHLET || (b == U_ROLLER && c == d)) return 0;
    }
  }
  return 1;
}

// 1 if flux DoF of component c at along-index ia is free (q.n = 0 is essential on no-flow faces)
__host__ __device__ inline int q_free(const Grid& g, int c, int ia) {
  if (ia == 0 && g.fbc[2 * c] == F_NOFLOW) return 0;
  if (ia == g.nu[c] - 1 && g.fbc[2 * c + 1] == F_NOFLOW) return 0;
  return 1;
}

// Coefficients of one slab-operator application.  For temporal output level k:
//   Y^u_k = au[k] * A u_k          + E   (sum_l ep[k][l] p_l)
//   Y^q_k = aq[k] * Mq q_k          + B^T (sum_l qp[k][l] p_l)
//   Y^p_k = E^T (sum_l pu[k][l] u_l) + Mp (sum_l pp[k][l] p_l) + pq[k] * B q_k
// on free rows; constrained u/q rows return the input (identity rows).
struct SlabCoef {
  int nt;  // r + 1
  double au[MAXR];
  double ep[MAXR][MAXR];
  double aq[MAXR];
  double qp[MAXR][MAXR];
  double pu[MAXR][MAXR];
  double pp[MAXR][MAXR];
  double pq[MAXR];
  double lam, mu;  // Lamé coefficients
  // elasticity kernels: number of columns processed and the divisor that maps a column
  // to its coefficient au[col / udiv] (0: nt * nb columns, divisor nb)
  int ucols, udiv;
};

}  // namespace biot
