// Device helpers for the displacement-pressure coupling E_{ij} = (phi^p_j, div v_i)
// of §Monolithic Approach (the -b E p block of A_s and the b E^T u storage term),
// evaluated pointwise and sum-factorised on the uniform Cartesian mesh:
//
//  * E_c = tensor product over the directions of 1-D Q2-node x Gauss-point
//    factors, the derivative factor (bd) along c and the value factor (bv)
//    along the others.
//  * A Q2 node sees the Gauss-point pressures of the (up to 2^d) cells sharing
//    it: a 4-wide window per direction at a vertex, 2 at a mid node.
//  * A Gauss point sees the 3^d Q2 nodes of its own cell.
//
// Everything stays in registers: fixed-size windows with zero weights on the
// missing taps (and an in-range index), no runtime-indexed local arrays.
#pragma once
#include "common.cuh"
#include "tables.h"

namespace biot {

// Face bit (2*dir + side) set when that face constrains displacement component c.
__device__ __forceinline__ int u_face_mask(const Grid& g, int c) {
  int m = 0;
  for (int f = 0; f < 2 * g.dim; ++f) {
    const int b = g.ubc[f];
    if (b == U_DIRICHLET || (b == U_ROLLER && c == f / 2)) m |= 1 << f;
  }
  return m;
}
__device__ __forceinline__ bool u_free_mask(int m, int gx, int gy, int gz, int nx, int ny, int nz) {
  return !(((m & 1) && gx == 0) || ((m & 2) && gx == nx - 1) || ((m & 4) && gy == 0) || ((m & 8) && gy == ny - 1) ||
           ((m & 16) && gz == 0) || ((m & 32) && gz == nz - 1));
}

// 1-D window of the E coupling along direction d for Q2 node index m: the
// Gauss-point pressures starting at s0 (4 slots), with value weights cv and
// derivative weights cd; slots of a missing cell carry zero weight.
template <typename T>
__device__ __forceinline__ void ep_window(const TabT<T>& tb, int d, int m, int ncell, int& s0, T (&cv)[4], T (&cd)[4]) {
  const int j = m >> 1;
  if (m & 1) {  // mid node: own cell only, local node 1
    s0 = 2 * j;
    cv[0] = tb.bv[d][1][0]; cv[1] = tb.bv[d][1][1]; cv[2] = T(0); cv[3] = T(0);
    cd[0] = tb.bd[d][1][0]; cd[1] = tb.bd[d][1][1]; cd[2] = T(0); cd[3] = T(0);
  } else {      // vertex: cell j-1 (local node 2) first if it exists, then cell j (local node 0)
    const bool lo = j >= 1, hi = j < ncell;
    s0 = lo ? 2 * j - 2 : 0;
    cv[0] = lo ? tb.bv[d][2][0] : (hi ? tb.bv[d][0][0] : T(0));
    cv[1] = lo ? tb.bv[d][2][1] : (hi ? tb.bv[d][0][1] : T(0));
    cv[2] = (lo && hi) ? tb.bv[d][0][0] : T(0);
    cv[3] = (lo && hi) ? tb.bv[d][0][1] : T(0);
    cd[0] = lo ? tb.bd[d][2][0] : (hi ? tb.bd[d][0][0] : T(0));
    cd[1] = lo ? tb.bd[d][2][1] : (hi ? tb.bd[d][0][1] : T(0));
    cd[2] = (lo && hi) ? tb.bd[d][0][0] : T(0);
    cd[3] = (lo && hi) ? tb.bd[d][0][1] : T(0);
  }
}

// The windows of one Q2 node in all directions.
template <typename T, int DIM>
struct EpNode {
  int ox[4], oy[4], oz[4];  // clamped pressure-grid coordinates of the window slots
  T vx[4], dx[4], vy[4], dy[4], vz[4], dz[4];
  int nsy, nsz;             // slots with nonzero weights along y and z: 2 unless a vertex between two cells

  __device__ __forceinline__ EpNode(const Grid& g, const TabT<T>& tb, int ix, int iy, int iz) {
    int sx, sy, sz = 0;
    ep_window<T>(tb, 0, ix, g.n[0], sx, vx, dx);
    ep_window<T>(tb, 1, iy, g.n[1], sy, vy, dy);
    if (DIM == 3) ep_window<T>(tb, 2, iz, g.n[2], sz, vz, dz);
    // (neighbouring threads share y and z, so these bounds are uniform across most warps)
    nsy = ((iy & 1) || iy == 0 || iy == 2 * g.n[1]) ? 2 : 4;
    nsz = DIM == 3 ? (((iz & 1) || iz == 0 || iz == 2 * g.n[2]) ? 2 : 4) : 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ox[e] = min(sx + e, g.ng[0] - 1);
      oy[e] = min(sy + e, g.ng[1] - 1);
      oz[e] = DIM == 3 ? min(sz + e, g.ng[2] - 1) : 0;
    }
  }

  // out[c] = (E_c p) at this node for one pressure level p (Gauss-point grid, x fastest)
  __device__ __forceinline__ void eval(const Grid& g, const T* __restrict__ p, T (&out)[DIM]) const {
    constexpr int NZ = DIM == 3 ? 4 : 1;
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int c2 = 0; c2 < NZ; ++c2) {
      if (c2 >= nsz) break;
      T b0 = 0, b1 = 0, b2 = 0;  // y-contracted partial sums
#pragma unroll
      for (int c1 = 0; c1 < 4; ++c1) {
        if (c1 >= nsy) break;
        const T* row = p + ((int64_t)oz[c2] * g.ng[1] + oy[c1]) * g.ng[0];
        T sv = 0, sd = 0;
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) {
          const T pv = __ldg(row + ox[c0]);
          sv += vx[c0] * pv;
          sd += dx[c0] * pv;
        }
        b0 += vy[c1] * sd;  // component 0: derivative along x
        b1 += dy[c1] * sv;  // component 1: derivative along y
        b2 += vy[c1] * sv;  // component 2: values along x and y
      }
      if (DIM == 3) {
        a0 += vz[c2] * b0;
        a1 += vz[c2] * b1;
        a2 += dz[c2] * b2;  // component 2: derivative along z
      } else {
        a0 += b0;
        a1 += b1;
      }
    }
    out[0] = a0;
    out[1] = a1;
    if (DIM == 3) out[DIM - 1] = a2;
  }
};

// E^T at one Gauss point: the 1-D factors f[c][d][a] of component c along
// direction d for the cell's local node a, and the cell's node block.
template <typename T, int DIM>
struct EtPoint {
  int cell[3];
  T f[DIM][3][3];
  int fm[3];
  bool interior;  // no node of the cell lies on the domain boundary: no constraint to test

  __device__ __forceinline__ EtPoint(const Grid& g, const TabT<T>& tb, const int (&co)[3]) {
    int gq[3];
    interior = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cell[d] = (d < DIM) ? co[d] >> 1 : 0;
      gq[d] = (d < DIM) ? (co[d] & 1) : 0;
      if (d < DIM) interior = interior && cell[d] > 0 && cell[d] < g.n[d] - 1;
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      fm[c] = u_face_mask(g, c);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          f[c][d][a] = (d < DIM) ? ((d == c) ? tb.bd[d][a][gq[d]] : tb.bv[d][a][gq[d]]) : (a == 0 ? T(1) : T(0));
    }
  }

  // (E^T u) at this point for one displacement level u ([u_0|u_1|u_2], stride nnode);
  // constrained displacement entries count as zero
  __device__ __forceinline__ T eval(const Grid& g, const T* __restrict__ u) const {
    const int nx = g.nu[0], ny = g.nu[1], nz = g.nu[2];
    constexpr int AZ = (DIM == 3) ? 3 : 1;
    T acc = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
#pragma unroll
      for (int az = 0; az < AZ; ++az)
#pragma unroll
        for (int ay = 0; ay < 3; ++ay) {
          const int iz = 2 * cell[2] + az, iy = 2 * cell[1] + ay;
          const T* row = u + c * g.nnode + ((int64_t)iz * ny + iy) * nx;
          T s = 0;
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            const int ix = 2 * cell[0] + ax;
            if (interior || u_free_mask(fm[c], ix, iy, iz, nx, ny, nz)) s += f[c][0][ax] * __ldg(row + ix);
          }
          acc += f[c][2][az] * f[c][1][ay] * s;
        }
    }
    return acc;
  }
};

// E^T u at the 2^DIM Gauss points of cell (cx, cy, cz) from the cell's 3^DIM nodes per
// component, sum-factorised (x, then y, then z contraction); u = one displacement level
// [u_0|u_1|u_2] (stride nnode); constrained displacement entries count as zero (`interior`:
// no node of the cell is on the domain boundary, nothing to test; fm: face masks per component).
// eu[p], p = gx + 2 gy + 4 gz.
template <typename T, int DIM>
__device__ __forceinline__ void cell_ETu(const Grid& g, const TabT<T>& tb, const T* __restrict__ u, int cx, int cy, int cz,
                                         bool interior, const int (&fm)[DIM], T (&eu)[1 << DIM]) {
  constexpr int NP = 1 << DIM;
  constexpr int NA = DIM == 3 ? 3 : 1;
  const int nx = g.nu[0], ny = g.nu[1], nz = g.nu[2];
#pragma unroll
  for (int p = 0; p < NP; ++p) eu[p] = T(0);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    // 1-D factors of component c: derivative along c, value across
    T fx[3][2], fy[3][2], fz[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        fx[a][q] = (c == 0) ? tb.bd[0][a][q] : tb.bv[0][a][q];
        fy[a][q] = (c == 1) ? tb.bd[1][a][q] : tb.bv[1][a][q];
        fz[a][q] = (DIM == 3) ? ((c == 2) ? tb.bd[2][a][q] : tb.bv[2][a][q]) : T(a == 0 ? 1 : 0);
      }
    const T* uc = u + c * g.nnode;
    T t2[NA][2][2];  // [az][gy][gx]
#pragma unroll
    for (int az = 0; az < NA; ++az)
#pragma unroll
      for (int q = 0; q < 4; ++q) t2[az][q >> 1][q & 1] = T(0);
#pragma unroll
    for (int az = 0; az < NA; ++az) {
      const int iz = 2 * cz + az;
#pragma unroll
      for (int ay = 0; ay < 3; ++ay) {
        const int iy = 2 * cy + ay;
        const T* row = uc + ((int64_t)iz * ny + iy) * nx + 2 * cx;
        T v[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
          v[ax] = (interior || u_free_mask(fm[c], 2 * cx + ax, iy, iz, nx, ny, nz)) ? __ldg(row + ax) : T(0);
#pragma unroll
        for (int gx = 0; gx < 2; ++gx) {
          const T t1 = fx[0][gx] * v[0] + fx[1][gx] * v[1] + fx[2][gx] * v[2];
#pragma unroll
          for (int gy = 0; gy < 2; ++gy) t2[az][gy][gx] += fy[ay][gy] * t1;
        }
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int gx = p & 1, gy = (p >> 1) & 1, gz = (p >> 2) & 1;
      T a2 = 0;
#pragma unroll
      for (int az = 0; az < NA; ++az) a2 += fz[az][gz] * t2[az][gy][gx];
      eu[p] += a2;
    }
  }
}

}  // namespace biot
