// Matrix-free slab operator kernels (paper §Monolithic Approach: the coupled
// operator of all r+1 temporal DoFs of one slab, D (x) S + tau M_t (x) A_s).
//
//  * apply_u : displacement rows.  The elasticity block is applied by global sum
//    factorisation: A = sum of 21 (3-D) / 8 (2-D) Kronecker products of banded
//    1-D Q2 matrices, evaluated tile by tile in shared memory in three passes
//    (z, then y, then x).  The E p coupling is added by a second per-node
//    kernel, sum-factorised over the node's block of Gauss-point pressures.
//  * apply_q : flux rows, Darcy mass with the cellwise eta/K_c and B^T p.
//  * apply_p : pressure rows, E^T u (storage of the volumetric strain),
//    Mp p and B q.
// Every output DoF is computed by exactly one thread (gather form): no atomics,
// bitwise reproducible.
#include <mutex>

#include "coupling.cuh"
#include "internal.h"

namespace biot {

// ---------------------------------------------------------------------------
// elasticity term tables: out comp i += coef * X_i(Y(Z(u_j)))
// ops: 0 M, 1 K, 2 G, 3 G^T ; coef: 0 -> 2mu+lam, 1 -> mu, 2 -> lam
struct Term3 { int j, i, xop, yop, zop, coef; };
// compile-time table (folded after unrolling, so per-thread accumulators stay in registers)
__host__ __device__ constexpr Term3 term3(int t) {
  constexpr Term3 tab[21] = {
      // output x
      {0, 0, 1, 0, 0, 0}, {0, 0, 0, 1, 0, 1}, {0, 0, 0, 0, 1, 1},
      {1, 0, 2, 3, 0, 1}, {2, 0, 2, 0, 3, 1}, {1, 0, 3, 2, 0, 2}, {2, 0, 3, 0, 2, 2},
      // output y
      {1, 1, 1, 0, 0, 1}, {1, 1, 0, 1, 0, 0}, {1, 1, 0, 0, 1, 1}, {2, 1, 0, 2, 3, 1}, {2, 1, 0, 3, 2, 2},
      {0, 1, 3, 2, 0, 1}, {0, 1, 2, 3, 0, 2},
      // output z
      {2, 2, 1, 0, 0, 1}, {2, 2, 0, 0, 1, 0}, {2, 2, 0, 1, 0, 1}, {1, 2, 0, 3, 2, 1}, {1, 2, 0, 2, 3, 2},
      {0, 2, 3, 0, 2, 1}, {0, 2, 2, 0, 3, 2}};
  return tab[t];
}

struct Term2 { int j, i, xop, yop, coef; };
__constant__ Term2 c_terms2[8] = {
    {0, 0, 1, 0, 0}, {0, 0, 0, 1, 1}, {1, 0, 2, 3, 1}, {1, 0, 3, 2, 2},
    {1, 1, 1, 0, 1}, {1, 1, 0, 1, 0}, {0, 1, 3, 2, 1}, {0, 1, 2, 3, 2}};

constexpr int T3 = 8;            // output tile edge (nodes), 3-D
constexpr int H3 = T3 + 4;       // with halo
constexpr int T2 = 16;           // output tile edge, 2-D
constexpr int H2 = T2 + 4;

template <typename T>
__device__ inline T tap5(const T* c, const T* v, int stride) {
  return c[0] * v[0] + c[1] * v[stride] + c[2] * v[2 * stride] + c[3] * v[3 * stride] + c[4] * v[4 * stride];
}

// Output stage of the elasticity kernels for one entry i (column offset included) of
// component-node cn: Ax is (tau A x)_i, x_i the input.  EPI_NONE stores Ax; EPI_CHEB does
// one Chebyshev-Jacobi smoothing step (r = b - Ax, d = c1 d + c2 Dinv r, xo = x + d; rows
// with Dinv = 0 are constrained: xo = b, d = 0); EPI_RESID stores the residual b - Ax.
template <typename T>
__device__ __forceinline__ void u_epilogue(int mode, const UEpi<T>& ep, T* __restrict__ y, int64_t i, int64_t cn, T Ax, T x) {
  if (mode == EPI_NONE) {
    y[i] = Ax;
  } else if (mode == EPI_RESID) {
    y[i] = ep.b[i] - Ax;
  } else {
    const T di = ep.dinv[cn], bi = ep.b[i];
    if (di == T(0)) {
      ep.xo[i] = bi;
      ep.d[i] = T(0);
    } else {
      T dn = ep.c2 * di * (bi - Ax);
      if (ep.c1 != T(0)) dn += ep.c1 * ep.d[i];
      ep.d[i] = dn;
      ep.xo[i] = x + dn;
    }
  }
}

// ---------------------------------------------------------------------------
// Y_k += E (sum_l ep[k][l] p_l) on the free displacement rows (§Monolithic
// Approach: the -b E p block of A_s and its time mixing), one thread per Q2 node
// for all components and temporal levels, sum-factorised over the node's block of
// Gauss-point pressures.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_add_Ep(Grid g, TabT<T> tb, SlabCoef sc, const T* __restrict__ p_in, int64_t sp,
                                                T* __restrict__ y, int64_t sy) {
  const int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (node >= g.nnode) return;
  int ix, iy, iz;
  unlex3(node, g.nu[0], g.nu[1], ix, iy, iz);
  if (DIM == 2) iz = 0;
  const EpNode<T, DIM> en(g, tb, ix, iy, iz);
  const int b = blockIdx.y, nb = g.nb;  // instance of a batched grid
  T s[MAXR][DIM];  // s[k][c] = sum_l ep[k][l] (E_c p_l)
#pragma unroll
  for (int k = 0; k < MAXR; ++k)
#pragma unroll
    for (int c = 0; c < DIM; ++c) s[k][c] = T(0);
#pragma unroll 1
  for (int l = 0; l < sc.nt; ++l) {
    T e[DIM];
    en.eval(g, p_in + (int64_t)(l * nb + b) * sp, e);
#pragma unroll
    for (int k = 0; k < MAXR; ++k) {
      const T w = T(l == 0 ? sc.ep[k][0] : (l == 1 ? sc.ep[k][1] : sc.ep[k][2]));
#pragma unroll
      for (int c = 0; c < DIM; ++c) s[k][c] += w * e[c];
    }
  }
  const int64_t nn = g.nnode;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    if (!u_free_mask(u_face_mask(g, c), ix, iy, iz, g.nu[0], g.nu[1], g.nu[2])) continue;
#pragma unroll
    for (int k = 0; k < MAXR; ++k)
      if (k < sc.nt) y[(int64_t)(k * nb + b) * sy + c * nn + node] += s[k][c];
  }
}

constexpr int U3_THREADS = 384;

// ---------------------------------------------------------------------------
// 3-D displacement rows.  grid: (tiles_x, tiles_y, tiles_z * nt); one block =
// one 8^3-node output tile of one temporal level k, staged with a 2-node halo
// (12^3) in shared memory; z, y, x passes of the 21 Kronecker terms.
// Y_k = au[k] A u_k on free rows, u_k on constrained rows (u_in: nt levels of
// [u_0|u_1|u_2] at stride su, y at stride sy; the E p term is added by k_add_Ep).
// Column form: every work item owns a whole line of the tile in registers: a z pass item loads its 12 staged values once and produces the
// 8 outputs of all 4 operators; a y pass item owns one pre-x target (output
// component i, x operator) along y; an x pass item owns one output component
// along x.  Vertex rows use 5 taps, mid rows 3; domain-boundary vertex rows
// differ only in the centre tap (zero padding outside the domain).
// ALLJ (FP32): the z pass runs for the three input components at once (12
// z-pass arrays); otherwise (FP64, twice the shared memory per value) component
// by component with the y pass accumulating into the pre-x arrays.
// Reference 1-D Q2 rows with integer taps (unit cell, before the per-direction scale):
// mass x30 (scale h/30), stiffness x3 (scale 1/(3h)), derivative coupling G and its
// transpose x6 (scale 1/6).  Vertex rows have 5 taps (offsets -2..2), mid rows 3; a
// vertex row on the domain boundary keeps only its own cell's centre entry.
template <int OP>
__host__ __device__ constexpr float ref_vertex(int k) {
  constexpr float M[5] = {-1.f, 2.f, 8.f, 2.f, -1.f}, K[5] = {1.f, -8.f, 14.f, -8.f, 1.f};
  constexpr float G[5] = {1.f, -4.f, 0.f, 4.f, -1.f}, Gt[5] = {-1.f, 4.f, 0.f, -4.f, 1.f};
  return OP == 0 ? M[k] : (OP == 1 ? K[k] : (OP == 2 ? G[k] : Gt[k]));
}
template <int OP>
__host__ __device__ constexpr float ref_mid(int k) {  // offsets -1, 0, 1
  constexpr float M[3] = {2.f, 16.f, 2.f}, K[3] = {-8.f, 16.f, -8.f}, G[3] = {-4.f, 0.f, 4.f}, Gt[3] = {4.f, 0.f, -4.f};
  return OP == 0 ? M[k] : (OP == 1 ? K[k] : (OP == 2 ? G[k] : Gt[k]));
}
template <int OP>
__host__ __device__ constexpr float ref_centre_lo() { return OP == 0 ? 4.f : (OP == 1 ? 7.f : -3.f); }
template <int OP>
__host__ __device__ constexpr float ref_centre_hi() { return OP == 0 ? 4.f : (OP == 1 ? 7.f : 3.f); }

template <int OP, typename T>
__device__ __forceinline__ void col8(int g0, int nn, const T* w, T* out) {
  // w[0..11]: staged line (offset -2), out[0..7]: unscaled outputs of operator OP along the line
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int gi = g0 + o;
    if ((o & 1) == 0) {
      const T cc = (gi == 0) ? T(ref_centre_lo<OP>()) : ((gi == nn - 1) ? T(ref_centre_hi<OP>()) : T(ref_vertex<OP>(2)));
      out[o] = T(ref_vertex<OP>(0)) * w[o] + T(ref_vertex<OP>(1)) * w[o + 1] + cc * w[o + 2] + T(ref_vertex<OP>(3)) * w[o + 3] +
               T(ref_vertex<OP>(4)) * w[o + 4];
    } else {
      out[o] = T(ref_mid<OP>(0)) * w[o + 1] + T(ref_mid<OP>(1)) * w[o + 2] + T(ref_mid<OP>(2)) * w[o + 3];
    }
  }
}

template <int Q, typename T>
__device__ __forceinline__ void ypass_target(const T* __restrict__ s_zo, T* __restrict__ s_px, const T (&sz)[4], const T (&sy)[4],
                                             int Y0, int ny, int lz, int lx, T cf0, T cf1, T cf2, int jonly) {
  constexpr int HH = H3 * H3, ZO = H3 * H3 * T3, PX = H3 * T3 * T3;
  T acc[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) acc[o] = 0;
#pragma unroll
  for (int t = 0; t < 21; ++t) {
    const Term3 tm = term3(t);
    if (tm.i * 4 + tm.xop != Q) continue;
    if (jonly >= 0 && tm.j != jonly) continue;
    const T* src = s_zo + (jonly >= 0 ? tm.zop : tm.j * 4 + tm.zop) * ZO + lz * HH + lx;
    T w[12];
#pragma unroll
    for (int y = 0; y < 12; ++y) w[y] = src[y * H3];
    T o8[8];
    switch (tm.yop) {
      case 0: col8<0>(Y0, ny, w, o8); break;
      case 1: col8<1>(Y0, ny, w, o8); break;
      case 2: col8<2>(Y0, ny, w, o8); break;
      default: col8<3>(Y0, ny, w, o8); break;
    }
    // the term's material coefficient with the z and y scales of its 1-D operators
    const T cfv = (tm.coef == 0 ? cf0 : (tm.coef == 1 ? cf1 : cf2)) * sz[tm.zop] * sy[tm.yop];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[o] += cfv * o8[o];
  }
  T* dst = s_px + Q * PX + lz * (T3 * H3) + lx;
  if (jonly <= 0) {
#pragma unroll
    for (int o = 0; o < 8; ++o) dst[o * H3] = acc[o];
  } else {
#pragma unroll
    for (int o = 0; o < 8; ++o) dst[o * H3] += acc[o];
  }
}

template <typename T, bool ALLJ>
__global__ void __launch_bounds__(U3_THREADS, ALLJ ? 2 : 1) k_apply_u3_col(Grid g, TabT<T> tb, SlabCoef sc,
                                                                            const T* __restrict__ u_in, int64_t su,
                                                                            T* __restrict__ y, int64_t sy, UEpi<T> ep) {
  constexpr int HH = H3 * H3, HHH = H3 * H3 * H3;
  constexpr int ZO = H3 * H3 * T3;
  constexpr int PX = H3 * T3 * T3;
  constexpr int NZO = ALLJ ? 12 : 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_in = reinterpret_cast<T*>(smem_raw);  // 3 * H3^3
  T* s_zo = s_in + 3 * HHH;                  // NZO * ZO
  T* s_px = s_zo + NZO * ZO;                 // 12 * PX
  const int tid = threadIdx.x;
  T scx[4], scy[4], scz[4];  // per-direction scales of the reference 1-D operators
#pragma unroll
  for (int op = 0; op < 4; ++op) {
    scx[op] = tb.opscale[0][op];
    scy[op] = tb.opscale[1][op];
    scz[op] = tb.opscale[2][op];
  }
  const int nx = g.nu[0], ny = g.nu[1], nz = g.nu[2];
  const int ntz = (nz + T3 - 1) / T3;
  const int k = blockIdx.z / ntz;  // column (temporal level x instance, level-major)
  const int X0 = blockIdx.x * T3, Y0 = blockIdx.y * T3, Z0 = (blockIdx.z - k * ntz) * T3;
  const T cf0 = T(2.0 * sc.mu + sc.lam), cf1 = T(sc.mu), cf2 = T(sc.lam);
  const int64_t nn = g.nnode;
  const T* u = u_in + k * su;
  const int fm0 = u_face_mask(g, 0), fm1 = u_face_mask(g, 1), fm2 = u_face_mask(g, 2);
  // staging: several independent loads in flight per thread (the loads hit L2)
  constexpr int NLD = (3 * HHH + U3_THREADS - 1) / U3_THREADS;
  T vals[NLD];
#pragma unroll
  for (int s8 = 0; s8 < NLD; ++s8) {
    const int i = tid + s8 * U3_THREADS;
    T v = 0;
    if (i < 3 * HHH) {
      const int c = i / HHH;
      const int rem = i - c * HHH;
      const int lz = rem / HH, ly = (rem / H3) % H3, lx = rem % H3;
      const int gx = X0 + lx - 2, gy = Y0 + ly - 2, gz = Z0 + lz - 2;
      const int fm = c == 0 ? fm0 : (c == 1 ? fm1 : fm2);
      if ((unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny && (unsigned)gz < (unsigned)nz &&
          u_free_mask(fm, gx, gy, gz, nx, ny, nz))
        v = __ldg(u + c * nn + ((int64_t)gz * ny + gy) * nx + gx);
    }
    vals[s8] = v;
  }
#pragma unroll
  for (int s8 = 0; s8 < NLD; ++s8) {
    const int i = tid + s8 * U3_THREADS;
    if (i < 3 * HHH) s_in[i] = vals[s8];
  }
  __syncthreads();
  constexpr int NJ = ALLJ ? 1 : 3;
  for (int jj = 0; jj < NJ; ++jj) {
    if (jj > 0) __syncthreads();
    // z pass: item = (component, y, x) line along z
    for (int it = tid; it < (ALLJ ? 3 : 1) * HH; it += U3_THREADS) {
      const int c = ALLJ ? it / HH : jj, rem = ALLJ ? it - (it / HH) * HH : it;
      const T* src = s_in + c * HHH + rem;
      T w[12];
#pragma unroll
      for (int z = 0; z < 12; ++z) w[z] = src[z * HH];
      T o8[8];
      T* dst = s_zo + (ALLJ ? c * 4 : 0) * ZO + rem;
      col8<0>(Z0, nz, w, o8);
#pragma unroll
      for (int o = 0; o < 8; ++o) dst[o * HH] = o8[o];
      col8<1>(Z0, nz, w, o8);
#pragma unroll
      for (int o = 0; o < 8; ++o) dst[ZO + o * HH] = o8[o];
      col8<2>(Z0, nz, w, o8);
#pragma unroll
      for (int o = 0; o < 8; ++o) dst[2 * ZO + o * HH] = o8[o];
      col8<3>(Z0, nz, w, o8);
#pragma unroll
      for (int o = 0; o < 8; ++o) dst[3 * ZO + o * HH] = o8[o];
    }
    __syncthreads();
    // y pass: item = (pre-x target q = 4 i + xop, z, x) line along y
    const int jo = ALLJ ? -1 : jj;
    for (int it = tid; it < 12 * T3 * H3; it += U3_THREADS) {
      const int q = it / (T3 * H3), rem = it - q * (T3 * H3);
      const int lz = rem / H3, lx = rem - lz * H3;
      switch (q) {
        case 0: ypass_target<0>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 1: ypass_target<1>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 2: ypass_target<2>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 3: ypass_target<3>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 4: ypass_target<4>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 5: ypass_target<5>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 6: ypass_target<6>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 7: ypass_target<7>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 8: ypass_target<8>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 9: ypass_target<9>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        case 10: ypass_target<10>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
        default: ypass_target<11>(s_zo, s_px, scz, scy, Y0, ny, lz, lx, cf0, cf1, cf2, jo); break;
      }
    }
  }
  __syncthreads();
  // x pass: item = (component, z, y) line along x; results staged in shared memory
  // (s_in is free again) so the output stage below runs on every thread with
  // consecutive threads on consecutive x
  T* s_out = s_in;  // [c][lz][ly][lx], 3 * T3^3
  const T au = T(sc.au[k / sc.udiv]);
  for (int it = tid; it < 3 * T3 * T3; it += U3_THREADS) {
    const int c = it / (T3 * T3), rem = it - c * (T3 * T3);
    const int lz = rem / T3, ly = rem - lz * T3;
    T acc[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[o] = 0;
    const T* src = s_px + (c * 4) * PX + (lz * T3 + ly) * H3;
#pragma unroll
    for (int op = 0; op < 4; ++op) {
      T w[12];
#pragma unroll
      for (int x = 0; x < 12; ++x) w[x] = src[op * PX + x];
      T o8[8];
      switch (op) {
        case 0: col8<0>(X0, nx, w, o8); break;
        case 1: col8<1>(X0, nx, w, o8); break;
        case 2: col8<2>(X0, nx, w, o8); break;
        default: col8<3>(X0, nx, w, o8); break;
      }
#pragma unroll
      for (int o = 0; o < 8; ++o) acc[o] += scx[op] * o8[o];
    }
    T* dst = s_out + it * T3;
#pragma unroll
    for (int o = 0; o < 8; ++o) dst[o] = au * acc[o];
  }
  __syncthreads();
  // output stage: constrained rows return the input; optional fused smoothing step / residual
  const int64_t ko = (int64_t)k * sy;  // column offset of the outputs (and of the epilogue arrays)
  for (int it = tid; it < 3 * T3 * T3 * T3; it += U3_THREADS) {
    const int c = it / (T3 * T3 * T3), rem = it - c * (T3 * T3 * T3);
    const int lz = rem / (T3 * T3), ly = (rem / T3) % T3, lx = rem % T3;
    const int gx = X0 + lx, gy = Y0 + ly, gz = Z0 + lz;
    if (gx >= nx || gy >= ny || gz >= nz) continue;
    const int fm = c == 0 ? fm0 : (c == 1 ? fm1 : fm2);
    const int64_t cn = c * nn + ((int64_t)gz * ny + gy) * nx + gx;
    const bool fr = u_free_mask(fm, gx, gy, gz, nx, ny, nz);
    const T xv = (ep.mode == EPI_CHEB || !fr) ? u[cn] : T(0);
    u_epilogue<T>(ep.mode, ep, y, ko + cn, cn, fr ? s_out[it] : xv, xv);
  }
}

// 2-D displacement rows: tiles of 16x16 nodes, passes y then x.
template <typename T>
__global__ void __launch_bounds__(256) k_apply_u2(Grid g, TabT<T> tb, SlabCoef sc, const T* __restrict__ u_in, int64_t su,
                                                  T* __restrict__ y, int64_t sy, UEpi<T> ep) {
  __shared__ T s_in[2][H2 * H2];
  __shared__ T s_px[8][T2 * H2];
  __shared__ T s_tab[2][4][4][5];
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int i = tid; i < 2 * 4 * 4 * 5; i += nth) (&s_tab[0][0][0][0])[i] = (&tb.q2[0][0][0][0])[i];
  const int X0 = blockIdx.x * T2, Y0 = blockIdx.y * T2;
  const int ex = min(T2, g.nu[0] - X0), ey = min(T2, g.nu[1] - Y0);
  const int rx = ex + 4, ry = ey + 4;
  const T cf[3] = {T(2.0 * sc.mu + sc.lam), T(sc.mu), T(sc.lam)};
  const int64_t nn = g.nnode;
  {
    const int k = blockIdx.z;  // column (temporal level x instance, level-major)
    const T* u = u_in + k * su;
    for (int i = tid; i < 2 * rx * ry; i += nth) {
      int c = i / (rx * ry);
      int rem = i - c * rx * ry;
      int ly = rem / rx, lx = rem - ly * rx;
      int gx = X0 + lx - 2, gy = Y0 + ly - 2;
      T v = 0;
      if (gx >= 0 && gx < g.nu[0] && gy >= 0 && gy < g.nu[1] && u_free(g, c, gx, gy, 0)) v = u[c * nn + (int64_t)gy * g.nu[0] + gx];
      s_in[c][ly * H2 + lx] = v;
    }
    for (int i = tid; i < 8 * T2 * H2; i += nth) (&s_px[0][0])[i] = 0;
    for (int j = 0; j < 2; ++j) {
      __syncthreads();
      for (int i = tid; i < rx * ey; i += nth) {
        int ly = i / rx, lx = i - ly * rx;
        int rt = rowtype(Y0 + ly, g.nu[1]);
        const T* v = &s_in[j][ly * H2 + lx];
        T w[4];
#pragma unroll
        for (int op = 0; op < 4; ++op) w[op] = tap5(s_tab[1][op][rt], v, H2);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const Term2 tm = c_terms2[t];
          if (tm.j != j) continue;
          s_px[tm.i * 4 + tm.xop][ly * H2 + lx] += cf[tm.coef] * w[tm.yop];
        }
      }
    }
    __syncthreads();
    const int64_t ko = (int64_t)k * sy;
    for (int i = tid; i < ex * ey; i += nth) {
      int ly = i / ex, lx = i - ly * ex;
      int gx = X0 + lx, gy = Y0 + ly;
      int rt = rowtype(gx, g.nu[0]);
      int64_t node = (int64_t)gy * g.nu[0] + gx;
      for (int c = 0; c < 2; ++c) {
        const int64_t cn = c * nn + node;
        const T xv = u[cn];
        T out;
        if (u_free(g, c, gx, gy, 0)) {
          T acc = 0;
#pragma unroll
          for (int op = 0; op < 4; ++op) acc += tap5(s_tab[0][op][rt], &s_px[c * 4 + op][ly * H2 + lx], 1);
          out = T(sc.au[k / sc.udiv]) * acc;
        } else {
          out = xv;
        }
        u_epilogue<T>(ep.mode, ep, y, ko + cn, cn, out, xv);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// flux rows: one thread per flux DoF (all components).
template <typename T, int DIM>
__global__ void k_apply_q(Grid g, TabT<T> tb, SlabCoef sc, const T* __restrict__ kscale, const T* __restrict__ x, int64_t sx,
                          T* __restrict__ y, int64_t sy) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (t >= nqt) return;
  const int bi = blockIdx.y, nb = g.nb;  // instance of a batched grid
  kscale += bi * g.ncells;
  int c = 0;
  int64_t r = t;
  while (r >= g.nq[c]) { r -= g.nq[c]; ++c; }
  // grid coordinates of this component's DoF grid
  int sh[3], co[3];
  for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
  unlex3(r, sh[0], sh[1], co[0], co[1], co[2]);
  const int64_t qoff = g.offq[c];
  const int64_t gidx = qoff + r;
  const int ia = co[c];
  // stride of the along-c index in this component's grid
  int64_t stride_c = 1;
  for (int d = 0; d < c; ++d) stride_c *= sh[d];
  // transverse weight and transverse cell indices
  T wt = T(1);
  int cell[3];
  for (int d = 0; d < 3; ++d) {
    if (d < DIM && d != c) { wt *= tb.wg[d]; cell[d] = co[d] >> 1; } else cell[d] = 0;
  }
  // adjacent cells along c: (cell index, local node a)
  int ce[2], la[2], ncell = 0;
  if (ia & 1) { ce[0] = ia >> 1; la[0] = 1; ncell = 1; }
  else {
    int j = ia >> 1;
    if (j >= 1) { ce[ncell] = j - 1; la[ncell] = 2; ++ncell; }
    if (j < g.n[c]) { ce[ncell] = j; la[ncell] = 0; ++ncell; }
  }
  const bool fr = q_free(g, c, ia);
  // p-grid strides
  int64_t pst[3] = {1, g.ng[0], (int64_t)g.ng[0] * g.ng[1]};
  int64_t pbase = 0;
  for (int d = 0; d < DIM; ++d) if (d != c) pbase += co[d] * pst[d];
  for (int k = 0; k < sc.nt; ++k) {
    const T* xk = x + (int64_t)(k * nb + bi) * sx;
    T out;
    if (!fr) out = xk[gidx];
    else {
      T acc = 0;
      for (int e = 0; e < ncell; ++e) {
        cell[c] = ce[e];
        int64_t cid = ((int64_t)cell[2] * g.n[1] + cell[1]) * g.n[0] + cell[0];
        T s = kscale[cid];
        T m = 0;
        for (int b = 0; b < 3; ++b) {
          int ib = 2 * ce[e] + b;
          if (!q_free(g, c, ib)) continue;
          m += tb.mq[c][la[e]][b] * xk[qoff + r + (int64_t)(ib - ia) * stride_c];
        }
        acc += s * m;
      }
      out = T(sc.aq[k]) * wt * acc;
      // B^T p
      for (int l = 0; l < sc.nt; ++l) {
        T w = T(sc.qp[k][l]);
        if (w == T(0)) continue;
        const T* pl = x + (int64_t)(l * nb + bi) * sx + g.offp + pbase;
        T bp = 0;
        for (int e = 0; e < ncell; ++e)
          for (int q = 0; q < 2; ++q) bp += tb.bd[c][la[e]][q] * pl[(int64_t)(2 * ce[e] + q) * pst[c]];
        out += w * wt * bp;
      }
    }
    y[(int64_t)(k * nb + bi) * sy + gidx] = out;
  }
}

// ---------------------------------------------------------------------------
// pressure rows: one thread per Gauss-point pressure DoF.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_apply_p(Grid g, TabT<T> tb, SlabCoef sc, const T* __restrict__ x, int64_t sx, T* __restrict__ y, int64_t sy) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  int co[3];
  unlex3(t, g.ng[0], g.ng[1], co[0], co[1], co[2]);
  int cell[3], gq[3];
  for (int d = 0; d < 3; ++d) { cell[d] = (d < DIM) ? co[d] >> 1 : 0; gq[d] = (d < DIM) ? (co[d] & 1) : 0; }
  T mp = T(1);
  for (int d = 0; d < DIM; ++d) mp *= tb.wg[d];
  T eu[MAXR], bq[MAXR], pv[MAXR];
  const EtPoint<T, DIM> et(g, tb, co);
  const int bi = blockIdx.y, nb = g.nb;  // instance of a batched grid
  for (int l = 0; l < sc.nt; ++l) {
    const T* xl = x + (int64_t)(l * nb + bi) * sx;
    const T acc = et.eval(g, xl);  // E^T u: the cell's 3^DIM nodes, all components
    eu[l] = acc;
    // B q: for each component c the 3 DoFs along c on this Gauss line
    T bacc = 0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      int sh[3];
      for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
      T wt = T(1);
      int64_t base = 0, mul = 1, stride_c = 1;
      for (int d = 0; d < 3; ++d) {
        if (d == c) stride_c = mul;
        else { base += co[d] * mul; if (d < DIM) wt *= tb.wg[d]; }
        mul *= sh[d];
      }
      const T* qc = xl + g.offq[c] + base;
      T s = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int ia = 2 * cell[c] + a;
        if (q_free(g, c, ia)) s += tb.bd[c][a][gq[c]] * qc[(int64_t)ia * stride_c];
      }
      bacc += wt * s;
    }
    bq[l] = bacc;
    pv[l] = xl[g.offp + t];
  }
  for (int k = 0; k < sc.nt; ++k) {
    T out = T(sc.pq[k]) * bq[k];
    for (int l = 0; l < sc.nt; ++l) out += T(sc.pu[k][l]) * eu[l] + T(sc.pp[k][l]) * mp * pv[l];
    y[(int64_t)(k * nb + bi) * sy + g.offp + t] = out;
  }
}

// ---------------------------------------------------------------------------
// pressure rows, one thread per cell and instance: the cell's 2^DIM Gauss points for every
// temporal output level.  E^T u is sum-factorised over the cell's 3^DIM nodes per component
// (x, then y, then z contraction), B q gathers the cell's flux DoFs line by line; every value
// of the cell is loaded once for all of its points.  Same arithmetic as k_apply_p:
//   Y^p_k = pq[k] B q_k + sum_l (pu[k][l] E^T u_l + pp[k][l] Mp p_l).
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_apply_p_cell(Grid g, TabT<T> tb, SlabCoef sc, const T* __restrict__ x, int64_t sx,
                                                      T* __restrict__ y, int64_t sy) {
  constexpr int NP = 1 << DIM;        // points per cell
  constexpr int NL = 1 << (DIM - 1);  // lines per cell and direction
  constexpr int NA = DIM == 3 ? 3 : 1;
  const int cid = blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= (int)g.ncells) return;
  const int bi = blockIdx.y, nb = g.nb;
  int cx, cy, cz;
  unlex3(cid, g.n[0], g.n[1], cx, cy, cz);
  if (DIM == 2) cz = 0;
  const int cc[3] = {cx, cy, cz};
  const int nx = g.nu[0], ny = g.nu[1], nz = g.nu[2];
  const int pst[3] = {1, g.ng[0], g.ng[0] * g.ng[1]};
  const int pbase = 2 * cx + pst[1] * 2 * cy + pst[2] * 2 * cz;
  bool interior = cx > 0 && cx < g.n[0] - 1 && cy > 0 && cy < g.n[1] - 1;
  if (DIM == 3) interior = interior && cz > 0 && cz < g.n[2] - 1;
  T mp = T(1);
#pragma unroll
  for (int d = 0; d < DIM; ++d) mp *= tb.wg[d];
  int fm[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) fm[c] = u_face_mask(g, c);
  T out[MAXR][NP];
#pragma unroll
  for (int k = 0; k < MAXR; ++k)
#pragma unroll
    for (int p = 0; p < NP; ++p) out[k][p] = T(0);
#pragma unroll
  for (int l = 0; l < MAXR; ++l) {
    if (l >= sc.nt) break;
    const T* xl = x + (int64_t)(l * nb + bi) * sx;
    // ---- E^T u at the cell's points
    T eu[NP];
    cell_ETu<T, DIM>(g, tb, xl, cx, cy, cz, interior, fm, eu);
    // ---- B q at the cell's points
    T bq[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) bq[p] = T(0);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      int mul = 1, stride_c = 1;
      int64_t base = g.offq[c];
      T wt = T(1);
#pragma unroll
      for (int k2 = 0; k2 < DIM; ++k2) {
        if (k2 == c) stride_c = mul;
        else wt *= tb.wg[k2];
        mul *= (k2 == c) ? g.nu[k2] : g.ng[k2];
      }
      bool fr[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) fr[a] = q_free(g, c, 2 * cc[c] + a);
#pragma unroll
      for (int l2 = 0; l2 < NL; ++l2) {
        // transverse Gauss-line coordinates of line l2, the point with along-c bit 0
        int64_t off = base + (int64_t)(2 * cc[c]) * stride_c;
        int p0 = 0, bit = 0, m2 = 1;
#pragma unroll
        for (int k2 = 0; k2 < DIM; ++k2) {
          if (k2 != c) {
            const int b = (l2 >> bit) & 1;
            off += (int64_t)(2 * cc[k2] + b) * m2;
            p0 |= b << k2;
            ++bit;
          }
          m2 *= (k2 == c) ? g.nu[k2] : g.ng[k2];
        }
        T qa[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) qa[a] = fr[a] ? xl[off + (int64_t)a * stride_c] : T(0);
#pragma unroll
        for (int gq = 0; gq < 2; ++gq)
          bq[p0 | (gq << c)] += wt * (tb.bd[c][0][gq] * qa[0] + tb.bd[c][1][gq] * qa[1] + tb.bd[c][2][gq] * qa[2]);
      }
    }
    // ---- pressure values and the level's contributions to every output level
    const T* pl = xl + g.offp + pbase;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int gx = p & 1, gy = (p >> 1) & 1, gz = (p >> 2) & 1;
      const T pv = pl[gx + gy * pst[1] + gz * pst[2]];
#pragma unroll
      for (int k = 0; k < MAXR; ++k) {
        if (k >= sc.nt) break;
        out[k][p] += T(sc.pu[k][l]) * eu[p] + T(sc.pp[k][l]) * mp * pv;
        if (k == l) out[k][p] += T(sc.pq[k]) * bq[p];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < MAXR; ++k) {
    if (k >= sc.nt) break;
    T* yk = y + (int64_t)(k * nb + bi) * sy + g.offp + pbase;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int gx = p & 1, gy = (p >> 1) & 1, gz = (p >> 2) & 1;
      yk[gx + gy * pst[1] + gz * pst[2]] = out[k][p];
    }
  }
}

// ---------------------------------------------------------------------------
// diagonal of the elasticity block A (unit tau) per node and component
template <typename T, int DIM>
__global__ void k_diag_A(Grid g, TabT<T> tb, double lam, double mu, T* __restrict__ d) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.nnode) return;
  int ix, iy, iz;
  unlex3(t, g.nu[0], g.nu[1], ix, iy, iz);
  int rt[3] = {rowtype(ix, g.nu[0]), rowtype(iy, g.nu[1]), DIM == 3 ? rowtype(iz, g.nu[2]) : 0};
  T Mc[3], Kc[3];
  for (int e = 0; e < DIM; ++e) { Mc[e] = tb.q2[e][0][rt[e]][2]; Kc[e] = tb.q2[e][1][rt[e]][2]; }
  for (int c = 0; c < DIM; ++c) {
    T acc = 0;
    for (int e = 0; e < DIM; ++e) {
      T term = (e == c) ? T(2 * mu + lam) : T(mu);
      for (int f = 0; f < DIM; ++f) term *= (f == e) ? Kc[f] : Mc[f];
      acc += term;
    }
    d[c * g.nnode + t] = u_free(g, c, ix, iy, iz) ? acc : T(1);
  }
}

// ---------------------------------------------------------------------------
// host launchers
template <typename T>
void launch_apply_u(const Grid& g, const TabT<T>& tb, const SlabCoef& sc, const T* u, int64_t su, const T* p, int64_t sp, T* y,
                    int64_t sy, cudaStream_t st, const UEpi<T>* epi) {
  UEpi<T> ep;
  if (epi) ep = *epi;
  else { ep = UEpi<T>(); ep.mode = EPI_NONE; }
  // columns: the nt temporal levels of every batched instance (or the caller's count)
  SlabCoef scu = sc;
  if (scu.ucols <= 0) { scu.ucols = sc.nt * g.nb; scu.udiv = g.nb; }
  if (scu.udiv <= 0) scu.udiv = 1;
  const int cols = scu.ucols;
  if (g.dim == 3 && sizeof(T) == 4 && g.nnode >= ELAST3_MIN_NODES) {
    // FP32 on the fine multigrid levels: the z-marching kernel (elast3.cu); the coarse levels,
    // where a serial march over the planes would be latency-bound, keep the 8^3-tile kernel
    launch_elast3_f32(g, *reinterpret_cast<const TabT<float>*>(&tb), scu, cols, reinterpret_cast<const float*>(u), su,
                      reinterpret_cast<float*>(y), sy, st, reinterpret_cast<const UEpi<float>*>(&ep));
  } else if (g.dim == 3) {
    constexpr bool ALLJ = sizeof(T) == 4;
    dim3 grid((g.nu[0] + T3 - 1) / T3, (g.nu[1] + T3 - 1) / T3, ((g.nu[2] + T3 - 1) / T3) * cols);
    size_t smem = sizeof(T) * (3 * H3 * H3 * H3 + (ALLJ ? 12 : 4) * H3 * H3 * T3 + 12 * H3 * T3 * T3);
    const int kind = sizeof(T) == 4 ? 3 : 1;
    prof_begin(st, kind, (double)g.nnode * cols);
    (note_launch(), k_apply_u3_col<T, ALLJ><<<grid, U3_THREADS, smem, st>>>(g, tb, scu, u, su, y, sy, ep));
    prof_end(st, kind);
  } else {
    dim3 grid((g.nu[0] + T2 - 1) / T2, (g.nu[1] + T2 - 1) / T2, cols);
    const int kind = sizeof(T) == 4 ? 0 : 1;
    prof_begin(st, kind, (double)g.nnode * cols);
    (note_launch(), k_apply_u2<T><<<grid, 256, 0, st>>>(g, tb, scu, u, su, y, sy, ep));
    prof_end(st, kind);
  }
  if (p) {
    bool any = false;
    for (int k = 0; k < sc.nt; ++k)
      for (int l = 0; l < sc.nt; ++l) any = any || sc.ep[k][l] != 0.0;
    if (any) {
      const dim3 blocks((unsigned)((g.nnode + 255) / 256), g.nb);
      if (g.dim == 3) (note_launch(), k_add_Ep<T, 3><<<blocks, 256, 0, st>>>(g, tb, sc, p, sp, y, sy));
      else (note_launch(), k_add_Ep<T, 2><<<blocks, 256, 0, st>>>(g, tb, sc, p, sp, y, sy));
    }
  }
}

template <typename T>
void launch_apply_q(const Grid& g, const TabT<T>& tb, const SlabCoef& sc, const T* kscale, const T* x, int64_t sx, T* y,
                    int64_t sy, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  const dim3 blocks((unsigned)((n + 255) / 256), g.nb);
  if (g.dim == 3) (note_launch(), k_apply_q<T, 3><<<blocks, 256, 0, st>>>(g, tb, sc, kscale, x, sx, y, sy));
  else (note_launch(), k_apply_q<T, 2><<<blocks, 256, 0, st>>>(g, tb, sc, kscale, x, sx, y, sy));
}

template <typename T>
void launch_apply_p(const Grid& g, const TabT<T>& tb, const SlabCoef& sc, const T* x, int64_t sx, T* y, int64_t sy,
                    cudaStream_t st) {
  const dim3 blocks((unsigned)((g.ncells + 127) / 128), g.nb);
  if (g.dim == 3) (note_launch(), k_apply_p_cell<T, 3><<<blocks, 128, 0, st>>>(g, tb, sc, x, sx, y, sy));
  else (note_launch(), k_apply_p_cell<T, 2><<<blocks, 128, 0, st>>>(g, tb, sc, x, sx, y, sy));
}

template <typename T>
void launch_diag_A(const Grid& g, const TabT<T>& tb, double lam, double mu, T* d, cudaStream_t st) {
  int blocks = (int)((g.nnode + 255) / 256);
  if (g.dim == 3) (note_launch(), k_diag_A<T, 3><<<blocks, 256, 0, st>>>(g, tb, lam, mu, d));
  else (note_launch(), k_diag_A<T, 2><<<blocks, 256, 0, st>>>(g, tb, lam, mu, d));
}

// opt-in shared memory sizes, set once per process before any launch (and so before any graph capture)
void apply_init_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
  elast3_init_attributes();
  cudaFuncSetAttribute(k_apply_u3_col<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(float) * (3 * H3 * H3 * H3 + 12 * H3 * H3 * T3 + 12 * H3 * T3 * T3)));
  cudaFuncSetAttribute(k_apply_u3_col<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(double) * (3 * H3 * H3 * H3 + 4 * H3 * H3 * T3 + 12 * H3 * T3 * T3)));
  });
}

#define INST(T)                                                                                                        \
  template void launch_apply_u<T>(const Grid&, const TabT<T>&, const SlabCoef&, const T*, int64_t, const T*, int64_t, T*, \
                                  int64_t, cudaStream_t, const UEpi<T>*);                                              \
  template void launch_apply_q<T>(const Grid&, const TabT<T>&, const SlabCoef&, const T*, const T*, int64_t, T*, int64_t, \
                                  cudaStream_t);                                                                       \
  template void launch_apply_p<T>(const Grid&, const TabT<T>&, const SlabCoef&, const T*, int64_t, T*, int64_t,         \
                                  cudaStream_t);                                                                       \
  template void launch_diag_A<T>(const Grid&, const TabT<T>&, double, double, T*, cudaStream_t);
INST(double)
INST(float)

}  // namespace biot
