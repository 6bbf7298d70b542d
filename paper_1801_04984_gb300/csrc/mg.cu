// Preconditioner kernels: geometric multigrid transfers and Chebyshev-Jacobi
// smoothing for the displacement block, a dense coarse solve, and the pieces of
// the flux-pressure (Darcy) block solve.
//
// Preconditioner (paper §Monolithic Approach and §Preconditioning technology):
// after the time transform each eigen-block is the dG(0)-type system
//   L(lam) = [[tau A, 0, -b tau E], [0, tau Mq, -tau B^T], [lam b E^T, tau B, (lam/M) Mp]]
// which is preconditioned block-triangularly in fixed-stress order: the flow
// block first, with the displacement coupling lam b E^T (tau A)^{-1} b tau E
// replaced by lam (b^2/K_dr) Mp, then the displacement from
// tau A u = r_u + b tau E p.
#include "coupling.cuh"
#include "internal.h"

namespace biot {

// ---------------------------------------------------------------------------
// Q2 -> Q2 embedding prolongation (coarse cell 2h -> two fine cells h):
// fine node 2c = coarse node c; fine nodes at 1/4 and 3/4 of a coarse cell take
// the coarse Q2 interpolant there: (3/8, 3/4, -1/8) and (-1/8, 3/4, 3/8).
template <typename T>
__device__ inline int prolong_taps(int f, int* ci, T* w) {
  if ((f & 1) == 0) { ci[0] = f >> 1; w[0] = T(1); return 1; }
  int m = f >> 2;
  if ((f & 3) == 1) { ci[0] = 2 * m; ci[1] = 2 * m + 1; ci[2] = 2 * m + 2; w[0] = T(0.375); w[1] = T(0.75); w[2] = T(-0.125); }
  else { ci[0] = 2 * m; ci[1] = 2 * m + 1; ci[2] = 2 * m + 2; w[0] = T(-0.125); w[1] = T(0.75); w[2] = T(0.375); }
  return 3;
}

// restriction = transpose of prolongation
template <typename T>
__device__ inline int restrict_taps(int c, int nf, int* fi, T* w) {
  int k = 0;
  if (c & 1) {
    int m = c >> 1;
    fi[k] = 4 * m + 1; w[k++] = T(0.75);
    fi[k] = 4 * m + 2; w[k++] = T(1);
    fi[k] = 4 * m + 3; w[k++] = T(0.75);
  } else {
    int m = c >> 1;
    const int off[5] = {-3, -1, 0, 1, 3};
    const T ww[5] = {T(-0.125), T(0.375), T(1), T(0.375), T(-0.125)};
    for (int t = 0; t < 5; ++t) {
      int f = 4 * m + off[t];
      if (f >= 0 && f < nf) { fi[k] = f; w[k++] = ww[t]; }
    }
  }
  return k;
}

template <typename T>
__global__ void k_prolong_add(Grid gf, Grid gc, const T* __restrict__ xc, int64_t sc, T* __restrict__ xf, int64_t sf, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= gf.nnode) return;
  const int c = blockIdx.y % gf.dim, r = blockIdx.y / gf.dim;
  int f[3];
  unlex3(t, gf.nu[0], gf.nu[1], f[0], f[1], f[2]);
  if (!u_free(gf, c, f[0], f[1], f[2])) return;
  // the coarse correction is zero on constrained coarse nodes (identity rows with zero data)
  int ci[3][3], cnt[3];
  T w[3][3];
  for (int d = 0; d < 3; ++d) {
    if (d < gf.dim) cnt[d] = prolong_taps<T>(f[d], ci[d], w[d]);
    else { cnt[d] = 1; ci[d][0] = 0; w[d][0] = T(1); }
  }
  const T* src = xc + r * sc + c * gc.nnode;
  T acc = 0;
  for (int a = 0; a < cnt[2]; ++a)
    for (int b = 0; b < cnt[1]; ++b) {
      const T* row = src + ((int64_t)ci[2][a] * gc.nu[1] + ci[1][b]) * gc.nu[0];
      T s = 0;
      for (int e = 0; e < cnt[0]; ++e) s += w[0][e] * row[ci[0][e]];
      acc += w[2][a] * w[1][b] * s;
    }
  xf[r * sf + c * gf.nnode + t] += acc;
}

template <typename T>
__global__ void k_restrict(Grid gf, Grid gc, const T* __restrict__ rf, int64_t sf, T* __restrict__ rc, int64_t sc, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= gc.nnode) return;
  const int c = blockIdx.y % gf.dim, r = blockIdx.y / gf.dim;
  int cidx[3];
  unlex3(t, gc.nu[0], gc.nu[1], cidx[0], cidx[1], cidx[2]);
  T acc = 0;
  // the fine residual is zero on constrained fine nodes (identity rows, x = b there)
  if (u_free(gc, c, cidx[0], cidx[1], cidx[2])) {
    int fi[3][5], cnt[3];
    T w[3][5];
    for (int d = 0; d < 3; ++d) {
      if (d < gf.dim) cnt[d] = restrict_taps<T>(cidx[d], gf.nu[d], fi[d], w[d]);
      else { cnt[d] = 1; fi[d][0] = 0; w[d][0] = T(1); }
    }
    const T* src = rf + r * sf + c * gf.nnode;
    for (int a = 0; a < cnt[2]; ++a)
      for (int b = 0; b < cnt[1]; ++b) {
        const T* row = src + ((int64_t)fi[2][a] * gf.nu[1] + fi[1][b]) * gf.nu[0];
        T s = 0;
        for (int e = 0; e < cnt[0]; ++e) s += w[0][e] * row[fi[0][e]];
        acc += w[2][a] * w[1][b] * s;
      }
  }
  rc[r * sc + c * gc.nnode + t] = acc;
}

template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, int64_t sc, T* xf, int64_t sf, int nrhs,
                        cudaStream_t st) {
  dim3 grid((unsigned)((fine.nnode + 255) / 256), fine.dim * nrhs);
  (note_launch(), k_prolong_add<T><<<grid, 256, 0, st>>>(fine, coarse, xc, sc, xf, sf, nrhs));
}
template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* rf, int64_t sf, T* rc, int64_t sc, int nrhs,
                     cudaStream_t st) {
  dim3 grid((unsigned)((coarse.nnode + 255) / 256), fine.dim * nrhs);
  (note_launch(), k_restrict<T><<<grid, 256, 0, st>>>(fine, coarse, rf, sf, rc, sc, nrhs));
}

// ---------------------------------------------------------------------------
// Chebyshev step.  dinv == 0 marks a constrained row: x = b there.
template <typename T>
__global__ void k_cheb_update(const T* __restrict__ b, const T* __restrict__ Ax, const T* __restrict__ dinv, T* __restrict__ d,
                              const T* __restrict__ x, T* __restrict__ xo, T c1, T c2, int first, int64_t n, int nrhs,
                              int64_t stride) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T di = dinv[e];
    for (int r = 0; r < nrhs; ++r) {
      int64_t i = r * stride + e;
      T bi = b[i];
      if (di == T(0)) { xo[i] = bi; d[i] = T(0); continue; }
      if (first) {
        T dn = c2 * di * bi;
        d[i] = dn;
        xo[i] = dn;
      } else {
        T res = bi - Ax[i];
        T dn = c2 * di * res;
        if (c1 != T(0)) dn += c1 * d[i];
        d[i] = dn;
        xo[i] = x[i] + dn;
      }
    }
  }
}
template <typename T>
void launch_cheb_update(const T* b, const T* Ax, const T* dinv, T* d, const T* x, T* xo, double c1, double c2, int first,
                        int64_t n, int nrhs, int64_t stride, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  (note_launch(), k_cheb_update<T><<<blocks, 256, 0, st>>>(b, Ax, dinv, d, x, xo, (T)c1, (T)c2, first, n, nrhs, stride));
}

// x[:, r] = s * Ainv b[:, r]; one warp per row
template <typename T>
__global__ void k_dense_gemv(const double* __restrict__ A, int n, const T* __restrict__ b, int64_t sb, T* __restrict__ x, int64_t sx,
                             double s) {
  int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  int r = blockIdx.y;
  if (row >= n) return;
  const double* a = A + (int64_t)row * n;
  const T* bb = b + r * sb;
  double acc = 0;
  for (int j = lane; j < n; j += 32) acc = fma(a[j], (double)bb[j], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[r * sx + row] = (T)(s * acc);
}
template <typename T>
void launch_dense_gemv(const double* Ainv, int n, const T* b, int64_t sb, T* x, int64_t sx, int nrhs, double s,
                       cudaStream_t st) {
  dim3 grid((n + 7) / 8, nrhs);
  (note_launch(), k_dense_gemv<T><<<grid, 256, 0, st>>>(Ainv, n, b, sb, x, sx, s));
}

// ---------------------------------------------------------------------------
// flux / pressure gathers
template <typename T>
struct QIdx {  // decoded flux DoF
  int c, ia;
  int co[3];
  int64_t r, stride_c, pbase;
  T wt;
  int ncell, ce[2], la[2];
};

template <int DIM, typename T>
__device__ inline bool decode_q(const Grid& g, const T* wg, int64_t t, QIdx<T>& q) {
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (t >= nqt) return false;
  int c = 0;
  int64_t r = t;
  while (r >= g.nq[c]) { r -= g.nq[c]; ++c; }
  int sh[3];
  for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
  unlex3(r, sh[0], sh[1], q.co[0], q.co[1], q.co[2]);
  q.c = c;
  q.r = r;
  q.ia = q.co[c];
  q.stride_c = 1;
  for (int d = 0; d < c; ++d) q.stride_c *= sh[d];
  q.wt = T(1);
  int64_t pst[3] = {1, g.ng[0], (int64_t)g.ng[0] * g.ng[1]};
  q.pbase = 0;
  for (int d = 0; d < DIM; ++d)
    if (d != c) { q.wt *= wg[d]; q.pbase += q.co[d] * pst[d]; }
  q.ncell = 0;
  if (q.ia & 1) { q.ce[0] = q.ia >> 1; q.la[0] = 1; q.ncell = 1; }
  else {
    int j = q.ia >> 1;
    if (j >= 1) { q.ce[q.ncell] = j - 1; q.la[q.ncell] = 2; ++q.ncell; }
    if (j < g.n[c]) { q.ce[q.ncell] = j; q.la[q.ncell] = 0; ++q.ncell; }
  }
  return true;
}

// (B^T p) at a flux DoF (without sign)
template <typename T>
__device__ inline T gather_BTp(const Grid& g, const TabT<T>& tb, const QIdx<T>& q, const T* p) {
  int64_t pst[3] = {1, g.ng[0], (int64_t)g.ng[0] * g.ng[1]};
  T bp = 0;
  for (int e = 0; e < q.ncell; ++e)
    for (int k = 0; k < 2; ++k) bp += tb.bd[q.c][q.la[e]][k] * p[q.pbase + (int64_t)(2 * q.ce[e] + k) * pst[q.c]];
  return q.wt * bp;
}

// (B q) at a pressure DoF t, flux input masked
template <typename T, int DIM>
__device__ inline T gather_Bq(const Grid& g, const TabT<T>& tb, int64_t t, const T* q, const T* dscale) {
  int co[3];
  unlex3(t, g.ng[0], g.ng[1], co[0], co[1], co[2]);
  T acc = 0;
  for (int c = 0; c < DIM; ++c) {
    int sh[3];
    for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
    T wt = 1;
    int64_t base = 0, mul = 1, stride_c = 1;
    for (int d = 0; d < 3; ++d) {
      if (d == c) stride_c = mul;
      else { base += co[d] * mul; if (d < DIM) wt *= tb.wg[d]; }
      mul *= sh[d];
    }
    const int64_t off = g.offq[c] - g.Nu + base;  // q arrays here are indexed from the start of the flux block
    int cell = co[c] >> 1, gq = co[c] & 1;
    T s = 0;
    for (int a = 0; a < 3; ++a) {
      int ia = 2 * cell + a;
      if (!q_free(g, c, ia)) continue;
      int64_t i = off + (int64_t)ia * stride_c;
      T v = q[i];
      if (dscale) v *= dscale[i];
      s += tb.bd[c][a][gq] * v;
    }
    acc += wt * s;
  }
  return acc;
}

// diag of Mq (unit tau) per flux DoF (1 on constrained DoFs)
template <typename T, int DIM>
__global__ void k_diag_Mq(Grid g, TabT<T> tb, const T* __restrict__ kscale, T* __restrict__ dmq) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx<double> q;
  double wg[3] = {(double)tb.wg[0], (double)tb.wg[1], (double)tb.wg[2]};
  if (!decode_q<DIM>(g, wg, t, q)) return;
  if (!q_free(g, q.c, q.ia)) { dmq[t] = T(1); return; }
  int cell[3];
  for (int d = 0; d < 3; ++d) cell[d] = (d < DIM && d != q.c) ? (q.co[d] >> 1) : 0;
  double acc = 0;
  for (int e = 0; e < q.ncell; ++e) {
    cell[q.c] = q.ce[e];
    int64_t cid = ((int64_t)cell[2] * g.n[1] + cell[1]) * g.n[0] + cell[0];
    acc += (double)kscale[cid] * (double)tb.mq[q.c][q.la[e]][q.la[e]];
  }
  dmq[t] = (T)(q.wt * acc);
}

// sum_q B_iq^2 / dmq_q at each pressure DoF
template <typename T, int DIM>
__global__ void k_diag_BDBt(Grid g, TabT<T> tb, const T* __restrict__ dmq, T* __restrict__ out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  int co[3];
  unlex3(t, g.ng[0], g.ng[1], co[0], co[1], co[2]);
  double acc = 0;
  for (int c = 0; c < DIM; ++c) {
    int sh[3];
    for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
    double wt = 1.0;
    int64_t base = 0, mul = 1, stride_c = 1;
    for (int d = 0; d < 3; ++d) {
      if (d == c) stride_c = mul;
      else { base += co[d] * mul; if (d < DIM) wt *= (double)tb.wg[d]; }
      mul *= sh[d];
    }
    const int64_t off = g.offq[c] - g.Nu + base;
    int cell = co[c] >> 1, gq = co[c] & 1;
    for (int a = 0; a < 3; ++a) {
      int ia = 2 * cell + a;
      if (!q_free(g, c, ia)) continue;
      double bcoef = wt * (double)tb.bd[c][a][gq];
      acc += bcoef * bcoef / (double)dmq[off + (int64_t)ia * stride_c];
    }
  }
  out[t] = (T)acc;
}

// --- flow solve steps (nrhs levels; flux arrays indexed from the flux block start, stride sq;
//     pressure arrays stride sp) ---
// q0 = Rq / (tau dmq) on free DoFs, Rq on constrained
template <typename T, int DIM>
__global__ void k_q_jacobi(Grid g, const T* __restrict__ rq, int64_t srq, const T* __restrict__ dmq, double tau,
                           T* __restrict__ q0, int64_t sq, int nrhs, TabT<T> tb) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx<T> q;
  if (!decode_q<DIM>(g, tb.wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  for (int r = 0; r < nrhs; ++r) {
    T v = rq[r * srq + t];
    q0[r * sq + t] = fr ? v / (T(tau) * dmq[(r % g.nb) * nqt + t]) : v;
  }
}

// out_p = rp - tau B q
template <typename T, int DIM>
__global__ void k_p_minus_Bq(Grid g, TabT<T> tb, const T* __restrict__ rp, int64_t srp, const T* __restrict__ q, int64_t sq,
                             double tau, T* __restrict__ out, int64_t so, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  for (int r = 0; r < nrhs; ++r)
    out[r * so + t] = rp[r * srp + t] - T(tau) * gather_Bq<T, DIM>(g, tb, t, q + r * sq, nullptr);
}

// tq = (B^T p) / dmq on free flux DoFs, 0 on constrained
template <typename T, int DIM>
__global__ void k_BTp_scaled(Grid g, TabT<T> tb, const T* __restrict__ p, int64_t spp, const T* __restrict__ dmq, T* __restrict__ tq,
                             int64_t sq, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx<T> q;
  if (!decode_q<DIM>(g, tb.wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  for (int r = 0; r < nrhs; ++r) {
    const T dinv = T(1) / dmq[(r % g.nb) * nqt + t];
    tq[r * sq + t] = fr ? gather_BTp<T>(g, tb, q, p + r * spp) * dinv : T(0);
  }
}

// out_p = cm[r] * mp * p + tau * B tq
struct RhsCoef {
  double c[MAXR];
};
template <typename T, int DIM>
__global__ void k_schur_out(Grid g, TabT<T> tb, const T* __restrict__ p, int64_t spp, const T* __restrict__ tq, int64_t sq,
                            double tau, RhsCoef cm, T* __restrict__ out, int64_t so, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  T mp = 1;
  for (int d = 0; d < DIM; ++d) mp *= tb.wg[d];
  for (int r = 0; r < nrhs; ++r)
    out[r * so + t] = T(cm.c[r / g.nb]) * mp * p[r * spp + t] + T(tau) * gather_Bq<T, DIM>(g, tb, t, tq + r * sq, nullptr);
}

// q = (Rq + bt B^T p) / (tau dmq) on free flux DoFs, Rq on constrained
template <typename T, int DIM>
__global__ void k_q_final(Grid g, TabT<T> tb, const T* __restrict__ rq, int64_t srq, const T* __restrict__ p, int64_t spp,
                          const T* __restrict__ dmq, double tau, double bt, T* __restrict__ qo, int64_t sq, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx<T> q;
  if (!decode_q<DIM>(g, tb.wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  for (int r = 0; r < nrhs; ++r) {
    const T den = T(1) / (T(tau) * dmq[(r % g.nb) * nqt + t]);
    T v = rq[r * srq + t];
    if (fr) v = (v + T(bt) * gather_BTp<T>(g, tb, q, p + r * spp)) * den;
    qo[r * sq + t] = v;
  }
}

// bu = ru + alpha * E p on free displacement DoFs, ru on constrained
// bu = ru + alpha E p on free displacement rows, ru on constrained rows; one
// thread per Q2 node, all components (sum-factorised E, see coupling.cuh)
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_u_rhs(Grid g, TabT<T> tb, const T* __restrict__ ru, int64_t sru,
                                               const T* __restrict__ p, int64_t spp, double alpha, T* __restrict__ bu,
                                               int64_t sbu, int nrhs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.nnode) return;
  int ix, iy, iz;
  unlex3(t, g.nu[0], g.nu[1], ix, iy, iz);
  if (DIM == 2) iz = 0;
  const EpNode<T, DIM> en(g, tb, ix, iy, iz);
  bool fr[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) fr[c] = u_free_mask(u_face_mask(g, c), ix, iy, iz, g.nu[0], g.nu[1], g.nu[2]);
  for (int r = 0; r < nrhs; ++r) {
    T ep[DIM];
    en.eval(g, p + r * spp, ep);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      T v = ru[r * sru + c * g.nnode + t];
      if (fr[c]) v += T(alpha) * ep[c];
      bu[r * sbu + c * g.nnode + t] = v;
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T>
void launch_diag_Mq(const Grid& g, const TabT<T>& tb, const T* kscale, T* dmq, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) (note_launch(), k_diag_Mq<T, 3><<<blocks, 256, 0, st>>>(g, tb, kscale, dmq));
  else (note_launch(), k_diag_Mq<T, 2><<<blocks, 256, 0, st>>>(g, tb, kscale, dmq));
}
template <typename T>
void launch_diag_BDBt(const Grid& g, const TabT<T>& tb, const T* dmq, T* out, cudaStream_t st) {
  int blocks = (int)((g.Np + 255) / 256);
  if (g.dim == 3) (note_launch(), k_diag_BDBt<T, 3><<<blocks, 256, 0, st>>>(g, tb, dmq, out));
  else (note_launch(), k_diag_BDBt<T, 2><<<blocks, 256, 0, st>>>(g, tb, dmq, out));
}
template <typename T>
void launch_q_jacobi(const Grid& g, const TabT<T>& tb, const T* rq, int64_t srq, const T* dmq, double tau, T* q0, int64_t sq,
                     int nrhs, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) (note_launch(), k_q_jacobi<T, 3><<<blocks, 256, 0, st>>>(g, rq, srq, dmq, tau, q0, sq, nrhs, tb));
  else (note_launch(), k_q_jacobi<T, 2><<<blocks, 256, 0, st>>>(g, rq, srq, dmq, tau, q0, sq, nrhs, tb));
}
template <typename T>
void launch_p_minus_Bq(const Grid& g, const TabT<T>& tb, const T* rp, int64_t srp, const T* q, int64_t sq, double tau, T* out,
                       int64_t so, int nrhs, cudaStream_t st) {
  int blocks = (int)((g.Np + 255) / 256);
  if (g.dim == 3) (note_launch(), k_p_minus_Bq<T, 3><<<blocks, 256, 0, st>>>(g, tb, rp, srp, q, sq, tau, out, so, nrhs));
  else (note_launch(), k_p_minus_Bq<T, 2><<<blocks, 256, 0, st>>>(g, tb, rp, srp, q, sq, tau, out, so, nrhs));
}
template <typename T>
void launch_schur_apply(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* dmq, T* tq, int64_t sq, double tau,
                        const double* cm, T* out, int64_t so, int nrhs, cudaStream_t st) {
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  RhsCoef rc;
  const int nlev = (nrhs + g.nb - 1) / g.nb;  // nrhs counts columns (level x instance)
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nlev) ? cm[r] : 0.0;
  if (g.dim == 3) {
    (note_launch(), k_BTp_scaled<T, 3><<<(int)((nqt + 255) / 256), 256, 0, st>>>(g, tb, p, spp, dmq, tq, sq, nrhs));
    (note_launch(), k_schur_out<T, 3><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(g, tb, p, spp, tq, sq, tau, rc, out, so, nrhs));
  } else {
    (note_launch(), k_BTp_scaled<T, 2><<<(int)((nqt + 255) / 256), 256, 0, st>>>(g, tb, p, spp, dmq, tq, sq, nrhs));
    (note_launch(), k_schur_out<T, 2><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(g, tb, p, spp, tq, sq, tau, rc, out, so, nrhs));
  }
}
template <typename T>
void launch_q_final(const Grid& g, const TabT<T>& tb, const T* rq, int64_t srq, const T* p, int64_t spp, const T* dmq,
                    double tau, double bt, T* qo, int64_t sq, int nrhs, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) (note_launch(), k_q_final<T, 3><<<blocks, 256, 0, st>>>(g, tb, rq, srq, p, spp, dmq, tau, bt, qo, sq, nrhs));
  else (note_launch(), k_q_final<T, 2><<<blocks, 256, 0, st>>>(g, tb, rq, srq, p, spp, dmq, tau, bt, qo, sq, nrhs));
}
template <typename T>
void launch_u_rhs(const Grid& g, const TabT<T>& tb, const T* ru, int64_t sru, const T* p, int64_t spp, double alpha, T* bu,
                  int64_t sbu, int nrhs, cudaStream_t st) {
  const unsigned grid = (unsigned)((g.nnode + 255) / 256);
  if (g.dim == 3) (note_launch(), k_u_rhs<T, 3><<<grid, 256, 0, st>>>(g, tb, ru, sru, p, spp, alpha, bu, sbu, nrhs));
  else (note_launch(), k_u_rhs<T, 2><<<grid, 256, 0, st>>>(g, tb, ru, sru, p, spp, alpha, bu, sbu, nrhs));
}


// out_p = rp + alpha E^T u at a pressure DoF (u masked)
// out = rp + alpha E^T u per pressure Gauss point (constrained displacements count as zero)
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_p_plus_ETu(Grid g, TabT<T> tb, const T* __restrict__ rp, int64_t srp,
                                                    const T* __restrict__ u, int64_t su, double alpha, T* __restrict__ out,
                                                    int64_t so, int nrhs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  int co[3];
  unlex3(t, g.ng[0], g.ng[1], co[0], co[1], co[2]);
  const EtPoint<T, DIM> et(g, tb, co);
  for (int r = 0; r < nrhs; ++r) out[r * so + t] = rp[r * srp + t] + T(alpha) * et.eval(g, u + r * su);
}
// the same, one thread per cell: E^T u sum-factorised over the cell's nodes for its 2^DIM points
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_p_plus_ETu_cell(Grid g, TabT<T> tb, const T* __restrict__ rp, int64_t srp,
                                                         const T* __restrict__ u, int64_t su, double alpha, T* __restrict__ out,
                                                         int64_t so, int nrhs) {
  constexpr int NP = 1 << DIM;
  const int cid = blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= (int)g.ncells) return;
  int cx, cy, cz;
  unlex3(cid, g.n[0], g.n[1], cx, cy, cz);
  if (DIM == 2) cz = 0;
  bool interior = cx > 0 && cx < g.n[0] - 1 && cy > 0 && cy < g.n[1] - 1;
  if (DIM == 3) interior = interior && cz > 0 && cz < g.n[2] - 1;
  int fm[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) fm[c] = u_face_mask(g, c);
  const int ng0 = g.ng[0], ng01 = g.ng[0] * g.ng[1];
  const int pbase = 2 * cx + ng0 * 2 * cy + ng01 * 2 * cz;
  for (int r = 0; r < nrhs; ++r) {
    T eu[NP];
    cell_ETu<T, DIM>(g, tb, u + r * su, cx, cy, cz, interior, fm, eu);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int off = pbase + (p & 1) + ((p >> 1) & 1) * ng0 + ((p >> 2) & 1) * ng01;
      out[r * so + off] = rp[r * srp + off] + T(alpha) * eu[p];
    }
  }
}
template <typename T>
void launch_p_plus_ETu(const Grid& g, const TabT<T>& tb, const T* rp, int64_t srp, const T* u, int64_t su, double alpha, T* out,
                       int64_t so, int nrhs, cudaStream_t st) {
  const int blocks = (int)((g.ncells + 127) / 128);
  if (g.dim == 3) (note_launch(), k_p_plus_ETu_cell<T, 3><<<blocks, 128, 0, st>>>(g, tb, rp, srp, u, su, alpha, out, so, nrhs));
  else (note_launch(), k_p_plus_ETu_cell<T, 2><<<blocks, 128, 0, st>>>(g, tb, rp, srp, u, su, alpha, out, so, nrhs));
}

// zero constrained entries of one-level vectors
template <typename T>
__global__ void k_mask(Grid g, T* __restrict__ x, int64_t s, int nrhs, int u_only) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < g.nnode) {
    int ix = (int)(t % g.nu[0]);
    int64_t rr = t / g.nu[0];
    int iy = (int)(rr % g.nu[1]);
    int iz = (int)(rr / g.nu[1]);
    for (int c = 0; c < g.dim; ++c)
      if (!u_free(g, c, ix, iy, iz))
        for (int r = 0; r < nrhs; ++r) x[r * s + c * g.nnode + t] = T(0);
  }
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (!u_only && t < nqt) {
    int c = 0;
    int64_t rq = t;
    while (rq >= g.nq[c]) { rq -= g.nq[c]; ++c; }
    int64_t stride_c = 1;
    for (int d = 0; d < c; ++d) stride_c *= (d < g.dim) ? g.ng[d] : 1;
    int ia = (int)((rq / stride_c) % g.nu[c]);
    if (!q_free(g, c, ia))
      for (int r = 0; r < nrhs; ++r) x[r * s + g.Nu + t] = T(0);
  }
}
template <typename T>
void launch_mask(const Grid& g, T* x, int64_t s, int nrhs, cudaStream_t st) {
  int64_t n = g.nnode > (g.nq[0] + g.nq[1] + g.nq[2]) ? g.nnode : (g.nq[0] + g.nq[1] + g.nq[2]);
  (note_launch(), k_mask<T><<<(int)((n + 255) / 256), 256, 0, st>>>(g, x, s, nrhs, 0));
}
template <typename T>
void launch_mask_u(const Grid& g, T* x, int64_t s, int nrhs, cudaStream_t st) {
  (note_launch(), k_mask<T><<<(int)((g.nnode + 255) / 256), 256, 0, st>>>(g, x, s, nrhs, 1));
}

// per-cell flux mass pairing (adjoint gradient): one thread per cell
template <int DIM>
__global__ void k_grad_pair(Grid g, TabT<double> tb, const double* __restrict__ kscale, const double* __restrict__ z,
                            const double* __restrict__ x, double w, double* __restrict__ grad) {
  int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cid >= g.ncells) return;
  int cell[3];
  cell[0] = (int)(cid % g.n[0]);
  int64_t rr = cid / g.n[0];
  cell[1] = (int)(rr % g.n[1]);
  cell[2] = (int)(rr / g.n[1]);
  double acc = 0;
  for (int c = 0; c < DIM; ++c) {
    int sh[3];
    int64_t st[3];
    int64_t mul = 1;
    for (int d = 0; d < 3; ++d) {
      sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
      st[d] = mul;
      mul *= sh[d];
    }
    // transverse Gauss lines of this cell: 2^(DIM-1)
    int tdims[2], nt = 0;
    for (int d = 0; d < DIM; ++d) if (d != c) tdims[nt++] = d;
    double wt = 1.0;
    for (int i = 0; i < nt; ++i) wt *= tb.wg[tdims[i]];
    for (int line = 0; line < (1 << nt); ++line) {
      int64_t base = g.offq[c];
      for (int i = 0; i < nt; ++i) base += (int64_t)(2 * cell[tdims[i]] + ((line >> i) & 1)) * st[tdims[i]];
      double zv[3], xv[3];
      for (int a = 0; a < 3; ++a) {
        int ia = 2 * cell[c] + a;
        bool fr = q_free(g, c, ia);
        int64_t i = base + (int64_t)ia * st[c];
        zv[a] = fr ? z[i] : 0.0;
        xv[a] = fr ? x[i] : 0.0;
      }
      double s = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += zv[a] * tb.mq[c][a][b] * xv[b];
      acc += wt * s;
    }
  }
  grad[cid] += w * kscale[cid] * acc;
}
void launch_grad_pair(const Grid& g, const TabT<double>& tb, const double* kscale, const double* z, const double* x, double w,
                      double* grad, cudaStream_t st) {
  int blocks = (int)((g.ncells + 255) / 256);
  if (g.dim == 3) (note_launch(), k_grad_pair<3><<<blocks, 256, 0, st>>>(g, tb, kscale, z, x, w, grad));
  else (note_launch(), k_grad_pair<2><<<blocks, 256, 0, st>>>(g, tb, kscale, z, x, w, grad));
}

// slab right-hand side from load terms and the jump term
struct RhsTab {
  double c[MAXR][8];
  double phi0[MAXR];
};
__global__ void k_slab_rhs(Grid g, const double* const* __restrict__ f, int nterms, RhsTab tab, int nt,
                           const double* __restrict__ sp, double* __restrict__ y, int64_t ys) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  for (int k = 0; k < nt; ++k) {
    double s = 0;
    for (int m = 0; m < nterms; ++m) s += tab.c[k][m] * f[m][e];
    if (e >= g.offp && sp) s += tab.phi0[k] * sp[e - g.offp];
    y[k * ys + e] = s;
  }
}
void launch_slab_rhs(const Grid& g, const double* const* f, int nterms, const double* c, const double* phi0, int nt,
                     const double* sp, double* y, int64_t ys, cudaStream_t st) {
  RhsTab tab;
  for (int k = 0; k < MAXR; ++k) {
    for (int m = 0; m < 8; ++m) tab.c[k][m] = (k < nt && m < nterms) ? c[k * nterms + m] : 0.0;
    tab.phi0[k] = (k < nt) ? phi0[k] : 0.0;
  }
  (note_launch(), k_slab_rhs<<<(int)((g.N + 255) / 256), 256, 0, st>>>(g, f, nterms, tab, nt, sp, y, ys));
}


// inverse Jacobi diagonal of the flux-pressure Schur approximation per rhs:
// dinv[r][i] = 1 / (cm[r] * mp + tau * sb2[i])
template <typename T>
__global__ void k_schur_dinv(const T* __restrict__ sb2, double mp, RhsCoef cm, double tau, T* __restrict__ dinv, int64_t np, int nrhs,
                             int nb) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= np) return;
  for (int r = 0; r < nrhs; ++r) dinv[r * np + t] = T(1) / (T(cm.c[r / nb] * mp) + T(tau) * sb2[(r % nb) * np + t]);
}
template <typename T>
void launch_schur_dinv(const Grid& g, const TabT<T>& tb, const T* sb2, const double* cm, double tau, T* dinv, int nrhs,
                       cudaStream_t st) {
  RhsCoef rc;
  const int nlev = (nrhs + g.nb - 1) / g.nb;  // nrhs counts columns (level x instance)
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nlev) ? cm[r] : 0.0;
  double mp = 1.0;
  for (int d = 0; d < g.dim; ++d) mp *= (double)tb.wg[d];
  (note_launch(), k_schur_dinv<T><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(sb2, mp, rc, tau, dinv, g.Np, nrhs, g.nb));
}

// Chebyshev step with a per-rhs diagonal (stride n between rhs for every array)
template <typename T>
__global__ void k_cheb_update_r(const T* __restrict__ b, const T* __restrict__ Ax, const T* __restrict__ dinv, T* __restrict__ d,
                                const T* __restrict__ x, T* __restrict__ xo, T c1, T c2, int first, int64_t n, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) {
      int64_t i = r * n + e;
      T di = dinv[i], bi = b[i];
      T dn;
      if (first) { dn = c2 * di * bi; d[i] = dn; xo[i] = dn; }
      else {
        dn = c2 * di * (bi - Ax[i]);
        if (c1 != T(0)) dn += c1 * d[i];
        d[i] = dn;
        xo[i] = x[i] + dn;
      }
    }
}
template <typename T>
void launch_cheb_update_r(const T* b, const T* Ax, const T* dinv, T* d, const T* x, T* xo, double c1, double c2, int first,
                          int64_t n, int nrhs, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  (note_launch(), k_cheb_update_r<T><<<blocks, 256, 0, st>>>(b, Ax, dinv, d, x, xo, (T)c1, (T)c2, first, n, nrhs));
}

// x += s * d (mixed precision update)
template <typename TX, typename TD>
__global__ void k_add_scaled(TX* __restrict__ x, const TD* __restrict__ d, double s, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = (TX)((double)x[e] + s * (double)d[e]);
}
template <typename TX, typename TD>
void launch_add_scaled(TX* x, const TD* d, double s, int64_t n, cudaStream_t st) {
  (note_launch(), k_add_scaled<TX, TD><<<2 * RED_BLOCKS, 256, 0, st>>>(x, d, s, n));
}
template void launch_add_scaled<double, float>(double*, const float*, double, int64_t, cudaStream_t);
template void launch_add_scaled<double, double>(double*, const double*, double, int64_t, cudaStream_t);


// ---------------------------------------------------------------------------
// Exact inverse of the Darcy mass Mq by lines.  Mq is block diagonal: component
// c couples only DoFs on one Gauss line along direction c, through the 1-D Q2
// mass of each cell scaled by eta/K_cell and the transverse Gauss weights.  The
// mid-cell DoF of every cell is condensed onto its two vertices, leaving a
// strictly diagonally dominant tridiagonal system on the vertex DoFs, solved
// by the Thomas algorithm (one thread per line).  No-flow vertices are
// eliminated (zero); on them the output is alpha * input (identity rows).
// out = (s * Mq)^{-1} in on free DoFs.
template <typename T, int DIM>
__global__ void k_mq_line_solve(Grid g, TabT<T> tb, const T* __restrict__ kscale, const T* __restrict__ in, int64_t sin,
                                T* __restrict__ out, int64_t sout, double s_scale, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // line decode: component c, transverse Gauss indices
  int64_t nl[3] = {0, 0, 0};
  for (int c = 0; c < DIM; ++c) nl[c] = g.nq[c] / g.nu[c];
  int c = 0;
  int64_t r = t;
  while (c < DIM && r >= nl[c]) { r -= nl[c]; ++c; }
  if (c >= DIM) return;
  int sh[3];
  for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
  int tr[3] = {0, 0, 0};
  int64_t rr = r;
  T wt = T(1);
  for (int d = 0; d < DIM; ++d) {
    if (d == c) continue;
    tr[d] = (int)(rr % sh[d]);
    rr /= sh[d];
    wt *= tb.wg[d];
  }
  int64_t base = 0, mul = 1, stride_c = 1;
  for (int d = 0; d < 3; ++d) {
    if (d == c) stride_c = mul;
    else base += (int64_t)tr[d] * mul;
    mul *= sh[d];
  }
  base += g.offq[c] - g.Nu;
  int cell[3];
  for (int d = 0; d < 3; ++d) cell[d] = (d < DIM && d != c) ? (tr[d] >> 1) : 0;
  const int n = g.n[c];
  const T hc = tb.mq[c][1][1] * T(30.0 / 16.0);  // = h_c
  const bool lo_fixed = !q_free(g, c, 0), hi_fixed = !q_free(g, c, 2 * n);
  for (int q = 0; q < nrhs; ++q) {
    const T* b = in + q * sin + base;
    T* x = out + q * sout + base;
    // forward sweep over vertices j = 0..n; c'_j kept in x[2j+1], d'_j in x[2j]
    T cprev = 0, dprev = 0;
    T s_left = 0, beta_left = 0;
    for (int j = 0; j <= n; ++j) {
      T s_right = 0, beta_right = 0;
      if (j < n) {
        cell[c] = j;
        int64_t cid = ((int64_t)cell[2] * g.n[1] + cell[1]) * g.n[0] + cell[0];
        s_right = T(s_scale) * kscale[cid] * wt;
        beta_right = T(30) * b[(int64_t)(2 * j + 1) * stride_c] / (hc * s_right);
      }
      bool fixed = (j == 0 && lo_fixed) || (j == n && hi_fixed);
      T a = T(-1.25) * s_left, dd = T(3.75) * (s_left + s_right), cc = T(-1.25) * s_right;
      T rhs = T(30) * b[(int64_t)(2 * j) * stride_c] / hc - (s_left * beta_left + s_right * beta_right) * T(0.125);
      if (fixed) { a = 0; dd = 1; cc = 0; rhs = 0; }
      // eliminate the sub-diagonal with the previous row
      T den = dd - a * cprev;
      T cp = cc / den;
      T dp = (rhs - a * dprev) / den;
      x[(int64_t)(2 * j) * stride_c] = dp;
      if (j < n) x[(int64_t)(2 * j + 1) * stride_c] = cp;
      cprev = cp;
      dprev = dp;
      s_left = s_right;
      beta_left = beta_right;
    }
    // back substitution on vertices, then the condensed mid DoFs
    T xnext = x[(int64_t)(2 * n) * stride_c];
    for (int j = n - 1; j >= 0; --j) {
      T cp = x[(int64_t)(2 * j + 1) * stride_c];
      T xv = x[(int64_t)(2 * j) * stride_c] - cp * xnext;
      x[(int64_t)(2 * j) * stride_c] = xv;
      cell[c] = j;
      int64_t cid = ((int64_t)cell[2] * g.n[1] + cell[1]) * g.n[0] + cell[0];
      T sj = T(s_scale) * kscale[cid] * wt;
      T beta = T(30) * b[(int64_t)(2 * j + 1) * stride_c] / (hc * sj);
      x[(int64_t)(2 * j + 1) * stride_c] = (beta - T(2) * xv - T(2) * xnext) * T(0.0625);
      xnext = xv;
    }
  }
}

// flux-grid gather tq = B^T p on free DoFs (0 on constrained)
// tq = base + coef B^T p on free DoFs (base may be null), 0 on constrained
template <typename T, int DIM>
__global__ void k_BTp(Grid g, TabT<T> tb, const T* __restrict__ p, int64_t spp, const T* __restrict__ base, int64_t sb,
                      T* __restrict__ tq, int64_t sq, T coef, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx<T> q;
  if (!decode_q<DIM>(g, tb.wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  for (int r = 0; r < nrhs; ++r) {
    T v = T(0);
    if (fr) {
      v = coef * gather_BTp<T>(g, tb, q, p + r * spp);
      if (base) v += base[r * sb + t];
    }
    tq[r * sq + t] = v;
  }
}

// out_q = alpha * in_q on constrained flux DoFs (restores the identity rows after a line solve)
template <typename T, int DIM>
__global__ void k_q_fix_constrained(Grid g, const T* __restrict__ in, int64_t sin, T* __restrict__ out, int64_t sout, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (t >= nqt) return;
  int c = 0;
  int64_t rq = t;
  while (rq >= g.nq[c]) { rq -= g.nq[c]; ++c; }
  int64_t stride_c = 1;
  for (int d = 0; d < c; ++d) stride_c *= (d < DIM) ? g.ng[d] : 1;
  int ia = (int)((rq / stride_c) % g.nu[c]);
  if (!q_free(g, c, ia))
    for (int r = 0; r < nrhs; ++r) out[r * sout + t] = in[r * sin + t];
}

template <typename T>
void launch_mq_line_solve(const Grid& g, const TabT<T>& tb, const T* kscale, const T* in, int64_t sin, T* out, int64_t sout,
                          double s_scale, int nrhs, cudaStream_t st) {
  int64_t lines = 0;
  for (int c = 0; c < g.dim; ++c) lines += g.nq[c] / g.nu[c];
  int blocks = (int)((lines + 127) / 128);
  if (g.dim == 3) (note_launch(), k_mq_line_solve<T, 3><<<blocks, 128, 0, st>>>(g, tb, kscale, in, sin, out, sout, s_scale, nrhs));
  else (note_launch(), k_mq_line_solve<T, 2><<<blocks, 128, 0, st>>>(g, tb, kscale, in, sin, out, sout, s_scale, nrhs));
}
template <typename T>
void launch_BTp(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* base, int64_t sb, T* tq, int64_t sq,
                double coef, int nrhs, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) (note_launch(), k_BTp<T, 3><<<blocks, 256, 0, st>>>(g, tb, p, spp, base, sb, tq, sq, T(coef), nrhs));
  else (note_launch(), k_BTp<T, 2><<<blocks, 256, 0, st>>>(g, tb, p, spp, base, sb, tq, sq, T(coef), nrhs));
}
template <typename T>
void launch_q_fix_constrained(const Grid& g, const T* in, int64_t sin, T* out, int64_t sout, int nrhs, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) (note_launch(), k_q_fix_constrained<T, 3><<<blocks, 256, 0, st>>>(g, in, sin, out, sout, nrhs));
  else (note_launch(), k_q_fix_constrained<T, 2><<<blocks, 256, 0, st>>>(g, in, sin, out, sout, nrhs));
}
// out_p = cm[r] mp p + tau B tq (tq on the flux grid, already M_q^{-1} B^T p)
template <typename T>
void launch_schur_out(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* tq, int64_t sq, double tau,
                      const double* cm, T* out, int64_t so, int nrhs, cudaStream_t st) {
  RhsCoef rc;
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nrhs) ? cm[r] : 0.0;
  if (g.dim == 3) (note_launch(), k_schur_out<T, 3><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(g, tb, p, spp, tq, sq, tau, rc, out, so, nrhs));
  else (note_launch(), k_schur_out<T, 2><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(g, tb, p, spp, tq, sq, tau, rc, out, so, nrhs));
}

// z = dinv * r over nrhs vectors (dinv per rhs when dstride != 0, shared otherwise)
template <typename T>
__global__ void k_dinv_mul(const T* __restrict__ dinv, int64_t dstride, const T* __restrict__ r, T* __restrict__ z, int64_t n,
                           int64_t stride, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    for (int q = 0; q < nrhs; ++q) z[q * stride + e] = dinv[q * dstride + e] * r[q * stride + e];
}
template <typename T>
void launch_dinv_mul(const T* dinv, int64_t dstride, const T* r, T* z, int64_t n, int64_t stride, int nrhs, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  (note_launch(), k_dinv_mul<T><<<blocks, 256, 0, st>>>(dinv, dstride, r, z, n, stride, nrhs));
}
template void launch_dinv_mul<double>(const double*, int64_t, const double*, double*, int64_t, int64_t, int, cudaStream_t);
template void launch_dinv_mul<float>(const float*, int64_t, const float*, float*, int64_t, int64_t, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Precomputed stencil of tau B diag(Mq)^{-1} B^T on the Gauss-point pressure grid:
// per point 16 coefficients [self, partner along x, y, z, then for x, y, z the
// two points of the lower and of the upper neighbour cell on the same line]
// (structure of arrays, coef[k * Np + t]; 2-D packs the 11 slots self, x and y
// partner, x lower and upper (2 each), y lower and upper (2 each) the same way).
// One Chebyshev-Jacobi step then costs no division and little index arithmetic.
template <typename T, int DIM>
__global__ void k_schur_stencil(Grid g, TabT<T> tb, const T* __restrict__ dmq, double tau, T* __restrict__ coef) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  const int64_t np = g.Np;
  int co[3];
  unlex3(t, g.ng[0], g.ng[1], co[0], co[1], co[2]);
  double self = 0, part[3] = {0, 0, 0}, lo[3][2] = {{0, 0}, {0, 0}, {0, 0}}, hi[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  for (int c = 0; c < DIM; ++c) {
    int sh[3];
    for (int k = 0; k < 3; ++k) sh[k] = (k < DIM) ? ((k == c) ? g.nu[k] : g.ng[k]) : 1;
    double wt = 1;
    int64_t qbase = 0, mul = 1, stride_c = 1;
    for (int k = 0; k < 3; ++k) {
      if (k == c) stride_c = mul;
      else { qbase += co[k] * mul; if (k < DIM) wt *= (double)tb.wg[k]; }
      mul *= sh[k];
    }
    qbase += g.offq[c] - g.Nu;
    const int cell = co[c] >> 1, gq = co[c] & 1;
    for (int a = 0; a < 3; ++a) {
      const int ia = 2 * cell + a;
      if (!q_free(g, c, ia)) continue;
      const double w = tau * wt * wt * (double)tb.bd[c][a][gq] / (double)dmq[qbase + (int64_t)ia * stride_c];
      // this flux DoF touches the own cell's two points (local a) ...
      for (int k = 0; k < 2; ++k) {
        const double v = w * (double)tb.bd[c][a][k];
        if (k == gq) self += v;
        else part[c] += v;
      }
      // ... and, on a face, the neighbour cell's two points (local 2 - a)
      if (a == 0 && cell >= 1)
        for (int k = 0; k < 2; ++k) lo[c][k] += w * (double)tb.bd[c][2][k];
      if (a == 2 && cell + 1 < g.n[c])
        for (int k = 0; k < 2; ++k) hi[c][k] += w * (double)tb.bd[c][0][k];
    }
  }
  coef[t] = (T)self;
  for (int c = 0; c < DIM; ++c) coef[(1 + c) * np + t] = (T)part[c];
  for (int c = 0; c < DIM; ++c)
    for (int k = 0; k < 2; ++k) {
      coef[(1 + DIM + 4 * c + k) * np + t] = (T)lo[c][k];
      coef[(1 + DIM + 4 * c + 2 + k) * np + t] = (T)hi[c][k];
    }
}

// (Shat_r x)_t with the precomputed stencil of one instance (coef) and the mass term of column r
template <typename T, int DIM>
__device__ __forceinline__ T schur_stencil_eval(const Grid& g, const T* __restrict__ coef, T mass, const T* __restrict__ xr,
                                                int64_t t) {
  const int64_t np = g.Np;
  const int ng0 = g.ng[0], ng1 = g.ng[1];
  const int c0 = (int)(t % ng0);
  const int64_t rr = t / ng0;
  const int co[3] = {c0, (int)(rr % ng1), (int)(rr / ng1)};
  const int64_t pst[3] = {1, ng0, (int64_t)ng0 * ng1};
  T acc = (mass + coef[t]) * xr[t];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int cc = co[c];
    const int64_t base = t - (int64_t)cc * pst[c];  // along-c coordinate 0 of this line
    acc += coef[(1 + c) * np + t] * xr[base + (int64_t)(cc ^ 1) * pst[c]];
    const int e2 = cc & ~1;  // 2 * cell
    if (e2 >= 2) {
      acc += coef[(1 + DIM + 4 * c) * np + t] * xr[base + (int64_t)(e2 - 2) * pst[c]];
      acc += coef[(1 + DIM + 4 * c + 1) * np + t] * xr[base + (int64_t)(e2 - 1) * pst[c]];
    }
    if (e2 + 2 < g.ng[c]) {
      acc += coef[(1 + DIM + 4 * c + 2) * np + t] * xr[base + (int64_t)(e2 + 2) * pst[c]];
      acc += coef[(1 + DIM + 4 * c + 3) * np + t] * xr[base + (int64_t)(e2 + 3) * pst[c]];
    }
  }
  return acc;
}

// Chebyshev-Jacobi step on Shat_r = cm[r] Mp + tau B diag(Mq)^{-1} B^T with the
// precomputed stencil; dinv per rhs (stride Np).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_schur_cheb_st(Grid g, const T* __restrict__ coef, const T* __restrict__ dinv, RhsCoef cm,
                                                       T mp, T c1, T c2, int first, const T* __restrict__ b,
                                                       const T* __restrict__ x, T* __restrict__ d, T* __restrict__ xo) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  const int r = blockIdx.y;  // column: level r / nb of instance r % nb
  const int64_t np = g.Np;
  const int64_t i = r * np + t;
  coef += (int64_t)(r % g.nb) * 16 * np;
  const T di = dinv[i];
  if (first) {
    const T dn = c2 * di * b[i];
    d[i] = dn;
    xo[i] = dn;
    return;
  }
  const T* xr = x + r * np;
  const T acc = schur_stencil_eval<T, DIM>(g, coef, T(cm.c[r / g.nb]) * mp, xr, t);
  T dn = c2 * di * (b[i] - acc);
  if (c1 != T(0)) dn += c1 * d[i];
  d[i] = dn;
  xo[i] = xr[t] + dn;
}

// ---------------------------------------------------------------------------
// Matrix-free form of the same lumped Schur complement.  Per flux DoF f one weight
//   wq_f = tau wt_f^2 / (Mq)_ff   (0 on no-flow DoFs),
// wt_f the transverse Gauss weight of f's line, so that
//   (Shat x)_p = cm mp x_p + sum_f B_pf/wt_f wq_f (B^T x)_f / wt_f
// with the 1-D divergence weights bd only.  A step then streams x, b, d and one flux-grid
// weight array shared by every column of the launch (about 3 values per point) instead of
// the 16 stencil coefficients per point and column, and forms the Jacobi diagonal
// sum_f wq_f bd^2 + cm mp on the fly.
template <typename T, int DIM>
__global__ void k_schur_wq(Grid g, TabT<T> tb, const T* __restrict__ dmq, double tau, T* __restrict__ wq) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx<double> q;
  double wg[3] = {(double)tb.wg[0], (double)tb.wg[1], (double)tb.wg[2]};
  if (!decode_q<DIM>(g, wg, t, q)) return;
  wq[t] = q_free(g, q.c, q.ia) ? (T)(tau * q.wt * q.wt / (double)dmq[t]) : T(0);
}

// One Chebyshev-Jacobi step on Shat for the nk temporal levels of one instance (grid y; column
// of level k = k * nb + instance, stride Np).  One thread owns one cell and its 2^DIM Gauss
// points: along each direction the cell holds 2^(DIM-1) lines of two points, and each line
// couples through its three flux DoFs (lower face, mid, upper face) to the two points of the
// neighbouring cells on the same line.  The cell's values and weights are loaded once for all
// of its points.  All index arithmetic is 32-bit (one level of one instance has fewer than
// 2^31 entries, checked at set-up).
template <typename T, int DIM>
__global__ void __launch_bounds__(256, 3) k_schur_cheb_mf(Grid g, TabT<T> tb, const T* __restrict__ wq, RhsCoef cm, T mp, T c1,
                                                       T c2, int first, int nk, const T* __restrict__ b,
                                                       const T* __restrict__ x, T* __restrict__ d, T* __restrict__ xo) {
  constexpr int NP = 1 << DIM;        // points per cell
  constexpr int NL = 1 << (DIM - 1);  // lines per cell and direction
  const int cid = blockIdx.x * blockDim.x + threadIdx.x;
  if (cid >= (int)g.ncells) return;
  const int inst = blockIdx.y, nb = g.nb;
  const int64_t np = g.Np;
  wq += (int64_t)inst * (g.nq[0] + g.nq[1] + g.nq[2]);
  int cx, cy, cz;
  unlex3(cid, g.n[0], g.n[1], cx, cy, cz);
  if (DIM == 2) cz = 0;
  const int cc[3] = {cx, cy, cz};
  const int pst[3] = {1, g.ng[0], g.ng[0] * g.ng[1]};
  const int pbase = 2 * cx + pst[1] * 2 * cy + pst[2] * 2 * cz;  // the cell's first point
  // point p of the cell (bits gx, gy, gz) at pbase + poff[p]
  int poff[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) poff[p] = (p & 1) + ((p >> 1) & 1) * pst[1] + ((p >> 2) & 1) * pst[2];
  // diagonal of the flux part per point
  T self[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) self[p] = 0;
  // flux-grid offset of line l of direction c at along-index 2 cc[c] (its lower face DoF), stride along c
  int qline[DIM][NL], qstr[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    int mul = 1, stride_c = 1, base = (int)(g.offq[c] - g.Nu);
#pragma unroll
    for (int k2 = 0; k2 < DIM; ++k2) {
      if (k2 == c) stride_c = mul;
      mul *= (k2 == c) ? g.nu[k2] : g.ng[k2];
    }
    qstr[c] = stride_c;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      // transverse Gauss-line coordinates of line l: the bits of l over the other directions
      int off = base + 2 * cc[c] * stride_c, bit = 0, m2 = 1;
#pragma unroll
      for (int k2 = 0; k2 < DIM; ++k2) {
        const int ext = (k2 == c) ? g.nu[k2] : g.ng[k2];
        if (k2 != c) {
          off += (2 * cc[k2] + ((l >> bit) & 1)) * m2;
          ++bit;
        }
        m2 *= ext;
      }
      qline[c][l] = off;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T wa = wq[off + a * stride_c];
#pragma unroll
        for (int gq = 0; gq < 2; ++gq) {
          // point of line l with along-c bit gq
          int p = 0, bb = 0;
#pragma unroll
          for (int k2 = 0; k2 < DIM; ++k2) {
            const int bitv = (k2 == c) ? gq : ((l >> bb) & 1);
            if (k2 != c) ++bb;
            p |= bitv << k2;
          }
          self[p] += wa * tb.bd[c][a][gq] * tb.bd[c][a][gq];
        }
      }
    }
  }
  // neighbour cells present below / above along each direction (bit c)
  const int has_lo = (cx >= 1 ? 1 : 0) | (cy >= 1 ? 2 : 0) | (DIM == 3 && cz >= 1 ? 4 : 0);
  const int has_hi = (cx + 1 < g.n[0] ? 1 : 0) | (cy + 1 < g.n[1] ? 2 : 0) | (DIM == 3 && cz + 1 < g.n[2] ? 4 : 0);
  for (int k = 0; k < nk; ++k) {
    const int64_t col = (int64_t)(k * nb + inst) * np;
    const T mass = T(cm.c[k]) * mp;
    const T* xr = x + col + pbase;
    if (first) {
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const int64_t i = col + pbase + poff[p];
        const T dn = c2 / (mass + self[p]) * b[i];
        d[i] = dn;
        xo[i] = dn;
      }
      continue;
    }
    T xv[NP], acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      xv[p] = xr[poff[p]];
      acc[p] = mass * xv[p];
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        int p0 = 0, bb = 0;  // the line's point with along-c bit 0
#pragma unroll
        for (int k2 = 0; k2 < DIM; ++k2) {
          const int bitv = (k2 == c) ? 0 : ((l >> bb) & 1);
          if (k2 != c) ++bb;
          p0 |= bitv << k2;
        }
        const int p1 = p0 | (1 << c);
        const T x0 = xv[p0], x1 = xv[p1];
        const T* xl = xr + poff[p0];
        T s0 = tb.bd[c][0][0] * x0 + tb.bd[c][0][1] * x1;
        const T s1 = tb.bd[c][1][0] * x0 + tb.bd[c][1][1] * x1;
        T s2 = tb.bd[c][2][0] * x0 + tb.bd[c][2][1] * x1;
        if ((has_lo >> c) & 1) s0 += tb.bd[c][2][0] * xl[-2 * pst[c]] + tb.bd[c][2][1] * xl[-pst[c]];
        if ((has_hi >> c) & 1) s2 += tb.bd[c][0][0] * xl[2 * pst[c]] + tb.bd[c][0][1] * xl[3 * pst[c]];
        const T w0 = wq[qline[c][l]], w1 = wq[qline[c][l] + qstr[c]], w2 = wq[qline[c][l] + 2 * qstr[c]];
        const T t0 = w0 * s0, t1 = w1 * s1, t2 = w2 * s2;
        acc[p0] += tb.bd[c][0][0] * t0 + tb.bd[c][1][0] * t1 + tb.bd[c][2][0] * t2;
        acc[p1] += tb.bd[c][0][1] * t0 + tb.bd[c][1][1] * t1 + tb.bd[c][2][1] * t2;
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int64_t i = col + pbase + poff[p];
      const T dinv = T(1) / (mass + self[p]);
      T dn = c2 * dinv * (b[i] - acc[p]);
      if (c1 != T(0)) dn += c1 * d[i];
      d[i] = dn;
      xo[i] = xv[p] + dn;
    }
  }
}

// ---------------------------------------------------------------------------
// Cell-centred multigrid for the lumped Schur complement (optional flow-block solver).
// Level 0 is the Gauss-point pressure grid with the 16-coefficient stencil above.
// Level 1 aggregates the 2^d points of each cell (piecewise-constant prolongation,
// restriction = its transpose); further levels aggregate 2^d cells.  Coarse operators
// are Galerkin products R S P: on the cell grids they are (2d+1)-point stencils stored
// as [diag | lower_0 | upper_0 | lower_1 | ...] per instance (the K-dependent part; the
// mass part cm[k] * mp * 2^(d l) is added per column).
template <typename T, int DIM>
__global__ void k_pmg_resid0(Grid g, const T* __restrict__ coef, RhsCoef cm, T mp, const T* __restrict__ b,
                             const T* __restrict__ x, T* __restrict__ r_out, int ncols) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  const int r = blockIdx.y;
  const int64_t np = g.Np;
  const T* cf = coef + (int64_t)(r % g.nb) * 16 * np;
  const T acc = schur_stencil_eval<T, DIM>(g, cf, T(cm.c[r / g.nb]) * mp, x + r * np, t);
  r_out[r * np + t] = b[r * np + t] - acc;
}

// level-1 stencil of every cell from the level-0 point stencil (one instance per grid y)
template <typename T, int DIM>
__global__ void k_pmg_build1(Grid g, const T* __restrict__ coef, T* __restrict__ st) {
  const int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cid >= g.ncells) return;
  const int b = blockIdx.y;
  const int64_t np = g.Np, nc = g.ncells;
  const T* cf = coef + (int64_t)b * 16 * np;
  T* so = st + (int64_t)b * (1 + 2 * DIM) * nc;
  const int cx = (int)(cid % g.n[0]);
  const int64_t rr = cid / g.n[0];
  const int cy = (int)(rr % g.n[1]), cz = DIM == 3 ? (int)(rr / g.n[1]) : 0;
  T diag = 0, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int q = 0; q < (1 << DIM); ++q) {
    const int px = 2 * cx + (q & 1), py = 2 * cy + ((q >> 1) & 1), pz = DIM == 3 ? 2 * cz + ((q >> 2) & 1) : 0;
    const int64_t t = ((int64_t)pz * g.ng[1] + py) * g.ng[0] + px;
    diag += cf[t];
    for (int c = 0; c < DIM; ++c) {
      diag += cf[(1 + c) * np + t];  // partner point of the same cell
      lo[c] += cf[(1 + DIM + 4 * c) * np + t] + cf[(1 + DIM + 4 * c + 1) * np + t];
      hi[c] += cf[(1 + DIM + 4 * c + 2) * np + t] + cf[(1 + DIM + 4 * c + 3) * np + t];
    }
  }
  so[cid] = diag;
  for (int c = 0; c < DIM; ++c) {
    so[(1 + 2 * c) * nc + cid] = lo[c];
    so[(2 + 2 * c) * nc + cid] = hi[c];
  }
}

// Galerkin stencil of level l+1 (cells cn) from level l (cells fn): aggregate 2^d children
template <typename T, int DIM>
__global__ void k_pmg_coarsen(PDims fd, PDims cd, const T* __restrict__ stf, T* __restrict__ stc) {
  const int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cid >= cd.nc) return;
  const int b = blockIdx.y;
  const T* sf = stf + (int64_t)b * (1 + 2 * DIM) * fd.nc;
  T* sc = stc + (int64_t)b * (1 + 2 * DIM) * cd.nc;
  const int cx = (int)(cid % cd.n[0]);
  const int64_t rr = cid / cd.n[0];
  const int cy = (int)(rr % cd.n[1]), cz = DIM == 3 ? (int)(rr / cd.n[1]) : 0;
  T diag = 0, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int q = 0; q < (1 << DIM); ++q) {
    const int f[3] = {2 * cx + (q & 1), 2 * cy + ((q >> 1) & 1), DIM == 3 ? 2 * cz + ((q >> 2) & 1) : 0};
    const int64_t fid = ((int64_t)f[2] * fd.n[1] + f[1]) * fd.n[0] + f[0];
    diag += sf[fid];
    for (int c = 0; c < DIM; ++c) {
      const T l = sf[(1 + 2 * c) * fd.nc + fid], h = sf[(2 + 2 * c) * fd.nc + fid];
      // a child's lower face is inside the parent when it is the upper child along c
      if ((f[c] & 1) == 1) diag += l; else lo[c] += l;
      if ((f[c] & 1) == 0) diag += h; else hi[c] += h;
    }
  }
  sc[cid] = diag;
  for (int c = 0; c < DIM; ++c) {
    sc[(1 + 2 * c) * cd.nc + cid] = lo[c];
    sc[(2 + 2 * c) * cd.nc + cid] = hi[c];
  }
}

// (2d+1)-point stencil apply at cell cid of one column (mass m added to the diagonal)
template <typename T, int DIM>
__device__ __forceinline__ T pmg_eval(const PDims& pd, const T* __restrict__ st, T m, const T* __restrict__ x, int64_t cid,
                                      T& diag) {
  const int cx = (int)(cid % pd.n[0]);
  const int64_t rr = cid / pd.n[0];
  const int c3[3] = {cx, (int)(rr % pd.n[1]), DIM == 3 ? (int)(rr / pd.n[1]) : 0};
  const int64_t str[3] = {1, pd.n[0], (int64_t)pd.n[0] * pd.n[1]};
  diag = st[cid] + m;
  T acc = diag * x[cid];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    if (c3[c] > 0) acc += st[(1 + 2 * c) * pd.nc + cid] * x[cid - str[c]];
    if (c3[c] + 1 < pd.n[c]) acc += st[(2 + 2 * c) * pd.nc + cid] * x[cid + str[c]];
  }
  return acc;
}

// Chebyshev-Jacobi step on a cell level (first: from x = 0) or its residual (resid = 1:
// xo = b - A x); columns on grid y, instance = column % nb
template <typename T, int DIM>
__global__ void k_pmg_step(PDims pd, const T* __restrict__ st, RhsCoef cm, T ml, int nb, T c1, T c2, int mode,
                           const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ d, T* __restrict__ xo) {
  const int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cid >= pd.nc) return;
  const int r = blockIdx.y;
  const int64_t i = r * pd.nc + cid;
  const T* s = st + (int64_t)(r % nb) * (1 + 2 * DIM) * pd.nc;
  const T m = T(cm.c[r / nb]) * ml;
  if (mode == 1) {  // first Chebyshev step from zero
    const T di = T(1) / (s[cid] + m);
    const T dn = c2 * di * b[i];
    d[i] = dn;
    xo[i] = dn;
    return;
  }
  T diag;
  const T ax = pmg_eval<T, DIM>(pd, s, m, x + r * pd.nc, cid, diag);
  if (mode == 2) {  // residual
    xo[i] = b[i] - ax;
    return;
  }
  T dn = c2 * (b[i] - ax) / diag;
  if (c1 != T(0)) dn += c1 * d[i];
  d[i] = dn;
  xo[i] = x[i] + dn;
}

// restriction (sum over the 2^d children: points of a cell at level 0 -> 1, or cells)
template <typename T, int DIM>
__global__ void k_pmg_restrict(PDims fd, PDims cd, const T* __restrict__ rf, T* __restrict__ rc) {
  const int64_t cid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cid >= cd.nc) return;
  const int r = blockIdx.y;
  const int cx = (int)(cid % cd.n[0]);
  const int64_t rr = cid / cd.n[0];
  const int cy = (int)(rr % cd.n[1]), cz = DIM == 3 ? (int)(rr / cd.n[1]) : 0;
  const T* src = rf + r * fd.nc;
  T s = 0;
  for (int q = 0; q < (1 << DIM); ++q) {
    const int64_t f = ((int64_t)(DIM == 3 ? 2 * cz + ((q >> 2) & 1) : 0) * fd.n[1] + 2 * cy + ((q >> 1) & 1)) * fd.n[0] + 2 * cx +
                      (q & 1);
    s += src[f];
  }
  rc[r * cd.nc + cid] = s;
}

// prolongation: x_f += alpha * x_c(parent), piecewise constant
template <typename T, int DIM>
__global__ void k_pmg_prolong(PDims fd, PDims cd, const T* __restrict__ xc, T* __restrict__ xf, T alpha) {
  const int64_t fid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (fid >= fd.nc) return;
  const int r = blockIdx.y;
  const int fx = (int)(fid % fd.n[0]);
  const int64_t rr = fid / fd.n[0];
  const int fy = (int)(rr % fd.n[1]), fz = DIM == 3 ? (int)(rr / fd.n[1]) : 0;
  const int64_t p = ((int64_t)(fz >> 1) * cd.n[1] + (fy >> 1)) * cd.n[0] + (fx >> 1);
  xf[r * fd.nc + fid] += alpha * xc[r * cd.nc + p];
}

template <typename T>
void launch_schur_stencil(const Grid& g, const TabT<T>& tb, const T* dmq, double tau, T* coef, cudaStream_t st) {
  int blocks = (int)((g.Np + 255) / 256);
  if (g.dim == 3) (note_launch(), k_schur_stencil<T, 3><<<blocks, 256, 0, st>>>(g, tb, dmq, tau, coef));
  else (note_launch(), k_schur_stencil<T, 2><<<blocks, 256, 0, st>>>(g, tb, dmq, tau, coef));
}
template <typename T>
void launch_schur_cheb_st(const Grid& g, const TabT<T>& tb, const T* coef, const T* dinv, const double* cm, double c1, double c2,
                          int first, const T* b, const T* x, T* d, T* xo, int nrhs, cudaStream_t st) {
  RhsCoef rc;
  const int nlev = (nrhs + g.nb - 1) / g.nb;  // nrhs counts columns (level x instance)
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nlev) ? cm[r] : 0.0;
  double mp = 1.0;
  for (int k = 0; k < g.dim; ++k) mp *= (double)tb.wg[k];
  dim3 grid((unsigned)((g.Np + 255) / 256), nrhs);
  if (sizeof(T) == 4) prof_begin(st, 2, (double)g.Np * nrhs);
  if (g.dim == 3) (note_launch(), k_schur_cheb_st<T, 3><<<grid, 256, 0, st>>>(g, coef, dinv, rc, T(mp), T(c1), T(c2), first, b, x, d, xo));
  else (note_launch(), k_schur_cheb_st<T, 2><<<grid, 256, 0, st>>>(g, coef, dinv, rc, T(mp), T(c1), T(c2), first, b, x, d, xo));
  if (sizeof(T) == 4) prof_end(st, 2);
}
template <typename T>
void launch_schur_wq(const Grid& g, const TabT<T>& tb, const T* dmq, double tau, T* wq, cudaStream_t st) {
  const int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  const int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) (note_launch(), k_schur_wq<T, 3><<<blocks, 256, 0, st>>>(g, tb, dmq, tau, wq));
  else (note_launch(), k_schur_wq<T, 2><<<blocks, 256, 0, st>>>(g, tb, dmq, tau, wq));
}
template <typename T>
void launch_schur_cheb_mf(const Grid& g, const TabT<T>& tb, const T* wq, const double* cm, double c1, double c2, int first,
                          const T* b, const T* x, T* d, T* xo, int nk, cudaStream_t st) {
  RhsCoef rc;
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nk) ? cm[r] : 0.0;
  double mp = 1.0;
  for (int k = 0; k < g.dim; ++k) mp *= (double)tb.wg[k];
  dim3 grid((unsigned)((g.ncells + 255) / 256), g.nb);
  if (sizeof(T) == 4) prof_begin(st, 2, (double)g.Np * nk * g.nb);
  if (g.dim == 3)
    (note_launch(), k_schur_cheb_mf<T, 3><<<grid, 256, 0, st>>>(g, tb, wq, rc, T(mp), T(c1), T(c2), first, nk, b, x, d, xo));
  else
    (note_launch(), k_schur_cheb_mf<T, 2><<<grid, 256, 0, st>>>(g, tb, wq, rc, T(mp), T(c1), T(c2), first, nk, b, x, d, xo));
  if (sizeof(T) == 4) prof_end(st, 2);
}
PDims pdims_points(const Grid& g) {
  PDims p;
  for (int d = 0; d < 3; ++d) p.n[d] = g.ng[d];
  p.nc = g.Np;
  return p;
}

template <typename T>
void launch_pmg_resid0(const Grid& g, const T* coef, const double* cm, const T* b, const T* x, T* r, int ncols, cudaStream_t st) {
  RhsCoef rc;
  const int nlev = (ncols + g.nb - 1) / g.nb;
  for (int k = 0; k < MAXR; ++k) rc.c[k] = (k < nlev) ? cm[k] : 0.0;
  double mp = 1.0;
  for (int d = 0; d < g.dim; ++d) mp *= 0.5 * g.h[d];
  dim3 grid((unsigned)((g.Np + 255) / 256), ncols);
  if (g.dim == 3) (note_launch(), k_pmg_resid0<T, 3><<<grid, 256, 0, st>>>(g, coef, rc, T(mp), b, x, r, ncols));
  else (note_launch(), k_pmg_resid0<T, 2><<<grid, 256, 0, st>>>(g, coef, rc, T(mp), b, x, r, ncols));
}
template <typename T>
void launch_pmg_build1(const Grid& g, const T* coef, T* st1, cudaStream_t st) {
  dim3 grid((unsigned)((g.ncells + 255) / 256), g.nb);
  if (g.dim == 3) (note_launch(), k_pmg_build1<T, 3><<<grid, 256, 0, st>>>(g, coef, st1));
  else (note_launch(), k_pmg_build1<T, 2><<<grid, 256, 0, st>>>(g, coef, st1));
}
template <typename T>
void launch_pmg_coarsen(int dim, const PDims& fd, const PDims& cd, int nb, const T* stf, T* stc, cudaStream_t st) {
  dim3 grid((unsigned)((cd.nc + 255) / 256), nb);
  if (dim == 3) (note_launch(), k_pmg_coarsen<T, 3><<<grid, 256, 0, st>>>(fd, cd, stf, stc));
  else (note_launch(), k_pmg_coarsen<T, 2><<<grid, 256, 0, st>>>(fd, cd, stf, stc));
}
template <typename T>
void launch_pmg_step(int dim, const PDims& pd, const T* stl, const double* cm, double ml, int nb, double c1, double c2, int mode,
                     const T* b, const T* x, T* d, T* xo, int ncols, cudaStream_t st) {
  RhsCoef rc;
  const int nlev = (ncols + nb - 1) / nb;
  for (int k = 0; k < MAXR; ++k) rc.c[k] = (k < nlev) ? cm[k] : 0.0;
  dim3 grid((unsigned)((pd.nc + 255) / 256), ncols);
  if (dim == 3) (note_launch(), k_pmg_step<T, 3><<<grid, 256, 0, st>>>(pd, stl, rc, T(ml), nb, T(c1), T(c2), mode, b, x, d, xo));
  else (note_launch(), k_pmg_step<T, 2><<<grid, 256, 0, st>>>(pd, stl, rc, T(ml), nb, T(c1), T(c2), mode, b, x, d, xo));
}
template <typename T>
void launch_pmg_restrict(int dim, const PDims& fd, const PDims& cd, const T* rf, T* rc, int ncols, cudaStream_t st) {
  dim3 grid((unsigned)((cd.nc + 255) / 256), ncols);
  if (dim == 3) (note_launch(), k_pmg_restrict<T, 3><<<grid, 256, 0, st>>>(fd, cd, rf, rc));
  else (note_launch(), k_pmg_restrict<T, 2><<<grid, 256, 0, st>>>(fd, cd, rf, rc));
}
template <typename T>
void launch_pmg_prolong(int dim, const PDims& fd, const PDims& cd, const T* xc, T* xf, double alpha, int ncols, cudaStream_t st) {
  dim3 grid((unsigned)((fd.nc + 255) / 256), ncols);
  if (dim == 3) (note_launch(), k_pmg_prolong<T, 3><<<grid, 256, 0, st>>>(fd, cd, xc, xf, T(alpha)));
  else (note_launch(), k_pmg_prolong<T, 2><<<grid, 256, 0, st>>>(fd, cd, xc, xf, T(alpha)));
}

#define INSTMG(T)                                                                                                   \
  template void launch_prolong_add<T>(const Grid&, const Grid&, const T*, int64_t, T*, int64_t, int, cudaStream_t); \
  template void launch_restrict<T>(const Grid&, const Grid&, const T*, int64_t, T*, int64_t, int, cudaStream_t);    \
  template void launch_cheb_update<T>(const T*, const T*, const T*, T*, const T*, T*, double, double, int, int64_t, int, \
                                      int64_t, cudaStream_t);                                                       \
  template void launch_dense_gemv<T>(const double*, int, const T*, int64_t, T*, int64_t, int, double, cudaStream_t);  \
  template void launch_diag_Mq<T>(const Grid&, const TabT<T>&, const T*, T*, cudaStream_t);                        \
  template void launch_diag_BDBt<T>(const Grid&, const TabT<T>&, const T*, T*, cudaStream_t);                      \
  template void launch_q_jacobi<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, double, T*, int64_t, int, \
                                   cudaStream_t);                                                                   \
  template void launch_p_minus_Bq<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, double, T*,   \
                                     int64_t, int, cudaStream_t);                                                   \
  template void launch_schur_apply<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, T*, int64_t, double,  \
                                      const double*, T*, int64_t, int, cudaStream_t);                               \
  template void launch_q_final<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, const T*, double, \
                                  double, T*, int64_t, int, cudaStream_t);                                          \
  template void launch_p_plus_ETu<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, double, T*,  \
                                     int64_t, int, cudaStream_t);                                                   \
  template void launch_mask<T>(const Grid&, T*, int64_t, int, cudaStream_t);                                        \
  template void launch_mask_u<T>(const Grid&, T*, int64_t, int, cudaStream_t);                                      \
  template void launch_schur_stencil<T>(const Grid&, const TabT<T>&, const T*, double, T*, cudaStream_t);          \
  template void launch_schur_cheb_st<T>(const Grid&, const TabT<T>&, const T*, const T*, const double*, double, double, \
                                        int, const T*, const T*, T*, T*, int, cudaStream_t);                        \
  template void launch_schur_wq<T>(const Grid&, const TabT<T>&, const T*, double, T*, cudaStream_t);                \
  template void launch_schur_cheb_mf<T>(const Grid&, const TabT<T>&, const T*, const double*, double, double, int,   \
                                        const T*, const T*, T*, T*, int, cudaStream_t);                              \
  template void launch_mq_line_solve<T>(const Grid&, const TabT<T>&, const T*, const T*, int64_t, T*, int64_t, double, int, \
                                        cudaStream_t);                                                              \
  template void launch_BTp<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, T*, int64_t, double, \
                              int, cudaStream_t);                                                                   \
  template void launch_q_fix_constrained<T>(const Grid&, const T*, int64_t, T*, int64_t, int, cudaStream_t);        \
  template void launch_schur_out<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, double,       \
                                    const double*, T*, int64_t, int, cudaStream_t);                                 \
  template void launch_schur_dinv<T>(const Grid&, const TabT<T>&, const T*, const double*, double, T*, int, cudaStream_t); \
  template void launch_cheb_update_r<T>(const T*, const T*, const T*, T*, const T*, T*, double, double, int, int64_t, int, \
                                        cudaStream_t);                                                              \
  template void launch_u_rhs<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, double, T*, int64_t, \
                                int, cudaStream_t);                                                                 \
  template void launch_pmg_resid0<T>(const Grid&, const T*, const double*, const T*, const T*, T*, int, cudaStream_t); \
  template void launch_pmg_build1<T>(const Grid&, const T*, T*, cudaStream_t);                                     \
  template void launch_pmg_coarsen<T>(int, const PDims&, const PDims&, int, const T*, T*, cudaStream_t);           \
  template void launch_pmg_step<T>(int, const PDims&, const T*, const double*, double, int, double, double, int,     \
                                   const T*, const T*, T*, T*, int, cudaStream_t);                                  \
  template void launch_pmg_restrict<T>(int, const PDims&, const PDims&, const T*, T*, int, cudaStream_t);          \
  template void launch_pmg_prolong<T>(int, const PDims&, const PDims&, const T*, T*, double, int, cudaStream_t);
INSTMG(double)
INSTMG(float)

}  // namespace biot
