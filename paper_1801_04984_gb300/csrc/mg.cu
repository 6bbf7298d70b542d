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
#include "internal.h"

namespace biot {

// ---------------------------------------------------------------------------
// Q2 -> Q2 embedding prolongation (coarse cell 2h -> two fine cells h):
// fine node 2c = coarse node c; fine nodes at 1/4 and 3/4 of a coarse cell take
// the coarse Q2 interpolant there: (3/8, 3/4, -1/8) and (-1/8, 3/4, 3/8).
__device__ inline int prolong_taps(int f, int* ci, double* w) {
  if ((f & 1) == 0) { ci[0] = f >> 1; w[0] = 1.0; return 1; }
  int m = f >> 2;
  if ((f & 3) == 1) { ci[0] = 2 * m; ci[1] = 2 * m + 1; ci[2] = 2 * m + 2; w[0] = 0.375; w[1] = 0.75; w[2] = -0.125; }
  else { ci[0] = 2 * m; ci[1] = 2 * m + 1; ci[2] = 2 * m + 2; w[0] = -0.125; w[1] = 0.75; w[2] = 0.375; }
  return 3;
}

// restriction = transpose of prolongation
__device__ inline int restrict_taps(int c, int nf, int* fi, double* w) {
  int k = 0;
  if (c & 1) {
    int m = c >> 1;
    fi[k] = 4 * m + 1; w[k++] = 0.75;
    fi[k] = 4 * m + 2; w[k++] = 1.0;
    fi[k] = 4 * m + 3; w[k++] = 0.75;
  } else {
    int m = c >> 1;
    const int off[5] = {-3, -1, 0, 1, 3};
    const double ww[5] = {-0.125, 0.375, 1.0, 0.375, -0.125};
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
  int f[3];
  f[0] = (int)(t % gf.nu[0]);
  int64_t rr = t / gf.nu[0];
  f[1] = (int)(rr % gf.nu[1]);
  f[2] = (int)(rr / gf.nu[1]);
  int ci[3][3], cnt[3];
  double w[3][3];
  for (int d = 0; d < 3; ++d) {
    if (d < gf.dim) cnt[d] = prolong_taps(f[d], ci[d], w[d]);
    else { cnt[d] = 1; ci[d][0] = 0; w[d][0] = 1.0; }
  }
  for (int r = 0; r < nrhs; ++r)
    for (int c = 0; c < gf.dim; ++c) {
      if (!u_free(gf, c, f[0], f[1], f[2])) continue;
      const T* src = xc + r * sc + c * gc.nnode;
      double acc = 0;
      for (int a = 0; a < cnt[2]; ++a)
        for (int b = 0; b < cnt[1]; ++b)
          for (int e = 0; e < cnt[0]; ++e) {
            if (!u_free(gc, c, ci[0][e], ci[1][b], ci[2][a])) continue;
            acc += w[2][a] * w[1][b] * w[0][e] * (double)src[((int64_t)ci[2][a] * gc.nu[1] + ci[1][b]) * gc.nu[0] + ci[0][e]];
          }
      T* dst = xf + r * sf + c * gf.nnode + t;
      *dst = (T)((double)*dst + acc);
    }
}

template <typename T>
__global__ void k_restrict(Grid gf, Grid gc, const T* __restrict__ rf, int64_t sf, T* __restrict__ rc, int64_t sc, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= gc.nnode) return;
  int cidx[3];
  cidx[0] = (int)(t % gc.nu[0]);
  int64_t rr = t / gc.nu[0];
  cidx[1] = (int)(rr % gc.nu[1]);
  cidx[2] = (int)(rr / gc.nu[1]);
  int fi[3][5], cnt[3];
  double w[3][5];
  for (int d = 0; d < 3; ++d) {
    if (d < gf.dim) cnt[d] = restrict_taps(cidx[d], gf.nu[d], fi[d], w[d]);
    else { cnt[d] = 1; fi[d][0] = 0; w[d][0] = 1.0; }
  }
  for (int r = 0; r < nrhs; ++r)
    for (int c = 0; c < gf.dim; ++c) {
      double acc = 0;
      if (u_free(gc, c, cidx[0], cidx[1], cidx[2])) {
        const T* src = rf + r * sf + c * gf.nnode;
        for (int a = 0; a < cnt[2]; ++a)
          for (int b = 0; b < cnt[1]; ++b)
            for (int e = 0; e < cnt[0]; ++e) {
              if (!u_free(gf, c, fi[0][e], fi[1][b], fi[2][a])) continue;
              acc += w[2][a] * w[1][b] * w[0][e] * (double)src[((int64_t)fi[2][a] * gf.nu[1] + fi[1][b]) * gf.nu[0] + fi[0][e]];
            }
      }
      rc[r * sc + c * gc.nnode + t] = (T)acc;
    }
}

template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, int64_t sc, T* xf, int64_t sf, int nrhs,
                        cudaStream_t st) {
  k_prolong_add<T><<<(int)((fine.nnode + 255) / 256), 256, 0, st>>>(fine, coarse, xc, sc, xf, sf, nrhs);
}
template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* rf, int64_t sf, T* rc, int64_t sc, int nrhs,
                     cudaStream_t st) {
  k_restrict<T><<<(int)((coarse.nnode + 255) / 256), 256, 0, st>>>(fine, coarse, rf, sf, rc, sc, nrhs);
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
  k_cheb_update<T><<<blocks, 256, 0, st>>>(b, Ax, dinv, d, x, xo, (T)c1, (T)c2, first, n, nrhs, stride);
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
  k_dense_gemv<T><<<grid, 256, 0, st>>>(Ainv, n, b, sb, x, sx, s);
}

// ---------------------------------------------------------------------------
// flux / pressure gathers
struct QIdx {  // decoded flux DoF
  int c, ia;
  int co[3];
  int64_t r, stride_c, pbase;
  double wt;
  int ncell, ce[2], la[2];
};

template <int DIM>
__device__ inline bool decode_q(const Grid& g, const double* wg, int64_t t, QIdx& q) {
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (t >= nqt) return false;
  int c = 0;
  int64_t r = t;
  while (r >= g.nq[c]) { r -= g.nq[c]; ++c; }
  int sh[3];
  for (int d = 0; d < 3; ++d) sh[d] = (d < DIM) ? ((d == c) ? g.nu[d] : g.ng[d]) : 1;
  q.co[0] = (int)(r % sh[0]);
  int64_t rr = r / sh[0];
  q.co[1] = (int)(rr % sh[1]);
  q.co[2] = (int)(rr / sh[1]);
  q.c = c;
  q.r = r;
  q.ia = q.co[c];
  q.stride_c = 1;
  for (int d = 0; d < c; ++d) q.stride_c *= sh[d];
  q.wt = 1.0;
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
__device__ inline double gather_BTp(const Grid& g, const TabT<T>& tb, const QIdx& q, const T* p) {
  int64_t pst[3] = {1, g.ng[0], (int64_t)g.ng[0] * g.ng[1]};
  double bp = 0;
  for (int e = 0; e < q.ncell; ++e)
    for (int k = 0; k < 2; ++k) bp += (double)tb.bd[q.c][q.la[e]][k] * (double)p[q.pbase + (int64_t)(2 * q.ce[e] + k) * pst[q.c]];
  return q.wt * bp;
}

// (B q) at a pressure DoF t, flux input masked
template <typename T, int DIM>
__device__ inline double gather_Bq(const Grid& g, const TabT<T>& tb, int64_t t, const T* q, const T* dscale) {
  int co[3];
  co[0] = (int)(t % g.ng[0]);
  int64_t rr = t / g.ng[0];
  co[1] = (int)(rr % g.ng[1]);
  co[2] = (int)(rr / g.ng[1]);
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
    const int64_t off = g.offq[c] - g.Nu + base;  // q arrays here are indexed from the start of the flux block
    int cell = co[c] >> 1, gq = co[c] & 1;
    double s = 0;
    for (int a = 0; a < 3; ++a) {
      int ia = 2 * cell + a;
      if (!q_free(g, c, ia)) continue;
      int64_t i = off + (int64_t)ia * stride_c;
      double v = (double)q[i];
      if (dscale) v *= (double)dscale[i];
      s += (double)tb.bd[c][a][gq] * v;
    }
    acc += wt * s;
  }
  return acc;
}

// diag of Mq (unit tau) per flux DoF (1 on constrained DoFs)
template <typename T, int DIM>
__global__ void k_diag_Mq(Grid g, TabT<T> tb, const T* __restrict__ kscale, T* __restrict__ dmq) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx q;
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
  co[0] = (int)(t % g.ng[0]);
  int64_t rr = t / g.ng[0];
  co[1] = (int)(rr % g.ng[1]);
  co[2] = (int)(rr / g.ng[1]);
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
  QIdx q;
  double wg[3] = {(double)tb.wg[0], (double)tb.wg[1], (double)tb.wg[2]};
  if (!decode_q<DIM>(g, wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  for (int r = 0; r < nrhs; ++r) {
    T v = rq[r * srq + t];
    q0[r * sq + t] = fr ? (T)((double)v / (tau * (double)dmq[t])) : v;
  }
}

// out_p = rp - tau B q
template <typename T, int DIM>
__global__ void k_p_minus_Bq(Grid g, TabT<T> tb, const T* __restrict__ rp, int64_t srp, const T* __restrict__ q, int64_t sq,
                             double tau, T* __restrict__ out, int64_t so, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  for (int r = 0; r < nrhs; ++r)
    out[r * so + t] = (T)((double)rp[r * srp + t] - tau * gather_Bq<T, DIM>(g, tb, t, q + r * sq, nullptr));
}

// tq = (B^T p) / dmq on free flux DoFs, 0 on constrained
template <typename T, int DIM>
__global__ void k_BTp_scaled(Grid g, TabT<T> tb, const T* __restrict__ p, int64_t spp, const T* __restrict__ dmq, T* __restrict__ tq,
                             int64_t sq, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx q;
  double wg[3] = {(double)tb.wg[0], (double)tb.wg[1], (double)tb.wg[2]};
  if (!decode_q<DIM>(g, wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  for (int r = 0; r < nrhs; ++r) tq[r * sq + t] = fr ? (T)(gather_BTp<T>(g, tb, q, p + r * spp) / (double)dmq[t]) : T(0);
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
  double mp = 1.0;
  for (int d = 0; d < DIM; ++d) mp *= (double)tb.wg[d];
  for (int r = 0; r < nrhs; ++r)
    out[r * so + t] = (T)(cm.c[r] * mp * (double)p[r * spp + t] + tau * gather_Bq<T, DIM>(g, tb, t, tq + r * sq, nullptr));
}

// q = (Rq + bt B^T p) / (tau dmq) on free flux DoFs, Rq on constrained
template <typename T, int DIM>
__global__ void k_q_final(Grid g, TabT<T> tb, const T* __restrict__ rq, int64_t srq, const T* __restrict__ p, int64_t spp,
                          const T* __restrict__ dmq, double tau, double bt, T* __restrict__ qo, int64_t sq, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  QIdx q;
  double wg[3] = {(double)tb.wg[0], (double)tb.wg[1], (double)tb.wg[2]};
  if (!decode_q<DIM>(g, wg, t, q)) return;
  bool fr = q_free(g, q.c, q.ia);
  for (int r = 0; r < nrhs; ++r) {
    double v = (double)rq[r * srq + t];
    if (fr) v = (v + bt * gather_BTp<T>(g, tb, q, p + r * spp)) / (tau * (double)dmq[t]);
    qo[r * sq + t] = (T)v;
  }
}

// bu = ru + alpha * E p on free displacement DoFs, ru on constrained
template <typename T, int DIM>
__global__ void k_u_rhs(Grid g, TabT<T> tb, const T* __restrict__ ru, int64_t sru, const T* __restrict__ p, int64_t spp,
                        double alpha, T* __restrict__ bu, int64_t sbu, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.nnode) return;
  int ix = (int)(t % g.nu[0]);
  int64_t rr = t / g.nu[0];
  int iy = (int)(rr % g.nu[1]);
  int iz = (int)(rr / g.nu[1]);
  int idx[3] = {ix, iy, iz};
  for (int c = 0; c < DIM; ++c) {
    bool fr = u_free(g, c, ix, iy, iz);
    // taps of E along each direction
    int pi[3][4], cnt[3];
    double pc[3][4];
    for (int d = 0; d < 3; ++d) {
      int k = 0;
      if (d < DIM) {
        int m = idx[d];
        const T(*tab)[2] = (d == c) ? tb.bd[d] : tb.bv[d];
        if (m & 1) { for (int q = 0; q < 2; ++q) { pi[d][k] = m - 1 + q; pc[d][k] = (double)tab[1][q]; ++k; } }
        else {
          int j = m >> 1;
          if (j >= 1) for (int q = 0; q < 2; ++q) { pi[d][k] = 2 * (j - 1) + q; pc[d][k] = (double)tab[2][q]; ++k; }
          if (j < g.n[d]) for (int q = 0; q < 2; ++q) { pi[d][k] = 2 * j + q; pc[d][k] = (double)tab[0][q]; ++k; }
        }
      } else { pi[d][0] = 0; pc[d][0] = 1.0; k = 1; }
      cnt[d] = k;
    }
    for (int r = 0; r < nrhs; ++r) {
      double v = (double)ru[r * sru + c * g.nnode + t];
      if (fr) {
        const T* pr = p + r * spp;
        double acc = 0;
        for (int a = 0; a < cnt[2]; ++a)
          for (int b = 0; b < cnt[1]; ++b)
            for (int e = 0; e < cnt[0]; ++e)
              acc += pc[2][a] * pc[1][b] * pc[0][e] * (double)pr[((int64_t)pi[2][a] * g.ng[1] + pi[1][b]) * g.ng[0] + pi[0][e]];
        v += alpha * acc;
      }
      bu[r * sbu + c * g.nnode + t] = (T)v;
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T>
void launch_diag_Mq(const Grid& g, const TabT<T>& tb, const T* kscale, T* dmq, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) k_diag_Mq<T, 3><<<blocks, 256, 0, st>>>(g, tb, kscale, dmq);
  else k_diag_Mq<T, 2><<<blocks, 256, 0, st>>>(g, tb, kscale, dmq);
}
template <typename T>
void launch_diag_BDBt(const Grid& g, const TabT<T>& tb, const T* dmq, T* out, cudaStream_t st) {
  int blocks = (int)((g.Np + 255) / 256);
  if (g.dim == 3) k_diag_BDBt<T, 3><<<blocks, 256, 0, st>>>(g, tb, dmq, out);
  else k_diag_BDBt<T, 2><<<blocks, 256, 0, st>>>(g, tb, dmq, out);
}
template <typename T>
void launch_q_jacobi(const Grid& g, const TabT<T>& tb, const T* rq, int64_t srq, const T* dmq, double tau, T* q0, int64_t sq,
                     int nrhs, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) k_q_jacobi<T, 3><<<blocks, 256, 0, st>>>(g, rq, srq, dmq, tau, q0, sq, nrhs, tb);
  else k_q_jacobi<T, 2><<<blocks, 256, 0, st>>>(g, rq, srq, dmq, tau, q0, sq, nrhs, tb);
}
template <typename T>
void launch_p_minus_Bq(const Grid& g, const TabT<T>& tb, const T* rp, int64_t srp, const T* q, int64_t sq, double tau, T* out,
                       int64_t so, int nrhs, cudaStream_t st) {
  int blocks = (int)((g.Np + 255) / 256);
  if (g.dim == 3) k_p_minus_Bq<T, 3><<<blocks, 256, 0, st>>>(g, tb, rp, srp, q, sq, tau, out, so, nrhs);
  else k_p_minus_Bq<T, 2><<<blocks, 256, 0, st>>>(g, tb, rp, srp, q, sq, tau, out, so, nrhs);
}
template <typename T>
void launch_schur_apply(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* dmq, T* tq, int64_t sq, double tau,
                        const double* cm, T* out, int64_t so, int nrhs, cudaStream_t st) {
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  RhsCoef rc;
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nrhs) ? cm[r] : 0.0;
  if (g.dim == 3) {
    k_BTp_scaled<T, 3><<<(int)((nqt + 255) / 256), 256, 0, st>>>(g, tb, p, spp, dmq, tq, sq, nrhs);
    k_schur_out<T, 3><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(g, tb, p, spp, tq, sq, tau, rc, out, so, nrhs);
  } else {
    k_BTp_scaled<T, 2><<<(int)((nqt + 255) / 256), 256, 0, st>>>(g, tb, p, spp, dmq, tq, sq, nrhs);
    k_schur_out<T, 2><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(g, tb, p, spp, tq, sq, tau, rc, out, so, nrhs);
  }
}
template <typename T>
void launch_q_final(const Grid& g, const TabT<T>& tb, const T* rq, int64_t srq, const T* p, int64_t spp, const T* dmq,
                    double tau, double bt, T* qo, int64_t sq, int nrhs, cudaStream_t st) {
  int64_t n = g.nq[0] + g.nq[1] + g.nq[2];
  int blocks = (int)((n + 255) / 256);
  if (g.dim == 3) k_q_final<T, 3><<<blocks, 256, 0, st>>>(g, tb, rq, srq, p, spp, dmq, tau, bt, qo, sq, nrhs);
  else k_q_final<T, 2><<<blocks, 256, 0, st>>>(g, tb, rq, srq, p, spp, dmq, tau, bt, qo, sq, nrhs);
}
template <typename T>
void launch_u_rhs(const Grid& g, const TabT<T>& tb, const T* ru, int64_t sru, const T* p, int64_t spp, double alpha, T* bu,
                  int64_t sbu, int nrhs, cudaStream_t st) {
  int blocks = (int)((g.nnode + 255) / 256);
  if (g.dim == 3) k_u_rhs<T, 3><<<blocks, 256, 0, st>>>(g, tb, ru, sru, p, spp, alpha, bu, sbu, nrhs);
  else k_u_rhs<T, 2><<<blocks, 256, 0, st>>>(g, tb, ru, sru, p, spp, alpha, bu, sbu, nrhs);
}


// out_p = rp + alpha E^T u at a pressure DoF (u masked)
template <typename T, int DIM>
__global__ void k_p_plus_ETu(Grid g, TabT<T> tb, const T* __restrict__ rp, int64_t srp, const T* __restrict__ u, int64_t su,
                             double alpha, T* __restrict__ out, int64_t so, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= g.Np) return;
  int co[3];
  co[0] = (int)(t % g.ng[0]);
  int64_t rr = t / g.ng[0];
  co[1] = (int)(rr % g.ng[1]);
  co[2] = (int)(rr / g.ng[1]);
  int cell[3], gq[3];
  for (int d = 0; d < 3; ++d) { cell[d] = (d < DIM) ? co[d] >> 1 : 0; gq[d] = (d < DIM) ? (co[d] & 1) : 0; }
  for (int r = 0; r < nrhs; ++r) {
    const T* ur = u + r * su;
    double acc = 0;
    for (int c = 0; c < DIM; ++c) {
      double f[3][3];
      for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a)
          f[d][a] = (d < DIM) ? (double)((d == c) ? tb.bd[d][a][gq[d]] : tb.bv[d][a][gq[d]]) : (a == 0 ? 1.0 : 0.0);
      const int az_n = (DIM == 3) ? 3 : 1;
      for (int az = 0; az < az_n; ++az)
        for (int ay = 0; ay < 3; ++ay) {
          int iz = 2 * cell[2] + az, iy = 2 * cell[1] + ay;
          const T* row = ur + c * g.nnode + ((int64_t)iz * g.nu[1] + iy) * g.nu[0];
          double s = 0;
          for (int ax = 0; ax < 3; ++ax) {
            int ix = 2 * cell[0] + ax;
            if (u_free(g, c, ix, iy, iz)) s += f[0][ax] * (double)row[ix];
          }
          acc += f[2][az] * f[1][ay] * s;
        }
    }
    out[r * so + t] = (T)((double)rp[r * srp + t] + alpha * acc);
  }
}
template <typename T>
void launch_p_plus_ETu(const Grid& g, const TabT<T>& tb, const T* rp, int64_t srp, const T* u, int64_t su, double alpha, T* out,
                       int64_t so, int nrhs, cudaStream_t st) {
  int blocks = (int)((g.Np + 255) / 256);
  if (g.dim == 3) k_p_plus_ETu<T, 3><<<blocks, 256, 0, st>>>(g, tb, rp, srp, u, su, alpha, out, so, nrhs);
  else k_p_plus_ETu<T, 2><<<blocks, 256, 0, st>>>(g, tb, rp, srp, u, su, alpha, out, so, nrhs);
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
  k_mask<T><<<(int)((n + 255) / 256), 256, 0, st>>>(g, x, s, nrhs, 0);
}
template <typename T>
void launch_mask_u(const Grid& g, T* x, int64_t s, int nrhs, cudaStream_t st) {
  k_mask<T><<<(int)((g.nnode + 255) / 256), 256, 0, st>>>(g, x, s, nrhs, 1);
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
  if (g.dim == 3) k_grad_pair<3><<<blocks, 256, 0, st>>>(g, tb, kscale, z, x, w, grad);
  else k_grad_pair<2><<<blocks, 256, 0, st>>>(g, tb, kscale, z, x, w, grad);
}

// slab right-hand side from load terms and the jump term
struct RhsTab {
  double c[MAXR][8];
  double phi0[MAXR];
};
__global__ void k_slab_rhs(Grid g, const double* const* __restrict__ f, int nterms, RhsTab tab, int nt,
                           const double* __restrict__ sp, double* __restrict__ y) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  for (int k = 0; k < nt; ++k) {
    double s = 0;
    for (int m = 0; m < nterms; ++m) s += tab.c[k][m] * f[m][e];
    if (e >= g.offp && sp) s += tab.phi0[k] * sp[e - g.offp];
    y[k * g.N + e] = s;
  }
}
void launch_slab_rhs(const Grid& g, const double* const* f, int nterms, const double* c, const double* phi0, int nt,
                     const double* sp, double* y, cudaStream_t st) {
  RhsTab tab;
  for (int k = 0; k < MAXR; ++k) {
    for (int m = 0; m < 8; ++m) tab.c[k][m] = (k < nt && m < nterms) ? c[k * nterms + m] : 0.0;
    tab.phi0[k] = (k < nt) ? phi0[k] : 0.0;
  }
  k_slab_rhs<<<(int)((g.N + 255) / 256), 256, 0, st>>>(g, f, nterms, tab, nt, sp, y);
}


// inverse Jacobi diagonal of the flux-pressure Schur approximation per rhs:
// dinv[r][i] = 1 / (cm[r] * mp + tau * sb2[i])
template <typename T>
__global__ void k_schur_dinv(const T* __restrict__ sb2, double mp, RhsCoef cm, double tau, T* __restrict__ dinv, int64_t np, int nrhs) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= np) return;
  for (int r = 0; r < nrhs; ++r) dinv[r * np + t] = (T)(1.0 / (cm.c[r] * mp + tau * (double)sb2[t]));
}
template <typename T>
void launch_schur_dinv(const Grid& g, const TabT<T>& tb, const T* sb2, const double* cm, double tau, T* dinv, int nrhs,
                       cudaStream_t st) {
  RhsCoef rc;
  for (int r = 0; r < MAXR; ++r) rc.c[r] = (r < nrhs) ? cm[r] : 0.0;
  double mp = 1.0;
  for (int d = 0; d < g.dim; ++d) mp *= (double)tb.wg[d];
  k_schur_dinv<T><<<(int)((g.Np + 255) / 256), 256, 0, st>>>(sb2, mp, rc, tau, dinv, g.Np, nrhs);
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
  k_cheb_update_r<T><<<blocks, 256, 0, st>>>(b, Ax, dinv, d, x, xo, (T)c1, (T)c2, first, n, nrhs);
}

// x += s * d (mixed precision update)
template <typename TX, typename TD>
__global__ void k_add_scaled(TX* __restrict__ x, const TD* __restrict__ d, double s, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = (TX)((double)x[e] + s * (double)d[e]);
}
template <typename TX, typename TD>
void launch_add_scaled(TX* x, const TD* d, double s, int64_t n, cudaStream_t st) {
  k_add_scaled<TX, TD><<<2 * RED_BLOCKS, 256, 0, st>>>(x, d, s, n);
}
template void launch_add_scaled<double, float>(double*, const float*, double, int64_t, cudaStream_t);
template void launch_add_scaled<double, double>(double*, const double*, double, int64_t, cudaStream_t);

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
  template void launch_schur_dinv<T>(const Grid&, const TabT<T>&, const T*, const double*, double, T*, int, cudaStream_t); \
  template void launch_cheb_update_r<T>(const T*, const T*, const T*, T*, const T*, T*, double, double, int, int64_t, int, \
                                        cudaStream_t);                                                              \
  template void launch_u_rhs<T>(const Grid&, const TabT<T>&, const T*, int64_t, const T*, int64_t, double, T*, int64_t, \
                                int, cudaStream_t);
INSTMG(double)
INSTMG(float)

}  // namespace biot
