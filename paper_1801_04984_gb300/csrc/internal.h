// Internal (not exported) declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#include "common.cuh"
#include "tables.h"

namespace biot {

// ---- tracing (prof.cu) ------------------------------------------------------
// 0 FP32 elasticity (displacement-row) operator (z-marching kernel on 3-D grids of >= 1e5
// nodes, the 2-D kernel), 1 FP64 elasticity operator, 2 FP32 Schur Chebyshev step, 3 FP32 3-D
// elasticity on grids below 1e5 nodes; units = the kernel's work units (node x right-hand side
// for the elasticity operator, pressure point x right-hand side for the Schur step)
constexpr int PROF_KINDS = 4;
void note_launch();
void note_launches(long long k);  // graph replays: add the kernels of the graph
long long launch_count();
void prof_enable(bool on);
bool prof_enabled();
void prof_begin(cudaStream_t st, int kind, double units);
void prof_end(cudaStream_t st, int kind);
void prof_collect(int kind, long long* n, double* ms, double* units);

// ---- slab operator pieces (apply.cu) --------------------------------------
// Optional fused output stage of the elasticity operator (multigrid smoothing and
// residuals; arrays share the output's column layout, dinv is one column shared by all)
enum { EPI_NONE = 0, EPI_CHEB = 1, EPI_RESID = 2 };
template <typename T>
struct UEpi {
  int mode = EPI_NONE;
  const T* b = nullptr;     // right-hand side (CHEB, RESID)
  const T* dinv = nullptr;  // inverse Jacobi diagonal, 0 on constrained rows (CHEB)
  T* d = nullptr;           // Chebyshev direction, updated in place (CHEB)
  T* xo = nullptr;          // new iterate (CHEB; y is not written then)
  T c1 = 0, c2 = 0;
};
template <typename T>
void launch_apply_u(const Grid& g, const TabT<T>& tb, const SlabCoef& sc, const T* u, int64_t su, const T* p, int64_t sp, T* y,
                    int64_t sy, cudaStream_t st, const UEpi<T>* epi = nullptr);
template <typename T>
void launch_apply_q(const Grid& g, const TabT<T>& tb, const SlabCoef& sc, const T* kscale, const T* x, int64_t sx, T* y,
                    int64_t sy, cudaStream_t st);
template <typename T>
void launch_apply_p(const Grid& g, const TabT<T>& tb, const SlabCoef& sc, const T* x, int64_t sx, T* y, int64_t sy,
                    cudaStream_t st);
void apply_init_attributes();
// FP32 3-D elasticity rows, z-marching sum-factorised kernel (elast3.cu), used on grids of at
// least ELAST3_MIN_NODES nodes per component (65^3 and finer)
constexpr int64_t ELAST3_MIN_NODES = 100000;
void elast3_init_attributes();
// measure the launch shape of the z-marching kernel for this grid and column count once (per
// GPU, cached in the tuning file); u and y: scratch of cols * g.Nu floats each
void elast3_tune(const Grid& g, const TabT<float>& tb, double lam, double mu, int cols, float* u, float* y, cudaStream_t st);

// ---- launch-shape autotuner (tune.cu): process table backed by a JSON cache file
bool tune_enabled();
int tune_get(const std::string& key);  // -1 when absent
void tune_put(const std::string& key, int value);
std::string tune_device_tag();
std::string tune_cache_path();
void launch_elast3_f32(const Grid& g, const TabT<float>& tb, const SlabCoef& sc, int cols, const float* u, int64_t su, float* y,
                       int64_t sy, cudaStream_t st, const UEpi<float>* epi);
template <typename T>
void launch_diag_A(const Grid& g, const TabT<T>& tb, double lam, double mu, T* d, cudaStream_t st);

// ---- vector kernels (blas.cu) ---------------------------------------------
// Deterministic reductions: per-block partials in a fixed order, then one
// block sums the partials in a fixed order.  Results land in device memory.
constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs
constexpr int MAXDOT = 64;       // max vectors in one multi-dot

// V: HOST array of nv device pointers, every vector 16-byte aligned (the pointers are passed
// to the kernel by value, so a captured graph keeps them)
template <typename TV>
void launch_multidot(const TV* const* V, int nv, const TV* w, int64_t n, double* partial, double* out, cudaStream_t st);
// w = w - sum_i V_i h_i  (h in device memory, double); optionally the dots
// V_i^T w_new into out (second Gram-Schmidt pass) or ||w_new||^2 into out[nv] when want_norm.
template <typename TV>
void launch_multiaxpy_dot(const TV* const* V, int nv, const double* h, TV* w, int64_t n, int mode, double* partial,
                          double* out, cudaStream_t st);
template <typename TA, typename TB>
void launch_convert(const TA* a, TB* b, int64_t n, cudaStream_t st);
template <typename T>
void launch_axpby(T* y, const T* x, double a, double b, int64_t n, cudaStream_t st);  // y = a x + b y
template <typename T>
void launch_scale_into(T* y, const T* x, const double* s, int inv, int64_t n, cudaStream_t st);  // y = x * s or x / s (s device)
// y += sum_i Z_i c_i  (c device, double; accumulated in double)
template <typename TY, typename TZ>
void launch_lincomb_add(TY* y, const TZ* const* Z, int nz, const double* c, int64_t n, cudaStream_t st);
void launch_residual(const double* b, const double* Ax, double* r, int64_t n, cudaStream_t st);  // r = b - Ax
// Segmented vectors of a batch of independent problems: element e (< len) of level k
// of instance b at k * lstride + b * istride + e.  Every segmented kernel runs on a
// (seg_gx(nb), nb) grid and keeps one result / scalar per instance.
struct Seg {
  int nb, nt;
  int64_t len, istride, lstride;
};
int seg_gx(int nb);
int64_t seg_partial_doubles(int nb);  // size of the partial buffer a segmented reduction needs
template <typename TV>
void launch_seg_multidot(const TV* const* V, int nv, const TV* w, const Seg& sg, double* partial, double* out, int ostride,
                         cudaStream_t st);  // out[b * ostride + i] = V_i^T w over instance b
template <typename TV>
void launch_seg_multiaxpy_dot(const TV* const* V, int nv, const double* h, int hstride, TV* w, const Seg& sg, int mode,
                              double* partial, double* out, int ostride, cudaStream_t st);
template <typename T>
void launch_seg_scale(T* y, const T* x, const double* s, int sstride, const Seg& sg, cudaStream_t st);
template <typename T>
void launch_seg_axpby(T* y, const T* x, const double* a, const double* c, const Seg& sg, cudaStream_t st);
template <typename TY, typename TZ>
void launch_seg_lincomb_add(TY* y, const TZ* const* Z, int nz, const double* c, int cstride, const Seg& sg, cudaStream_t st);
template <typename TX, typename TD>
void launch_seg_add_scaled(TX* x, const TD* d, const double* s, int sstride, const Seg& sg, cudaStream_t st);
// y_r = a x_r + b y_r for rows r < rows of length n at stride s
template <typename T>
void launch_axpby_rows(T* y, const T* x, double a, double b, int64_t n, int rows, int64_t s, cudaStream_t st);
// out[k] = sum_l C[k][l] in[l], k < nout, l < nin (C row-major nout x nin, both <= MAXR)
void launch_time_embed(const double* in, int64_t sin, int nin, double* out, int64_t sout, int nout, const double* C, int64_t n,
                       cudaStream_t st);
// time transform: out[k] = sum_l C[k][l] in[l] over nt levels of length n (strided)
template <typename TI, typename TO>
void launch_time_mix(const TI* in, int64_t sin, TO* out, int64_t sout, int nt, const double* C, int64_t n, cudaStream_t st);

// ---- multigrid / preconditioner pieces (mg.cu) ----------------------------
template <typename T>
void launch_prolong_add(const Grid& fine, const Grid& coarse, const T* xc, int64_t sc, T* xf, int64_t sf, int nrhs,
                        cudaStream_t st);
template <typename T>
void launch_restrict(const Grid& fine, const Grid& coarse, const T* rf, int64_t sf, T* rc, int64_t sc, int nrhs,
                     cudaStream_t st);
// Chebyshev step on nrhs vectors of length n (u block only):
// r = b - Ax ; d = c1 d + c2 Dinv r ; xo = x + d   (first step: d = c2 Dinv b, xo = d)
template <typename T>
void launch_cheb_update(const T* b, const T* Ax, const T* dinv, T* d, const T* x, T* xo, double c1, double c2, int first,
                        int64_t n, int nrhs, int64_t stride, cudaStream_t st);
// x = Ainv * b for nrhs columns (dense FP64 inverse, n x n), scale s
template <typename T>
void launch_dense_gemv(const double* Ainv, int n, const T* b, int64_t sb, T* x, int64_t sx, int nrhs, double s,
                       cudaStream_t st);

// flow-block pieces (mg.cu); flux arrays start at the flux block (offset Nu of a
// temporal level), pressure arrays at the pressure block.
template <typename T>
void launch_diag_Mq(const Grid& g, const TabT<T>& tb, const T* kscale, T* dmq, cudaStream_t st);
template <typename T>
void launch_diag_BDBt(const Grid& g, const TabT<T>& tb, const T* dmq, T* out, cudaStream_t st);
template <typename T>
void launch_q_jacobi(const Grid& g, const TabT<T>& tb, const T* rq, int64_t srq, const T* dmq, double tau, T* q0, int64_t sq,
                     int nrhs, cudaStream_t st);
template <typename T>
void launch_p_minus_Bq(const Grid& g, const TabT<T>& tb, const T* rp, int64_t srp, const T* q, int64_t sq, double tau, T* out,
                       int64_t so, int nrhs, cudaStream_t st);
template <typename T>
void launch_schur_apply(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* dmq, T* tq, int64_t sq, double tau,
                        const double* cm, T* out, int64_t so, int nrhs, cudaStream_t st);
template <typename T>
void launch_q_final(const Grid& g, const TabT<T>& tb, const T* rq, int64_t srq, const T* p, int64_t spp, const T* dmq,
                    double tau, double bt, T* qo, int64_t sq, int nrhs, cudaStream_t st);  // (Rq + bt B^T p)/(tau dmq)
template <typename T>
void launch_u_rhs(const Grid& g, const TabT<T>& tb, const T* ru, int64_t sru, const T* p, int64_t spp, double alpha, T* bu,
                  int64_t sbu, int nrhs, cudaStream_t st);
// out_p = rp + alpha E^T u (u masked)
template <typename T>
void launch_p_plus_ETu(const Grid& g, const TabT<T>& tb, const T* rp, int64_t srp, const T* u, int64_t su, double alpha, T* out,
                       int64_t so, int nrhs, cudaStream_t st);
// zero the constrained entries of nrhs spatial vectors (stride s)
template <typename T>
void launch_mask(const Grid& g, T* x, int64_t s, int nrhs, cudaStream_t st);
// displacement block only (buffers of nrhs * Nu)
template <typename T>
void launch_mask_u(const Grid& g, T* x, int64_t s, int nrhs, cudaStream_t st);
// per-cell flux-mass pairing: g[c] += w * kscale[c] * z_c^T Mq_ref x_c (both masked)
void launch_grad_pair(const Grid& g, const TabT<double>& tb, const double* kscale, const double* z, const double* x, double w,
                      double* grad, cudaStream_t st);
// y_k = sum_m c[k][m] f_m (masked) + phi0[k] * sp (pressure block only), k < nt
void launch_slab_rhs(const Grid& g, const double* const* f, int nterms, const double* c, const double* phi0, int nt,
                     const double* sp, double* y, int64_t ys, cudaStream_t st);  // level k at y + k * ys

template <typename T>
void launch_schur_dinv(const Grid& g, const TabT<T>& tb, const T* sb2, const double* cm, double tau, T* dinv, int nrhs,
                       cudaStream_t st);
template <typename T>
void launch_cheb_update_r(const T* b, const T* Ax, const T* dinv, T* d, const T* x, T* xo, double c1, double c2, int first,
                          int64_t n, int nrhs, cudaStream_t st);
template <typename TX, typename TD>
void launch_add_scaled(TX* x, const TD* d, double s, int64_t n, cudaStream_t st);
// precomputed lumped flux-pressure Schur stencil (16 coefficients per pressure point) and one
// fused Chebyshev-Jacobi step using it (pressure arrays, stride Np)
template <typename T>
void launch_schur_stencil(const Grid& g, const TabT<T>& tb, const T* dmq, double tau, T* coef, cudaStream_t st);
template <typename T>
void launch_schur_cheb_st(const Grid& g, const TabT<T>& tb, const T* coef, const T* dinv, const double* cm, double c1, double c2,
                          int first, const T* b, const T* x, T* d, T* xo, int nrhs, cudaStream_t st);
// matrix-free form of the same step: per-flux-DoF weights tau wt^2 / Mq_ff (0 on no-flow DoFs,
// instance-major like dmq) and one Chebyshev-Jacobi step for nk levels x nb instances
// (columns level-major, stride Np; cm indexed by level) with the Jacobi diagonal formed on the fly
template <typename T>
void launch_schur_wq(const Grid& g, const TabT<T>& tb, const T* dmq, double tau, T* wq, cudaStream_t st);
template <typename T>
void launch_schur_cheb_mf(const Grid& g, const TabT<T>& tb, const T* wq, const double* cm, double c1, double c2, int first,
                          const T* b, const T* x, T* d, T* xo, int nk, cudaStream_t st);
// cell-centred multigrid for the lumped Schur complement (mg.cu): grid sizes of one level
struct PDims {
  int n[3];
  int64_t nc;
};
PDims pdims_points(const Grid& g);  // the Gauss-point pressure grid (level 0)
template <typename T>
void launch_pmg_resid0(const Grid& g, const T* coef, const double* cm, const T* b, const T* x, T* r, int ncols, cudaStream_t st);
template <typename T>
void launch_pmg_build1(const Grid& g, const T* coef, T* st1, cudaStream_t st);
template <typename T>
void launch_pmg_coarsen(int dim, const PDims& fd, const PDims& cd, int nb, const T* stf, T* stc, cudaStream_t st);
// mode 0: Chebyshev-Jacobi step, 1: first step from zero, 2: residual b - A x into xo
template <typename T>
void launch_pmg_step(int dim, const PDims& pd, const T* stl, const double* cm, double ml, int nb, double c1, double c2, int mode,
                     const T* b, const T* x, T* d, T* xo, int ncols, cudaStream_t st);
template <typename T>
void launch_pmg_restrict(int dim, const PDims& fd, const PDims& cd, const T* rf, T* rc, int ncols, cudaStream_t st);
template <typename T>
void launch_pmg_prolong(int dim, const PDims& fd, const PDims& cd, const T* xc, T* xf, double alpha, int ncols, cudaStream_t st);
template <typename T>
void launch_dinv_mul(const T* dinv, int64_t dstride, const T* r, T* z, int64_t n, int64_t stride, int nrhs, cudaStream_t st);
// exact (s Mq)^{-1} by line solves (flux-block arrays); constrained entries untouched
template <typename T>
void launch_mq_line_solve(const Grid& g, const TabT<T>& tb, const T* kscale, const T* in, int64_t sin, T* out, int64_t sout,
                          double s_scale, int nrhs, cudaStream_t st);
template <typename T>
void launch_BTp(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* base, int64_t sb, T* tq, int64_t sq,
                double coef, int nrhs, cudaStream_t st);
template <typename T>
void launch_q_fix_constrained(const Grid& g, const T* in, int64_t sin, T* out, int64_t sout, int nrhs, cudaStream_t st);
template <typename T>
void launch_schur_out(const Grid& g, const TabT<T>& tb, const T* p, int64_t spp, const T* tq, int64_t sq, double tau,
                      const double* cm, T* out, int64_t so, int nrhs, cudaStream_t st);

}  // namespace biot
