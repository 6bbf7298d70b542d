// C ABI of the space-time Biot library: context set-up, slab apply, the
// time-spectral block preconditioner, flexible GMRES, mixed-precision
// refinement, slab marching and the adjoint gradient.
//
// Paper references: §Poroelasticity (the coupled system), §Discretisation in
// Time (dG(r) slabs, marching), §Discretisation in Space (Q2 / RT1 / DGQ1),
// §Monolithic Approach (slab block system, spectral decomposition of the time
// matrix, diagonal blocks L_j of dG(0) type), §Preconditioning technology
// (GMRES with truncated fixed-stress preconditioning).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <cstdlib>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/biot.h"
#include "internal.h"

using namespace biot;

namespace {
// NVTX range of one phase (march, slab, slab solve, inner FP32 solve) for timeline tools;
// without an attached tool the calls return at once
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

// ---------------------------------------------------------------------------
// helpers
namespace {

struct Err {
  int code;
};

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      throw_cuda(e_, #call, __LINE__);                                                           \
    }                                                                                            \
  } while (0)

thread_local std::string g_err_msg;

[[noreturn]] void throw_cuda(cudaError_t e, const char* what, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "CUDA error %s (%d) at api.cu:%d in %s", cudaGetErrorString(e), (int)e, line, what);
  g_err_msg = buf;
  throw Err{e == cudaErrorMemoryAllocation ? BIOT_ENOMEM : BIOT_ECUDA};
}

[[noreturn]] void fail(int code, const std::string& msg) {
  g_err_msg = msg;
  throw Err{code};
}

void check_launch(int line) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw_cuda(e, "kernel launch", line);
}
#define CKL() check_launch(__LINE__)

template <typename T>
T* dalloc(size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  CK(cudaMalloc(&p, n * sizeof(T)));
  return reinterpret_cast<T*>(p);
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- time basis (right-Radau Lagrange) --------------------------------------
struct TimeBasis {
  int nt;
  double nodes[MAXR], w[MAXR], D[MAXR][MAXR], phi0[MAXR];
  double V[MAXR][MAXR], W[MAXR][MAXR];  // M_t^{-1} D = V Lambda_R V^{-1};  W = V^{-1} M_t^{-1}
  double lam[MAXR];                      // real part of the eigenvalue owning each transformed component
  int pair;                              // first transformed component of the complex pair (-1: none)
  double pair_beta;                      // beta of the pair: block [[alpha, beta], [-beta, alpha]]
};

long double lagr(const long double* x, int n, int i, long double s) {
  long double v = 1;
  for (int j = 0; j < n; ++j)
    if (j != i) v *= (s - x[j]) / (x[i] - x[j]);
  return v;
}
long double lagr_d(const long double* x, int n, int i, long double s) {
  long double tot = 0;
  for (int k = 0; k < n; ++k) {
    if (k == i) continue;
    long double v = 1 / (x[i] - x[k]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != k) v *= (s - x[j]) / (x[i] - x[j]);
    tot += v;
  }
  return tot;
}

void invert_small(int n, const long double A[MAXR][MAXR], long double Ai[MAXR][MAXR]) {
  long double M[MAXR][2 * MAXR];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = (j < n) ? A[i][j] : (j - n == i ? 1 : 0);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs((double)M[i][c]) > std::fabs((double)M[p][c])) p = i;
    for (int j = 0; j < 2 * n; ++j) std::swap(M[c][j], M[p][j]);
    long double d = M[c][c];
    for (int j = 0; j < 2 * n; ++j) M[c][j] /= d;
    for (int i = 0; i < n; ++i)
      if (i != c) {
        long double f = M[i][c];
        for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[c][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ai[i][j] = M[i][j + n];
}

TimeBasis make_time_basis(int r) {
  TimeBasis tb;
  std::memset(&tb, 0, sizeof(tb));
  tb.pair = -1;
  int nt = r + 1;
  tb.nt = nt;
  long double x[MAXR];
  if (r == 0) x[0] = 1;
  if (r == 1) { x[0] = 1.0L / 3; x[1] = 1; }
  if (r == 2) { x[0] = (4 - std::sqrt(6.0L)) / 10; x[1] = (4 + std::sqrt(6.0L)) / 10; x[2] = 1; }
  // 5-point Gauss on [0,1] (exact to degree 9)
  const long double gx[5] = {-0.9061798459386639927976L, -0.5384693101056830910363L, 0.0L, 0.5384693101056830910363L,
                             0.9061798459386639927976L};
  const long double gw[5] = {0.2369268850561890875143L, 0.4786286704993664680413L, 0.5688888888888888888889L,
                             0.4786286704993664680413L, 0.2369268850561890875143L};
  long double M[MAXR][MAXR] = {}, D[MAXR][MAXR] = {};
  for (int k = 0; k < nt; ++k)
    for (int l = 0; l < nt; ++l) {
      long double m = 0, d = 0;
      for (int q = 0; q < 5; ++q) {
        long double s = (gx[q] + 1) / 2, w = gw[q] / 2;
        m += w * lagr(x, nt, l, s) * lagr(x, nt, k, s);
        d += w * lagr_d(x, nt, l, s) * lagr(x, nt, k, s);
      }
      M[k][l] = m;
      D[k][l] = d + lagr(x, nt, l, 0) * lagr(x, nt, k, 0);
    }
  for (int k = 0; k < nt; ++k) {
    tb.nodes[k] = (double)x[k];
    tb.w[k] = (double)M[k][k];
    tb.phi0[k] = (double)lagr(x, nt, k, 0);
    for (int l = 0; l < nt; ++l) tb.D[k][l] = (double)D[k][l];
  }
  // T = M^{-1} D (M diagonal)
  typedef std::complex<long double> cx;
  long double T[MAXR][MAXR];
  for (int k = 0; k < nt; ++k)
    for (int l = 0; l < nt; ++l) T[k][l] = D[k][l] / M[k][k];
  // eigenvalues: characteristic polynomial z^n + c1 z^{n-1} + ... via Faddeev-LeVerrier
  std::vector<cx> ev;
  if (nt == 1) ev.push_back(T[0][0]);
  else if (nt == 2) {
    long double tr = T[0][0] + T[1][1], det = T[0][0] * T[1][1] - T[0][1] * T[1][0];
    cx disc = std::sqrt(cx(tr * tr - 4 * det));
    ev.push_back((tr + disc) / 2.0L);
    ev.push_back((tr - disc) / 2.0L);
  } else {
    long double tr = T[0][0] + T[1][1] + T[2][2];
    long double m2 = T[0][0] * T[1][1] - T[0][1] * T[1][0] + T[0][0] * T[2][2] - T[0][2] * T[2][0] + T[1][1] * T[2][2] -
                     T[1][2] * T[2][1];
    long double det = T[0][0] * (T[1][1] * T[2][2] - T[1][2] * T[2][1]) - T[0][1] * (T[1][0] * T[2][2] - T[1][2] * T[2][0]) +
                      T[0][2] * (T[1][0] * T[2][1] - T[1][1] * T[2][0]);
    // p(z) = z^3 - tr z^2 + m2 z - det ; one real root by Newton from an upper bound
    long double z = tr + 1;
    for (int it = 0; it < 200; ++it) {
      long double p = ((z - tr) * z + m2) * z - det, dp = (3 * z - 2 * tr) * z + m2;
      long double nz = z - p / dp;
      if (std::fabs((double)(nz - z)) < 1e-30) break;
      z = nz;
    }
    // deflate: z^2 + (z0 - tr) z + det/z0
    long double bq = z - tr, cq = det / z;
    cx disc = std::sqrt(cx(bq * bq - 4 * cq));
    ev.push_back(z);
    ev.push_back((-bq + disc) / 2.0L);
    ev.push_back((-bq - disc) / 2.0L);
  }
  // real block form: columns of V
  long double V[MAXR][MAXR] = {};
  int col = 0;
  for (size_t i = 0; i < ev.size(); ++i) {
    cx lam = ev[i];
    if (std::fabs((double)lam.imag()) > 1e-12 && lam.imag() < 0) continue;  // conjugate handled with its partner
    // null vector of (T - lam I)
    cx A[MAXR][MAXR];
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b) A[a][b] = cx(T[a][b]) - (a == b ? lam : cx(0));
    cx v[MAXR];
    if (nt == 1) v[0] = 1;
    else if (nt == 2) { v[0] = A[0][1]; v[1] = -A[0][0]; if (std::abs(v[0]) + std::abs(v[1]) < 1e-20L) { v[0] = -A[1][1]; v[1] = A[1][0]; } }
    else {  // cross product of two rows
      v[0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
      v[1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
      v[2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    }
    if (std::fabs((double)lam.imag()) <= 1e-12) {
      long double nr = 0;
      for (int a = 0; a < nt; ++a) nr += std::norm(v[a]);
      nr = std::sqrt(nr);
      // make real: divide by the phase of the largest entry
      int am = 0;
      for (int a = 1; a < nt; ++a) if (std::abs(v[a]) > std::abs(v[am])) am = a;
      cx ph = v[am] / std::abs(v[am]);
      for (int a = 0; a < nt; ++a) V[a][col] = (v[a] / ph).real() / nr;
      tb.lam[col] = (double)lam.real();
      ++col;
    } else {
      // T (a + ib) = (alpha + i beta)(a + ib): V = [a, b] gives block [[alpha, beta], [-beta, alpha]]
      for (int a = 0; a < nt; ++a) { V[a][col] = v[a].real(); V[a][col + 1] = v[a].imag(); }
      tb.lam[col] = tb.lam[col + 1] = (double)lam.real();
      tb.pair = col;
      tb.pair_beta = (double)lam.imag();
      col += 2;
    }
  }
  long double Vi[MAXR][MAXR];
  invert_small(nt, V, Vi);
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      tb.V[a][b] = (double)V[a][b];
      tb.W[a][b] = (double)(Vi[a][b] / M[b][b]);
    }
  return tb;
}

}  // namespace

// ---------------------------------------------------------------------------
// context
template <typename T>
struct LevelWork {
  T *x = nullptr, *xo = nullptr, *d = nullptr, *Ax = nullptr, *b = nullptr;
};

struct Level {
  Grid g;
  TabT<double> t64;
  TabT<float> t32;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double lmax = 2.0;
  LevelWork<double> w64;
  LevelWork<float> w32;
};

template <typename T>
struct Krylov {
  int m = 0;
  std::vector<T*> V, Z;
  const T** dV = nullptr;  // device array of basis pointers
  T* tmp = nullptr;        // slab temporary
};

template <typename T>
struct PrecWork {
  T *tA = nullptr, *tB = nullptr;  // slab
  T *fq = nullptr, *tq = nullptr, *fq2 = nullptr;  // nt * Nq
  T *gp = nullptr, *pp = nullptr, *pd = nullptr, *pAx = nullptr, *pxo = nullptr, *pdinv = nullptr;  // nt * Np
  T* scoef = nullptr;  // 16 * Np per instance: lumped Schur stencil for schur_tau (multigrid path only)
  T* wq = nullptr;     // nqt per instance: flux weights tau wt^2 / Mq_ff of the matrix-free Schur step
  double schur_tau = -1.0;
  // cell-centred multigrid of the Schur complement: level l >= 1 stencils (per instance) and
  // level vectors (per column); pmr0 holds the level-0 residual
  std::vector<PDims> pml;
  std::vector<T*> pms, pmb, pmx, pmd, pmt;
  T* pmr0 = nullptr;
};

struct GraphKey {
  int prec, transpose, j;
  bool operator<(const GraphKey& o) const {
    return prec != o.prec ? prec < o.prec : (transpose != o.transpose ? transpose < o.transpose : j < o.j);
  }
};
struct GraphEntry {
  cudaGraphExec_t exec;
  double tau;
  long long kernels;  // kernel nodes in the graph (for the launch counter)
};

// per-instance scalar block of the Krylov reductions in hdev / hhost (instance b at b * HS):
// [0, 64) first Gram-Schmidt dots, [64, 128) second, 128 ||w||^2, 129 1/||w||, [160, 224) the
// least-squares coefficients y
constexpr int HS = 256;

struct biot_ctx {
  Grid g;
  int nb = 1;                  // independent instances batched in this context (level-major vectors)
  int lumped_flux = 1;
  bool use_graphs = true;
  bool tuned = false;          // launch shapes of this context's kernels looked up / measured
  std::map<GraphKey, GraphEntry> graphs;
  cudaStream_t ws = nullptr;   // the library's own work stream (graphs need a capturable stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int r = 0, nt = 1;
  double b, invM, Kdr, lam, mu, eta, beta;
  std::vector<double> Kcell;
  TabT<double> t64;
  TabT<float> t32;
  double* kscale64 = nullptr;
  float* kscale32 = nullptr;
  double *dmq64 = nullptr, *sb2_64 = nullptr;
  float *dmq32 = nullptr, *sb2_32 = nullptr;
  std::vector<Level> lv;
  double* Ainv = nullptr;
  int ncoarse = 0;
  TimeBasis tb;
  biot_opts opts;
  double schur_lmax = 0, schur_lmax_tau = -1, schur_lmin = 0;
  double schur_kappa = 1;      // Lanczos estimate of cond(Dinv Shat) for schur_lmax_tau
  Krylov<double> k64;
  Krylov<float> k32;
  PrecWork<double> p64;
  PrecWork<float> p32;
  void** ptrbuf = nullptr;     // device array of vector pointers for small reductions
  void** hptr = nullptr;       // pinned staging for ptrbuf
  double* hdev = nullptr;      // device scalars for the Krylov reductions (HS per instance)
  double* hhost = nullptr;     // pinned mirror
  double* bdev = nullptr;      // per-column scalars of batched kernels (4 * nt * nb + 64)
  double* bhost = nullptr;     // pinned mirror
  std::vector<int> it_b, ref_b, rc_b;   // batched solve: per-instance statistics of the last call
  std::vector<double> res_b;
  double* partial = nullptr;   // reduction partials
  double* r64 = nullptr;       // FP64 slab temporaries (refinement / march)
  double* a64 = nullptr;
  float* d32 = nullptr;
  float* r32 = nullptr;
  double* m_f[8] = {nullptr};  // march buffers (load terms, state, rhs, slab solution)
  const double** m_fdev = nullptr;
  double *m_U = nullptr, *m_SU = nullptr, *m_rhs = nullptr, *m_X = nullptr;
  double* bm_f = nullptr;      // batched march buffers: load terms [b][m][N], state [b][N],
  const double** bm_fdev = nullptr;  // per-instance term tables (8 each), jump term, rhs and
  double *bm_U = nullptr, *bm_SU = nullptr, *bm_rhs = nullptr, *bm_X = nullptr;  // solution [k][b][N]
  int bm_terms = 0;
  double* lvl64 = nullptr;     // one-level temporaries
  double* lvl64b = nullptr;
  std::vector<void*> extra;    // other allocations
  std::string err;

  int64_t lvN() const { return g.N * nb; }  // stride between temporal levels of a slab vector
  template <typename T> Krylov<T>& kry();
  template <typename T> PrecWork<T>& pw();
  template <typename T> const TabT<T>& tab() const;
  template <typename T> const T* kscale() const;
  template <typename T> const T* dmq() const;
  template <typename T> const T* sb2() const;
};
template <> Krylov<double>& biot_ctx::kry<double>() { return k64; }
template <> Krylov<float>& biot_ctx::kry<float>() { return k32; }
template <> PrecWork<double>& biot_ctx::pw<double>() { return p64; }
template <> PrecWork<float>& biot_ctx::pw<float>() { return p32; }
template <> const TabT<double>& biot_ctx::tab<double>() const { return t64; }
template <> const TabT<float>& biot_ctx::tab<float>() const { return t32; }
template <> const double* biot_ctx::kscale<double>() const { return kscale64; }
template <> const float* biot_ctx::kscale<float>() const { return kscale32; }
template <> const double* biot_ctx::dmq<double>() const { return dmq64; }
template <> const float* biot_ctx::dmq<float>() const { return dmq32; }
template <> const double* biot_ctx::sb2<double>() const { return sb2_64; }
template <> const float* biot_ctx::sb2<float>() const { return sb2_32; }

template <typename T> LevelWork<T>& lwork(Level& L);
template <> LevelWork<double>& lwork<double>(Level& L) { return L.w64; }
template <> LevelWork<float>& lwork<float>(Level& L) { return L.w32; }
template <typename T> const T* ldinv(const Level& L);
template <> const double* ldinv<double>(const Level& L) { return L.dinv64; }
template <> const float* ldinv<float>(const Level& L) { return L.dinv32; }
template <typename T> const TabT<T>& ltab(const Level& L);
template <> const TabT<double>& ltab<double>(const Level& L) { return L.t64; }
template <> const TabT<float>& ltab<float>(const Level& L) { return L.t32; }

namespace {

// ---- slab coefficients ------------------------------------------------------
SlabCoef slab_coef(const biot_ctx& c, double tau, int transpose) {
  SlabCoef s;
  std::memset(&s, 0, sizeof(s));
  s.nt = c.nt;
  s.lam = c.lam;
  s.mu = c.mu;
  for (int k = 0; k < c.nt; ++k) {
    double tw = tau * c.tb.w[k];
    s.au[k] = tw;
    s.aq[k] = tw;
    if (!transpose) {
      s.ep[k][k] = -c.b * tw;
      s.qp[k][k] = -tw;
      s.pq[k] = tw;
      for (int l = 0; l < c.nt; ++l) {
        s.pu[k][l] = c.b * c.tb.D[k][l];
        s.pp[k][l] = c.invM * c.tb.D[k][l];
      }
    } else {
      s.qp[k][k] = tw;
      s.pq[k] = -tw;
      s.pu[k][k] = -c.b * tw;
      for (int l = 0; l < c.nt; ++l) {
        s.ep[k][l] = c.b * c.tb.D[l][k];
        s.pp[k][l] = c.invM * c.tb.D[l][k];
      }
    }
  }
  return s;
}

// segments of a (batched) slab vector: instance b, level k at (k * nb + b) * N
Seg slab_seg(const biot_ctx& c) {
  Seg sg;
  sg.nb = c.nb;
  sg.nt = c.nt;
  sg.len = c.g.N;
  sg.istride = c.g.N;
  sg.lstride = c.g.N * c.nb;
  return sg;
}

template <typename T>
void apply_slab_T(biot_ctx& c, double tau, const T* x, T* y, int transpose, cudaStream_t st) {
  SlabCoef sc = slab_coef(c, tau, transpose);
  const Grid& g = c.g;
  launch_apply_u<T>(g, c.tab<T>(), sc, x, g.N, x + g.offp, g.N, y, g.N, st);
  CKL();
  launch_apply_q<T>(g, c.tab<T>(), sc, c.kscale<T>(), x, g.N, y, g.N, st);
  CKL();
  launch_apply_p<T>(g, c.tab<T>(), sc, x, g.N, y, g.N, st);
  CKL();
}

// tau A x on one MG level, nrhs vectors of stride Nu (epi: fused smoothing step or residual)
template <typename T>
void apply_A(const Level& L, double lam, double mu, double tau, const T* x, T* y, int nrhs, cudaStream_t st,
             const UEpi<T>* epi = nullptr) {
  SlabCoef sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.nt = 1;
  sc.lam = lam;
  sc.mu = mu;
  sc.au[0] = tau;
  sc.ucols = nrhs;  // every column (temporal level x batched instance) takes tau A
  sc.udiv = nrhs;
  launch_apply_u<T>(L.g, ltab<T>(L), sc, x, L.g.Nu, nullptr, 0, y, L.g.Nu, st, epi);
  CKL();
}

// ---- workspace -------------------------------------------------------------------
template <typename T>
void ensure_prec(biot_ctx& c) {
  PrecWork<T>& w = c.pw<T>();
  if (w.tA) return;
  const Grid& g = c.g;
  const int nt = c.nt * c.nb;  // columns: temporal levels x instances
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  w.tA = dalloc<T>(nt * g.N);
  w.tB = dalloc<T>(nt * g.N);
  w.fq = dalloc<T>(nt * nqt);
  w.tq = dalloc<T>(nt * nqt);
  w.fq2 = dalloc<T>(nt * nqt);
  w.gp = dalloc<T>(nt * g.Np);
  w.pp = dalloc<T>(nt * g.Np);
  w.pd = dalloc<T>(nt * g.Np);
  w.pAx = dalloc<T>(nt * g.Np);
  w.pxo = dalloc<T>(nt * g.Np);
  w.pdinv = dalloc<T>(nt * g.Np);
  w.scoef = dalloc<T>(16 * g.Np * c.nb);
  w.wq = dalloc<T>(nqt * c.nb);
  for (Level& L : c.lv) {
    LevelWork<T>& lw = lwork<T>(L);
    int64_t n = (int64_t)nt * L.g.Nu;
    lw.x = dalloc<T>(n);
    lw.xo = dalloc<T>(n);
    lw.d = dalloc<T>(n);
    lw.Ax = dalloc<T>(n);
    lw.b = dalloc<T>(n);
  }
}

template <typename T>
void ensure_krylov(biot_ctx& c, int m) {
  Krylov<T>& K = c.kry<T>();
  if (K.m >= m) return;
  for (T* p : K.V) cudaFree(p);
  for (T* p : K.Z) cudaFree(p);
  if (K.dV) cudaFree((void*)K.dV);
  if (K.tmp) cudaFree(K.tmp);
  K.V.clear();
  K.Z.clear();
  const int64_t n = c.g.N * c.nt * c.nb;
  for (int i = 0; i <= m; ++i) K.V.push_back(dalloc<T>(n));
  for (int i = 0; i < m; ++i) K.Z.push_back(dalloc<T>(n));
  K.tmp = dalloc<T>(n);
  K.dV = (const T**)dalloc<T*>(2 * m + 1);
  std::vector<T*> ptrs(K.V.begin(), K.V.end());
  ptrs.insert(ptrs.end(), K.Z.begin(), K.Z.end());
  // pageable copy on the legacy stream: wait for it, the solver's streams do not order after it
  CK(cudaMemcpy((void*)K.dV, ptrs.data(), ptrs.size() * sizeof(T*), cudaMemcpyHostToDevice));
  CK(cudaDeviceSynchronize());
  K.m = m;
}

double dev_dot(biot_ctx& c, const double* a, const double* b, int64_t n, cudaStream_t st) {
  const double* va[1] = {a};  // host array of vector pointers (passed to the kernel by value)
  launch_multidot<double>(va, 1, b, n, c.partial, c.hdev + 100, st);
  CKL();
  CK(cudaMemcpyAsync(c.hhost + 100, c.hdev + 100, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return c.hhost[100];
}


// ---- eigenvalue bounds ----------------------------------------------------------
// Largest eigenvalue of Dinv Op (Op symmetric positive semi-definite, Dinv >= 0
// diagonal) by `steps` preconditioned-CG steps, from the Lanczos tridiagonal
// matrix built out of the CG coefficients (FP64).  nrhs independent systems
// of length n (stride between them), the maximum over them is returned.
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, bool want_max);
double tridiag_lmax(const std::vector<double>& d, const std::vector<double>& e) { return tridiag_eig(d, e, true); }
double tridiag_lmin(const std::vector<double>& d, const std::vector<double>& e) { return tridiag_eig(d, e, false); }
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, bool want_max) {
  // bisection with Sturm counts on the symmetric tridiagonal (d, e)
  int k = (int)d.size();
  if (k == 0) return 1.0;
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    double rad = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - rad);
    hi = std::max(hi, d[i] + rad);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < k; ++i) {
      double qq = (q == 0.0) ? 1e-300 : q;
      q = d[i] - x - e[i - 1] * e[i - 1] / qq;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  // bisection on the Sturm count: the largest eigenvalue is the smallest x with count(x) = k,
  // the smallest eigenvalue the smallest x with count(x) >= 1
  const int target = want_max ? k : 1;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= target) hi = mid;
    else lo = mid;
  }
  return hi;
}

template <class OpF>
double lanczos_lmax(biot_ctx& c, OpF op, const double* dinv, int64_t dstride, int64_t n, int64_t stride, int nrhs, int steps,
                    double* r, double* z, double* p, double* q, cudaStream_t st, double* lmin_out = nullptr, int per_level = 1) {
  // start vector of rhs k depends on its temporal level k / per_level only, so every batched
  // instance starts from the vector a single context would use
  std::vector<double> h((size_t)stride * nrhs, 0.0);
  for (int k = 0; k < nrhs; ++k)
    for (int64_t i = 0; i < n; ++i)
      h[k * stride + i] = 1.0 + 0.3 * std::sin(0.91 * (double)i + 0.7 * (k / per_level)) + 0.2 * std::cos(2.3 * (double)i);
  CK(cudaMemcpyAsync(r, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  // z = Dinv r, p = z (rows with Dinv = 0, the constrained ones, never enter the Krylov space)
  launch_dinv_mul<double>(dinv, dstride, r, z, n, stride, nrhs, st);
  CK(cudaMemcpyAsync(p, z, (size_t)stride * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CKL();
  // every rhs at once: segmented dots (one result per rhs) and per-rhs axpbys with
  // coefficient columns staged through pinned memory (each staging write follows a
  // stream synchronisation, so no copy still reads it)
  Seg sg;
  sg.nb = nrhs;
  sg.nt = 1;
  sg.len = n;
  sg.istride = stride;
  sg.lstride = 0;
  double* out = c.bdev;                 // nrhs dots
  double* ca = c.bdev + nrhs;           // coefficient columns
  double* cb = c.bdev + 2 * nrhs;
  double* one = c.bdev + 3 * nrhs;
  c.hptr[8] = (void*)r;
  c.hptr[9] = (void*)p;
  CK(cudaMemcpyAsync(c.ptrbuf + 8, c.hptr + 8, 2 * sizeof(void*), cudaMemcpyHostToDevice, st));
  const double* const* vr = reinterpret_cast<const double* const*>(c.ptrbuf + 8);
  const double* const* vp = reinterpret_cast<const double* const*>(c.ptrbuf + 9);
  auto dots = [&](const double* const* V, const double* w, std::vector<double>& res) {
    launch_seg_multidot<double>(V, 1, w, sg, c.partial, out, 1, st);
    CKL();
    CK(cudaMemcpyAsync(c.bhost, out, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    res.assign(c.bhost, c.bhost + nrhs);
  };
  double best = 0.0;
  std::vector<double> rz, pq, rzn, alpha_prev(nrhs, 0.0), beta_prev(nrhs, 0.0);
  std::vector<std::vector<double>> dd(nrhs), ee(nrhs);
  dots(vr, z, rz);
  for (int k = 0; k < nrhs; ++k) c.bhost[3 * nrhs + k] = 1.0;
  for (int it = 0; it < steps; ++it) {
    op(p, q);
    dots(vp, q, pq);
    bool stop = false;
    for (int k = 0; k < nrhs; ++k)
      if (!(pq[k] > 0) || !(rz[k] > 0)) stop = true;
    if (stop) break;
    for (int k = 0; k < nrhs; ++k) {
      const double alpha = rz[k] / pq[k];
      dd[k].push_back(1.0 / alpha + (it > 0 ? beta_prev[k] / alpha_prev[k] : 0.0));
      alpha_prev[k] = alpha;
      c.bhost[nrhs + k] = -alpha;
      c.bhost[3 * nrhs + k] = 1.0;
    }
    CK(cudaMemcpyAsync(ca, c.bhost + nrhs, nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(one, c.bhost + 3 * nrhs, nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_seg_axpby<double>(r, q, ca, one, sg, st);  // r -= alpha q
    launch_dinv_mul<double>(dinv, dstride, r, z, n, stride, nrhs, st);
    CKL();
    dots(vr, z, rzn);
    for (int k = 0; k < nrhs; ++k) {
      const double beta = rzn[k] / rz[k];
      ee[k].push_back(std::sqrt(std::max(beta, 0.0)) / alpha_prev[k]);
      beta_prev[k] = beta;
      rz[k] = rzn[k];
      c.bhost[2 * nrhs + k] = beta;
    }
    CK(cudaMemcpyAsync(cb, c.bhost + 2 * nrhs, nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_seg_axpby<double>(p, z, one, cb, sg, st);  // p = z + beta p
    CKL();
  }
  CK(cudaStreamSynchronize(st));
  double worst_min = 1e300;
  for (int k = 0; k < nrhs; ++k) {
    std::vector<double> e(ee[k].begin(), ee[k].end());
    if (e.size() >= dd[k].size() && !e.empty()) e.resize(dd[k].size() - 1);
    best = std::max(best, tridiag_lmax(dd[k], e));
    worst_min = std::min(worst_min, tridiag_lmin(dd[k], e));
  }
  if (lmin_out) *lmin_out = worst_min;
  return best;
}

// ---- Chebyshev smoothing -----------------------------------------------------
constexpr int MAX_CHEB = 128;
struct ChebCoef {
  int n;
  double c1[MAX_CHEB], c2[MAX_CHEB];
};
ChebCoef cheb_coefs(int degree, double lmin, double lmax) {
  ChebCoef cc;
  cc.n = degree;
  double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho_old = 1.0 / sigma;
  cc.c1[0] = 0.0;
  cc.c2[0] = 1.0 / theta;
  for (int k = 1; k < degree && k < MAX_CHEB; ++k) {
    double rho = 1.0 / (2.0 * sigma - rho_old);
    cc.c1[k] = rho * rho_old;
    cc.c2[k] = 2.0 * rho / delta;
    rho_old = rho;
  }
  return cc;
}

// smooth tau A x = b on level l; x_in_zero: start from 0.  Result pointer in w.x.
template <typename T>
void smooth(biot_ctx& c, Level& L, double tau, int nrhs, bool zero_start, cudaStream_t st) {
  LevelWork<T>& w = lwork<T>(L);
  ChebCoef cc = cheb_coefs(c.opts.cheb_degree, L.lmax / 20.0, 1.1 * L.lmax);
  const int64_t n = L.g.Nu;
  for (int k = 0; k < cc.n; ++k) {
    bool first = (k == 0 && zero_start);
    if (first) {
      launch_cheb_update<T>(w.b, w.Ax, ldinv<T>(L), w.d, w.x, w.xo, cc.c1[k], cc.c2[k] / tau, 1, n, nrhs, n, st);
    } else {
      // the operator's output stage does the Chebyshev-Jacobi update (no separate pass)
      UEpi<T> ep;
      ep.mode = EPI_CHEB;
      ep.b = w.b;
      ep.dinv = ldinv<T>(L);
      ep.d = w.d;
      ep.xo = w.xo;
      ep.c1 = (T)cc.c1[k];
      ep.c2 = (T)(cc.c2[k] / tau);
      apply_A<T>(L, c.lam, c.mu, tau, w.x, nullptr, nrhs, st, &ep);
    }
    CKL();
    std::swap(w.x, w.xo);
  }
}

// V-cycle on levels[0..]: b in lv[0].w.b, result in lv[0].w.x
template <typename T>
void vcycle(biot_ctx& c, double tau, int nrhs, cudaStream_t st) {
  const int nl = (int)c.lv.size();
  for (int l = 0; l < nl - 1; ++l) {
    Level& L = c.lv[l];
    LevelWork<T>& w = lwork<T>(L);
    smooth<T>(c, L, tau, nrhs, true, st);
    UEpi<T> ep;  // residual b - tau A x in Ax, fused into the operator's output stage
    ep.mode = EPI_RESID;
    ep.b = w.b;
    apply_A<T>(L, c.lam, c.mu, tau, w.x, w.Ax, nrhs, st, &ep);
    CKL();
    Level& C = c.lv[l + 1];
    launch_restrict<T>(L.g, C.g, w.Ax, L.g.Nu, lwork<T>(C).b, C.g.Nu, nrhs, st);
    CKL();
  }
  Level& Lc = c.lv[nl - 1];
  if (c.Ainv) {
    launch_dense_gemv<T>(c.Ainv, c.ncoarse, lwork<T>(Lc).b, Lc.g.Nu, lwork<T>(Lc).x, Lc.g.Nu, nrhs, 1.0 / tau, st);
    CKL();
  } else {
    smooth<T>(c, Lc, tau, nrhs, true, st);
  }
  for (int l = nl - 2; l >= 0; --l) {
    Level& L = c.lv[l];
    Level& C = c.lv[l + 1];
    launch_prolong_add<T>(L.g, C.g, lwork<T>(C).x, C.g.Nu, lwork<T>(L).x, L.g.Nu, nrhs, st);
    CKL();
    smooth<T>(c, L, tau, nrhs, false, st);
  }
}

// ---- flux-pressure Schur complement ---------------------------------------------
// Shat p = cm Mp p + tau B Mq^{-1} B^T p, with Mq^{-1} exact (line solves) or lumped (diagonal)
template <typename T>
void schur_apply(biot_ctx& c, double tau, const double* cm, const T* p, T* out, int nrhs, cudaStream_t st) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (c.lumped_flux) {
    launch_schur_apply<T>(g, c.tab<T>(), p, g.Np, c.dmq<T>(), w.tq, nqt, tau, cm, out, g.Np, nrhs, st);
  } else {
    launch_BTp<T>(g, c.tab<T>(), p, g.Np, nullptr, 0, w.tq, nqt, 1.0, nrhs, st);
    launch_mq_line_solve<T>(g, c.tab<T>(), c.kscale<T>(), w.tq, nqt, w.fq2, nqt, 1.0, nrhs, st);
    launch_schur_out<T>(g, c.tab<T>(), p, g.Np, w.fq2, nqt, tau, cm, out, g.Np, nrhs, st);
  }
  CKL();
}

// q = (tau Mq)^{-1} (base + coef B^T p) on free flux DoFs, base on constrained ones
template <typename T>
void flux_solve(biot_ctx& c, double tau, const T* base, int64_t sb, const T* p, double coef, T* qo, int64_t so, int nrhs,
                cudaStream_t st) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  if (c.lumped_flux) {
    if (p) launch_q_final<T>(g, c.tab<T>(), base, sb, p, g.Np, c.dmq<T>(), tau, coef, qo, so, nrhs, st);
    else launch_q_jacobi<T>(g, c.tab<T>(), base, sb, c.dmq<T>(), tau, qo, so, nrhs, st);
  } else {
    const T* rhs = base;
    int64_t sr = sb;
    if (p) {
      launch_BTp<T>(g, c.tab<T>(), p, g.Np, base, sb, w.tq, nqt, coef, nrhs, st);
      rhs = w.tq;
      sr = nqt;
    }
    launch_mq_line_solve<T>(g, c.tab<T>(), c.kscale<T>(), rhs, sr, qo, so, tau, nrhs, st);
    launch_q_fix_constrained<T>(g, base, sb, qo, so, nrhs, st);
  }
  CKL();
}

void schur_cm(const biot_ctx& c, double* cm) {
  for (int k = 0; k < c.nt; ++k) cm[k] = c.tb.lam[k] * (c.invM + c.beta);
}

// Chebyshev interval of the Schur solve: [max(0.7 lmin_ritz, lmax / SCHUR_KAPPA_MAX), 1.1 lmax]
constexpr double SCHUR_KAPPA_MAX = 4000.0;

// largest eigenvalue of Dinv Shat (CG-Lanczos in FP64 on every rhs, max over rhs), cached per tau
double schur_lmax(biot_ctx& c, double tau, cudaStream_t st) {
  if (c.schur_lmax_tau == tau) return c.schur_lmax;
  ensure_prec<double>(c);
  PrecWork<double>& w = c.p64;
  const Grid& g = c.g;
  double cm[MAXR];
  schur_cm(c, cm);
  const int cols = c.nt * c.nb;  // every temporal level of every batched instance
  launch_schur_dinv<double>(g, c.t64, c.sb2_64, cm, tau, w.pdinv, cols, st);
  CKL();
  auto op = [&](const double* x, double* y) { schur_apply<double>(c, tau, cm, x, y, cols, st); };
  double lmin = 0;
  double lm = lanczos_lmax(c, op, w.pdinv, g.Np, g.Np, g.Np, cols, 30, w.gp, w.pp, w.pd, w.pAx, st, &lmin, c.nb);
  c.schur_lmax = lm;
  c.schur_kappa = lmin > 0 ? lm / lmin : 1e300;
  // Ritz values converge from inside the spectrum: widen the lower end, keep it positive
  c.schur_lmin = std::max(0.7 * lmin, lm / SCHUR_KAPPA_MAX);
  c.schur_lmax_tau = tau;
  return lm;
}

// Flow-block solver choice (after schur_lmax for this tau).  Chebyshev(degree) converges
// at a rate set by sqrt(kappa) of the Jacobi-scaled Schur complement; when the Darcy part
// dominates the storage part (large tau K / h^2) kappa grows like h^-2 and the multigrid
// V-cycle wins.  Measured on the 2-D batching workload (kappa 173, 400, 918, 2004 for
// n = 16, 32, 64, 128): multigrid faster from kappa ~900 on; in 3-D (32^3 dG(1) and
// 64^3 dG(2)) Chebyshev was faster in every case measured.
constexpr double PMG_KAPPA_2D = 600.0;
bool use_schur_mg(const biot_ctx& c) {
  if (c.opts.schur_mg > 0) return true;
  if (c.opts.schur_mg < 0 || !c.lumped_flux) return false;
  return c.g.dim == 2 && c.schur_kappa > PMG_KAPPA_2D;
}

// Jacobi diagonal of every column and the lumped Schur stencil of every instance for this tau
template <typename T>
void schur_prepare(biot_ctx& c, double tau, cudaStream_t st) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  double cm_all[MAXR];
  schur_cm(c, cm_all);
  launch_schur_dinv<T>(g, c.tab<T>(), c.sb2<T>(), cm_all, tau, w.pdinv, c.nt * c.nb, st);
  for (int b = 0; b < c.nb; ++b) {
    // FP32 runs the matrix-free step; FP64 (a small share of the work, on the slow FP64 pipe)
    // keeps the precomputed stencil, which needs no divisions
    if (sizeof(T) == 4) launch_schur_wq<T>(g, c.tab<T>(), c.dmq<T>() + b * nqt, tau, w.wq + (int64_t)b * nqt, st);
    if (use_schur_mg(c) || sizeof(T) == 8)
      launch_schur_stencil<T>(g, c.tab<T>(), c.dmq<T>() + b * nqt, tau, w.scoef + (int64_t)b * 16 * g.Np, st);
  }
  CKL();
  if (use_schur_mg(c)) {
    // Galerkin stencils of the cell levels: 2^d Gauss points -> cell, then 2^d cells -> cell
    if (w.pml.empty()) {
      const int cols = c.nt * c.nb;
      PDims p;
      for (int d = 0; d < 3; ++d) p.n[d] = g.n[d];
      p.nc = g.ncells;
      while (true) {
        w.pml.push_back(p);
        w.pms.push_back(dalloc<T>((int64_t)(1 + 2 * g.dim) * p.nc * c.nb));
        for (auto* v : {&w.pmb, &w.pmx, &w.pmd, &w.pmt}) v->push_back(dalloc<T>(p.nc * cols));
        bool can = true;
        for (int d = 0; d < g.dim; ++d)
          if (p.n[d] % 2 != 0 || p.n[d] / 2 < 2) can = false;
        if (!can) break;
        for (int d = 0; d < g.dim; ++d) p.n[d] /= 2;
        p.nc = 1;
        for (int d = 0; d < g.dim; ++d) p.nc *= p.n[d];
      }
      w.pmr0 = dalloc<T>(g.Np * cols);
    }
    launch_pmg_build1<T>(g, w.scoef, w.pms[0], st);
    for (size_t l = 1; l < w.pml.size(); ++l)
      launch_pmg_coarsen<T>(g.dim, w.pml[l - 1], w.pml[l], c.nb, w.pms[l - 1], w.pms[l], st);
    CKL();
  }
}

// One V-cycle of the cell-centred multigrid on the lumped Schur complement for the
// columns k0.. (nk levels x nb instances): right-hand side w.gp, result w.pp.  Chebyshev-
// Jacobi smoothing on every level (level 0 with the Lanczos bound, cell levels with the
// Gershgorin bound 2 of the Jacobi-scaled diagonally dominant stencils); coarse corrections
// are scaled by PMG_ALPHA, which offsets the stiffness that piecewise-constant aggregation
// gives the Galerkin operators of a Laplacian-type block.
constexpr int PMG_NU = 2;          // smoothing steps before and after the coarse correction
constexpr int PMG_COARSE = 8;      // Chebyshev steps on the coarsest level
constexpr double PMG_ALPHA = 1.6;  // coarse-correction scale (measured best of 1.0, 1.3, 1.6 in 2-D)
template <typename T>
void schur_vcycle(biot_ctx& c, double tau, const double* cm, double lmax0, int k0, int nk, cudaStream_t st) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  const int cols = nk * c.nb;
  const int dim = g.dim;
  const T* dinv = w.pdinv + (int64_t)k0 * c.nb * g.Np;
  ChebCoef c0 = cheb_coefs(PMG_NU, lmax0 / 6.0, 1.1 * lmax0);
  ChebCoef cl = cheb_coefs(PMG_NU, 2.2 / 6.0, 2.2);
  ChebCoef cc = cheb_coefs(PMG_COARSE, 0.02, 2.2);
  double mp = 1.0;
  for (int d = 0; d < dim; ++d) mp *= c.t64.wg[d];
  // level 0 pre-smoothing from zero (w.gp -> w.pp)
  for (int k = 0; k < PMG_NU; ++k) {
    launch_schur_cheb_st<T>(g, c.tab<T>(), w.scoef, dinv, cm, c0.c1[k], c0.c2[k], k == 0 ? 1 : 0, w.gp, w.pp, w.pd, w.pxo, cols, st);
    std::swap(w.pp, w.pxo);
  }
  launch_pmg_resid0<T>(g, w.scoef, cm, w.gp, w.pp, w.pmr0, cols, st);
  const PDims p0 = pdims_points(g);
  launch_pmg_restrict<T>(dim, p0, w.pml[0], w.pmr0, w.pmb[0], cols, st);
  CKL();
  const int L = (int)w.pml.size();
  double ml = mp * (1 << dim);  // mass of a level-1 cell (Galerkin sum of its points)
  std::vector<double> mls(L);
  for (int l = 0; l < L; ++l) {
    mls[l] = ml;
    ml *= (1 << dim);
  }
  // down: smooth from zero, residual, restrict
  for (int l = 0; l < L - 1; ++l) {
    const PDims& pd = w.pml[l];
    for (int k = 0; k < PMG_NU; ++k) {
      launch_pmg_step<T>(dim, pd, w.pms[l], cm, mls[l], c.nb, cl.c1[k], cl.c2[k], k == 0 ? 1 : 0, w.pmb[l], w.pmx[l], w.pmd[l],
                         w.pmt[l], cols, st);
      std::swap(w.pmx[l], w.pmt[l]);
    }
    launch_pmg_step<T>(dim, pd, w.pms[l], cm, mls[l], c.nb, 0.0, 0.0, 2, w.pmb[l], w.pmx[l], w.pmd[l], w.pmt[l], cols, st);
    launch_pmg_restrict<T>(dim, pd, w.pml[l + 1], w.pmt[l], w.pmb[l + 1], cols, st);
    CKL();
  }
  // coarsest level: Chebyshev from zero
  {
    const int l = L - 1;
    for (int k = 0; k < cc.n; ++k) {
      launch_pmg_step<T>(dim, w.pml[l], w.pms[l], cm, mls[l], c.nb, cc.c1[k], cc.c2[k], k == 0 ? 1 : 0, w.pmb[l], w.pmx[l],
                         w.pmd[l], w.pmt[l], cols, st);
      std::swap(w.pmx[l], w.pmt[l]);
    }
    CKL();
  }
  // up: prolong the correction, smooth
  for (int l = L - 2; l >= 0; --l) {
    const PDims& pd = w.pml[l];
    launch_pmg_prolong<T>(dim, pd, w.pml[l + 1], w.pmx[l + 1], w.pmx[l], PMG_ALPHA, cols, st);
    for (int k = 0; k < PMG_NU; ++k) {
      launch_pmg_step<T>(dim, pd, w.pms[l], cm, mls[l], c.nb, cl.c1[k], cl.c2[k], 0, w.pmb[l], w.pmx[l], w.pmd[l], w.pmt[l], cols,
                         st);
      std::swap(w.pmx[l], w.pmt[l]);
    }
    CKL();
  }
  launch_pmg_prolong<T>(dim, p0, w.pml[0], w.pmx[0], w.pp, PMG_ALPHA, cols, st);
  for (int k = 0; k < PMG_NU; ++k) {
    launch_schur_cheb_st<T>(g, c.tab<T>(), w.scoef, dinv, cm, c0.c1[k], c0.c2[k], 0, w.gp, w.pp, w.pd, w.pxo, cols, st);
    std::swap(w.pp, w.pxo);
  }
  CKL();
}

// Chebyshev degree of the flux-pressure Schur solve: the caller's, else the degree at which
// the Chebyshev error bound 2 rho^k, rho = (sqrt(kappa) - 1) / (sqrt(kappa) + 1), on the
// solve's interval (kappa = its hi / lo) falls to about 0.07, i.e. k ~ 1.7 sqrt(kappa).
// Measured on the layered 3-D problems: at 32^3 dG(1) (kappa 218, degree 26) degrees 20-40
// give the same time to solution; at 64^3 dG(2) (kappa ~950, degree 53) 52 was fastest of
// 32-96, 68 3 % and 84 6 % slower, 32 29 % slower.  Called after schur_lmax for this tau.
int schur_degree(const biot_ctx& c) {
  if (c.opts.schur_degree > 0) return c.opts.schur_degree;
  const double kappa = 1.1 * c.schur_lmax / c.schur_lmin;
  const int k = (int)std::ceil(1.7 * std::sqrt(kappa));
  return std::max(16, std::min(k, MAX_CHEB));
}

// p = Shat^{-1} g by Chebyshev-Jacobi (w.gp -> w.pp)
template <typename T>
void schur_solve(biot_ctx& c, double tau, cudaStream_t st, int k0, int nk) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  double cm_all[MAXR];
  schur_cm(c, cm_all);
  const double* cm = cm_all + k0;
  double lmax = schur_lmax(c, tau, st);
  ChebCoef cc = cheb_coefs(schur_degree(c), c.schur_lmin, 1.1 * lmax);
  if (c.lumped_flux) {
    if (w.schur_tau != tau) {  // stencil and diagonal of this tau (prec_prepare normally did this)
      schur_prepare<T>(c, tau, st);
      w.schur_tau = tau;
    }
    const T* dinv = w.pdinv + (int64_t)k0 * c.nb * g.Np;
    if (use_schur_mg(c) && !w.pml.empty()) {
      schur_vcycle<T>(c, tau, cm, lmax, k0, nk, st);
      return;
    }
    for (int k = 0; k < cc.n; ++k) {
      if (sizeof(T) == 4)
        launch_schur_cheb_mf<T>(g, c.tab<T>(), w.wq, cm, cc.c1[k], cc.c2[k], k == 0 ? 1 : 0, w.gp, w.pp, w.pd, w.pxo, nk, st);
      else
        launch_schur_cheb_st<T>(g, c.tab<T>(), w.scoef, dinv, cm, cc.c1[k], cc.c2[k], k == 0 ? 1 : 0, w.gp, w.pp, w.pd, w.pxo,
                                nk * c.nb, st);
      CKL();
      std::swap(w.pp, w.pxo);
    }
    return;
  }
  launch_schur_dinv<T>(g, c.tab<T>(), c.sb2<T>(), cm, tau, w.pdinv, nk, st);
  CKL();
  for (int k = 0; k < cc.n; ++k) {
    bool first = (k == 0);
    if (!first) schur_apply<T>(c, tau, cm, w.pp, w.pAx, nk, st);
    launch_cheb_update_r<T>(w.gp, w.pAx, w.pdinv, w.pd, w.pp, w.pxo, cc.c1[k], cc.c2[k], first ? 1 : 0, g.Np, nk, st);
    CKL();
    std::swap(w.pp, w.pxo);
  }
}

template <typename T>
void copy2d(T* dst, int64_t dpitch, const T* src, int64_t spitch, int64_t width, int rows, cudaStream_t st) {
  CK(cudaMemcpy2DAsync(dst, dpitch * sizeof(T), src, spitch * sizeof(T), width * sizeof(T), rows, cudaMemcpyDeviceToDevice, st));
}

// Block-triangular solve of the transformed diagonal blocks for components k0 .. k0+nk-1
// (w.tA -> w.tB): flux-pressure block first (lumped Schur, Chebyshev), then the
// displacement by one V-cycle for tau A u = r_u + b tau E p.
template <typename T>
void block_solve(biot_ctx& c, double tau, int k0, int nk, cudaStream_t st) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  const int64_t N = g.N, Nu = g.Nu, Np = g.Np;
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  LevelWork<T>& lw = lwork<T>(c.lv[0]);
  // levels k0 .. k0+nk-1 of every instance are the consecutive columns from k0 * nb on
  const int cols = nk * c.nb;
  T* tA = w.tA + (int64_t)k0 * c.lvN();
  T* tB = w.tB + (int64_t)k0 * c.lvN();
  flux_solve<T>(c, tau, tA + Nu, N, nullptr, 0.0, w.fq, nqt, cols, st);
  launch_p_minus_Bq<T>(g, c.tab<T>(), tA + g.offp, N, w.fq, nqt, tau, w.gp, Np, cols, st);
  CKL();
  schur_solve<T>(c, tau, st, k0, nk);
  flux_solve<T>(c, tau, tA + Nu, N, w.pp, tau, tB + Nu, N, cols, st);
  copy2d<T>(tB + g.offp, N, w.pp, Np, Np, cols, st);
  launch_u_rhs<T>(g, c.tab<T>(), tA, N, w.pp, Np, c.b * tau, lw.b, Nu, cols, st);
  CKL();
  vcycle<T>(c, tau, cols, st);
  copy2d<T>(tB, N, lw.x, Nu, Nu, cols, st);
}

// z = P r  (or P^T r)
template <typename T>
void precondition_T(biot_ctx& c, double tau, const T* R, T* Z, int transpose, cudaStream_t st) {
  PrecWork<T>& w = c.pw<T>();
  const Grid& g = c.g;
  const int nt = c.nt;
  const int64_t N = g.N, Nu = g.Nu, Np = g.Np;
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  Level& L0 = c.lv[0];
  LevelWork<T>& lw = lwork<T>(L0);
  // the Schur eigenvalue bounds use the FP64 flow-block buffers: obtain them before any of
  // those buffers holds data of this application (a no-op once cached for this tau)
  (void)schur_lmax(c, tau, st);
  double Wm[MAXR * MAXR], Vm[MAXR * MAXR];
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      Wm[a * nt + b] = transpose ? c.tb.V[b][a] : c.tb.W[a][b];
      Vm[a * nt + b] = transpose ? c.tb.W[b][a] : c.tb.V[a][b];
    }
  // the time transform mixes the levels of each DoF: with level-major batched vectors
  // the instances just extend the spatial index (nb * N entries per level)
  const int64_t LN = c.lvN();
  const int cols = nt * c.nb;
  launch_time_mix<T, T>(R, LN, w.tA, LN, nt, Wm, LN, st);
  CKL();
  if (!transpose) {
    const int p0 = c.tb.pair;
    if (c.opts.pair_coupling && p0 >= 0) {
      // one block Gauss-Seidel sweep on the 2x2 real block of the complex pair
      // [[L, beta S], [-beta S, L]]: y_p0 = L^{-1} r_p0, y_p0+1 = L^{-1} (r_p0+1 + beta S y_p0)
      block_solve<T>(c, tau, 0, p0 + 1, st);
      const double beta = c.tb.pair_beta;
      T* r1 = w.tA + (int64_t)(p0 + 1) * LN;
      const T* y0 = w.tB + (int64_t)p0 * LN;
      launch_p_plus_ETu<T>(g, c.tab<T>(), r1 + g.offp, N, y0, N, beta * c.b, r1 + g.offp, N, c.nb, st);
      double mp = 1.0;
      for (int d = 0; d < g.dim; ++d) mp *= c.t64.wg[d];
      if (c.nb == 1) launch_axpby<T>(r1 + g.offp, y0 + g.offp, beta * c.invM * mp, 1.0, Np, st);
      else launch_axpby_rows<T>(r1 + g.offp, y0 + g.offp, beta * c.invM * mp, 1.0, Np, c.nb, N, st);
      CKL();
      block_solve<T>(c, tau, p0 + 1, nt - p0 - 1, st);
    } else {
      block_solve<T>(c, tau, 0, nt, st);
    }
  } else {
    copy2d<T>(lw.b, Nu, w.tA, N, Nu, cols, st);
    vcycle<T>(c, tau, cols, st);
    copy2d<T>(w.tB, N, lw.x, Nu, Nu, cols, st);
    launch_p_plus_ETu<T>(g, c.tab<T>(), w.tA + g.offp, N, lw.x, Nu, c.b * tau, w.gp, Np, cols, st);
    CKL();
    flux_solve<T>(c, tau, w.tA + Nu, N, nullptr, 0.0, w.fq, nqt, cols, st);
    launch_p_minus_Bq<T>(g, c.tab<T>(), w.gp, Np, w.fq, nqt, -tau, w.gp, Np, cols, st);
    CKL();
    schur_solve<T>(c, tau, st, 0, nt);
    flux_solve<T>(c, tau, w.tA + Nu, N, w.pp, -tau, w.tB + Nu, N, cols, st);
    copy2d<T>(w.tB + g.offp, N, w.pp, Np, Np, cols, st);
  }
  launch_time_mix<T, T>(w.tB, LN, Z, LN, nt, Vm, LN, st);
  CKL();
}

// ---- flexible GMRES(m), right preconditioned -------------------------------------
// One Arnoldi step j: z_j = P v_j, w = calA z_j, classical Gram-Schmidt twice
// with fused multi-dot / multi-axpy, normalisation by a device-side 1/||w||.
// Results: h1 in hdev[0..j], h2 in hdev[64..64+j], ||w||^2 in hdev[128].
template <typename T>
void arnoldi_step_body(biot_ctx& c, double tau, int transpose, int j, cudaStream_t st) {
  Krylov<T>& K = c.kry<T>();
  const int64_t n = c.g.N * c.nt;
  double* hd = c.hdev;
  precondition_T<T>(c, tau, K.V[j], K.Z[j], transpose, st);
  apply_slab_T<T>(c, tau, K.Z[j], K.V[j + 1], transpose, st);
  T* w = K.V[j + 1];
  if (c.nb > 1) {
    // batched instances: every reduction and scalar per instance (block of HS scalars each)
    const Seg sg = slab_seg(c);
    launch_seg_multidot<T>(K.dV, j + 1, w, sg, c.partial, hd, HS, st);
    launch_seg_multiaxpy_dot<T>(K.dV, j + 1, hd, HS, w, sg, 1, c.partial, hd + 64, HS, st);
    launch_seg_multiaxpy_dot<T>(K.dV, j + 1, hd + 64, HS, w, sg, 2, c.partial, hd + 128, HS, st);
    launch_seg_scale<T>(w, w, hd + 129, HS, sg, st);
    CKL();
    return;
  }
  const T* const* Vh = K.V.data();  // host array of basis pointers (kernel parameters)
  launch_multidot<T>(Vh, j + 1, w, n, c.partial, hd, st);
  launch_multiaxpy_dot<T>(Vh, j + 1, hd, w, n, 1, c.partial, hd + 64, st);
  launch_multiaxpy_dot<T>(Vh, j + 1, hd + 64, w, n, 2, c.partial, hd + 128, st);
  launch_scale_into<T>(w, w, hd + 129, 0, n, st);  // hd[129] = 1/||w|| from the norm reduction
  CKL();
}

template <typename T> constexpr int prec_id();
template <> constexpr int prec_id<double>() { return 0; }
template <> constexpr int prec_id<float>() { return 1; }

// launch shapes of the FP32 z-marching elasticity kernel on every level that uses it, for each
// column count the solver launches (once per context; measured once per GPU and shape)
template <typename T>
void tune_levels(biot_ctx&, cudaStream_t) {}
template <>
void tune_levels<float>(biot_ctx& c, cudaStream_t st) {
  if (c.tuned || c.g.dim != 3) return;
  c.tuned = true;
  for (Level& L : c.lv) {
    if (L.g.nnode < ELAST3_MIN_NODES) continue;
    for (int k = 1; k <= c.nt; ++k) elast3_tune(L.g, L.t32, c.lam, c.mu, k * c.nb, L.w32.x, L.w32.Ax, st);
  }
  CKL();
}

// precompute what the preconditioner needs for this tau (host syncs, so never inside a capture)
template <typename T>
void prec_prepare(biot_ctx& c, double tau, cudaStream_t st) {
  ensure_prec<T>(c);
  tune_levels<T>(c, st);
  PrecWork<T>& w = c.pw<T>();
  double lm = schur_lmax(c, tau, st);
  (void)lm;
  if (w.schur_tau != tau) {
    schur_prepare<T>(c, tau, st);
    w.schur_tau = tau;
  }
}

template <typename T>
void arnoldi_step(biot_ctx& c, double tau, int transpose, int j, cudaStream_t st) {
  if (!c.use_graphs || prof_enabled()) {
    arnoldi_step_body<T>(c, tau, transpose, j, st);
    return;
  }
  GraphKey key{prec_id<T>(), transpose, j};
  auto it = c.graphs.find(key);
  if (it != c.graphs.end() && it->second.tau != tau) {
    cudaGraphExecDestroy(it->second.exec);
    c.graphs.erase(it);
    it = c.graphs.end();
  }
  if (it == c.graphs.end()) {
    cudaGraph_t gr;
    long long k0 = launch_count();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    arnoldi_step_body<T>(c, tau, transpose, j, st);
    CK(cudaStreamEndCapture(st, &gr));
    long long nk = launch_count() - k0;
    note_launches(-nk);  // captured, not launched
    cudaGraphExec_t ex;
    CK(cudaGraphInstantiate(&ex, gr, 0));
    cudaGraphDestroy(gr);
    GraphEntry e{ex, tau, nk};
    it = c.graphs.emplace(key, e).first;
  }
  CK(cudaGraphLaunch(it->second.exec, st));
  note_launches(it->second.kernels);
}

// Solves calA x = b (precision T) to ||b - calA x|| <= tol_abs.  Returns BIOT_OK,
// BIOT_ENOCONV or BIOT_EBREAKDOWN.  single_cycle: x = 0 on entry, one Arnoldi
// cycle only, no closing true residual (the mixed-precision inner solve; the
// outer FP64 refinement measures the true residual).
template <typename T>
int gmres(biot_ctx& c, double tau, int transpose, const T* b, T* x, double tol_abs, int maxit, int& iters, int& restarts,
          double& resnorm, cudaStream_t st, bool single_cycle = false) {
  const int m = c.opts.gmres_restart;
  ensure_krylov<T>(c, m);
  prec_prepare<T>(c, tau, st);
  Krylov<T>& K = c.kry<T>();
  const int64_t n = c.g.N * c.nt;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  double* hd = c.hdev;
  auto norm2 = [&](T* v) -> double {
    const T* vp[1] = {v};
    launch_multidot<T>(vp, 1, v, n, c.partial, hd + 128, st);
    CKL();
    CK(cudaMemcpyAsync(c.hhost + 128, hd + 128, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return c.hhost[128];
  };
  if (single_cycle) {
    CK(cudaMemcpyAsync(K.V[0], b, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  } else {
    apply_slab_T<T>(c, tau, x, K.V[0], transpose, st);
    launch_axpby<T>(K.V[0], b, 1.0, -1.0, n, st);
    CKL();
  }
  double beta = std::sqrt(norm2(K.V[0]));
  resnorm = beta;
  while (true) {
    if (!std::isfinite(beta)) return BIOT_EBREAKDOWN;
    if (beta <= tol_abs) return BIOT_OK;
    if (iters >= maxit) return BIOT_ENOCONV;
    launch_axpby<T>(K.V[0], K.V[0], 0.0, 1.0 / beta, n, st);
    CKL();
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jl = -1;
    for (int j = 0; j < m; ++j) {
      arnoldi_step<T>(c, tau, transpose, j, st);
      CK(cudaMemcpyAsync(c.hhost, hd, 130 * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i <= j; ++i) H[i * m + j] = c.hhost[i] + c.hhost[64 + i];
      double hn = std::sqrt(std::max(c.hhost[128], 0.0));
      if (!std::isfinite(hn)) return BIOT_EBREAKDOWN;
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double rr = std::hypot(a, bb);
      cs[j] = (rr > 0) ? a / rr : 1.0;
      sn[j] = (rr > 0) ? bb / rr : 0.0;
      H[j * m + j] = rr;
      H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++iters;
      jl = j;
      if (std::fabs(gv[j + 1]) <= tol_abs || iters >= maxit || hn == 0.0) break;
    }
    // y = H^{-1} g, x += Z y
    for (int i = jl; i >= 0; --i) {
      double s = gv[i];
      for (int k = i + 1; k <= jl; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    CK(cudaMemcpyAsync(hd + 160, y.data(), (jl + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    launch_lincomb_add<T, T>(x, K.dV + (m + 1), jl + 1, hd + 160, n, st);
    CKL();
    if (single_cycle) {
      resnorm = std::fabs(gv[jl + 1]);
      return BIOT_OK;
    }
    apply_slab_T<T>(c, tau, x, K.V[0], transpose, st);
    launch_axpby<T>(K.V[0], b, 1.0, -1.0, n, st);
    CKL();
    beta = std::sqrt(norm2(K.V[0]));
    resnorm = beta;
    ++restarts;
  }
}

// ---- batched solves ------------------------------------------------------------------
// Per-instance scalars round trip through the pinned bhost / device bdev columns: the
// first 4 nt nb entries serve the eigenvalue estimates, then slots of nb values each.
int64_t bslot(const biot_ctx& c, int slot) { return 4 * (int64_t)c.nt * c.nb + (int64_t)slot * c.nb; }
int64_t bdev_doubles(int nt, int nb) { return 4 * (int64_t)nt * nb + 10 * (int64_t)nb + 64; }
void put_scalars(biot_ctx& c, const std::vector<double>& v, int slot, cudaStream_t st) {
  // callers synchronise the stream before rewriting a slot
  std::memcpy(c.bhost + bslot(c, slot), v.data(), c.nb * sizeof(double));
  CK(cudaMemcpyAsync(c.bdev + bslot(c, slot), c.bhost + bslot(c, slot), c.nb * sizeof(double), cudaMemcpyHostToDevice, st));
}

// per-instance squared norms of a batched slab vector (synchronises st)
template <typename T>
std::vector<double> seg_norms2(biot_ctx& c, const T* v, int slot, cudaStream_t st) {
  c.hptr[16 + slot] = (void*)v;
  CK(cudaMemcpyAsync(c.ptrbuf + 16 + slot, c.hptr + 16 + slot, sizeof(void*), cudaMemcpyHostToDevice, st));
  launch_seg_multidot<T>(reinterpret_cast<const T* const*>(c.ptrbuf + 16 + slot), 1, v, slab_seg(c), c.partial,
                         c.bdev + bslot(c, 8), 1, st);
  CKL();
  CK(cudaMemcpyAsync(c.bhost + bslot(c, 8), c.bdev + bslot(c, 8), c.nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return std::vector<double>(c.bhost + bslot(c, 8), c.bhost + bslot(c, 9));
}

// One cycle of right-preconditioned FGMRES for every batched instance at once (x = 0 on
// entry).  All instances share the Arnoldi steps (each a graph of batch-wide launches);
// each keeps its own Hessenberg matrix, Givens rotations and stopping point: an instance
// stops contributing once its residual estimate falls below tol_abs[b] (inactive
// instances enter with b = 0 and stay at x = 0).  iters[b] counts the steps it used.
template <typename T>
void gmres_batch(biot_ctx& c, double tau, int transpose, const T* b, T* x, const std::vector<double>& tol_abs, int maxit,
                 std::vector<int>& iters, cudaStream_t st) {
  const int m = c.opts.gmres_restart;
  const int nb = c.nb;
  ensure_krylov<T>(c, m);
  prec_prepare<T>(c, tau, st);
  Krylov<T>& K = c.kry<T>();
  const int64_t n = c.g.N * c.nt * nb;
  const Seg sg = slab_seg(c);
  double* hd = c.hdev;
  CK(cudaMemcpyAsync(K.V[0], b, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  launch_seg_multidot<T>(K.dV, 1, K.V[0], sg, c.partial, hd + 128, HS, st);
  CKL();
  CK(cudaMemcpy2DAsync(c.hhost, HS * sizeof(double), hd, HS * sizeof(double), 130 * sizeof(double), nb,
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<double> beta(nb), scale(nb, 0.0);
  std::vector<char> alive(nb, 0);
  for (int i = 0; i < nb; ++i) {
    beta[i] = std::sqrt(std::max(c.hhost[(int64_t)i * HS + 128], 0.0));
    if (beta[i] > 0 && std::isfinite(beta[i]) && beta[i] > tol_abs[i]) {
      alive[i] = 1;
      scale[i] = 1.0 / beta[i];
    }
  }
  put_scalars(c, scale, 0, st);
  launch_seg_scale<T>(K.V[0], K.V[0], c.bdev + bslot(c, 0), 1, sg, st);
  CKL();
  std::vector<double> H((size_t)nb * (m + 1) * m, 0.0), cs((size_t)nb * m), sn((size_t)nb * m), gv((size_t)nb * (m + 1), 0.0);
  std::vector<int> jl(nb, -1);
  for (int i = 0; i < nb; ++i) gv[(size_t)i * (m + 1)] = alive[i] ? beta[i] : 0.0;
  int steps = 0;
  for (int j = 0; j < m && steps < maxit; ++j) {
    bool any = false;
    for (int i = 0; i < nb; ++i) any = any || alive[i];
    if (!any) break;
    arnoldi_step<T>(c, tau, transpose, j, st);
    CK(cudaMemcpy2DAsync(c.hhost, HS * sizeof(double), hd, HS * sizeof(double), 130 * sizeof(double), nb,
                         cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ++steps;
    for (int ib = 0; ib < nb; ++ib) {
      if (!alive[ib]) continue;
      const double* hh = c.hhost + (int64_t)ib * HS;
      double* Hb = H.data() + (size_t)ib * (m + 1) * m;
      double* csb = cs.data() + (size_t)ib * m;
      double* snb = sn.data() + (size_t)ib * m;
      double* gb = gv.data() + (size_t)ib * (m + 1);
      for (int i = 0; i <= j; ++i) Hb[i * m + j] = hh[i] + hh[64 + i];
      double hn = std::sqrt(std::max(hh[128], 0.0));
      if (!std::isfinite(hn)) { alive[ib] = 0; continue; }
      Hb[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        double a = Hb[i * m + j], bb = Hb[(i + 1) * m + j];
        Hb[i * m + j] = csb[i] * a + snb[i] * bb;
        Hb[(i + 1) * m + j] = -snb[i] * a + csb[i] * bb;
      }
      double a = Hb[j * m + j], bb = Hb[(j + 1) * m + j];
      double rr = std::hypot(a, bb);
      csb[j] = (rr > 0) ? a / rr : 1.0;
      snb[j] = (rr > 0) ? bb / rr : 0.0;
      Hb[j * m + j] = rr;
      Hb[(j + 1) * m + j] = 0.0;
      gb[j + 1] = -snb[j] * gb[j];
      gb[j] = csb[j] * gb[j];
      ++iters[ib];
      jl[ib] = j;
      if (std::fabs(gb[j + 1]) <= tol_abs[ib] || hn == 0.0) alive[ib] = 0;
    }
  }
  // y_b = H_b^{-1} g_b per instance, x += Z y (coefficients beyond an instance's last step are 0)
  int jmax = -1;
  for (int ib = 0; ib < nb; ++ib) jmax = std::max(jmax, jl[ib]);
  if (jmax < 0) return;
  for (int ib = 0; ib < nb; ++ib) {
    double* yb = c.hhost + (int64_t)ib * HS + 160;
    for (int i = 0; i <= jmax; ++i) yb[i] = 0.0;
    const double* Hb = H.data() + (size_t)ib * (m + 1) * m;
    const double* gb = gv.data() + (size_t)ib * (m + 1);
    for (int i = jl[ib]; i >= 0; --i) {
      double s = gb[i];
      for (int k = i + 1; k <= jl[ib]; ++k) s -= Hb[i * m + k] * yb[k];
      yb[i] = (Hb[i * m + i] != 0.0) ? s / Hb[i * m + i] : 0.0;
    }
  }
  CK(cudaMemcpy2DAsync(hd + 160, HS * sizeof(double), c.hhost + 160, HS * sizeof(double), (jmax + 1) * sizeof(double), nb,
                       cudaMemcpyHostToDevice, st));
  launch_seg_lincomb_add<T, T>(x, K.dV + (m + 1), jmax + 1, hd + 160, HS, sg, st);
  CKL();
  CK(cudaStreamSynchronize(st));  // hhost is rewritten by the next call
}

// Mixed-precision refinement of every batched instance (FP64 true residual and update,
// one FP32 FGMRES cycle per refinement step), each to its own relative tolerance.
// Per-instance results go to c.it_b / c.ref_b / c.res_b / c.rc_b.
int solve_slab_batch(biot_ctx& c, double tau, const double* rhs, double* x, const biot_solve_opts& o, biot_stats& s,
                     cudaStream_t st) {
  double t0 = now_s();
  const int nb = c.nb;
  const int64_t n = c.g.N * c.nt * nb;
  const Seg sg = slab_seg(c);
  if (o.mode != BIOT_MIXED) fail(BIOT_EINVAL, "batched contexts solve in BIOT_MIXED mode");
  c.it_b.assign(nb, 0);
  c.ref_b.assign(nb, 0);
  c.res_b.assign(nb, 0.0);
  c.rc_b.assign(nb, BIOT_OK);
  std::vector<double> bn = seg_norms2<double>(c, rhs, 0, st);
  for (double& v : bn) v = std::sqrt(v);
  for (int i = 0; i < nb; ++i)
    if (!std::isfinite(bn[i])) fail(BIOT_EINVAL, "non-finite right-hand side");
  if (!c.r64) c.r64 = dalloc<double>(n);
  if (!c.d32) c.d32 = dalloc<float>(n);
  if (!c.r32) c.r32 = dalloc<float>(n);
  {  // instances with a zero right-hand side have the zero solution
    std::vector<double> keep(nb);
    for (int i = 0; i < nb; ++i) keep[i] = bn[i] == 0.0 ? 0.0 : 1.0;
    put_scalars(c, keep, 1, st);
    launch_seg_scale<double>(x, x, c.bdev + bslot(c, 1), 1, sg, st);
    CKL();
  }
  std::vector<char> done(nb, 0);
  for (int i = 0; i < nb; ++i) done[i] = bn[i] == 0.0;
  int total = 0;
  while (true) {
    apply_slab_T<double>(c, tau, x, c.r64, o.transpose, st);
    launch_axpby<double>(c.r64, rhs, 1.0, -1.0, n, st);
    CKL();
    std::vector<double> rn = seg_norms2<double>(c, c.r64, 1, st);
    std::vector<double> sc(nb, 0.0), tol_in(nb, 0.0);
    bool any = false;
    for (int i = 0; i < nb; ++i) {
      rn[i] = std::sqrt(std::max(rn[i], 0.0));
      if (done[i]) continue;
      c.res_b[i] = rn[i] / bn[i];
      if (!std::isfinite(rn[i])) { c.rc_b[i] = BIOT_EBREAKDOWN; done[i] = 1; continue; }
      if (rn[i] <= o.tol * bn[i]) { done[i] = 1; continue; }
      if (c.it_b[i] >= o.max_iters || c.ref_b[i] >= 50) { c.rc_b[i] = BIOT_ENOCONV; done[i] = 1; continue; }
      sc[i] = 1.0 / rn[i];
      tol_in[i] = o.inner_tol;
      any = true;
    }
    if (!any) break;
    put_scalars(c, sc, 2, st);
    launch_seg_scale<double>(c.r64, c.r64, c.bdev + bslot(c, 2), 1, sg, st);
    launch_convert<double, float>(c.r64, c.r32, n, st);
    CK(cudaMemsetAsync(c.d32, 0, n * sizeof(float), st));
    CKL();
    std::vector<int> it_in(nb, 0);
    int budget = std::min(o.max_iters, c.opts.gmres_restart);
    gmres_batch<float>(c, tau, o.transpose, c.r32, c.d32, tol_in, budget, it_in, st);
    for (int i = 0; i < nb; ++i) {
      if (sc[i] == 0.0) { rn[i] = 0.0; continue; }
      c.it_b[i] += it_in[i];
      c.ref_b[i] += 1;
      total = std::max(total, c.it_b[i]);
    }
    put_scalars(c, rn, 3, st);  // x_b += ||r_b|| d_b (0 for finished instances)
    launch_seg_add_scaled<double, float>(x, c.d32, c.bdev + bslot(c, 3), 1, sg, st);
    CKL();
  }
  CK(cudaStreamSynchronize(st));
  int rc = BIOT_OK;
  double worst = 0;
  int refs_max = 0;
  for (int i = 0; i < nb; ++i) {
    if (c.rc_b[i] != BIOT_OK && rc == BIOT_OK) rc = c.rc_b[i];
    worst = std::max(worst, c.res_b[i]);
    refs_max = std::max(refs_max, c.ref_b[i]);
  }
  s.iterations = total;
  s.restarts = 0;
  s.refinements = refs_max;
  s.rel_residual = worst;
  s.seconds = now_s() - t0;
  return rc;
}

// Fixed-stress iterative coupling (paper §Iterative Coupling Approach): each sweep solves the
// flow problem with the volumetric mean stress held fixed (the beta Mp stabilisation of the
// flux-pressure block) and then the deformation problem with the pressure held fixed.  Here a
// sweep applies the block preconditioner's flow and displacement solves (for all temporal DoFs
// of the slab, through the time transform) to the current residual, z = P r, and relaxes it by
// the residual-minimising factor alpha = (r, calA z) / (calA z, calA z), so the residual norm
// never grows; x <- x + alpha z, all in FP64, until ||b - calA x|| <= tol ||b||.
int solve_fixed_stress(biot_ctx& c, double tau, const double* rhs, double* x, const biot_solve_opts& o, biot_stats& s,
                       cudaStream_t st) {
  const double t0 = now_s();
  const int64_t n = c.g.N * c.nt;
  if (c.nb > 1) fail(BIOT_EINVAL, "fixed-stress solves take a single instance");
  if (o.transpose) fail(BIOT_EINVAL, "fixed-stress solves are forward solves");
  ensure_prec<double>(c);
  prec_prepare<double>(c, tau, st);
  if (!c.r64) c.r64 = dalloc<double>(n);
  if (!c.a64) c.a64 = dalloc<double>(n);
  Krylov<double>& K = c.kry<double>();
  if (!K.tmp) ensure_krylov<double>(c, 1);
  double* r = c.r64;
  double* z = c.a64;
  double* w = K.tmp;
  const double bn = std::sqrt(dev_dot(c, rhs, rhs, n, st));
  if (!std::isfinite(bn)) fail(BIOT_EINVAL, "non-finite right-hand side");
  int it = 0, rc = BIOT_OK;
  apply_slab_T<double>(c, tau, x, r, 0, st);
  launch_axpby<double>(r, rhs, 1.0, -1.0, n, st);  // r = b - calA x
  CKL();
  double rn = std::sqrt(dev_dot(c, r, r, n, st));
  while (bn > 0 && rn > o.tol * bn) {
    if (!std::isfinite(rn)) { rc = BIOT_EBREAKDOWN; break; }
    if (it >= o.max_iters) { rc = BIOT_ENOCONV; break; }
    precondition_T<double>(c, tau, r, z, 0, st);  // flow with fixed mean stress, then deformation
    apply_slab_T<double>(c, tau, z, w, 0, st);
    const double rw = dev_dot(c, r, w, n, st), ww = dev_dot(c, w, w, n, st);
    const double alpha = ww > 0 ? rw / ww : 0.0;
    if (!(alpha != 0.0) || !std::isfinite(alpha)) { rc = BIOT_EBREAKDOWN; break; }
    launch_axpby<double>(x, z, alpha, 1.0, n, st);
    launch_axpby<double>(r, w, -alpha, 1.0, n, st);
    CKL();
    rn = std::sqrt(dev_dot(c, r, r, n, st));
    ++it;
  }
  if (bn == 0) CK(cudaMemsetAsync(x, 0, n * sizeof(double), st));
  // the true residual of the result (the recursively updated one drifts by rounding only)
  apply_slab_T<double>(c, tau, x, r, 0, st);
  launch_axpby<double>(r, rhs, 1.0, -1.0, n, st);
  CKL();
  rn = std::sqrt(dev_dot(c, r, r, n, st));
  s.iterations = it;
  s.restarts = 0;
  s.refinements = 0;
  s.rel_residual = bn > 0 ? rn / bn : 0.0;
  s.seconds = now_s() - t0;
  return rc;
}

// ---- slab solve ---------------------------------------------------------------------
int solve_slab_impl(biot_ctx& c, double tau, const double* rhs, double* x, const biot_solve_opts& o, biot_stats& s,
                    cudaStream_t st_user) {
  double t0 = now_s();
  // all solver work runs on the library's own (capturable) stream, ordered after the caller's stream
  CK(cudaEventRecord(c.ev_in, st_user));
  CK(cudaStreamWaitEvent(c.ws, c.ev_in, 0));
  cudaStream_t st = c.ws;
  struct Rejoin {
    biot_ctx& c;
    cudaStream_t su;
    ~Rejoin() {
      cudaEventRecord(c.ev_out, c.ws);
      cudaStreamWaitEvent(su, c.ev_out, 0);
    }
  } rejoin{c, st_user};
  NvtxRange range_solve("biot solve_slab");
  if (c.nb > 1) return solve_slab_batch(c, tau, rhs, x, o, s, st);
  if (o.mode == BIOT_FIXED_STRESS) return solve_fixed_stress(c, tau, rhs, x, o, s, st);
  const int64_t n = c.g.N * c.nt;
  int iters = 0, restarts = 0, refs = 0;
  double res = 0;
  int rc = BIOT_OK;
  // ||b||
  double bn = std::sqrt(dev_dot(c, rhs, rhs, n, st));
  if (!std::isfinite(bn)) fail(BIOT_EINVAL, "non-finite right-hand side");
  if (bn == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    s = biot_stats{0, 0, 0, 0.0, now_s() - t0};
    return BIOT_OK;
  }
  if (o.mode == BIOT_FP64) {
    rc = gmres<double>(c, tau, o.transpose, rhs, x, o.tol * bn, o.max_iters, iters, restarts, res, st);
  } else {
    if (!c.r64) c.r64 = dalloc<double>(n);
    if (!c.d32) c.d32 = dalloc<float>(n);
    if (!c.r32) c.r32 = dalloc<float>(n);
    while (true) {
      apply_slab_T<double>(c, tau, x, c.r64, o.transpose, st);
      launch_axpby<double>(c.r64, rhs, 1.0, -1.0, n, st);
      CKL();
      double rn = std::sqrt(dev_dot(c, c.r64, c.r64, n, st));
      res = rn;
      if (!std::isfinite(rn)) { rc = BIOT_EBREAKDOWN; break; }
      if (rn <= o.tol * bn) { rc = BIOT_OK; break; }
      if (iters >= o.max_iters || refs >= 50) { rc = BIOT_ENOCONV; break; }
      NvtxRange range_ref("biot FP32 inner solve");
      launch_axpby<double>(c.r64, c.r64, 0.0, 1.0 / rn, n, st);
      launch_convert<double, float>(c.r64, c.r32, n, st);
      CK(cudaMemsetAsync(c.d32, 0, n * sizeof(float), st));
      CKL();
      int it_in = 0, rs_in = 0;
      double res_in = 0;
      int budget = std::min(o.max_iters - iters, c.opts.gmres_restart);
      int rci = gmres<float>(c, tau, o.transpose, c.r32, c.d32, o.inner_tol, budget, it_in, rs_in, res_in, st, true);
      iters += it_in;
      restarts += rs_in;
      if (rci == BIOT_EBREAKDOWN) { rc = rci; break; }
      launch_add_scaled<double, float>(x, c.d32, rn, n, st);
      CKL();
      ++refs;
    }
  }
  s.iterations = iters;
  s.restarts = restarts;
  s.refinements = refs;
  s.rel_residual = res / bn;
  CK(cudaStreamSynchronize(st));
  s.seconds = now_s() - t0;
  return rc;
}

// ---- multigrid set-up ----------------------------------------------------------------
double level_lmax(biot_ctx& c, Level& L, cudaStream_t st) {
  LevelWork<double>& w = L.w64;
  auto op = [&](const double* x, double* y) { apply_A<double>(L, c.lam, c.mu, 1.0, x, y, 1, st); };
  return lanczos_lmax(c, op, L.dinv64, 0, L.g.Nu, L.g.Nu, 1, 24, w.x, w.xo, w.d, w.Ax, st);
}

void build_levels(biot_ctx& c, cudaStream_t st) {
  Grid g = c.g;
  int minc = std::max(1, c.opts.mg_min_cells);
  c.lv.clear();
  while (true) {
    Level L;
    L.g = g;
    build_tables(g, L.t64);
    L.t32 = cast_tables<float>(L.t64);
    c.lv.push_back(L);
    bool can = true;
    for (int d = 0; d < g.dim; ++d)
      if (g.n[d] % 2 != 0 || g.n[d] / 2 < minc) can = false;
    if (!can) break;
    g = coarsen(g);
  }
  for (Level& L : c.lv) {
    int64_t n = L.g.Nu;
    L.dinv64 = dalloc<double>(n);
    L.dinv32 = dalloc<float>(n);
    launch_diag_A<double>(L.g, L.t64, c.lam, c.mu, L.dinv64, st);
    CKL();
    // invert (constrained -> 0)
    std::vector<double> h(n);
    CK(cudaMemcpy(h.data(), L.dinv64, n * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> hm(n, 1.0);
    {
      // constraint flags from a masked vector of ones
      double* ones = dalloc<double>(L.g.N);
      std::vector<double> o(L.g.N, 1.0);
      CK(cudaMemcpy(ones, o.data(), L.g.N * sizeof(double), cudaMemcpyHostToDevice));
      launch_mask<double>(L.g, ones, L.g.N, 1, st);
      CKL();
      CK(cudaMemcpy(hm.data(), ones, n * sizeof(double), cudaMemcpyDeviceToHost));
      cudaFree(ones);
    }
    std::vector<float> hf(n);
    for (int64_t i = 0; i < n; ++i) {
      h[i] = hm[i] != 0.0 ? 1.0 / h[i] : 0.0;
      hf[i] = (float)h[i];
    }
    CK(cudaMemcpy(L.dinv64, h.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.dinv32, hf.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  }
  ensure_prec<double>(c);
  for (Level& L : c.lv) L.lmax = level_lmax(c, L, st);
  // dense coarse inverse when the coarsest level is small
  Level& Lc = c.lv.back();
  int64_t nc = Lc.g.Nu;
  c.Ainv = nullptr;
  c.ncoarse = 0;
  if (nc <= 1500) {
    std::vector<double> A(nc * nc);
    double* e = dalloc<double>(3 * nc);
    double* ae = dalloc<double>(3 * nc);
    std::vector<double> eh(3 * nc), aeh(3 * nc);
    for (int64_t j0 = 0; j0 < nc; j0 += 3) {
      int cnt = (int)std::min<int64_t>(3, nc - j0);
      std::fill(eh.begin(), eh.end(), 0.0);
      for (int k = 0; k < cnt; ++k) eh[k * nc + j0 + k] = 1.0;
      CK(cudaMemcpy(e, eh.data(), 3 * nc * sizeof(double), cudaMemcpyHostToDevice));
      apply_A<double>(Lc, c.lam, c.mu, 1.0, e, ae, cnt, st);
      CK(cudaMemcpy(aeh.data(), ae, 3 * nc * sizeof(double), cudaMemcpyDeviceToHost));
      for (int k = 0; k < cnt; ++k)
        for (int64_t i = 0; i < nc; ++i) A[i * nc + j0 + k] = aeh[k * nc + i];
    }
    cudaFree(e);
    cudaFree(ae);
    // Cholesky-based inverse (FP64, host, set-up only)
    std::vector<double> Lm(nc * nc, 0.0);
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t j = 0; j <= i; ++j) {
        double s = 0.5 * (A[i * nc + j] + A[j * nc + i]);
        for (int64_t k = 0; k < j; ++k) s -= Lm[i * nc + k] * Lm[j * nc + k];
        if (i == j) {
          if (s <= 0) fail(BIOT_EINVAL, "coarse elasticity matrix is not positive definite (check boundary conditions)");
          Lm[i * nc + i] = std::sqrt(s);
        } else
          Lm[i * nc + j] = s / Lm[j * nc + j];
      }
    // inverse of L (lower), then A^{-1} = L^{-T} L^{-1}
    std::vector<double> Li(nc * nc, 0.0);
    for (int64_t j = 0; j < nc; ++j) {
      Li[j * nc + j] = 1.0 / Lm[j * nc + j];
      for (int64_t i = j + 1; i < nc; ++i) {
        double s = 0;
        for (int64_t k = j; k < i; ++k) s -= Lm[i * nc + k] * Li[k * nc + j];
        Li[i * nc + j] = s / Lm[i * nc + i];
      }
    }
    std::vector<double> Ai(nc * nc);
    for (int64_t i = 0; i < nc; ++i)
      for (int64_t j = 0; j <= i; ++j) {
        double s = 0;
        for (int64_t k = i; k < nc; ++k) s += Li[k * nc + i] * Li[k * nc + j];
        Ai[i * nc + j] = Ai[j * nc + i] = (double)s;
      }
    c.Ainv = dalloc<double>(nc * nc);
    CK(cudaMemcpy(c.Ainv, Ai.data(), nc * nc * sizeof(double), cudaMemcpyHostToDevice));
    c.ncoarse = (int)nc;
  }
}

// K: nb * n_cells values (instance-major for a batched context)
void set_permeability(biot_ctx& c, const double* K, cudaStream_t st) {
  const int64_t nc = c.g.ncells * c.nb;
  std::vector<double> ks(nc);
  std::vector<float> kf(nc);
  for (int64_t i = 0; i < nc; ++i) {
    if (!(K[i] > 0.0) || !std::isfinite(K[i])) fail(BIOT_EINVAL, "permeability must be positive and finite");
    ks[i] = c.eta / K[i];
    kf[i] = (float)ks[i];
  }
  c.Kcell.assign(K, K + nc);
  CK(cudaMemcpyAsync(c.kscale64, ks.data(), nc * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c.kscale32, kf.data(), nc * sizeof(float), cudaMemcpyHostToDevice, st));
  const Grid& g = c.g;
  const int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  for (int b = 0; b < c.nb; ++b) {
    launch_diag_Mq<double>(g, c.t64, c.kscale64 + b * g.ncells, c.dmq64 + b * nqt, st);
    launch_diag_Mq<float>(g, c.t32, c.kscale32 + b * g.ncells, c.dmq32 + b * nqt, st);
    launch_diag_BDBt<double>(g, c.t64, c.dmq64 + b * nqt, c.sb2_64 + b * g.Np, st);
    launch_diag_BDBt<float>(g, c.t32, c.dmq32 + b * nqt, c.sb2_32 + b * g.Np, st);
  }
  CKL();
  CK(cudaStreamSynchronize(st));
  c.schur_lmax_tau = -1;
  c.p64.schur_tau = -1;
  c.p32.schur_tau = -1;
  // captured Arnoldi steps carry the Chebyshev coefficients of the old Schur bounds
  for (auto& kv : c.graphs) cudaGraphExecDestroy(kv.second.exec);
  c.graphs.clear();
}

// ---- loads ---------------------------------------------------------------------------
// time integrals c[k][m] = tau int_0^1 g_m(t0 + tau s) l_k(s) ds (6-point Gauss, exact for the cubic profiles)
void time_load_coefs(const biot_ctx& c, double t0, double tau, int nterms, const double* tcoef, double* out) {
  static const double gx[6] = {-0.9324695142031521, -0.6612093864662645, -0.2386191860831969,
                               0.2386191860831969, 0.6612093864662645, 0.9324695142031521};
  static const double gw[6] = {0.1713244923791704, 0.3607615730481386, 0.4679139345726910,
                               0.4679139345726910, 0.3607615730481386, 0.1713244923791704};
  long double x[MAXR];
  for (int k = 0; k < c.nt; ++k) x[k] = c.tb.nodes[k];
  for (int k = 0; k < c.nt; ++k)
    for (int m = 0; m < nterms; ++m) {
      double s = 0;
      for (int q = 0; q < 6; ++q) {
        double sq = 0.5 * (gx[q] + 1.0), w = 0.5 * gw[q];
        double t = t0 + tau * sq;
        const double* a = tcoef + 4 * m;
        double gm = a[0] + t * (a[1] + t * (a[2] + t * a[3]));
        s += w * gm * (double)lagr(x, c.nt, k, sq);
      }
      out[k * nterms + m] = tau * s;
    }
}

struct MarchBufs {
  const double** fdev = nullptr;
  double* U = nullptr;
  double* SU = nullptr;  // one level
  double* rhs = nullptr;
  double* X = nullptr;
};

// The march buffers live in the context (allocated on first use, reused by every later
// march, freed by biot_destroy), so repeated marches allocate nothing.
void march_prepare(biot_ctx& c, int nterms, const double* const* f_terms, const double* U0, MarchBufs& mb, cudaStream_t st) {
  const Grid& g = c.g;
  if (nterms < 0 || nterms > 8) fail(BIOT_EINVAL, "nterms must be in 0..8");
  if (!c.m_U) {
    for (int m = 0; m < 8; ++m) c.m_f[m] = dalloc<double>(g.N);
    c.m_fdev = (const double**)dalloc<double*>(8);
    CK(cudaMemcpy((void*)c.m_fdev, c.m_f, 8 * sizeof(double*), cudaMemcpyHostToDevice));
    CK(cudaDeviceSynchronize());  // the pageable copy above runs on the legacy stream
    c.m_U = dalloc<double>(g.N);
    c.m_SU = dalloc<double>(g.N);
    c.m_rhs = dalloc<double>(g.N * c.nt);
    c.m_X = dalloc<double>(g.N * c.nt);
  }
  for (int m = 0; m < nterms; ++m) {
    if (!f_terms[m]) fail(BIOT_EINVAL, "NULL load term");
    CK(cudaMemcpyAsync(c.m_f[m], f_terms[m], g.N * sizeof(double),
                       is_device_ptr(f_terms[m]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    launch_mask<double>(g, c.m_f[m], g.N, 1, st);
    CKL();
  }
  mb.fdev = c.m_fdev;
  mb.U = c.m_U;
  mb.SU = c.m_SU;
  mb.rhs = c.m_rhs;
  mb.X = c.m_X;
  if (U0) CK(cudaMemcpyAsync(mb.U, U0, g.N * sizeof(double), is_device_ptr(U0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  else CK(cudaMemsetAsync(mb.U, 0, g.N * sizeof(double), st));
  CK(cudaStreamSynchronize(st));
}

// rhs of slab n from the loads and the jump term of the state mb.U
void build_slab_rhs(biot_ctx& c, double t0, double tau, int nterms, const double* tcoef, MarchBufs& mb, cudaStream_t st) {
  const Grid& g = c.g;
  SlabCoef s;
  std::memset(&s, 0, sizeof(s));
  s.nt = 1;
  s.pu[0][0] = c.b;
  s.pp[0][0] = c.invM;
  launch_apply_p<double>(g, c.t64, s, mb.U, g.N, mb.SU, g.N, st);
  CKL();
  std::vector<double> coef(c.nt * std::max(1, nterms), 0.0);
  if (nterms) time_load_coefs(c, t0, tau, nterms, tcoef, coef.data());
  launch_slab_rhs(g, mb.fdev, nterms, coef.data(), c.tb.phi0, c.nt, mb.SU + g.offp, mb.rhs, g.N, st);
  CKL();
}

// Slabs first .. first + count - 1 of the uniform partition of (0, T] into `slabs` slabs, from
// the state U0 = U(t_first^-).  X_all, ckpt and iters are indexed from the first marched slab.
void march_impl(biot_ctx& c, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                const double* U0, double* U_end, double* X_all, double* ckpt, const biot_solve_opts& o, int* iters,
                biot_stats& st_out, cudaStream_t st, int& rc_out, int first = 0, int count = -1) {
  double t_start = now_s();
  const Grid& g = c.g;
  NvtxRange range_march("biot march");
  MarchBufs mb;
  march_prepare(c, nterms, f_terms, U0, mb, st);
  const double tau = T / slabs;
  if (count < 0) count = slabs - first;
  biot_stats tot{0, 0, 0, 0.0, 0.0};
  rc_out = BIOT_OK;
  for (int nsl = 0; nsl < count; ++nsl) {
    NvtxRange range_slab("biot slab");
    if (ckpt) CK(cudaMemcpyAsync(ckpt + (int64_t)nsl * g.N, mb.U, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    build_slab_rhs(c, (first + nsl) * tau, tau, nterms, tcoef, mb, st);
    for (int k = 0; k < c.nt; ++k) CK(cudaMemcpyAsync(mb.X + k * g.N, mb.U, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    biot_stats s;
    int rc = solve_slab_impl(c, tau, mb.rhs, mb.X, o, s, st);
    if (rc != BIOT_OK && rc_out == BIOT_OK) rc_out = rc;
    tot.iterations += s.iterations;
    tot.refinements += s.refinements;
    tot.restarts += s.restarts;
    tot.rel_residual = std::max(tot.rel_residual, s.rel_residual);
    if (iters) iters[nsl] = s.iterations;
    if (X_all) CK(cudaMemcpyAsync(X_all + (int64_t)nsl * g.N * c.nt, mb.X, g.N * c.nt * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(mb.U, mb.X + (int64_t)(c.nt - 1) * g.N, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  if (ckpt) CK(cudaMemcpyAsync(ckpt + (int64_t)count * g.N, mb.U, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (U_end) CK(cudaMemcpyAsync(U_end, mb.U, g.N * sizeof(double), is_device_ptr(U_end) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  tot.seconds = now_s() - t_start;
  st_out = tot;
}

// March every batched instance over the same slabs (paper §Discretisation in Time).
// Instance b has its own load terms f_terms[b * nterms + m] (n_space each, host or device),
// initial state U0[b] and end state U_end[b]; the time profiles tcoef are shared.
void march_batch_impl(biot_ctx& c, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                      const double* const* U0, double* const* U_end, const biot_solve_opts& o, int* iters, biot_stats* sb,
                      int* status, cudaStream_t st) {
  const Grid& g = c.g;
  const int nb = c.nb;
  const int64_t N = g.N, LN = c.lvN();
  if (nterms < 0 || nterms > 8) fail(BIOT_EINVAL, "nterms must be in 0..8");
  const int mt = std::max(1, nterms);
  if (!c.bm_U || c.bm_terms < mt) {
    if (c.bm_f) cudaFree(c.bm_f);
    c.bm_f = dalloc<double>((int64_t)nb * mt * N);
    c.bm_terms = mt;
  }
  if (!c.bm_U) {
    c.bm_fdev = (const double**)dalloc<double*>((int64_t)nb * 8);
    c.bm_U = dalloc<double>(LN);
    c.bm_SU = dalloc<double>(LN);
    c.bm_rhs = dalloc<double>(LN * c.nt);
    c.bm_X = dalloc<double>(LN * c.nt);
  }
  std::vector<const double*> tab((size_t)nb * 8, nullptr);
  for (int b = 0; b < nb; ++b)
    for (int m = 0; m < nterms; ++m) {
      const double* src = f_terms[(size_t)b * nterms + m];
      if (!src) fail(BIOT_EINVAL, "NULL load term");
      double* dst = c.bm_f + ((int64_t)b * mt + m) * N;
      CK(cudaMemcpyAsync(dst, src, N * sizeof(double), is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      tab[(size_t)b * 8 + m] = dst;
    }
  // pageable source: the copy is staged before the call returns and ordered on st
  CK(cudaMemcpyAsync((void*)c.bm_fdev, tab.data(), tab.size() * sizeof(double*), cudaMemcpyHostToDevice, st));
  launch_mask<double>(g, c.bm_f, N, nb * mt, st);
  CKL();
  for (int b = 0; b < nb; ++b) {
    const double* u0 = U0 ? U0[b] : nullptr;
    if (u0) CK(cudaMemcpyAsync(c.bm_U + b * N, u0, N * sizeof(double), is_device_ptr(u0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    else CK(cudaMemsetAsync(c.bm_U + b * N, 0, N * sizeof(double), st));
  }
  CK(cudaStreamSynchronize(st));
  const double tau = T / slabs;
  for (int b = 0; b < nb; ++b) {
    sb[b] = biot_stats{0, 0, 0, 0.0, 0.0};
    status[b] = BIOT_OK;
    if (iters) iters[b] = 0;
  }
  double t_start = now_s();
  SlabCoef sj;
  std::memset(&sj, 0, sizeof(sj));
  sj.nt = 1;
  sj.pu[0][0] = c.b;
  sj.pp[0][0] = c.invM;
  std::vector<double> coef(c.nt * mt, 0.0);
  for (int nsl = 0; nsl < slabs; ++nsl) {
    // right-hand sides: loads integrated over the slab plus the jump term S U(t_{n-1}^-)
    launch_apply_p<double>(g, c.t64, sj, c.bm_U, N, c.bm_SU, N, st);
    if (nterms) time_load_coefs(c, nsl * tau, tau, nterms, tcoef, coef.data());
    for (int b = 0; b < nb; ++b)
      launch_slab_rhs(g, c.bm_fdev + (size_t)b * 8, nterms, coef.data(), c.tb.phi0, c.nt, c.bm_SU + b * N + g.offp,
                      c.bm_rhs + b * N, LN, st);
    CKL();
    for (int k = 0; k < c.nt; ++k) CK(cudaMemcpyAsync(c.bm_X + k * LN, c.bm_U, LN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    biot_stats s;
    solve_slab_impl(c, tau, c.bm_rhs, c.bm_X, o, s, st);
    for (int b = 0; b < nb; ++b) {
      sb[b].iterations += c.it_b[b];
      sb[b].refinements += c.ref_b[b];
      sb[b].rel_residual = std::max(sb[b].rel_residual, c.res_b[b]);
      if (iters) iters[b] += c.it_b[b];
      if (c.rc_b[b] != BIOT_OK && status[b] == BIOT_OK) status[b] = c.rc_b[b];  // first failing slab's code
    }
    CK(cudaMemcpyAsync(c.bm_U, c.bm_X + (int64_t)(c.nt - 1) * LN, LN * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  for (int b = 0; b < nb; ++b)
    if (U_end && U_end[b])
      CK(cudaMemcpyAsync(U_end[b], c.bm_U + b * N, N * sizeof(double),
                         is_device_ptr(U_end[b]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double secs = now_s() - t_start;
  for (int b = 0; b < nb; ++b) sb[b].seconds = secs;
}

biot_solve_opts solve_defaults(const biot_solve_opts* o) {
  biot_solve_opts d;
  d.tol = 1e-10;
  d.max_iters = 2000;
  d.mode = BIOT_FP64;
  d.inner_tol = 1e-5;
  d.transpose = 0;
  if (o) {
    d = *o;
    if (d.tol <= 0) d.tol = 1e-10;
    if (d.max_iters <= 0) d.max_iters = 2000;
    if (d.inner_tol <= 0) d.inner_tol = 1e-5;
  }
  if (d.mode != BIOT_FP64 && d.mode != BIOT_MIXED && d.mode != BIOT_FIXED_STRESS)
    fail(BIOT_EINVAL, "solve mode must be BIOT_FP64, BIOT_MIXED or BIOT_FIXED_STRESS");
  return d;
}


}  // namespace

// ---------------------------------------------------------------------------
// exported entry points
#define API_BEGIN(ctx)         \
  try {                        \
    if (!(ctx)) { g_err_msg = "NULL context"; return BIOT_EINVAL; }
#define API_END(ctx)                                  \
  }                                                   \
  catch (const Err& e) {                              \
    (ctx)->err = g_err_msg;                           \
    return e.code;                                    \
  }                                                   \
  catch (const std::exception& e) {                   \
    (ctx)->err = e.what();                            \
    return BIOT_ENOMEM;                               \
  }

namespace {
int setup_impl(const biot_mesh* mesh, const biot_coeffs* co, int r, const biot_opts* opts, int nb, biot_t* out) {
  if (!out || !mesh || !co) return BIOT_EINVAL;
  *out = nullptr;
  biot_ctx* c = new biot_ctx();
  try {
    if (nb < 1 || nb > 4096) fail(BIOT_EINVAL, "batch size must be in 1..4096");
    c->nb = nb;
    if (mesh->dim != 2 && mesh->dim != 3) fail(BIOT_EINVAL, "dim must be 2 or 3");
    for (int d = 0; d < mesh->dim; ++d) {
      if (mesh->n[d] < 1) fail(BIOT_EINVAL, "n must be >= 1");
      if (!(mesh->hi[d] > mesh->lo[d])) fail(BIOT_EINVAL, "hi must exceed lo");
    }
    for (int f = 0; f < 2 * mesh->dim; ++f) {
      if (mesh->u_bc[f] < 0 || mesh->u_bc[f] > 2) fail(BIOT_EINVAL, "bad u_bc code");
      if (mesh->f_bc[f] < 0 || mesh->f_bc[f] > 1) fail(BIOT_EINVAL, "bad f_bc code");
    }
    if (r < 0 || r > 2) fail(BIOT_EINVAL, "r must be 0, 1 or 2");
    if (!(co->b > 0 && co->b < 1)) fail(BIOT_EINVAL, "b must lie in (0, 1)");
    if (!(co->invM >= 0) || !(co->K_dr > 0) || !(co->mu > 0) || !(co->lambda >= 0) || !(co->eta > 0))
      fail(BIOT_EINVAL, "coefficients out of range");
    if (!co->K_cell) fail(BIOT_EINVAL, "K_cell is NULL");
    for (double v : {co->b, co->invM, co->K_dr, co->lambda, co->mu, co->eta})
      if (!std::isfinite(v)) fail(BIOT_EINVAL, "coefficients must be finite");
    {
      // every permeability is checked on the host before the first CUDA call
      int64_t ncell_all = nb;
      for (int d = 0; d < mesh->dim; ++d) ncell_all *= mesh->n[d];
      for (int64_t i = 0; i < ncell_all; ++i)
        if (!(co->K_cell[i] > 0.0) || !std::isfinite(co->K_cell[i])) {
          char buf[128];
          snprintf(buf, sizeof(buf), "K_cell[%lld] = %g: permeabilities must be positive and finite", (long long)i,
                   co->K_cell[i]);
          fail(BIOT_EINVAL, buf);
        }
    }
    apply_init_attributes();
    {
      const char* ng = std::getenv("BIOT_NO_GRAPHS");
      c->use_graphs = !(ng && ng[0] == '1');
    }
    c->g = make_grid(mesh->dim, mesh->n, mesh->lo, mesh->hi, mesh->u_bc, mesh->f_bc);
    c->g.nb = nb;
    // the kernels index one temporal level of one instance with 32-bit integers
    if (c->g.N >= (int64_t)1 << 31) fail(BIOT_EINVAL, "mesh too large: 2^31 or more unknowns per temporal level");
    c->r = r;
    c->nt = r + 1;
    c->b = co->b;
    c->invM = co->invM;
    c->Kdr = co->K_dr;
    c->lam = co->lambda;
    c->mu = co->mu;
    c->eta = co->eta;
    biot_opts d;
    d.gmres_restart = 30;
    d.cheb_degree = 3;
    d.schur_degree = 0;  // chosen per tau from the spectral bounds
    d.mg_min_cells = 2;
    d.beta_fs = -1;
    d.flux_mass_exact = 0;
    d.pair_coupling = 1;
    d.schur_mg = 0;
    if (opts) {
      if (opts->gmres_restart > 0) d.gmres_restart = std::min(opts->gmres_restart, 60);
      if (opts->cheb_degree > 0) d.cheb_degree = std::min(opts->cheb_degree, MAX_CHEB);
      if (opts->schur_degree > 0) d.schur_degree = std::min(opts->schur_degree, MAX_CHEB);
      if (opts->mg_min_cells > 0) d.mg_min_cells = opts->mg_min_cells;
      d.beta_fs = opts->beta_fs;
      d.flux_mass_exact = opts->flux_mass_exact ? 1 : 0;
      d.pair_coupling = opts->pair_coupling >= 0 ? 1 : 0;
      d.schur_mg = opts->schur_mg > 0 ? 1 : (opts->schur_mg < 0 ? -1 : 0);
    }
    c->opts = d;
    c->lumped_flux = d.flux_mass_exact ? 0 : 1;
    if (nb > 1 && !c->lumped_flux) fail(BIOT_EINVAL, "batched contexts use the lumped Darcy mass (flux_mass_exact = 0)");
    c->beta = (d.beta_fs > 0) ? d.beta_fs : c->b * c->b / c->Kdr;
    build_tables(c->g, c->t64);
    c->t32 = cast_tables<float>(c->t64);
    c->tb = make_time_basis(r);
    const Grid& g = c->g;
    int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
    c->kscale64 = dalloc<double>(g.ncells * nb);
    c->kscale32 = dalloc<float>(g.ncells * nb);
    c->dmq64 = dalloc<double>(nqt * nb);
    c->dmq32 = dalloc<float>(nqt * nb);
    c->sb2_64 = dalloc<double>(g.Np * nb);
    c->sb2_32 = dalloc<float>(g.Np * nb);
    c->hdev = dalloc<double>((int64_t)HS * nb + 256);
    c->bdev = dalloc<double>(bdev_doubles(c->nt, nb));

    CK(cudaStreamCreateWithFlags(&c->ws, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    c->ptrbuf = dalloc<void*>(64);
    CK(cudaMallocHost((void**)&c->hptr, 64 * sizeof(void*)));
    CK(cudaMallocHost((void**)&c->hhost, ((int64_t)HS * nb + 256) * sizeof(double)));
    CK(cudaMallocHost((void**)&c->bhost, bdev_doubles(c->nt, nb) * sizeof(double)));
    c->partial = dalloc<double>(
        std::max<int64_t>(RED_BLOCKS * 32, std::max(seg_partial_doubles(c->nt * nb), seg_partial_doubles(nb))));
    c->lvl64 = dalloc<double>(g.N);
    c->lvl64b = dalloc<double>(g.N);
    cudaStream_t st = 0;  // set-up runs on the legacy stream, ordered with its synchronous copies
    set_permeability(*c, co->K_cell, st);
    build_levels(*c, st);
    CK(cudaStreamSynchronize(st));
  } catch (const Err& e) {
    biot_destroy(c);
    return e.code;
  } catch (const std::exception& e) {
    g_err_msg = e.what();
    biot_destroy(c);
    return BIOT_ENOMEM;
  }
  *out = c;
  return BIOT_OK;
}
}  // namespace

extern "C" int biot_time_tables(int r, double* nodes, double* w, double* phi0, double* D, double* V, double* W, double* lam,
                                int* pair, double* pair_beta) {
  if (r < 0 || r > 2) return BIOT_EINVAL;
  const TimeBasis tb = make_time_basis(r);
  const int nt = r + 1;
  for (int k = 0; k < nt; ++k) {
    if (nodes) nodes[k] = tb.nodes[k];
    if (w) w[k] = tb.w[k];
    if (phi0) phi0[k] = tb.phi0[k];
    if (lam) lam[k] = tb.lam[k];
    for (int l = 0; l < nt; ++l) {
      if (D) D[k * nt + l] = tb.D[k][l];
      if (V) V[k * nt + l] = tb.V[k][l];
      if (W) W[k * nt + l] = tb.W[k][l];
    }
  }
  if (pair) *pair = tb.pair;
  if (pair_beta) *pair_beta = tb.pair_beta;
  return BIOT_OK;
}

extern "C" int biot_setup(const biot_mesh* mesh, const biot_coeffs* co, int r, const biot_opts* opts, biot_t* out) {
  return setup_impl(mesh, co, r, opts, 1, out);
}

extern "C" int biot_setup_batch(const biot_mesh* mesh, const biot_coeffs* co, int r, const biot_opts* opts, int nb,
                                biot_t* out) {
  return setup_impl(mesh, co, r, opts, nb, out);
}

extern "C" int biot_sizes(biot_t c, int64_t* n_space, int64_t* n_slab, int64_t* n_cells) {
  if (!c) return BIOT_EINVAL;
  if (n_space) *n_space = c->g.N;
  if (n_slab) *n_slab = c->g.N * c->nt;
  if (n_cells) *n_cells = c->g.ncells;
  return BIOT_OK;
}

extern "C" int biot_set_permeability(biot_t c, const double* K) {
  API_BEGIN(c)
  if (!K) fail(BIOT_EINVAL, "K is NULL");
  set_permeability(*c, K, 0);
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_set_log_permeability(biot_t c, const double* g, double K0) {
  API_BEGIN(c)
  if (!g) fail(BIOT_EINVAL, "log-permeability is NULL");
  if (!(K0 > 0) || !std::isfinite(K0)) fail(BIOT_EINVAL, "K0 must be positive and finite");
  const int64_t nc = c->g.ncells * c->nb;
  std::vector<double> K(nc);
  for (int64_t i = 0; i < nc; ++i) K[i] = K0 * std::exp(g[i]);  // non-finite results are rejected below
  set_permeability(*c, K.data(), 0);
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_apply_slab(biot_t c, double tau, const void* x, void* y, int prec, int transpose, void* stream) {
  API_BEGIN(c)
  if (!x || !y || !(tau > 0)) fail(BIOT_EINVAL, "apply_slab: NULL vector or tau <= 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == BIOT_FP64) apply_slab_T<double>(*c, tau, (const double*)x, (double*)y, transpose, st);
  else if (prec == BIOT_FP32) apply_slab_T<float>(*c, tau, (const float*)x, (float*)y, transpose, st);
  else fail(BIOT_EINVAL, "prec must be BIOT_FP64 or BIOT_FP32");
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_precondition(biot_t c, double tau, const void* r, void* z, int prec, int transpose, void* stream) {
  API_BEGIN(c)
  if (!r || !z || !(tau > 0)) fail(BIOT_EINVAL, "precondition: NULL vector or tau <= 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == BIOT_FP64) {
    ensure_prec<double>(*c);
    precondition_T<double>(*c, tau, (const double*)r, (double*)z, transpose, st);
  } else if (prec == BIOT_FP32) {
    ensure_prec<float>(*c);
    precondition_T<float>(*c, tau, (const float*)r, (float*)z, transpose, st);
  } else
    fail(BIOT_EINVAL, "prec must be BIOT_FP64 or BIOT_FP32");
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_solve_slab(biot_t c, double tau, const double* rhs, double* x, const biot_solve_opts* opts, biot_stats* stats,
                               void* stream) {
  API_BEGIN(c)
  if (!rhs || !x || !(tau > 0)) fail(BIOT_EINVAL, "solve_slab: NULL vector or tau <= 0");
  biot_solve_opts o = solve_defaults(opts);
  biot_stats s{0, 0, 0, 0.0, 0.0};
  int rc = solve_slab_impl(*c, tau, rhs, x, o, s, (cudaStream_t)stream);
  if (stats) *stats = s;
  if (rc != BIOT_OK) c->err = (rc == BIOT_ENOCONV) ? "iteration limit reached" : "breakdown (non-finite values)";
  return rc;
  API_END(c)
}

extern "C" int biot_march(biot_t c, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                          const double* U0, double* U_end, double* X_all, const biot_solve_opts* opts, int* iters_per_slab,
                          biot_stats* stats, void* stream) {
  API_BEGIN(c)
  if (!(T > 0) || slabs < 1) fail(BIOT_EINVAL, "march: T must be > 0 and slabs >= 1");
  if (nterms > 0 && (!f_terms || !tcoef)) fail(BIOT_EINVAL, "march: load terms missing");
  if (c->nb > 1) fail(BIOT_EINVAL, "march: batched context (use biot_march_batch)");
  biot_solve_opts o = solve_defaults(opts);
  biot_stats s{0, 0, 0, 0.0, 0.0};
  int rc = BIOT_OK;
  march_impl(*c, T, slabs, nterms, f_terms, tcoef, U0, U_end, X_all, nullptr, o, iters_per_slab, s, (cudaStream_t)stream, rc);
  if (stats) *stats = s;
  return rc;
  API_END(c)
}

extern "C" int biot_march_resume(biot_t c, double T, int slabs, int first, int count, int nterms, const double* const* f_terms,
                                 const double* tcoef, const double* U_first, double* U_end, double* X_all,
                                 const biot_solve_opts* opts, int* iters_per_slab, biot_stats* stats, void* stream) {
  API_BEGIN(c)
  if (!(T > 0) || slabs < 1) fail(BIOT_EINVAL, "march_resume: T must be > 0 and slabs >= 1");
  if (first < 0 || count < 1 || first + count > slabs) fail(BIOT_EINVAL, "march_resume: need 0 <= first < first + count <= slabs");
  if (nterms > 0 && (!f_terms || !tcoef)) fail(BIOT_EINVAL, "march_resume: load terms missing");
  if (c->nb > 1) fail(BIOT_EINVAL, "march_resume: batched context");
  biot_solve_opts o = solve_defaults(opts);
  biot_stats s{0, 0, 0, 0.0, 0.0};
  int rc = BIOT_OK;
  march_impl(*c, T, slabs, nterms, f_terms, tcoef, U_first, U_end, X_all, nullptr, o, iters_per_slab, s, (cudaStream_t)stream, rc,
             first, count);
  if (stats) *stats = s;
  return rc;
  API_END(c)
}

extern "C" int biot_march_batch(biot_t c, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                                const double* const* U0, double* const* U_end, const biot_solve_opts* opts, int* iters,
                                biot_stats* stats, int* status, void* stream) {
  API_BEGIN(c)
  if (!(T > 0) || slabs < 1) fail(BIOT_EINVAL, "march: T must be > 0 and slabs >= 1");
  if (nterms > 0 && (!f_terms || !tcoef)) fail(BIOT_EINVAL, "march: load terms missing");
  biot_solve_opts o = solve_defaults(opts);
  if (c->nb > 1 && o.mode != BIOT_MIXED) fail(BIOT_EINVAL, "batched contexts solve in BIOT_MIXED mode");
  if (o.transpose) fail(BIOT_EINVAL, "march: transpose is not a forward march");
  std::vector<biot_stats> sb(c->nb);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = BIOT_OK;
  if (c->nb == 1) {
    march_impl(*c, T, slabs, nterms, f_terms, tcoef, U0 ? U0[0] : nullptr, U_end ? U_end[0] : nullptr, nullptr, nullptr, o,
               nullptr, sb[0], st, rc);
    if (iters) iters[0] = sb[0].iterations;
    if (status) status[0] = rc;
  } else {
    std::vector<int> code(c->nb, BIOT_OK);
    march_batch_impl(*c, T, slabs, nterms, f_terms, tcoef, U0, U_end, o, iters, sb.data(), code.data(), st);
    for (int b = 0; b < c->nb; ++b) {
      if (status) status[b] = code[b];
      if (code[b] != BIOT_OK && rc == BIOT_OK) rc = code[b];
    }
  }
  if (stats)
    for (int b = 0; b < c->nb; ++b) stats[b] = sb[b];
  return rc;
  API_END(c)
}

extern "C" int biot_adjoint_grad(biot_t c, double T, int slabs, int nterms, const double* const* f_terms, const double* tcoef,
                                 const double* U0, const double* j_goal, const biot_solve_opts* opts, int recompute,
                                 double* J_out, double* dJ, void* stream) {
  API_BEGIN(c)
  if (!(T > 0) || slabs < 1 || !j_goal || !dJ) fail(BIOT_EINVAL, "adjoint_grad: bad arguments");
  if (c->nb > 1) fail(BIOT_EINVAL, "adjoint_grad: batched context");
  cudaStream_t st = (cudaStream_t)stream;
  biot_solve_opts o = solve_defaults(opts);
  const Grid& g = c->g;
  const int nt = c->nt;
  const int64_t ns = g.N * nt;
  const double tau = T / slabs;
  // forward march with end-state checkpoints (and all slabs when not recomputing)
  double* ck = dalloc<double>((int64_t)(slabs + 1) * g.N);
  double* Xall = recompute ? nullptr : dalloc<double>((int64_t)slabs * ns);
  biot_stats s;
  int rc = BIOT_OK;
  march_impl(*c, T, slabs, nterms, f_terms, tcoef, U0, nullptr, Xall, ck, o, nullptr, s, st, rc);
  double J = dev_dot(*c, j_goal, ck + (int64_t)slabs * g.N, g.N, st);
  if (J_out) *J_out = J;
  CK(cudaMemsetAsync(dJ, 0, g.ncells * sizeof(double), st));
  MarchBufs mb;
  march_prepare(*c, nterms, f_terms, nullptr, mb, st);
  double* Z = dalloc<double>(ns);
  double* zr = dalloc<double>(ns);
  double* tmp = dalloc<double>(g.N);
  double* zero = dalloc<double>(g.N);
  CK(cudaMemsetAsync(zero, 0, g.N * sizeof(double), st));
  // terminal adjoint rhs: level r gets j
  CK(cudaMemsetAsync(zr, 0, ns * sizeof(double), st));
  CK(cudaMemcpyAsync(zr + (int64_t)(nt - 1) * g.N, j_goal, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_mask<double>(g, zr, g.N, nt, st);
  biot_solve_opts oa = o;
  oa.transpose = 1;
  double mp = 1.0;
  for (int d = 0; d < g.dim; ++d) mp *= c->t64.wg[d];
  for (int nsl = slabs - 1; nsl >= 0; --nsl) {
    const double* X;
    if (recompute) {
      CK(cudaMemcpyAsync(mb.U, ck + (int64_t)nsl * g.N, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
      build_slab_rhs(*c, nsl * tau, tau, nterms, tcoef, mb, st);
      for (int k = 0; k < nt; ++k) CK(cudaMemcpyAsync(mb.X + k * g.N, mb.U, g.N * sizeof(double), cudaMemcpyDeviceToDevice, st));
      biot_stats s2;
      int rc2 = solve_slab_impl(*c, tau, mb.rhs, mb.X, o, s2, st);
      if (rc2 != BIOT_OK && rc == BIOT_OK) rc = rc2;
      X = mb.X;
    } else {
      X = Xall + (int64_t)nsl * ns;
    }
    CK(cudaMemsetAsync(Z, 0, ns * sizeof(double), st));
    biot_stats s3;
    int rc3 = solve_slab_impl(*c, tau, zr, Z, oa, s3, st);
    if (rc3 != BIOT_OK && rc == BIOT_OK) rc = rc3;
    for (int k = 0; k < nt; ++k) {
      launch_grad_pair(g, c->t64, c->kscale64, Z + k * g.N, X + k * g.N, tau * c->tb.w[k], dJ, st);
      CKL();
    }
    if (nsl > 0) {
      // next rhs: level r = M S^T (sum_k phi_k(0) Z_k), others 0
      CK(cudaMemsetAsync(tmp, 0, g.N * sizeof(double), st));
      for (int k = 0; k < nt; ++k) launch_axpby<double>(tmp, Z + k * g.N, c->tb.phi0[k], 1.0, g.N, st);
      CKL();
      CK(cudaMemsetAsync(zr, 0, ns * sizeof(double), st));
      double* zl = zr + (int64_t)(nt - 1) * g.N;
      launch_u_rhs<double>(g, c->t64, zero, g.N, tmp + g.offp, g.N, c->b, zl, g.N, 1, st);
      launch_axpby<double>(zl + g.offp, tmp + g.offp, c->invM * mp, 0.0, g.Np, st);
      CKL();
    }
  }
  CK(cudaStreamSynchronize(st));
  cudaFree(Z);
  cudaFree(zr);
  cudaFree(tmp);
  cudaFree(zero);
  cudaFree(ck);
  if (Xall) cudaFree(Xall);
  return rc;
  API_END(c)
}

// Dual-weighted residual estimate of the dG(r) time error of J = j^T U(T^-) against dG(r+1)
// (paper §Abstract: goal-oriented, duality-based adaptivity).  The dG(r) slab solution X_n
// embeds into the dG(r+1) system as Y_n = (Pi (x) I) X_n with Pi[k][l] = phi_l^(r)(s_k^(r+1));
// with the dG(r+1) dual Z_n, eta_n = Z_n^T (F_n + C Y_{n-1} - calA Y_n) and sum eta_n equals
// J(U_{r+1}) - J(U_r) up to the solver tolerances.
extern "C" int biot_dwr_time_estimate(biot_t c, biot_t c1, double T, int slabs, int nterms, const double* const* f_terms,
                                      const double* tcoef, const double* U0, const double* j_goal, const biot_solve_opts* opts,
                                      double* eta_slab, double* eta_out, double* J_out, void* stream) {
  API_BEGIN(c)
  if (!c1 || !(T > 0) || slabs < 1 || !j_goal) fail(BIOT_EINVAL, "dwr: bad arguments");
  if (c->nb > 1 || c1->nb > 1) fail(BIOT_EINVAL, "dwr: batched context");
  if (c1->r != c->r + 1) fail(BIOT_EINVAL, "dwr: the second context must have time order r + 1");
  const Grid& g = c->g;
  {
    const Grid& g1 = c1->g;
    bool same = g.dim == g1.dim && g.N == g1.N;
    for (int d = 0; d < 3; ++d) same = same && g.n[d] == g1.n[d] && g.h[d] == g1.h[d];
    for (int f = 0; f < 6; ++f) same = same && g.ubc[f] == g1.ubc[f] && g.fbc[f] == g1.fbc[f];
    same = same && c->b == c1->b && c->invM == c1->invM && c->lam == c1->lam && c->mu == c1->mu && c->eta == c1->eta &&
           c->Kcell == c1->Kcell;
    if (!same) fail(BIOT_EINVAL, "dwr: the two contexts must share mesh, boundary codes and coefficients");
  }
  cudaStream_t st = (cudaStream_t)stream;
  biot_solve_opts o = solve_defaults(opts);
  o.transpose = 0;
  const int nt = c->nt, nt1 = c1->nt;
  const int64_t N = g.N, ns = N * nt, ns1 = N * nt1;
  const double tau = T / slabs;
  // forward dG(r) march keeping every slab solution and the end states
  double* ck = dalloc<double>((int64_t)(slabs + 1) * N);
  double* Xall = dalloc<double>((int64_t)slabs * ns);
  biot_stats s;
  int rc = BIOT_OK;
  march_impl(*c, T, slabs, nterms, f_terms, tcoef, U0, nullptr, Xall, ck, o, nullptr, s, st, rc);
  const double J = dev_dot(*c, j_goal, ck + (int64_t)slabs * N, N, st);
  // embedding of the dG(r) Radau-Lagrange basis into the dG(r+1) nodes
  double Pi[MAXR * MAXR];
  {
    long double xr[MAXR];
    for (int l = 0; l < nt; ++l) xr[l] = c->tb.nodes[l];
    for (int k = 0; k < nt1; ++k)
      for (int l = 0; l < nt; ++l) Pi[k * nt + l] = (double)lagr(xr, nt, l, (long double)c1->tb.nodes[k]);
  }
  MarchBufs mb1;
  march_prepare(*c1, nterms, f_terms, nullptr, mb1, st);
  double* Z = dalloc<double>(ns1);
  double* zr = dalloc<double>(ns1);
  double* Y = dalloc<double>(ns1);
  double* R = dalloc<double>(ns1);
  double* tmp = dalloc<double>(N);
  double* zero = dalloc<double>(N);
  CK(cudaMemsetAsync(zero, 0, N * sizeof(double), st));
  CK(cudaMemsetAsync(zr, 0, ns1 * sizeof(double), st));
  CK(cudaMemcpyAsync(zr + (int64_t)(nt1 - 1) * N, j_goal, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_mask<double>(g, zr, N, nt1, st);
  biot_solve_opts oa = o;
  oa.transpose = 1;
  double mp = 1.0;
  for (int d = 0; d < g.dim; ++d) mp *= c1->t64.wg[d];
  double eta = 0.0;
  for (int nsl = slabs - 1; nsl >= 0; --nsl) {
    // dG(r+1) dual of this slab
    CK(cudaMemsetAsync(Z, 0, ns1 * sizeof(double), st));
    biot_stats s3;
    const int rc3 = solve_slab_impl(*c1, tau, zr, Z, oa, s3, st);
    if (rc3 != BIOT_OK && rc == BIOT_OK) rc = rc3;
    // residual of the embedded dG(r) solution in the dG(r+1) slab system
    launch_time_embed(Xall + (int64_t)nsl * ns, N, nt, Y, N, nt1, Pi, N, st);
    CK(cudaMemcpyAsync(mb1.U, ck + (int64_t)nsl * N, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    build_slab_rhs(*c1, nsl * tau, tau, nterms, tcoef, mb1, st);
    apply_slab_T<double>(*c1, tau, Y, R, 0, st);
    launch_axpby<double>(R, mb1.rhs, 1.0, -1.0, ns1, st);  // R = rhs - calA Y
    CKL();
    const double en = dev_dot(*c1, Z, R, ns1, st);
    if (eta_slab) eta_slab[nsl] = en;
    eta += en;
    if (nsl > 0) {  // next dual right-hand side: C^T Z (level r+1 = S^T sum_k phi_k(0) Z_k)
      CK(cudaMemsetAsync(tmp, 0, N * sizeof(double), st));
      for (int k = 0; k < nt1; ++k) launch_axpby<double>(tmp, Z + k * N, c1->tb.phi0[k], 1.0, N, st);
      CKL();
      CK(cudaMemsetAsync(zr, 0, ns1 * sizeof(double), st));
      double* zl = zr + (int64_t)(nt1 - 1) * N;
      launch_u_rhs<double>(g, c1->t64, zero, N, tmp + g.offp, N, c1->b, zl, N, 1, st);
      launch_axpby<double>(zl + g.offp, tmp + g.offp, c1->invM * mp, 0.0, g.Np, st);
      CKL();
    }
  }
  CK(cudaStreamSynchronize(st));
  for (double* p : {Z, zr, Y, R, tmp, zero, ck, Xall}) cudaFree(p);
  if (eta_out) *eta_out = eta;
  if (J_out) *J_out = J;
  return rc;
  API_END(c)
}

extern "C" int biot_goal_mean_pressure(biot_t c, const double* lo, const double* hi, double* j, void* stream) {
  API_BEGIN(c)
  if (!lo || !hi || !j) fail(BIOT_EINVAL, "goal: NULL argument");
  const Grid& g = c->g;
  std::vector<double> h(g.N, 0.0);
  double vol = 1.0;
  for (int d = 0; d < g.dim; ++d) {
    if (!(hi[d] > lo[d])) fail(BIOT_EINVAL, "goal box is empty");
    vol *= hi[d] - lo[d];
  }
  const double gs[2] = {0.5 - std::sqrt(3.0) / 6.0, 0.5 + std::sqrt(3.0) / 6.0};
  // int over [sa, sb] (reference) of the Gauss-point Lagrange function psi_q
  auto psi_int = [&](int q, double sa, double sb) {
    double mid = 0.5 * (sa + sb);
    double v = (q == 0) ? (mid - gs[1]) / (gs[0] - gs[1]) : (mid - gs[0]) / (gs[1] - gs[0]);
    return v * (sb - sa);
  };
  for (int64_t cid = 0; cid < g.ncells; ++cid) {
    int cell[3] = {(int)(cid % g.n[0]), (int)((cid / g.n[0]) % g.n[1]), (int)(cid / ((int64_t)g.n[0] * g.n[1]))};
    double I[3][2];
    bool inside = true;
    for (int d = 0; d < 3; ++d) {
      if (d >= g.dim) { I[d][0] = 1; I[d][1] = 0; continue; }
      double a = std::max(lo[d], cell[d] * g.h[d]), b = std::min(hi[d], (cell[d] + 1) * g.h[d]);
      if (!(b > a)) { inside = false; break; }
      double sa = a / g.h[d] - cell[d], sb = b / g.h[d] - cell[d];
      for (int q = 0; q < 2; ++q) I[d][q] = psi_int(q, sa, sb) * g.h[d];
    }
    if (!inside) continue;
    for (int qz = 0; qz < (g.dim == 3 ? 2 : 1); ++qz)
      for (int qy = 0; qy < 2; ++qy)
        for (int qx = 0; qx < 2; ++qx) {
          int64_t idx = g.offp + ((int64_t)(2 * cell[2] + qz) * g.ng[1] + (2 * cell[1] + qy)) * g.ng[0] + 2 * cell[0] + qx;
          double v = I[0][qx] * I[1][qy] * (g.dim == 3 ? I[2][qz] : 1.0);
          h[idx] += v / vol;
        }
  }
  CK(cudaMemcpyAsync(j, h.data(), g.N * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_load_preset(biot_t c, int kind, double value, double* f, void* stream) {
  API_BEGIN(c)
  if (!f) fail(BIOT_EINVAL, "load: NULL output");
  const Grid& g = c->g;
  std::vector<double> h(g.N, 0.0);
  const double PI = 3.14159265358979323846;
  auto q2 = [](int a, double s) {
    return a == 0 ? 2 * (s - 0.5) * (s - 1) : (a == 1 ? 4 * s * (1 - s) : 2 * s * (s - 0.5));
  };
  const double gs[2] = {0.5 - std::sqrt(3.0) / 6.0, 0.5 + std::sqrt(3.0) / 6.0};
  auto gl = [&](int q, double s) { return q == 0 ? (s - gs[1]) / (gs[0] - gs[1]) : (s - gs[0]) / (gs[1] - gs[0]); };
  static const double g4x[4] = {0.0694318442029737, 0.3300094782075719, 0.6699905217924281, 0.9305681557970263};
  static const double g4w[4] = {0.1739274225687269, 0.3260725774312731, 0.3260725774312731, 0.1739274225687269};
  if (kind == BIOT_LOAD_TRACTION_TOP) {
    int d = g.dim - 1;
    int top = 2 * d + 1;
    if (g.ubc[top] != U_NATURAL) fail(BIOT_EINVAL, "top face is not a traction face");
    // -value * int_top phi_node ds on component d
    int iz = g.nu[d] - 1;
    for (int64_t node = 0; node < g.nnode; ++node) {
      int ix = (int)(node % g.nu[0]);
      int iy = (int)((node / g.nu[0]) % g.nu[1]);
      int iw = (int)(node / ((int64_t)g.nu[0] * g.nu[1]));
      int idx[3] = {ix, iy, iw};
      if (idx[d] != iz) continue;
      double w = 1.0;
      for (int e = 0; e < g.dim; ++e) {
        if (e == d) continue;
        int m = idx[e];
        double one;
        if (m & 1) one = 2.0 / 3.0;
        else one = ((m > 0) ? 1.0 / 6.0 : 0.0) + ((m < g.nu[e] - 1) ? 1.0 / 6.0 : 0.0);
        w *= one * g.h[e];
      }
      h[d * g.nnode + node] = -value * w;
    }
  } else if (kind == BIOT_LOAD_MMS2D_CONST || kind == BIOT_LOAD_MMS2D_LINEAR) {
    if (g.dim != 2) fail(BIOT_EINVAL, "MMS preset is 2-D");
    const double b = c->b, invM = c->invM, mu = c->mu, lam = c->lam;
    const double kov = c->Kcell[0] / c->eta;
    const bool lin = (kind == BIOT_LOAD_MMS2D_LINEAR);
    for (int cy = 0; cy < g.n[1]; ++cy)
      for (int cx = 0; cx < g.n[0]; ++cx)
        for (int qy = 0; qy < 4; ++qy)
          for (int qx = 0; qx < 4; ++qx) {
            double sx = g4x[qx], sy = g4x[qy];
            double x = (cx + sx) * g.h[0], y = (cy + sy) * g.h[1];
            double W = g4w[qx] * g4w[qy] * g.h[0] * g.h[1];
            double S = std::sin(PI * x) * std::sin(PI * y), C = std::cos(PI * x) * std::cos(PI * y);
            double fu[2] = {0, 0}, fp;
            if (lin) {
              double cxy = std::cos(PI * (x + y));
              fu[0] = 2 * mu * PI * PI * S - (mu + lam) * PI * PI * cxy - b * PI * std::sin(PI * x) * std::cos(PI * y);
              fu[1] = 2 * mu * PI * PI * S - (mu + lam) * PI * PI * cxy - b * PI * std::cos(PI * x) * std::sin(PI * y);
              fp = 2 * PI * PI * kov * C;
            } else {
              fp = b * PI * std::sin(PI * (x + y)) + invM * C;
            }
            for (int ay = 0; ay < 3; ++ay)
              for (int ax = 0; ax < 3; ++ax) {
                double ph = q2(ax, sx) * q2(ay, sy) * W;
                int64_t node = (int64_t)(2 * cy + ay) * g.nu[0] + 2 * cx + ax;
                h[node] += fu[0] * ph;
                h[g.nnode + node] += fu[1] * ph;
              }
            for (int gy = 0; gy < 2; ++gy)
              for (int gx = 0; gx < 2; ++gx) {
                int64_t idx = g.offp + (int64_t)(2 * cy + gy) * g.ng[0] + 2 * cx + gx;
                h[idx] += fp * gl(gx, sx) * gl(gy, sy) * W;
              }
          }
    if (lin) {
      // natural pressure: -<p_exact, z.n> with p_exact = C t on every natural-flow face
      for (int f = 0; f < 4; ++f) {
        if (g.fbc[f] != F_NATURAL) continue;
        int dn = f / 2, side = f % 2;
        int dt = 1 - dn;
        double nsign = side ? 1.0 : -1.0;
        int ia = side ? g.nu[dn] - 1 : 0;  // along-normal index of the face DoFs
        for (int ct = 0; ct < g.n[dt]; ++ct)
          for (int q = 0; q < 4; ++q) {
            double s = g4x[q];
            double xt = (ct + s) * g.h[dt];
            double xn = side ? 1.0 * g.n[dn] * g.h[dn] : 0.0;
            double x = dn == 0 ? xn : xt, y = dn == 0 ? xt : xn;
            double pD = std::cos(PI * x) * std::cos(PI * y);
            double W = g4w[q] * g.h[dt];
            for (int gq = 0; gq < 2; ++gq) {
              // q component dn: grid (along dn: nu, across: ng)
              int64_t it = 2 * ct + gq;
              int64_t local = (dn == 0) ? (it * g.nu[0] + ia) : ((int64_t)ia * g.ng[0] + it);
              h[g.offq[dn] + local] += -pD * nsign * gl(gq, s) * W;
            }
          }
      }
    }
  } else {
    fail(BIOT_EINVAL, "unknown load preset");
  }
  CK(cudaMemcpyAsync(f, h.data(), g.N * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return BIOT_OK;
  API_END(c)
}

namespace {
template <typename T>
void apply_part_T(biot_ctx& c, int part, double tau, const T* in, T* out, cudaStream_t st) {
  ensure_prec<T>(c);
  const Grid& g = c.g;
  PrecWork<T>& w = c.pw<T>();
  int64_t nqt = g.nq[0] + g.nq[1] + g.nq[2];
  CK(cudaMemsetAsync(out, 0, g.N * sizeof(T), st));
  if (part == BIOT_PART_FLUX_MASS_INV) {
    launch_mq_line_solve<T>(g, c.tab<T>(), c.kscale<T>(), in + g.Nu, nqt, out + g.Nu, nqt, tau, 1, st);
    launch_q_fix_constrained<T>(g, in + g.Nu, nqt, out + g.Nu, nqt, 1, st);
  } else if (part == BIOT_PART_SCHUR) {
    double cm[1] = {c.invM + c.beta};
    schur_apply<T>(c, tau, cm, in + g.offp, out + g.offp, 1, st);
  } else if (part == BIOT_PART_VCYCLE) {
    LevelWork<T>& lw = lwork<T>(c.lv[0]);
    CK(cudaMemcpyAsync(lw.b, in, g.Nu * sizeof(T), cudaMemcpyDeviceToDevice, st));
    vcycle<T>(c, tau, 1, st);
    CK(cudaMemcpyAsync(out, lw.x, g.Nu * sizeof(T), cudaMemcpyDeviceToDevice, st));
  } else if (part == BIOT_PART_ELASTICITY) {
    apply_A<T>(c.lv[0], c.lam, c.mu, tau, in, out, 1, st);
  } else if (part == BIOT_PART_SCHUR_STEP) {
    if (!c.lumped_flux || c.nb != 1) fail(BIOT_EINVAL, "apply_part: BIOT_PART_SCHUR_STEP needs a lumped, unbatched context");
    prec_prepare<T>(c, tau, st);
    double cm[1] = {c.invM + c.beta};
    // one step of the kernel the solver runs in this precision, with c1 = 0, c2 = 1 and b = 0:
    // out_p = in_p - diag(Shat)^{-1} Shat in_p
    CK(cudaMemsetAsync(w.gp, 0, g.Np * sizeof(T), st));
    if (sizeof(T) == 4) {
      launch_schur_cheb_mf<T>(g, c.tab<T>(), w.wq, cm, 0.0, 1.0, 0, w.gp, in + g.offp, w.pd, out + g.offp, 1, st);
    } else {
      launch_schur_dinv<T>(g, c.tab<T>(), c.sb2<T>(), cm, tau, w.pdinv, 1, st);
      launch_schur_cheb_st<T>(g, c.tab<T>(), w.scoef, w.pdinv, cm, 0.0, 1.0, 0, w.gp, in + g.offp, w.pd, out + g.offp, 1, st);
      w.schur_tau = -1;  // the solver's diagonals of this tau were overwritten
    }
  } else {
    fail(BIOT_EINVAL, "unknown part");
  }
  CKL();
  (void)w;
}
}  // namespace

extern "C" int biot_apply_part(biot_t c, int part, double tau, const void* in, void* out, int prec, void* stream) {
  API_BEGIN(c)
  if (!in || !out || !(tau > 0)) fail(BIOT_EINVAL, "apply_part: NULL vector or tau <= 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == BIOT_FP64) apply_part_T<double>(*c, part, tau, (const double*)in, (double*)out, st);
  else if (prec == BIOT_FP32) apply_part_T<float>(*c, part, tau, (const float*)in, (float*)out, st);
  else fail(BIOT_EINVAL, "prec must be BIOT_FP64 or BIOT_FP32");
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_schur_bounds(biot_t c, double tau, double* bounds, int* degree, void* stream) {
  API_BEGIN(c)
  if (!bounds || !(tau > 0)) fail(BIOT_EINVAL, "schur_bounds: NULL bounds or tau <= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const double lm = schur_lmax(*c, tau, st);
  bounds[0] = lm / c->schur_kappa;
  bounds[1] = lm;
  bounds[2] = c->schur_lmin;
  bounds[3] = 1.1 * lm;
  if (degree) *degree = use_schur_mg(*c) ? 0 : schur_degree(*c);
  return BIOT_OK;
  API_END(c)
}

extern "C" int biot_counters(biot_t c, int64_t* launches, int64_t* op_launches, double* op_ms) {
  if (!c) return BIOT_EINVAL;
  if (launches) *launches = (int64_t)launch_count();
  long long n = 0;
  double ms = 0;
  prof_collect(0, &n, &ms, nullptr);
  if (op_launches) *op_launches = n;
  if (op_ms) *op_ms = ms;
  return BIOT_OK;
}

extern "C" int biot_kernel_stats(biot_t c, int kind, int64_t* launches, double* ms, double* units) {
  if (!c || kind < 0 || kind >= PROF_KINDS) return BIOT_EINVAL;
  long long n = 0;
  double t = 0, u = 0;
  prof_collect(kind, &n, &t, &u);
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (units) *units = u;
  return BIOT_OK;
}

extern "C" int biot_profile(biot_t c, int enable) {
  if (!c) return BIOT_EINVAL;
  prof_enable(enable != 0);
  return BIOT_OK;
}

// read-only view of a context for the allocation-free entry point (noalloc.cu)
namespace biot {
struct CtxView {
  const Grid* g;
  const TabT<double>* t64;
  const double* dmq64;
  double invM, beta;
  int nb;           // batched instances (1: a context of biot_setup)
  int lumped_flux;  // 1: the Schur complement uses the diagonal of the Darcy mass
};
bool ctx_view(biot_t c, CtxView* v) {
  if (!c || !v) return false;
  v->g = &c->g;
  v->t64 = &c->t64;
  v->dmq64 = c->dmq64;
  v->invM = c->invM;
  v->beta = c->beta;
  v->nb = c->nb;
  v->lumped_flux = c->lumped_flux;
  return true;
}
void ctx_set_error(biot_t c, const char* msg) {
  if (c) c->err = msg ? msg : "";
}
}  // namespace biot

extern "C" const char* biot_last_error(biot_t c) {
  if (!c) return g_err_msg.c_str();
  return c->err.c_str();
}

extern "C" void biot_destroy(biot_t c) {
  if (!c) return;
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(c->kscale64); F(c->kscale32); F(c->dmq64); F(c->dmq32); F(c->sb2_64); F(c->sb2_32);
  F(c->hdev); F(c->partial); F(c->r64); F(c->a64); F(c->d32); F(c->r32); F(c->lvl64); F(c->lvl64b); F(c->Ainv);
  if (c->hhost) cudaFreeHost(c->hhost);
  if (c->bhost) cudaFreeHost(c->bhost);
  F(c->bdev);

  if (c->hptr) cudaFreeHost(c->hptr);
  F(c->ptrbuf);
  for (Level& L : c->lv) {
    F(L.dinv64); F(L.dinv32);
    F(L.w64.x); F(L.w64.xo); F(L.w64.d); F(L.w64.Ax); F(L.w64.b);
    F(L.w32.x); F(L.w32.xo); F(L.w32.d); F(L.w32.Ax); F(L.w32.b);
  }
  auto FK = [&](auto& K) {
    for (auto p : K.V) F(p);
    for (auto p : K.Z) F(p);
    F((void*)K.dV); F(K.tmp);
  };
  FK(c->k64); FK(c->k32);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ws) cudaStreamDestroy(c->ws);
  auto FP = [&](auto& w) {
    F(w.tA); F(w.tB); F(w.fq); F(w.tq); F(w.fq2); F(w.gp); F(w.pp); F(w.pd); F(w.pAx); F(w.pxo); F(w.pdinv); F(w.scoef); F(w.wq);
    for (auto* v : {&w.pms, &w.pmb, &w.pmx, &w.pmd, &w.pmt})
      for (auto p : *v) F(p);
    F(w.pmr0);
  };
  FP(c->p64); FP(c->p32);
  for (void* p : c->extra) F(p);
  for (int m = 0; m < 8; ++m) F(c->m_f[m]);
  F((void*)c->m_fdev); F(c->m_U); F(c->m_SU); F(c->m_rhs); F(c->m_X);
  F(c->bm_f); F((void*)c->bm_fdev); F(c->bm_U); F(c->bm_SU); F(c->bm_rhs); F(c->bm_X);
  delete c;
}
