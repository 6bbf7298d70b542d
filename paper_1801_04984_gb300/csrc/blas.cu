// Vector kernels of the Krylov solver: fused multi-dot, fused multi-axpy with
// the second Gram-Schmidt pass or the norm folded in, conversions, time-basis
// mixing.  All reductions are deterministic: fixed grid, per-thread partials
// reduced in a fixed order, then one block sums the per-block partials.
//
// FP32 vectors are reduced with exact products (two-product by fma) and
// compensated (two-sum) single-precision accumulation per thread, converted to
// double for the cross-thread reduction, so inner products of FP32 Krylov
// vectors carry FP64-level accuracy without using the (slow) FP64 pipe per
// element.
#include "internal.h"

namespace biot {

constexpr int NV = 8;  // vectors per multi-dot pass

struct Acc {  // compensated accumulator
  float hi, lo;
};

__device__ __forceinline__ void acc_add(Acc& a, float x) {
  float s = __fadd_rn(a.hi, x);
  float bb = __fsub_rn(s, a.hi);
  float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, err);
}
__device__ __forceinline__ void acc_fma(Acc& a, float x, float y) {
  float p = __fmul_rn(x, y);
  float e = __fmaf_rn(x, y, -p);
  acc_add(a, p);
  a.lo = __fadd_rn(a.lo, e);
}

template <typename TV>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s;
  __device__ void init() { s = 0.0; }
  __device__ void add(double x, double y) { s = fma(x, y, s); }
  __device__ void add_plain(double x) { s += x; }
  __device__ double get() const { return s; }
};
template <>
struct DotAcc<float> {
  Acc a;
  __device__ void init() { a.hi = 0.f; a.lo = 0.f; }
  __device__ void add(float x, float y) { acc_fma(a, x, y); }
  __device__ void add_plain(float x) { a.hi += x; }  // uncompensated
  __device__ double get() const { return (double)a.hi + (double)a.lo; }
};

// block-reduce `cnt` doubles per thread (in smem), write to partial[bid * stride + i]
__device__ inline void block_reduce_store(double* vals, int cnt, double* partial, int stride, int64_t bid) {
  __shared__ double sh[NV + 1][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = 0; i < cnt; ++i) {
    double v = vals[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
    partial[bid * stride + threadIdx.x] = s;
  }
}

// Basis pointers travel as a kernel parameter (constant bank): no pointer loads per element,
// and a CUDA graph that captures the launch keeps them.
template <typename TV>
struct PtrPack {
  const TV* p[MAXDOT];
};
// 16-byte vectors of the element type
template <typename TV>
struct Vec16;
template <>
struct Vec16<float> {
  using T = float4;
  static constexpr int W = 4;
  __device__ static void get(const T& v, float (&o)[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  __device__ static T make(const float (&o)[4]) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec16<double> {
  using T = double2;
  static constexpr int W = 2;
  __device__ static void get(const T& v, double (&o)[2]) { o[0] = v.x; o[1] = v.y; }
  __device__ static T make(const double (&o)[2]) { return make_double2(o[0], o[1]); }
};

// block-reduce `cnt` (<= NVM) doubles per thread, write to partial[bid * stride + i]
template <int NVM>
__device__ inline void block_reduce_store_n(const double* vals, int cnt, double* partial, int stride, int64_t bid) {
  __shared__ double sh[NVM][8];  // 256 threads = 8 warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NVM; ++i) {
    if (i >= cnt) break;
    double v = vals[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
    partial[bid * stride + threadIdx.x] = s;
  }
}

// dots V_i^T w, i < nv <= NVM, in one pass over w: 16-byte loads, per-thread compensated
// FP32 (or plain FP64) accumulation, partials per block
template <typename TV, int NVM, bool VEC>
__global__ void __launch_bounds__(256) k_multidot(const __grid_constant__ PtrPack<TV> V, int nv, const TV* __restrict__ w, int64_t n,
                                                  double* __restrict__ partial) {
  using VT = typename Vec16<TV>::T;
  constexpr int W = Vec16<TV>::W;
  DotAcc<TV> acc[NVM];
#pragma unroll
  for (int i = 0; i < NVM; ++i) acc[i].init();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nvec = VEC ? n / W : 0;
  for (int64_t e = t0; e < nvec; e += stride) {
    TV wv[W];
    Vec16<TV>::get(reinterpret_cast<const VT*>(w)[e], wv);
#pragma unroll
    for (int i = 0; i < NVM; ++i) {
      if (i >= nv) break;
      TV vv[W];
      Vec16<TV>::get(__ldg(reinterpret_cast<const VT*>(V.p[i]) + e), vv);
#pragma unroll
      for (int q = 0; q < W; ++q) acc[i].add(vv[q], wv[q]);
    }
  }
  for (int64_t e = nvec * W + t0; e < n; e += stride) {  // tail
    const TV we = w[e];
#pragma unroll
    for (int i = 0; i < NVM; ++i) {
      if (i >= nv) break;
      acc[i].add(V.p[i][e], we);
    }
  }
  double vals[NVM];
#pragma unroll
  for (int i = 0; i < NVM; ++i) vals[i] = acc[i].get();
  block_reduce_store_n<NVM>(vals, nv, partial, NVM, blockIdx.x);
}

// sum partial[b][i] over blocks b (fixed order) -> out[i]
// rsq (optional): receives 1/sqrt(out[0]) (0 when out[0] <= 0), the normalisation factor of a squared norm
__global__ void k_final_reduce(const double* __restrict__ partial, int nblocks, int cnt, int stride, double* __restrict__ out,
                               double* __restrict__ rsq = nullptr) {
  __shared__ double sh[256];
  for (int i = 0; i < cnt; ++i) {
    double s = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)b * stride + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[i] = sh[0];
      if (rsq && i == 0) rsq[0] = sh[0] > 0.0 ? 1.0 / sqrt(sh[0]) : 0.0;
    }
    __syncthreads();
  }
}

constexpr int DOT_PASS = 32;  // vectors per pass of the multi-dot / multi-axpy

template <typename TV>
bool aligned16(const TV* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// V: HOST array of nv device pointers (every vector 16-byte aligned)
template <typename TV>
void launch_multidot(const TV* const* V, int nv, const TV* w, int64_t n, double* partial, double* out, cudaStream_t st) {
  for (int c0 = 0; c0 < nv; c0 += DOT_PASS) {
    const int cnt = (nv - c0 < DOT_PASS) ? nv - c0 : DOT_PASS;
    PtrPack<TV> pk;
    bool vec = aligned16(w);
    for (int i = 0; i < MAXDOT; ++i) {
      pk.p[i] = (i < cnt) ? V[c0 + i] : nullptr;
      if (i < cnt) vec = vec && aligned16(pk.p[i]);
    }
    // 16-byte loads when every vector allows them (library buffers always do; caller
    // vectors at an offset may not)
    if (vec) {
      if (cnt <= 8) (note_launch(), k_multidot<TV, 8, true><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, w, n, partial));
      else if (cnt <= 16) (note_launch(), k_multidot<TV, 16, true><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, w, n, partial));
      else (note_launch(), k_multidot<TV, 32, true><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, w, n, partial));
    } else {
      if (cnt <= 8) (note_launch(), k_multidot<TV, 8, false><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, w, n, partial));
      else if (cnt <= 16) (note_launch(), k_multidot<TV, 16, false><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, w, n, partial));
      else (note_launch(), k_multidot<TV, 32, false><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, w, n, partial));
    }
    const int stride = cnt <= 8 ? 8 : (cnt <= 16 ? 16 : 32);
    (note_launch(), k_final_reduce<<<1, 256, 0, st>>>(partial, RED_BLOCKS, cnt, stride, out + c0));
  }
}

// mode 0: w -= V h ; mode 1: also dots V^T w_new ; mode 2: also ||w_new||^2.  The update runs
// in the vectors' precision; mode 1 reads the basis a second time right after (cache hits).
template <typename TV, int NVM, bool VEC>
__global__ void __launch_bounds__(256) k_multiaxpy(const __grid_constant__ PtrPack<TV> V, int nv, const double* __restrict__ h,
                                                   TV* __restrict__ w, int64_t n, int mode, double* __restrict__ partial) {
  using VT = typename Vec16<TV>::T;
  constexpr int W = Vec16<TV>::W;
  __shared__ TV hs[NVM];
  if (threadIdx.x < NVM) hs[threadIdx.x] = (threadIdx.x < nv) ? (TV)h[threadIdx.x] : TV(0);
  __syncthreads();
  DotAcc<TV> acc[NVM];
#pragma unroll
  for (int i = 0; i < NVM; ++i) acc[i].init();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nvec = VEC ? n / W : 0;
  for (int64_t e = t0; e < nvec; e += stride) {
    TV wv[W];
    Vec16<TV>::get(reinterpret_cast<const VT*>(w)[e], wv);
#pragma unroll
    for (int i = 0; i < NVM; ++i) {
      if (i >= nv) break;
      TV vv[W];
      Vec16<TV>::get(__ldg(reinterpret_cast<const VT*>(V.p[i]) + e), vv);
      const TV hi = hs[i];
#pragma unroll
      for (int q = 0; q < W; ++q) wv[q] -= hi * vv[q];
    }
    reinterpret_cast<VT*>(w)[e] = Vec16<TV>::make(wv);
    if (mode == 1) {
      // second Gram-Schmidt coefficients: w is already orthogonal to the basis up to the
      // first pass's rounding, so these dots only need accuracy relative to ||v|| ||w||;
      // plain per-thread accumulation (then FP64 across threads) is enough
#pragma unroll
      for (int i = 0; i < NVM; ++i) {
        if (i >= nv) break;
        TV vv[W];
        Vec16<TV>::get(__ldg(reinterpret_cast<const VT*>(V.p[i]) + e), vv);
        TV sdot = TV(0);
#pragma unroll
        for (int q = 0; q < W; ++q) sdot = fma(vv[q], wv[q], sdot);
        acc[i].add_plain(sdot);
      }
    } else if (mode == 2) {
#pragma unroll
      for (int q = 0; q < W; ++q) acc[0].add(wv[q], wv[q]);
    }
  }
  for (int64_t e = nvec * W + t0; e < n; e += stride) {  // tail
    TV we = w[e];
#pragma unroll
    for (int i = 0; i < NVM; ++i) {
      if (i >= nv) break;
      we -= hs[i] * V.p[i][e];
    }
    w[e] = we;
    if (mode == 1) {
#pragma unroll
      for (int i = 0; i < NVM; ++i) {
        if (i >= nv) break;
        acc[i].add(V.p[i][e], we);
      }
    } else if (mode == 2) {
      acc[0].add(we, we);
    }
  }
  if (mode == 0) return;
  double vals[NVM];
#pragma unroll
  for (int i = 0; i < NVM; ++i) vals[i] = acc[i].get();
  block_reduce_store_n<NVM>(vals, mode == 1 ? nv : 1, partial, NVM, blockIdx.x);
}

template <typename TV>
void launch_multiaxpy_dot(const TV* const* V, int nv, const double* h, TV* w, int64_t n, int mode, double* partial,
                          double* out, cudaStream_t st) {
  // mode 1 needs every pass's dots against the final w: with more than one pass apply all
  // updates first, then dot in a separate pass
  const int npass = (nv + DOT_PASS - 1) / DOT_PASS;
  for (int c0 = 0; c0 < nv; c0 += DOT_PASS) {
    const int cnt = (nv - c0 < DOT_PASS) ? nv - c0 : DOT_PASS;
    const bool last = c0 + DOT_PASS >= nv;
    const int m = (mode == 2 && last) ? 2 : ((mode == 1 && npass == 1) ? 1 : 0);
    PtrPack<TV> pk;
    bool vec = aligned16(w);
    for (int i = 0; i < MAXDOT; ++i) {
      pk.p[i] = (i < cnt) ? V[c0 + i] : nullptr;
      if (i < cnt) vec = vec && aligned16(pk.p[i]);
    }
    const int nvm = cnt <= 8 ? 8 : (cnt <= 16 ? 16 : 32);
#define BIOT_MAXPY(NVM, VEC) (note_launch(), k_multiaxpy<TV, NVM, VEC><<<RED_BLOCKS, 256, 0, st>>>(pk, cnt, h + c0, w, n, m, partial))
    if (vec) {
      if (nvm == 8) BIOT_MAXPY(8, true);
      else if (nvm == 16) BIOT_MAXPY(16, true);
      else BIOT_MAXPY(32, true);
    } else {
      if (nvm == 8) BIOT_MAXPY(8, false);
      else if (nvm == 16) BIOT_MAXPY(16, false);
      else BIOT_MAXPY(32, false);
    }
#undef BIOT_MAXPY
    if (m == 1) (note_launch(), k_final_reduce<<<1, 256, 0, st>>>(partial, RED_BLOCKS, cnt, nvm, out));
    if (m == 2) (note_launch(), k_final_reduce<<<1, 256, 0, st>>>(partial, RED_BLOCKS, 1, nvm, out, out + 1));
  }
  if (mode == 1 && npass > 1) launch_multidot<TV>(V, nv, w, n, partial, out, st);
}

template <typename TA, typename TB>
__global__ void k_convert(const TA* __restrict__ a, TB* __restrict__ b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) b[e] = (TB)a[e];
}
template <typename TA, typename TB>
void launch_convert(const TA* a, TB* b, int64_t n, cudaStream_t st) {
  (note_launch(), k_convert<TA, TB><<<RED_BLOCKS * 2, 256, 0, st>>>(a, b, n));
}

template <typename T>
__global__ void k_axpby(T* __restrict__ y, const T* __restrict__ x, T a, T b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + b * y[e];
}
template <typename T>
void launch_axpby(T* y, const T* x, double a, double b, int64_t n, cudaStream_t st) {
  (note_launch(), k_axpby<T><<<RED_BLOCKS * 2, 256, 0, st>>>(y, x, (T)a, (T)b, n));
}

template <typename T>
__global__ void k_scale_into(T* __restrict__ y, const T* __restrict__ x, const double* __restrict__ s, int inv, int64_t n) {
  T f = (T)(*s);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) y[e] = x[e] * f;
}
// y = x * (*s) (s in device memory; `inv` is kept for the signature and ignored)
template <typename T>
void launch_scale_into(T* y, const T* x, const double* s, int inv, int64_t n, cudaStream_t st) {
  (note_launch(), k_scale_into<T><<<RED_BLOCKS * 2, 256, 0, st>>>(y, x, s, inv, n));
}

template <typename TY, typename TZ>
__global__ void k_lincomb_add(TY* __restrict__ y, const TZ* const* __restrict__ Z, int nz, const double* __restrict__ c,
                              int64_t n) {
  // arithmetic in the precision of y (the FP32 inner solver never touches the FP64 pipe per element)
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    TY s = y[e];
    for (int i = 0; i < nz; ++i) s += TY(c[i]) * TY(Z[i][e]);
    y[e] = s;
  }
}
template <typename TY, typename TZ>
void launch_lincomb_add(TY* y, const TZ* const* Z, int nz, const double* c, int64_t n, cudaStream_t st) {
  (note_launch(), k_lincomb_add<TY, TZ><<<RED_BLOCKS * 2, 256, 0, st>>>(y, Z, nz, c, n));
}

__global__ void k_residual(const double* __restrict__ b, const double* __restrict__ Ax, double* __restrict__ r, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) r[e] = b[e] - Ax[e];
}
void launch_residual(const double* b, const double* Ax, double* r, int64_t n, cudaStream_t st) {
  (note_launch(), k_residual<<<RED_BLOCKS * 2, 256, 0, st>>>(b, Ax, r, n));
}

template <typename T>
struct Mix {
  T c[MAXR][MAXR];
};
// arithmetic in the output precision
template <typename TI, typename TO>
__global__ void k_time_mix(const TI* __restrict__ in, int64_t sin, TO* __restrict__ out, int64_t sout, int nt, Mix<TO> m, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    TO v[MAXR];
    for (int l = 0; l < nt; ++l) v[l] = (TO)in[l * sin + e];
    for (int k = 0; k < nt; ++k) {
      TO s = 0;
      for (int l = 0; l < nt; ++l) s += m.c[k][l] * v[l];
      out[k * sout + e] = s;
    }
  }
}
template <typename TI, typename TO>
void launch_time_mix(const TI* in, int64_t sin, TO* out, int64_t sout, int nt, const double* C, int64_t n, cudaStream_t st) {
  Mix<TO> m;
  for (int k = 0; k < MAXR; ++k)
    for (int l = 0; l < MAXR; ++l) m.c[k][l] = (TO)((k < nt && l < nt) ? C[k * nt + l] : 0.0);
  (note_launch(), k_time_mix<TI, TO><<<RED_BLOCKS * 2, 256, 0, st>>>(in, sin, out, sout, nt, m, n));
}

// ---------------------------------------------------------------------------
// Segmented (per-instance) vector kernels of a batch of independent problems.
// Element e of level k of instance b sits at k * lstride + b * istride + e
// (e < len); block (x, b) of a (gx, nb) grid works on instance b only, so
// every instance gets its own inner products and its own scalars (Krylov
// coefficients, normalisations), in the same deterministic order as above.
int seg_gx(int nb) {
  int gx = (RED_BLOCKS + nb - 1) / nb;
  return gx < 2 ? 2 : (gx > RED_BLOCKS ? RED_BLOCKS : gx);
}
int64_t seg_partial_doubles(int nb) { return (int64_t)seg_gx(nb) * nb * (NV + 1); }

template <typename TV>
__global__ void __launch_bounds__(256) k_seg_multidot(const TV* const* __restrict__ V, int nv, const TV* __restrict__ w, Seg sg,
                                                      double* __restrict__ partial) {
  const int b = blockIdx.y;
  DotAcc<TV> acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i].init();
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < sg.nt; ++k) {
    const int64_t base = k * sg.lstride + b * sg.istride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.len; e += step) {
      const TV we = w[base + e];
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nv) acc[i].add(V[i][base + e], we);
    }
  }
  double vals[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) vals[i] = acc[i].get();
  block_reduce_store(vals, nv, partial, NV + 1, (int64_t)b * gridDim.x + blockIdx.x);
}

// per instance b (one block each): out[b * ostride + i] = sum over its gx partials;
// with rsq, out[b * ostride + 1] = 1/sqrt(out[b * ostride]) (0 when not positive)
__global__ void k_seg_final(const double* __restrict__ partial, int gx, int cnt, double* __restrict__ out, int ostride, int rsq) {
  __shared__ double sh[256];
  const int b = blockIdx.x;
  for (int i = 0; i < cnt; ++i) {
    double s = 0;
    for (int x = threadIdx.x; x < gx; x += blockDim.x) s += partial[((int64_t)b * gx + x) * (NV + 1) + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[(int64_t)b * ostride + i] = sh[0];
      if (rsq && i == 0) out[(int64_t)b * ostride + 1] = sh[0] > 0.0 ? 1.0 / sqrt(sh[0]) : 0.0;
    }
    __syncthreads();
  }
}

template <typename TV>
void launch_seg_multidot(const TV* const* V, int nv, const TV* w, const Seg& sg, double* partial, double* out, int ostride,
                         cudaStream_t st) {
  const int gx = seg_gx(sg.nb);
  for (int c0 = 0; c0 < nv; c0 += NV) {
    int cnt = (nv - c0 < NV) ? nv - c0 : NV;
    (note_launch(), k_seg_multidot<TV><<<dim3(gx, sg.nb), 256, 0, st>>>(V + c0, cnt, w, sg, partial));
    (note_launch(), k_seg_final<<<sg.nb, 256, 0, st>>>(partial, gx, cnt, out + c0, ostride, 0));
  }
}

// w -= sum_i V_i h[b * hstride + i]; mode 1: partial dots V^T w_new; mode 2: ||w_new||^2
template <typename TV>
__global__ void __launch_bounds__(256) k_seg_multiaxpy(const TV* const* __restrict__ V, int nv, const double* __restrict__ h,
                                                       int hstride, TV* __restrict__ w, Seg sg, int mode, double* __restrict__ partial) {
  const int b = blockIdx.y;
  TV hv[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) hv[i] = (i < nv) ? (TV)h[(int64_t)b * hstride + i] : TV(0);
  DotAcc<TV> acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i].init();
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < sg.nt; ++k) {
    const int64_t base = k * sg.lstride + b * sg.istride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.len; e += step) {
      TV v[NV];
      TV we = w[base + e];
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nv) { v[i] = V[i][base + e]; we -= hv[i] * v[i]; }
      w[base + e] = we;
      if (mode == 1) {
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (i < nv) acc[i].add(v[i], we);
      } else if (mode == 2) {
        acc[0].add(we, we);
      }
    }
  }
  if (mode == 0) return;
  double vals[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) vals[i] = acc[i].get();
  block_reduce_store(vals, mode == 1 ? nv : 1, partial, NV + 1, (int64_t)b * gridDim.x + blockIdx.x);
}

template <typename TV>
void launch_seg_multiaxpy_dot(const TV* const* V, int nv, const double* h, int hstride, TV* w, const Seg& sg, int mode,
                              double* partial, double* out, int ostride, cudaStream_t st) {
  const int gx = seg_gx(sg.nb);
  const dim3 grid(gx, sg.nb);
  if (nv <= NV) {
    (note_launch(), k_seg_multiaxpy<TV><<<grid, 256, 0, st>>>(V, nv, h, hstride, w, sg, mode, partial));
    if (mode == 1) (note_launch(), k_seg_final<<<sg.nb, 256, 0, st>>>(partial, gx, nv, out, ostride, 0));
    if (mode == 2) (note_launch(), k_seg_final<<<sg.nb, 256, 0, st>>>(partial, gx, 1, out, ostride, 1));
    return;
  }
  for (int c0 = 0; c0 < nv; c0 += NV) {
    int cnt = (nv - c0 < NV) ? nv - c0 : NV;
    bool last = c0 + NV >= nv;
    int m = (last && mode == 2) ? 2 : 0;
    (note_launch(), k_seg_multiaxpy<TV><<<grid, 256, 0, st>>>(V + c0, cnt, h + c0, hstride, w, sg, m, partial));
    if (m == 2) (note_launch(), k_seg_final<<<sg.nb, 256, 0, st>>>(partial, gx, 1, out, ostride, 1));
  }
  if (mode == 1) launch_seg_multidot<TV>(V, nv, w, sg, partial, out, ostride, st);
}

// y = x * s[b * sstride] per instance
template <typename T>
__global__ void k_seg_scale(T* __restrict__ y, const T* __restrict__ x, const double* __restrict__ s, int sstride, Seg sg) {
  const int b = blockIdx.y;
  const T f = (T)s[(int64_t)b * sstride];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < sg.nt; ++k) {
    const int64_t base = k * sg.lstride + b * sg.istride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.len; e += step) y[base + e] = x[base + e] * f;
  }
}
template <typename T>
void launch_seg_scale(T* y, const T* x, const double* s, int sstride, const Seg& sg, cudaStream_t st) {
  (note_launch(), k_seg_scale<T><<<dim3(seg_gx(sg.nb), sg.nb), 256, 0, st>>>(y, x, s, sstride, sg));
}

// y = a[b] x + c[b] y per instance (a, c device arrays, one value per instance)
template <typename T>
__global__ void k_seg_axpby(T* __restrict__ y, const T* __restrict__ x, const double* __restrict__ a, const double* __restrict__ c,
                            Seg sg) {
  const int b = blockIdx.y;
  const T av = (T)a[b], cv = (T)c[b];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < sg.nt; ++k) {
    const int64_t base = k * sg.lstride + b * sg.istride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.len; e += step)
      y[base + e] = av * x[base + e] + cv * y[base + e];
  }
}
template <typename T>
void launch_seg_axpby(T* y, const T* x, const double* a, const double* c, const Seg& sg, cudaStream_t st) {
  (note_launch(), k_seg_axpby<T><<<dim3(seg_gx(sg.nb), sg.nb), 256, 0, st>>>(y, x, a, c, sg));
}

// y += sum_i Z_i c[b * cstride + i] per instance (arithmetic in the precision of y)
template <typename TY, typename TZ>
__global__ void k_seg_lincomb_add(TY* __restrict__ y, const TZ* const* __restrict__ Z, int nz, const double* __restrict__ c,
                                  int cstride, Seg sg) {
  const int b = blockIdx.y;
  const double* cb = c + (int64_t)b * cstride;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < sg.nt; ++k) {
    const int64_t base = k * sg.lstride + b * sg.istride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.len; e += step) {
      TY s = y[base + e];
      for (int i = 0; i < nz; ++i) s += TY(cb[i]) * TY(Z[i][base + e]);
      y[base + e] = s;
    }
  }
}
template <typename TY, typename TZ>
void launch_seg_lincomb_add(TY* y, const TZ* const* Z, int nz, const double* c, int cstride, const Seg& sg, cudaStream_t st) {
  (note_launch(), k_seg_lincomb_add<TY, TZ><<<dim3(seg_gx(sg.nb), sg.nb), 256, 0, st>>>(y, Z, nz, c, cstride, sg));
}

// x += s[b * sstride] * d per instance (mixed-precision refinement update)
template <typename TX, typename TD>
__global__ void k_seg_add_scaled(TX* __restrict__ x, const TD* __restrict__ d, const double* __restrict__ s, int sstride, Seg sg) {
  const int b = blockIdx.y;
  const double f = s[(int64_t)b * sstride];
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k < sg.nt; ++k) {
    const int64_t base = k * sg.lstride + b * sg.istride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.len; e += step)
      x[base + e] = (TX)((double)x[base + e] + f * (double)d[base + e]);
  }
}
template <typename TX, typename TD>
void launch_seg_add_scaled(TX* x, const TD* d, const double* s, int sstride, const Seg& sg, cudaStream_t st) {
  (note_launch(), k_seg_add_scaled<TX, TD><<<dim3(seg_gx(sg.nb), sg.nb), 256, 0, st>>>(x, d, s, sstride, sg));
}

// rectangular time map: out[k] = sum_l C[k][l] in[l] for nt_out output and nt_in input
// levels (the embedding of a dG(r) slab polynomial into the dG(r+1) nodal basis)
template <typename T>
__global__ void k_time_embed(const T* __restrict__ in, int64_t sin, int nin, T* __restrict__ out, int64_t sout, int nout,
                             Mix<T> m, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T v[MAXR];
    for (int l = 0; l < nin; ++l) v[l] = in[l * sin + e];
    for (int k = 0; k < nout; ++k) {
      T s = 0;
      for (int l = 0; l < nin; ++l) s += m.c[k][l] * v[l];
      out[k * sout + e] = s;
    }
  }
}
void launch_time_embed(const double* in, int64_t sin, int nin, double* out, int64_t sout, int nout, const double* C, int64_t n,
                       cudaStream_t st) {
  Mix<double> m;
  for (int k = 0; k < MAXR; ++k)
    for (int l = 0; l < MAXR; ++l) m.c[k][l] = (k < nout && l < nin) ? C[k * nin + l] : 0.0;
  (note_launch(), k_time_embed<double><<<RED_BLOCKS * 2, 256, 0, st>>>(in, sin, nin, out, sout, nout, m, n));
}

template void launch_multidot<double>(const double* const*, int, const double*, int64_t, double*, double*, cudaStream_t);
template void launch_multidot<float>(const float* const*, int, const float*, int64_t, double*, double*, cudaStream_t);
template void launch_multiaxpy_dot<double>(const double* const*, int, const double*, double*, int64_t, int, double*, double*,
                                           cudaStream_t);
template void launch_multiaxpy_dot<float>(const float* const*, int, const double*, float*, int64_t, int, double*, double*,
                                          cudaStream_t);
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);
template void launch_convert<float, float>(const float*, float*, int64_t, cudaStream_t);
template void launch_axpby<double>(double*, const double*, double, double, int64_t, cudaStream_t);
template void launch_axpby<float>(float*, const float*, double, double, int64_t, cudaStream_t);
template void launch_scale_into<double>(double*, const double*, const double*, int, int64_t, cudaStream_t);
template void launch_scale_into<float>(float*, const float*, const double*, int, int64_t, cudaStream_t);
template void launch_lincomb_add<double, double>(double*, const double* const*, int, const double*, int64_t, cudaStream_t);
template void launch_lincomb_add<double, float>(double*, const float* const*, int, const double*, int64_t, cudaStream_t);
template void launch_lincomb_add<float, float>(float*, const float* const*, int, const double*, int64_t, cudaStream_t);
template void launch_time_mix<double, double>(const double*, int64_t, double*, int64_t, int, const double*, int64_t,
                                              cudaStream_t);
template void launch_time_mix<float, float>(const float*, int64_t, float*, int64_t, int, const double*, int64_t, cudaStream_t);
template void launch_time_mix<double, float>(const double*, int64_t, float*, int64_t, int, const double*, int64_t, cudaStream_t);

// y_r = a x_r + b y_r on `rows` vectors of length n at stride s (one row per grid y)
template <typename T>
__global__ void k_axpby_rows(T* __restrict__ y, const T* __restrict__ x, T a, T b, int64_t n, int64_t s) {
  const int64_t off = (int64_t)blockIdx.y * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[off + e] = a * x[off + e] + b * y[off + e];
}
template <typename T>
void launch_axpby_rows(T* y, const T* x, double a, double b, int64_t n, int rows, int64_t s, cudaStream_t st) {
  int gx = (int)((n + 255) / 256);
  const int cap = seg_gx(rows) * 2;
  if (gx > cap) gx = cap;
  (note_launch(), k_axpby_rows<T><<<dim3(gx, rows), 256, 0, st>>>(y, x, (T)a, (T)b, n, s));
}

template void launch_seg_multidot<double>(const double* const*, int, const double*, const Seg&, double*, double*, int, cudaStream_t);
template void launch_seg_multidot<float>(const float* const*, int, const float*, const Seg&, double*, double*, int, cudaStream_t);
template void launch_seg_multiaxpy_dot<double>(const double* const*, int, const double*, int, double*, const Seg&, int, double*,
                                               double*, int, cudaStream_t);
template void launch_seg_multiaxpy_dot<float>(const float* const*, int, const double*, int, float*, const Seg&, int, double*,
                                              double*, int, cudaStream_t);
template void launch_seg_scale<double>(double*, const double*, const double*, int, const Seg&, cudaStream_t);
template void launch_seg_scale<float>(float*, const float*, const double*, int, const Seg&, cudaStream_t);
template void launch_seg_axpby<double>(double*, const double*, const double*, const double*, const Seg&, cudaStream_t);
template void launch_seg_axpby<float>(float*, const float*, const double*, const double*, const Seg&, cudaStream_t);
template void launch_seg_lincomb_add<double, double>(double*, const double* const*, int, const double*, int, const Seg&, cudaStream_t);
template void launch_seg_lincomb_add<double, float>(double*, const float* const*, int, const double*, int, const Seg&, cudaStream_t);
template void launch_seg_lincomb_add<float, float>(float*, const float* const*, int, const double*, int, const Seg&, cudaStream_t);
template void launch_seg_add_scaled<double, float>(double*, const float*, const double*, int, const Seg&, cudaStream_t);
template void launch_seg_add_scaled<double, double>(double*, const double*, const double*, int, const Seg&, cudaStream_t);

template void launch_axpby_rows<double>(double*, const double*, double, double, int64_t, int, int64_t, cudaStream_t);
template void launch_axpby_rows<float>(float*, const float*, double, double, int64_t, int, int64_t, cudaStream_t);

}  // namespace biot
