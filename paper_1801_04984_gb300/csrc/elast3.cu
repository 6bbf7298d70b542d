// FP32 3-D displacement rows of the slab operator (paper §Monolithic Approach: the
// elasticity block A of A_s, applied to every temporal level of the slab), the kernel
// every FP32 elasticity apply of the solver runs (slab applies, multigrid smoothing
// steps and residuals on every level).
//
// A is the sum of 21 Kronecker products X (x) Y (x) Z of banded 1-D Q2 operators (mass,
// stiffness, derivative coupling and its transpose) mapping input component j to output
// component i.  The kernel evaluates them by sum factorisation while it marches along z:
//
//  * a block owns an xy tile of TX x TY output nodes and a run of z planes of one column
//    (temporal level x instance);
//  * every thread owns one z line of the tile's xy halo (TX+4 x TY+4 lines, two nodes
//    each side) and keeps a 5-plane window of the three input components in registers:
//    the z pass (4 operators x 3 components) runs on that window, and the plane three
//    ahead is already being loaded while the current plane is processed;
//  * the 12 z-pass results of the plane go to shared memory; the y pass (21 terms into
//    12 pre-x arrays: output component x x operator) runs one warp per pre-x array with
//    a y line of TY outputs per lane; the x pass (4 operators per output component) and
//    the output stage follow.
//
// The z pass uses the integer taps of the reference rows (mass x30, stiffness x3,
// derivative couplings x6); the y and x passes take taps that already carry the term's
// material coefficient and every direction's scale, so each output costs 5 (vertex rows)
// or 3 (mid rows) fused multiply-adds per term.  A vertex row on the domain boundary
// differs from an interior one only in its centre tap (inputs outside the domain are
// zero), so boundary tiles add that difference after the interior formula.  Inputs on
// constrained rows are read as zero; constrained output rows return the input.  Every
// output is computed by one thread: no atomics, bitwise reproducible.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace biot {
namespace {

constexpr int TX = 28, TY = 8;        // output tile (nodes)
constexpr int HX = TX + 4, HY = TY + 4;  // z lines of the halo: 32 x 12 = 384, one per thread
constexpr int NTH = HX * HY;          // 384 threads = 12 warps: one warp per pre-x array in the y pass
constexpr int XSEG = 4;               // x-pass outputs per item
constexpr int NXSEG = TX / XSEG;      // 7 segments per row

struct Term3z { int j, i, xop, yop, zop, coef; };
// out comp i += coef * X_xop(Y_yop(Z_zop(u_j))); ops 0 M, 1 K, 2 G, 3 G^T; coef 0 -> 2mu+lam, 1 -> mu, 2 -> lam
__host__ __device__ constexpr Term3z term(int t) {
  constexpr Term3z tab[21] = {
      {0, 0, 1, 0, 0, 0}, {0, 0, 0, 1, 0, 1}, {0, 0, 0, 0, 1, 1}, {1, 0, 2, 3, 0, 1}, {2, 0, 2, 0, 3, 1},
      {1, 0, 3, 2, 0, 2}, {2, 0, 3, 0, 2, 2}, {1, 1, 1, 0, 0, 1}, {1, 1, 0, 1, 0, 0}, {1, 1, 0, 0, 1, 1},
      {2, 1, 0, 2, 3, 1}, {2, 1, 0, 3, 2, 2}, {0, 1, 3, 2, 0, 1}, {0, 1, 2, 3, 0, 2}, {2, 2, 1, 0, 0, 1},
      {2, 2, 0, 0, 1, 0}, {2, 2, 0, 1, 0, 1}, {1, 2, 0, 3, 2, 1}, {1, 2, 0, 2, 3, 2}, {0, 2, 3, 0, 2, 1},
      {0, 2, 2, 0, 3, 2}};
  return tab[t];
}

// integer taps of the reference 1-D rows: vertex (offsets -2..2), mid (-1..1), and the
// centre tap of a vertex row on the lower / upper domain boundary
__host__ __device__ constexpr float tap_v(int op, int k) {
  constexpr float v[4][5] = {{-1, 2, 8, 2, -1}, {1, -8, 14, -8, 1}, {1, -4, 0, 4, -1}, {-1, 4, 0, -4, 1}};
  return v[op][k];
}
__host__ __device__ constexpr float tap_m(int op, int k) {
  constexpr float m[4][3] = {{2, 16, 2}, {-8, 16, -8}, {-4, 0, 4}, {4, 0, -4}};
  return m[op][k];
}
__host__ __device__ constexpr float tap_lo(int op) { return op == 0 ? 4.f : (op == 1 ? 7.f : -3.f); }
__host__ __device__ constexpr float tap_hi(int op) { return op == 0 ? 4.f : (op == 1 ? 7.f : 3.f); }

// scaled taps of the y pass (per term) and of the x pass (per operator); dlo / dhi are the
// boundary-row centre-tap differences (boundary minus interior)
// One y-pass term in the order the warps run them: source z-pass array, destination pre-x
// slot, whether the accumulator is stored (and restarted) after it, and its scaled taps.
struct YEnt {
  int src, slot, flush, pad;
  float v[5], m[3], dlo, dhi;
};
struct ElastTaps {
  YEnt ye[21];
  int wbeg[13];  // warp w runs terms wbeg[w] .. wbeg[w+1]-1 (at most two)
  float xv[4][5], xm[4][3], xdlo[4], xdhi[4];
};

struct ElastArgs {
  int nx, ny, nz, ntx;
  int64_t nn;      // nodes per component
  int fm[3];       // constrained-face bits per component (bit 2*dir+side)
  int zchunk;      // planes per block
  float au[MAXR];  // column scale tau * w_k, indexed by column / udiv
  int udiv;
};

__device__ __forceinline__ bool face_free(int m, int gx, int gy, int gz, int nx, int ny, int nz) {
  return !(((m & 1) && gx == 0) || ((m & 2) && gx == nx - 1) || ((m & 4) && gy == 0) || ((m & 8) && gy == ny - 1) ||
           ((m & 16) && gz == 0) || ((m & 32) && gz == nz - 1));
}

// asynchronous 4-byte global -> shared copies (completed per thread by cp_async_wait_all)
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// z pass of one component's window w[0..4] (planes z-2..z+2) into 4 operator outputs
template <bool VERTEX>
__device__ __forceinline__ void zpass(const float (&w)[5], float (&o)[4], int bnd) {
#pragma unroll
  for (int op = 0; op < 4; ++op) {
    float a;
    if (VERTEX) {
      a = tap_v(op, 0) * w[0] + tap_v(op, 1) * w[1] + tap_v(op, 2) * w[2] + tap_v(op, 3) * w[3] + tap_v(op, 4) * w[4];
      if (bnd < 0) a += (tap_lo(op) - tap_v(op, 2)) * w[2];
      if (bnd > 0) a += (tap_hi(op) - tap_v(op, 2)) * w[2];
    } else {
      a = tap_m(op, 0) * w[1] + tap_m(op, 1) * w[2] + tap_m(op, 2) * w[3];
    }
    o[op] = a;
  }
}

// pre-x slots: array Q in slot Q; the 4-term arrays 4 and 8 are split into two partial slots
// (4, 12) and (8, 13) so that no warp of the y pass carries more than two terms
constexpr int NSLOT = 14;

// y pass of one warp, lane = halo column hx: the warp's terms from the table (the same code for
// every warp keeps the kernel small for the instruction cache; the table index is warp-uniform),
// a y line of TY outputs per term, accumulated per destination slot.  ylo / yhi >= 0: tile
// output row that is the lower / upper domain boundary.
__device__ __forceinline__ void ypass_warp(int warp, const ElastTaps& tp, const float* __restrict__ zp, float* __restrict__ px, int hx,
                                           int ylo, int yhi) {
  const int e0 = tp.wbeg[warp], e1 = tp.wbeg[warp + 1];
  float acc[TY];
#pragma unroll
  for (int o = 0; o < TY; ++o) acc[o] = 0.f;
  for (int e = e0; e < e1; ++e) {
    const YEnt& t = tp.ye[e];
    const float* src = zp + t.src * (HY * HX) + hx;
    float w[HY];
#pragma unroll
    for (int y = 0; y < HY; ++y) w[y] = src[y * HX];
    const float v0 = t.v[0], v1 = t.v[1], v2 = t.v[2], v3 = t.v[3], v4 = t.v[4];
    const float m0 = t.m[0], m1 = t.m[1], m2 = t.m[2];
#pragma unroll
    for (int o = 0; o < TY; ++o) {
      if ((o & 1) == 0) {
        acc[o] = fmaf(v0, w[o], acc[o]);
        acc[o] = fmaf(v1, w[o + 1], acc[o]);
        acc[o] = fmaf(v2, w[o + 2], acc[o]);
        acc[o] = fmaf(v3, w[o + 3], acc[o]);
        acc[o] = fmaf(v4, w[o + 4], acc[o]);
      } else {
        acc[o] = fmaf(m0, w[o + 1], acc[o]);
        acc[o] = fmaf(m1, w[o + 2], acc[o]);
        acc[o] = fmaf(m2, w[o + 3], acc[o]);
      }
    }
    if (ylo >= 0 || yhi >= 0) {
#pragma unroll
      for (int o = 0; o < TY; o += 2) {
        if (o == ylo) acc[o] = fmaf(t.dlo, w[o + 2], acc[o]);
        if (o == yhi) acc[o] = fmaf(t.dhi, w[o + 2], acc[o]);
      }
    }
    if (t.flush) {
      float* dst = px + t.slot * (TY * HX) + hx;
#pragma unroll
      for (int o = 0; o < TY; ++o) {
        dst[o * HX] = acc[o];
        acc[o] = 0.f;
      }
    }
  }
}

// x-pass items (output component, row, segment of XSEG outputs) run on the first warps;
// the output stage of the previous plane runs on the others at the same time
constexpr int NXITEM = 3 * TY * NXSEG;          // 168
constexpr int XWARPS = (NXITEM + 31) / 32;      // 6
constexpr int OUT_T0 = XWARPS * 32;             // first output-stage thread (192)
constexpr int NOUT_T = NTH - OUT_T0;            // 192 output-stage threads
constexpr int NOUT = 3 * TY * TX;               // 672 outputs per plane
constexpr int OUT_PER_T = (NOUT + NOUT_T - 1) / NOUT_T;  // 4

template <typename EPI>
__global__ void __launch_bounds__(NTH, 2) k_elast3_zm(const __grid_constant__ ElastTaps tp, const __grid_constant__ ElastArgs a,
                                                      const float* __restrict__ u_in, int64_t su, float* __restrict__ y,
                                                      int64_t sy, const __grid_constant__ EPI ep) {
  extern __shared__ __align__(16) float smem_e3[];
  float* zp = smem_e3;                        // z-pass results of the plane: [4 j + zop][hy][hx]
  float* px = zp + 12 * HY * HX;              // pre-x slots: [slot][y][hx]
  float* so_base = px + NSLOT * TY * HX;      // outputs of two planes: [buf][i][y][x]
  float* eb = so_base + 2 * 3 * TY * TX;      // output-stage operands of one plane: [op][item]
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int X0 = (tile % a.ntx) * TX, Y0 = (tile / a.ntx) * TY;
  const int Z0 = blockIdx.y * a.zchunk;
  const int Z1 = min(Z0 + a.zchunk, a.nz);
  const int k = blockIdx.z;  // column
  const float au = a.au[k / a.udiv];
  const float* u = u_in + k * su;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t nn = a.nn;
  const int64_t pstride = (int64_t)nx * ny;
  const int64_t ko = (int64_t)k * sy;

  // ---- this thread's z line of the halo (z pass)
  const int hx = tid % HX, hy = tid / HX;
  const int gx = X0 + hx - 2, gy = Y0 + hy - 2;
  const bool inside = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
  bool cfree[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) cfree[c] = inside && face_free(a.fm[c] & 15, gx, gy, 1, nx, ny, 3);
  const float* ucol = u + (inside ? (int64_t)gy * nx + gx : 0);
  // plane q of component c is read unless it is outside the domain or a constrained z face
  auto zok = [&](int c, int q) {
    return q >= 0 && q < nz && !(((a.fm[c] >> 4) & 1) && q == 0) && !(((a.fm[c] >> 5) & 1) && q == nz - 1);
  };
  auto load_plane = [&](int q, float (&v)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = (cfree[c] && zok(c, q)) ? __ldg(ucol + c * nn + q * pstride) : 0.f;
  };
  float win[3][5], nxt[3];
  {
    float v[3];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      load_plane(Z0 - 2 + s, v);
#pragma unroll
      for (int c = 0; c < 3; ++c) win[c][s] = v[c];
    }
    load_plane(Z0 + 2, nxt);
  }

  // boundary rows of the tile (y pass rows, x pass outputs), -1 if none
  const int ylo = (Y0 == 0) ? 0 : -1;
  const int yhi = (ny - 1 - Y0 >= 0 && ny - 1 - Y0 < TY) ? ny - 1 - Y0 : -1;
  const int warp = tid >> 5, lane = tid & 31;

  // ---- x-pass item of this thread (plane independent)
  const bool xitem = tid < NXITEM;
  const int xi = tid / (TY * NXSEG), xrem = tid - xi * (TY * NXSEG);
  const int xyy = xrem / NXSEG, x0 = (xrem - xyy * NXSEG) * XSEG;
  bool xlo_here = false, xhi_here = false;
  int xlo_o = 0, xhi_o = 0;
  if (X0 == 0 && x0 == 0) { xlo_here = true; xlo_o = 0; }
  {
    const int xb = nx - 1 - X0 - x0;  // tile-local boundary output relative to this segment
    if (xb >= 0 && xb < XSEG) { xhi_here = true; xhi_o = xb; }
  }

  // ---- output-stage items of this thread (plane independent): in-plane offset (-1 outside the
  // domain) and a meta word: smem slot (bits 0-9), component (10-11), free on the x / y faces
  // (12), constrained on the lower / upper z face (13, 14)
  int oin[OUT_PER_T], ometa[OUT_PER_T];
#pragma unroll
  for (int q = 0; q < OUT_PER_T; ++q) {
    const int it = tid - OUT_T0 + q * NOUT_T;
    oin[q] = -1;
    ometa[q] = 0;
    if (tid >= OUT_T0 && it < NOUT) {
      const int i = it / (TY * TX), rem = it - i * (TY * TX);
      const int yy = rem / TX, xx = rem - yy * TX;
      const int ox = X0 + xx, oy = Y0 + yy;
      if (ox < nx && oy < ny) {
        const int m = i == 0 ? a.fm[0] : (i == 1 ? a.fm[1] : a.fm[2]);
        oin[q] = oy * nx + ox;
        ometa[q] = it | (i << 10) | (face_free(m & 15, ox, oy, 1, nx, ny, 3) ? 1 << 12 : 0) | (((m >> 4) & 1) << 13) |
                   (((m >> 5) & 1) << 14);
      }
    }
  }
  const int64_t coff[3] = {0, nn, 2 * nn};
  auto item_cn = [&](int q, int64_t planeoff) {
    const int i = (ometa[q] >> 10) & 3;
    return (i == 0 ? coff[0] : (i == 1 ? coff[1] : coff[2])) + planeoff + oin[q];
  };
  auto prefetch_stage = [&](int izo) {
    if (EPI::NPF == 0) return;
    const int64_t planeoff = (int64_t)izo * pstride;
#pragma unroll
    for (int q = 0; q < OUT_PER_T; ++q) {
      if (oin[q] < 0) continue;
      ep.prefetch(eb, ometa[q] & 1023, ko, item_cn(q, planeoff), u);
    }
    cp_async_commit();
  };
  auto output_stage = [&](int izo, const float* sob) {
    if (EPI::NPF > 0) cp_async_wait_all();
    const int64_t planeoff = (int64_t)izo * pstride;
    const bool zlo_plane = izo == 0, zhi_plane = izo == nz - 1;
#pragma unroll
    for (int q = 0; q < OUT_PER_T; ++q) {
      if (oin[q] < 0) continue;
      const int mt = ometa[q], it = mt & 1023;
      const bool fr = ((mt >> 12) & 1) && !(((mt >> 13) & 1) && zlo_plane) && !(((mt >> 14) & 1) && zhi_plane);
      ep.store(y, ko, item_cn(q, planeoff), fr, sob[it], u, eb, it);
    }
  };

  int buf = 0;
  for (int iz = Z0; iz < Z1; ++iz) {
    // window plane z+2 arrives; request plane z+3
#pragma unroll
    for (int c = 0; c < 3; ++c) win[c][4] = nxt[c];
    load_plane(iz + 3, nxt);
    // operands of the previous plane's output stage, which runs after the y pass
    if (tid >= OUT_T0 && iz > Z0) prefetch_stage(iz - 1);
    // ---- z pass (registers -> zp)
    {
      const int bnd = (iz == 0) ? -1 : (iz == nz - 1 ? 1 : 0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float o[4];
        if ((iz & 1) == 0) zpass<true>(win[c], o, bnd);
        else zpass<false>(win[c], o, 0);
#pragma unroll
        for (int op = 0; op < 4; ++op) zp[(c * 4 + op) * (HY * HX) + hy * HX + hx] = o[op];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int s = 0; s < 4; ++s) win[c][s] = win[c][s + 1];
      }
    }
    __syncthreads();
    // ---- y pass
    ypass_warp(warp, tp, zp, px, lane, ylo, yhi);
    __syncthreads();
    // ---- x pass of this plane on the first warps, output stage of the previous plane on the rest
    if (xitem) {
      float acc[XSEG];
#pragma unroll
      for (int o = 0; o < XSEG; ++o) acc[o] = 0.f;
#pragma unroll
      for (int op = 0; op < 4; ++op) {
        const int Q = xi * 4 + op;
        const float4* src = reinterpret_cast<const float4*>(px + (Q * TY + xyy) * HX + x0);
        float4 lo4 = src[0], hi4 = src[1];
        if (Q == 4 || Q == 8) {  // sum of the two partial slots
          const float4* s2 = reinterpret_cast<const float4*>(px + ((Q == 4 ? 12 : 13) * TY + xyy) * HX + x0);
          const float4 l2 = s2[0], h2 = s2[1];
          lo4.x += l2.x; lo4.y += l2.y; lo4.z += l2.z; lo4.w += l2.w;
          hi4.x += h2.x; hi4.y += h2.y; hi4.z += h2.z; hi4.w += h2.w;
        }
        const float w[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
#pragma unroll
        for (int o = 0; o < XSEG; ++o) {
          if ((o & 1) == 0) {
            acc[o] = fmaf(tp.xv[op][0], w[o], acc[o]);
            acc[o] = fmaf(tp.xv[op][1], w[o + 1], acc[o]);
            acc[o] = fmaf(tp.xv[op][2], w[o + 2], acc[o]);
            acc[o] = fmaf(tp.xv[op][3], w[o + 3], acc[o]);
            acc[o] = fmaf(tp.xv[op][4], w[o + 4], acc[o]);
          } else {
            acc[o] = fmaf(tp.xm[op][0], w[o + 1], acc[o]);
            acc[o] = fmaf(tp.xm[op][1], w[o + 2], acc[o]);
            acc[o] = fmaf(tp.xm[op][2], w[o + 3], acc[o]);
          }
        }
        if (xlo_here) {
#pragma unroll
          for (int o = 0; o < XSEG; o += 2)
            if (o == xlo_o) acc[o] = fmaf(tp.xdlo[op], w[o + 2], acc[o]);
        }
        if (xhi_here) {
#pragma unroll
          for (int o = 0; o < XSEG; o += 2)
            if (o == xhi_o) acc[o] = fmaf(tp.xdhi[op], w[o + 2], acc[o]);
        }
      }
      float4 r;
      r.x = au * acc[0];
      r.y = au * acc[1];
      r.z = au * acc[2];
      r.w = au * acc[3];
      *reinterpret_cast<float4*>(so_base + buf * (3 * TY * TX) + (xi * TY + xyy) * TX + x0) = r;
    } else if (iz > Z0) {
      output_stage(iz - 1, so_base + (buf ^ 1) * (3 * TY * TX));
    }
    __syncthreads();
    buf ^= 1;
  }
  // the last plane's outputs
  if (tid >= OUT_T0 && Z1 > Z0) {
    prefetch_stage(Z1 - 1);
    output_stage(Z1 - 1, so_base + (buf ^ 1) * (3 * TY * TX));
  }
}

// Output stages (the same as the generic kernels': plain, Chebyshev-Jacobi step, residual).
// NPF operands per output are copied to shared memory (slot `it` of each of NPF arrays of NOUT)
// one plane ahead, so the stage does not wait on global loads; constrained rows read the input
// directly (they are few).
struct EpiPlain {
  static constexpr int NPF = 0;
  __device__ __forceinline__ void prefetch(float*, int, int64_t, int64_t, const float*) const {}
  __device__ __forceinline__ void store(float* y, int64_t ko, int64_t cn, bool fr, float Ax, const float* u, const float*, int) const {
    y[ko + cn] = fr ? Ax : u[cn];
  }
};
struct EpiResid {
  static constexpr int NPF = 1;
  const float* b;
  __device__ __forceinline__ void prefetch(float* eb, int it, int64_t ko, int64_t cn, const float*) const {
    cp_async4(eb + it, b + ko + cn);
  }
  __device__ __forceinline__ void store(float* y, int64_t ko, int64_t cn, bool fr, float Ax, const float* u, const float* eb,
                                        int it) const {
    y[ko + cn] = __fsub_rn(eb[it], fr ? Ax : u[cn]);
  }
};
struct EpiCheb {
  static constexpr int NPF = 4;  // b, Dinv, x, d
  const float *b, *dinv;
  float *d, *xo;
  float c1, c2;
  __device__ __forceinline__ void prefetch(float* eb, int it, int64_t ko, int64_t cn, const float* u) const {
    cp_async4(eb + it, b + ko + cn);
    cp_async4(eb + NOUT + it, dinv + cn);
    cp_async4(eb + 2 * NOUT + it, u + cn);
    if (c1 != 0.f) cp_async4(eb + 3 * NOUT + it, d + ko + cn);
  }
  __device__ __forceinline__ void store(float*, int64_t ko, int64_t cn, bool fr, float Ax, const float*, const float* eb,
                                        int it) const {
    const float bi = eb[it], di = eb[NOUT + it];
    if (!fr || di == 0.f) {
      xo[ko + cn] = bi;
      d[ko + cn] = 0.f;
      return;
    }
    // explicit roundings: the stage is inlined twice (inside the plane loop and for a run's last
    // plane), and both copies must compute the same sequence whatever the compiler contracts
    float dn = __fmul_rn(__fmul_rn(c2, di), __fsub_rn(bi, Ax));
    if (c1 != 0.f) dn = __fmaf_rn(c1, eb[3 * NOUT + it], dn);
    d[ko + cn] = dn;
    xo[ko + cn] = __fadd_rn(eb[2 * NOUT + it], dn);
  }
};

template <typename EPI>
constexpr size_t elast3_smem_bytes() {
  return sizeof(float) * (12 * HY * HX + NSLOT * TY * HX + 2 * 3 * TY * TX + (EPI::NPF > 0 ? EPI::NPF : 1) * NOUT);
}

ElastTaps make_taps(const TabT<float>& tb, double lam, double mu) {
  ElastTaps t;
  std::memset(&t, 0, sizeof(t));
  const double cf[3] = {2.0 * mu + lam, mu, lam};
  // warps of the y pass: (pre-x array Q, first and last rank of its terms, slot) runs; every
  // warp carries at most two terms (warp 11 none)
  struct Run { int Q, r0, r1, slot; };
  const std::vector<std::vector<Run>> plan = {
      {{0, 0, 4, 0}}, {{2, 0, 4, 2}}, {{3, 0, 4, 3}}, {{4, 0, 2, 4}}, {{4, 2, 4, 12}}, {{8, 0, 2, 8}}, {{8, 2, 4, 13}},
      {{1, 0, 4, 1}, {5, 0, 4, 5}}, {{6, 0, 4, 6}, {7, 0, 4, 7}}, {{9, 0, 4, 9}, {10, 0, 4, 10}}, {{11, 0, 4, 11}}, {}};
  int ne = 0;
  for (int w = 0; w < 12; ++w) {
    t.wbeg[w] = ne;
    for (const Run& run : plan[w]) {
      int rank = 0;
      const int first = ne;
      for (int q = 0; q < 21; ++q) {
        const Term3z tm = term(q);
        if (tm.i * 4 + tm.xop != run.Q) continue;
        const int rk = rank++;
        if (rk < run.r0 || rk >= run.r1) continue;
        YEnt& e = t.ye[ne++];
        const double sc = cf[tm.coef] * (double)tb.opscale[2][tm.zop] * (double)tb.opscale[1][tm.yop];
        e.src = tm.j * 4 + tm.zop;
        e.slot = run.slot;
        e.flush = 0;
        for (int k = 0; k < 5; ++k) e.v[k] = (float)(sc * tap_v(tm.yop, k));
        for (int k = 0; k < 3; ++k) e.m[k] = (float)(sc * tap_m(tm.yop, k));
        e.dlo = (float)(sc * (tap_lo(tm.yop) - tap_v(tm.yop, 2)));
        e.dhi = (float)(sc * (tap_hi(tm.yop) - tap_v(tm.yop, 2)));
      }
      if (ne > first) t.ye[ne - 1].flush = 1;  // the run's last term stores its slot
    }
  }
  t.wbeg[12] = ne;
  for (int op = 0; op < 4; ++op) {
    const double s = (double)tb.opscale[0][op];
    for (int k = 0; k < 5; ++k) t.xv[op][k] = (float)(s * tap_v(op, k));
    for (int k = 0; k < 3; ++k) t.xm[op][k] = (float)(s * tap_m(op, k));
    t.xdlo[op] = (float)(s * (tap_lo(op) - tap_v(op, 2)));
    t.xdhi[op] = (float)(s * (tap_hi(op) - tap_v(op, 2)));
  }
  return t;
}

}  // namespace

// tuned planes per block by (device, nx, ny, nz, columns); filled from the tuning table on
// first use of a shape (0: none, use the heuristic)
std::mutex g_zrun_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_zrun;
thread_local int g_zrun_force = 0;  // set only while elast3_tune (on this thread) times a candidate

std::string zrun_key(int nx, int ny, int nz, int cols) {
  return "elast3_zrun|" + tune_device_tag() + "|" + std::to_string(nx) + "x" + std::to_string(ny) + "x" + std::to_string(nz) +
         "|cols" + std::to_string(cols);
}

int zrun_lookup(int nx, int ny, int nz, int cols) {
  int dev = 0;
  cudaGetDevice(&dev);
  const auto k = std::make_tuple(dev, nx, ny, nz, cols);
  std::lock_guard<std::mutex> lk(g_zrun_mu);
  auto it = g_zrun.find(k);
  if (it != g_zrun.end()) return it->second;
  const int v = std::max(0, tune_get(zrun_key(nx, ny, nz, cols)));
  g_zrun[k] = v;
  return v;
}

// host launcher (FP32, 3-D): `cols` columns of stride su / sy; column k takes au[k / udiv]
void launch_elast3_f32(const Grid& g, const TabT<float>& tb, const SlabCoef& sc, int cols, const float* u, int64_t su, float* y,
                       int64_t sy, cudaStream_t st, const UEpi<float>* epi) {
  ElastTaps tp = make_taps(tb, sc.lam, sc.mu);
  ElastArgs a;
  a.nx = g.nu[0];
  a.ny = g.nu[1];
  a.nz = g.nu[2];
  a.ntx = (a.nx + TX - 1) / TX;
  const int nty = (a.ny + TY - 1) / TY;
  a.nn = g.nnode;
  for (int c = 0; c < 3; ++c) {
    int m = 0;
    for (int f = 0; f < 6; ++f) {
      const int b = g.ubc[f];
      if (b == U_DIRICHLET || (b == U_ROLLER && c == f / 2)) m |= 1 << f;
    }
    a.fm[c] = m;
  }
  for (int k = 0; k < MAXR; ++k) a.au[k] = (float)sc.au[k];
  a.udiv = sc.udiv > 0 ? sc.udiv : 1;
  // planes per block: the tuned value for this shape, else enough blocks for about four waves
  // of two blocks per SM with runs of at least 6 planes (a run reloads 4 window planes)
  const int tiles = a.ntx * nty;
  const int tuned = g_zrun_force > 0 ? g_zrun_force : zrun_lookup(a.nx, a.ny, a.nz, cols);
  if (tuned > 0) {
    a.zchunk = std::min(tuned, a.nz);
  } else {
    int nc = (4 * 2 * 152 + tiles * cols - 1) / (tiles * cols);
    nc = std::max(1, std::min(nc, a.nz / 6));
    a.zchunk = (a.nz + nc - 1) / nc;
  }
  const int nchunk = (a.nz + a.zchunk - 1) / a.zchunk;
  const dim3 grid((unsigned)tiles, (unsigned)nchunk, (unsigned)cols);
  const int mode = epi ? epi->mode : EPI_NONE;
  prof_begin(st, 0, (double)g.nnode * cols);
  if (mode == EPI_CHEB) {
    EpiCheb e{epi->b, epi->dinv, epi->d, epi->xo, epi->c1, epi->c2};
    (note_launch(), k_elast3_zm<EpiCheb><<<grid, NTH, elast3_smem_bytes<EpiCheb>(), st>>>(tp, a, u, su, y, sy, e));
  } else if (mode == EPI_RESID) {
    EpiResid e{epi->b};
    (note_launch(), k_elast3_zm<EpiResid><<<grid, NTH, elast3_smem_bytes<EpiResid>(), st>>>(tp, a, u, su, y, sy, e));
  } else {
    (note_launch(), k_elast3_zm<EpiPlain><<<grid, NTH, elast3_smem_bytes<EpiPlain>(), st>>>(tp, a, u, su, y, sy, EpiPlain{}));
  }
  prof_end(st, 0);
}

// Time every candidate run length (planes per block) of the plain apply on this shape and keep
// the fastest (median of 5 launches after 2 warm-ups, CUDA events on `st`).  All candidates give
// bitwise-identical results.  Not to be called inside a stream capture.
void elast3_tune(const Grid& g, const TabT<float>& tb, double lam, double mu, int cols, float* u, float* y, cudaStream_t st) {
  if (g.dim != 3 || g.nnode < ELAST3_MIN_NODES || !tune_enabled()) return;
  const int nx = g.nu[0], ny = g.nu[1], nz = g.nu[2];
  if (zrun_lookup(nx, ny, nz, cols) > 0) return;
  SlabCoef sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.nt = 1;
  sc.lam = lam;
  sc.mu = mu;
  sc.au[0] = 0.1;
  sc.ucols = cols;
  sc.udiv = cols;
  if (cudaMemsetAsync(u, 0, sizeof(float) * cols * g.Nu, st) != cudaSuccess) return;
  std::vector<int> cand;
  for (int z : {4, 6, 8, 11, 16, 22, 32, 43, 65, 129, 257})
    if (z <= nz && (cand.empty() || (nz + z - 1) / z != (nz + cand.back() - 1) / cand.back())) cand.push_back(z);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  int best = 0;
  float best_ms = 1e30f;
  for (int z : cand) {
    g_zrun_force = z;
    for (int w = 0; w < 2; ++w) launch_elast3_f32(g, tb, sc, cols, u, g.Nu, y, g.Nu, st, nullptr);
    float ts[5];
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(e0, st);
      launch_elast3_f32(g, tb, sc, cols, u, g.Nu, y, g.Nu, st, nullptr);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ts[rep], e0, e1);
    }
    std::sort(ts, ts + 5);
    if (ts[2] < best_ms) {
      best_ms = ts[2];
      best = z;
    }
  }
  g_zrun_force = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // peek, not get: an error of a timed launch stays pending for the caller's launch check
  if (cudaPeekAtLastError() != cudaSuccess || best <= 0) return;
  tune_put(zrun_key(nx, ny, nz, cols), best);
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_zrun_mu);
  g_zrun[std::make_tuple(dev, nx, ny, nz, cols)] = best;
}

// opt-in dynamic shared memory of the three instantiations (called once, before any capture)
void elast3_init_attributes() {
  cudaFuncSetAttribute(k_elast3_zm<EpiCheb>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elast3_smem_bytes<EpiCheb>());
  cudaFuncSetAttribute(k_elast3_zm<EpiResid>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elast3_smem_bytes<EpiResid>());
  cudaFuncSetAttribute(k_elast3_zm<EpiPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)elast3_smem_bytes<EpiPlain>());
}

}  // namespace biot
