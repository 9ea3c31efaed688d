// Kernels of the Dirichlet-BC solver: the sine-transform passes of the UNO preconditioner
// (Algorithm 2 with T the DST, Dirichlet row of Table (fnocg-mode-selection-2d)) fused with the
// CG vector updates of Algorithm 1, the non-periodic K d, the residual evaluations and the
// post-processing.  Layouts and the two-lines-per-complex-transform scheme: dargs.h.
//
// One UNO-CG iteration is six kernels:
//   k_dpass<DP_MID>    DST axis 2 of r_hat
//   k_dpass<DP_QMUL>   DST axis 1, s_hat = Q r_hat, gamma = r.s (Parseval), DST axis 1, beta
//   k_dpass<DP_MID>    DST axis 2
//   k_dpass<DP_LAST>   DST axis 3, p = s + beta p
//   k_ku               q = K p, p.q, alpha (the periodic kernel on the embedding grid)
//   k_dpass<DP_FIRST>  r -= alpha q, u += alpha p, ||r||_inf, stopping test, DST axis 3 of r
#include <algorithm>

#include "../fft.cuh"
#include "../df64.cuh"
#include "../kargs.h"
#include "../stencil.cuh"
#include "../replace_elastic.cuh"
#include "dargs.h"

namespace unocg {

constexpr int kDThreads = 256;

// line addressing of one pass: `lines` lines per block, line l of length M = N_axis - 1
struct DTile {
  long long base;   // first element of this (instance, load)
  int ax, M, lines, W;
  // axis 3: rows [row0, row0 + lines) of the c M1 M2 rows
  long long row0, rows;
  // axes 1, 2: positions i3 in [i30, i30 + W)
  int i1, i2, comp, i30;
};

__device__ __forceinline__ DTile dtile(const DGrid& g, int c, int ax, int lines, int bl, int t) {
  DTile d;
  d.base = (long long)bl * c * g.ne;
  d.ax = ax;
  d.lines = ax == 1 ? c * lines : lines;
  d.W = lines;
  d.M = ax == 3 ? g.m3 : ax == 2 ? g.m2 : g.m1;  // free points per line
  d.row0 = 0; d.rows = 0; d.i1 = d.i2 = d.comp = d.i30 = 0;
  const int nb3 = (g.m3 + lines - 1) / lines;
  if (ax == 3) {
    d.row0 = (long long)t * lines;
    d.rows = (long long)c * g.m1 * g.m2;
  } else if (ax == 2) {
    d.i30 = (t % nb3) * lines;
    const int rest = t / nb3;
    d.i1 = rest % g.m1;
    d.comp = rest / g.m1;
  } else {
    d.i30 = (t % nb3) * lines;
    d.i2 = t / nb3;
  }
  return d;
}

// embedding-grid index of free point j of line l, or -1 when the line lies outside the field
// (free index j is node j + o_a on axis a)
__device__ __forceinline__ long long daddr(const DGrid& g, const DTile& d, int l, int j) {
  const int o1 = g.o[0], o2 = g.o[1], o3 = g.o[2];
  if (d.ax == 3) {
    const long long row = d.row0 + l;
    if (row >= d.rows) return -1LL;
    const int comp = (int)(row / ((long long)g.m1 * g.m2));
    const int r2 = (int)(row - (long long)comp * g.m1 * g.m2);
    const int j1 = r2 / g.m2, j2 = r2 - j1 * g.m2;
    return d.base + (((long long)comp * g.n1 + j1 + o1) * g.n2 + j2 + o2) * g.n3 + j + o3;
  }
  const int w = l % d.W, grp = l / d.W;
  const int i3 = d.i30 + w;
  if (i3 >= g.m3) return -1LL;
  if (d.ax == 2) return d.base + (((long long)d.comp * g.n1 + d.i1 + o1) * g.n2 + j + o2) * g.n3 + i3 + o3;
  return d.base + (((long long)grp * g.n1 + j + o1) * g.n2 + d.i2 + o2) * g.n3 + i3 + o3;
}

// element (l, j) of the loop over a tile: j fastest along axis 3 (contiguous rows), the
// position fastest along axes 1 and 2 (contiguous i3) -- coalesced either way
__device__ __forceinline__ void dtile_item(const DTile& d, int idx, int& l, int& j) {
  if (d.ax == 3) {
    l = idx / d.M;
    j = idx - l * d.M;
  } else {
    const int w = idx % d.W, rest = idx / d.W;
    j = rest % d.M;
    l = (rest / d.M) * d.W + w;
  }
}

// Pair buffers of one axis with N voxels: line l of a pair in the real (l even) or imaginary
// (l odd) part.  Sine transform (Dirichlet axis, dst = true): N - 1 points odd-extended to a
// complex sequence of 2N, X[k] = -Im Z[k+1] / 2 (even l), Re Z[k+1] / 2 (odd l).  Hartley
// transform (periodic axis): N points as they are, H = Re A - Im A of the line's own DFT A,
// A = (Z[k] + conj Z[-k]) / 2 (even l) or (Z[k] - conj Z[-k]) / 2i (odd l).
template <typename T>
__device__ __forceinline__ void dput(cplx<T>* buf, int P, int N, int l, int j, T x, bool dst = true) {
  T* a = reinterpret_cast<T*>(buf + (long long)(dst ? j + 1 : j) * P + (l >> 1)) + (l & 1);
  *a = x;
  if (dst) *(reinterpret_cast<T*>(buf + (long long)(2 * N - 1 - j) * P + (l >> 1)) + (l & 1)) = -x;
}
template <typename T>
__device__ __forceinline__ T dget(const cplx<T>* buf, int P, int l, int k, bool dst = true, int N = 0) {
  if (dst) {
    const cplx<T> z = buf[(long long)(k + 1) * P + (l >> 1)];
    return (l & 1) ? (T)0.5 * z.x : (T)-0.5 * z.y;
  }
  const cplx<T> z = buf[(long long)k * P + (l >> 1)];
  const cplx<T> w = buf[(long long)(k == 0 ? 0 : N - k) * P + (l >> 1)];
  return (l & 1) ? (T)0.5 * ((z.y + w.y) - (w.x - z.x)) : (T)0.5 * ((z.x + w.x) - (z.y - w.y));
}
template <typename T>
__device__ __forceinline__ void dzero_ends(cplx<T>* buf, int P, int N, bool dst = true) {
  if (!dst) return;
  for (int m = threadIdx.x; m < P; m += blockDim.x) {
    buf[m] = mk<T>((T)0, (T)0);
    buf[(long long)N * P + m] = mk<T>((T)0, (T)0);
  }
}

template <typename T> __device__ __forceinline__ T dabs(T x) { return x < (T)0 ? -x : x; }

template <typename T, int CC>
__device__ __forceinline__ void qmul(const T* __restrict__ q, const T* x, T* y) {
  if (CC == 1) {
    y[0] = q[0] * x[0];
  } else {
    // paper order v1 = Q11, v2 = Q22, v3 = Q12, v4 = Q33, v5 = Q23, v6 = Q13
    y[0] = q[0] * x[0] + q[2] * x[1] + q[5] * x[2];
    y[1] = q[2] * x[0] + q[1] * x[1] + q[4] * x[2];
    y[2] = q[5] * x[0] + q[4] * x[1] + q[3] * x[2];
  }
}

// ============================================================================ transform passes
template <typename T, int MODE, int CC>
__global__ void __launch_bounds__(kDThreads) k_dpass(DPassArgs<T> a) {
  using C = cplx<T>;
  constexpr int AX = (MODE == DP_FIRST || MODE == DP_LAST) ? 3 : (MODE == DP_MID ? 2 : 1);
  static_assert(MODE != DP_MID1 || AX == 1, "axis of the plain axis-1 pass");
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int N = AX == 3 ? g.n3 : (AX == 2 ? g.n2 : g.n1);
  const bool dst = g.bc[AX - 1] != 0;  // sine (Dirichlet axis) or Hartley (periodic axis)
  const int Lt = dst ? 2 * N : N;      // transform length
  const DTile d = dtile(g, CC, AX, a.lines, bl, blockIdx.x);
  const int P = d.lines >> 1;
  C* A = reinterpret_cast<C*>(dsm);
  C* B = A + (long long)2 * N * P;
  C* tw = B + (long long)2 * N * P;

  bool active = true;
  if (!a.standalone) {
    const CgScal& s = a.sc[bl];
    active = !s.done && (MODE != DP_FIRST || !a.after_replace || s.need_replace);
  }
  double bval = 0.0;  // rmax (DP_FIRST) or gamma partial (DP_QMUL)
  if (active) {
    load_tw<T>(tw, a.t.tw[AX - 1], Lt);
    dzero_ends<T>(A, P, N, dst);
    const int total = d.lines * d.M;
    if (MODE == DP_FIRST && !a.standalone) {
      const CgScal& s = a.sc[bl];
      const T alpha = (T)s.alpha;
      const bool upd = !a.after_replace && s.started;
      T rm = (T)0;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int l, j;
        dtile_item(d, idx, l, j);
        const long long ga = daddr(g, d, l, j);
        T x = (T)0;
        if (ga >= 0) {
          x = a.r[ga];
          if (upd) {
            x -= alpha * a.q[ga];
            a.r[ga] = x;
            a.u[ga] += alpha * a.p[ga];
          }
          rm = rm > dabs(x) ? rm : dabs(x);
        }
        dput<T>(A, P, N, l, j, x, dst);
      }
      bval = (double)rm;
    } else {
      const T* src = (MODE == DP_FIRST && a.standalone) ? a.src : a.hat;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int l, j;
        dtile_item(d, idx, l, j);
        const long long ga = daddr(g, d, l, j);
        dput<T>(A, P, N, l, j, ga >= 0 ? src[ga] : (T)0, dst);
      }
    }
    __syncthreads();
    C* res = fft_lines<T, -1>(A, B, P, 1, P, a.t.p[AX - 1], tw);
    if (MODE == DP_QMUL) {
      // block multiply on the modes (k1, k2 = i2, k3 = i3) of this tile, then the second transform
      C* oth = res == A ? B : A;
      dzero_ends<T>(oth, P, N, dst);
      DotAcc<T> acc;
      const int W = d.W;
      for (int idx = threadIdx.x; idx < W * d.M; idx += blockDim.x) {
        const int w = idx % W, k = idx / W;
        T x[CC], y[CC];
#pragma unroll
        for (int i = 0; i < CC; ++i) x[i] = dget<T>(res, P, i * W + w, k, dst, N);
        const int i3 = d.i30 + w;
        if (i3 < g.m3) {
          const long long mode = ((long long)k * g.m2 + d.i2) * g.m3 + i3;
          const T* qp = reinterpret_cast<const T*>(a.Q) + (long long)(bl / a.L) * a.q_inst_stride +
                        mode * (CC == 1 ? 1 : 6);
          qmul<T, CC>(qp, x, y);
#pragma unroll
          for (int i = 0; i < CC; ++i) acc.add_prod(x[i], y[i]);
        } else {
#pragma unroll
          for (int i = 0; i < CC; ++i) y[i] = (T)0;
        }
#pragma unroll
        for (int i = 0; i < CC; ++i) dput<T>(oth, P, N, i * W + w, k, y[i], dst);
      }
      bval = block_sum_acc(acc, red_sh);
      __syncthreads();
      res = fft_lines<T, -1>(oth, res, P, 1, P, a.t.p[AX - 1], tw);
    }
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      int l, j;
      dtile_item(d, idx, l, j);
      const long long ga = daddr(g, d, l, j);
      if (ga < 0) continue;
      const T x = dget<T>(res, P, l, j, dst, N);
      if (MODE == DP_LAST) {
        if (a.standalone) a.out[ga] = x;
        else a.p[ga] = x + (T)a.sc[bl].beta * a.p[ga];
      } else {
        a.hat[ga] = x;
      }
    }
  }
  if (a.standalone) return;
  if (MODE == DP_FIRST) {
    const double bm = block_max(active ? bval : 0.0, red_sh);
    if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bm);
    if (last_block(a.red.ticket)) {
      residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
      if (threadIdx.x == 0) *a.red.ticket = 0u;
    }
  } else if (MODE == DP_QMUL) {
    if (threadIdx.x == 0) a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bval;
    if (last_block(a.red.ticket)) {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int q = warp; q < a.BL; q += blockDim.x / 32) {
        if (a.sc[q].done) continue;
        const double gam = warp_sum_partials(a.red.part + (long long)q * gridDim.x, gridDim.x, 1);
        if (lane == 0) direction_update(a.sc[q], gam, 0.0, 0);
      }
      __syncthreads();
      if (threadIdx.x == 0) *a.red.ticket = 0u;
    }
  }
}

// ============================================================================ plane passes
// Axes 3 and 2 of one interior plane (instance-load, component, i1) in one block, the plane held
// in shared memory between the two transforms.  FWD: rows (axis 3; with the residual update,
// ||r||_inf and the stopping test in loop mode), then columns (axis 2), written to hat.  INV:
// columns of hat, then rows, written as p = s + beta p (or to out).  The row pairs (j2, j2+1)
// and column pairs (k3, k3+1) are odd-extended lines of length 2 N3 and 2 N2.
constexpr int kDPlaneThreads = 512;

template <typename T, int FWD>
__global__ void __launch_bounds__(kDPlaneThreads) k_dplane(DPassArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int c = a.c;
  const int comp = blockIdx.x / g.m1, j1 = blockIdx.x - comp * g.m1;
  const int N2 = g.n2, N3 = g.n3, M2 = g.m2, M3 = g.m3;
  const bool d2 = g.bc[1] != 0, d3 = g.bc[2] != 0;  // sine or Hartley per axis
  const int Pr = (M2 + 1) >> 1, Pc = (M3 + 1) >> 1;
  const long long half = (long long)(2 * N3 * Pr > 2 * N2 * Pc ? 2 * N3 * Pr : 2 * N2 * Pc);
  C* A = reinterpret_cast<C*>(dsm);
  C* B = A + half;
  C* tw3 = B + half;
  C* tw2 = tw3 + 2 * N3;
  // element (j2, j3) of the plane
  const long long base = (long long)bl * c * g.ne + ((long long)comp * g.n1 + j1 + g.o[0]) * g.n2 * g.n3;
  auto at = [&](int j2, int j3) { return base + (long long)(j2 + g.o[1]) * N3 + j3 + g.o[2]; };

  bool active = true;
  if (!a.standalone) {
    const CgScal& s = a.sc[bl];
    active = !s.done && (!FWD || !a.after_replace || s.need_replace);
  }
  double bval = 0.0;
  if (active) {
    load_tw<T>(tw3, a.t.tw[2], d3 ? 2 * N3 : N3);
    load_tw<T>(tw2, a.t.tw[1], d2 ? 2 * N2 : N2);
    const int total = M2 * M3;
    if (FWD) {
      // rows into A: line j2 (pair j2 / 2), point j3
      dzero_ends<T>(A, Pr, N3, d3);
      if (M2 & 1)  // the unpaired last row: its partner line is zero
        for (int j = threadIdx.x; j < M3; j += blockDim.x) dput<T>(A, Pr, N3, M2, j, (T)0, d3);
      if (!a.standalone) {
        const CgScal& s = a.sc[bl];
        const T alpha = (T)s.alpha;
        const bool upd = !a.after_replace && s.started;
        T rm = (T)0;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
          const int j2 = idx / M3, j3 = idx - j2 * M3;
          const long long ga = at(j2, j3);
          T x = a.r[ga];
          if (upd) {
            x -= alpha * a.q[ga];
            a.r[ga] = x;
            a.u[ga] += alpha * a.p[ga];
          }
          rm = rm > dabs(x) ? rm : dabs(x);
          dput<T>(A, Pr, N3, j2, j3, x, d3);
        }
        bval = (double)rm;
      } else {
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
          const int j2 = idx / M3, j3 = idx - j2 * M3;
          dput<T>(A, Pr, N3, j2, j3, a.src[at(j2, j3)], d3);
        }
      }
      __syncthreads();
      C* res = fft_lines<T, -1>(A, B, Pr, 1, Pr, a.t.p[2], tw3);
      C* oth = res == A ? B : A;
      // columns: line k3 (pair k3 / 2), point j2
      dzero_ends<T>(oth, Pc, N2, d2);
      if (M3 & 1)
        for (int j = threadIdx.x; j < M2; j += blockDim.x) dput<T>(oth, Pc, N2, M3, j, (T)0, d2);
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int j2 = idx / M3, k3 = idx - j2 * M3;
        dput<T>(oth, Pc, N2, k3, j2, dget<T>(res, Pr, j2, k3, d3, N3), d2);
      }
      __syncthreads();
      res = fft_lines<T, -1>(oth, res, Pc, 1, Pc, a.t.p[1], tw2);
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k2 = idx / M3, k3 = idx - k2 * M3;
        a.hat[at(k2, k3)] = dget<T>(res, Pc, k3, k2, d2, N2);
      }
    } else {
      // columns of hat into A: line k3, point k2
      dzero_ends<T>(A, Pc, N2, d2);
      if (M3 & 1)
        for (int j = threadIdx.x; j < M2; j += blockDim.x) dput<T>(A, Pc, N2, M3, j, (T)0, d2);
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k2 = idx / M3, k3 = idx - k2 * M3;
        dput<T>(A, Pc, N2, k3, k2, a.hat[at(k2, k3)], d2);
      }
      __syncthreads();
      C* res = fft_lines<T, -1>(A, B, Pc, 1, Pc, a.t.p[1], tw2);
      C* oth = res == A ? B : A;
      dzero_ends<T>(oth, Pr, N3, d3);
      if (M2 & 1)
        for (int j = threadIdx.x; j < M3; j += blockDim.x) dput<T>(oth, Pr, N3, M2, j, (T)0, d3);
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int j2 = idx / M3, k3 = idx - j2 * M3;
        dput<T>(oth, Pr, N3, j2, k3, dget<T>(res, Pc, k3, j2, d2, N2), d3);
      }
      __syncthreads();
      res = fft_lines<T, -1>(oth, res, Pr, 1, Pr, a.t.p[2], tw3);
      const T beta = a.standalone ? (T)0 : (T)a.sc[bl].beta;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int j2 = idx / M3, j3 = idx - j2 * M3;
        const long long ga = at(j2, j3);
        const T x = dget<T>(res, Pr, j2, j3, d3, N3);
        if (a.standalone) a.out[ga] = x;
        else a.p[ga] = x + beta * a.p[ga];
      }
    }
  }
  if (a.standalone || !FWD) return;
  const double bm = block_max(active ? bval : 0.0, red_sh);
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bm);
  if (last_block(a.red.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// ============================================================================ two periodic axes
// With periodic axes a < b the separable Hartley passes give H = (H_a x H_b) r, whose basis
// functions cas(k_a x_a) cas(k_b x_b) are not those of the Fourier transform the paper uses
// along both axes.  The true two-dimensional Hartley coefficients, cas(k_a x_a + k_b x_b), are
// T = B H over the four modes (+-k_a, +-k_b) with the orthogonal involution
// B = 1/2 [[1, 1, 1, -1], [1, 1, -1, 1], [1, -1, 1, 1], [-1, 1, 1, 1]] in the order
// (++, -+, +-, --).  For real blocks with Q(-k) = Q(k) (conjugate modes) T^T Q T equals the
// Fourier-domain F^H Q F, so this pass applies s_hat = B Q B r_hat with gamma = r.s (Parseval;
// coinciding mirror modes counted once).  One thread per canonical quadruple and third-axis mode.
template <typename T, int CC>
__global__ void __launch_bounds__(kDThreads) k_dmixq(DPassArgs<T> a, int pa, int pb) {
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int n[3] = {g.n1, g.n2, g.n3};
  const int m[3] = {g.m1, g.m2, g.m3};
  const int pc = 3 - pa - pb;  // the Dirichlet axis
  const int ha = n[pa] / 2 + 1, hb = n[pb] / 2 + 1;
  const long long total = (long long)ha * hb * m[pc];
  // consecutive threads step along axis 3 (contiguous in memory): the mirrored entries of a
  // warp then fall into a few segments (reversed order for -k3)
  const bool c_fast = pc == 2;
  const bool active = a.standalone || !a.sc[bl].done;
  DotAcc<T> acc;
  if (active) {
    const T* Qb = reinterpret_cast<const T*>(a.Q) + (long long)(bl / a.L) * a.q_inst_stride;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
      int ka, kb, kc;
      if (c_fast) {
        kc = (int)(t % m[pc]);
        const long long r = t / m[pc];
        kb = (int)(r % hb);
        ka = (int)(r / hb);
      } else {  // pb == 2: axis 3 periodic
        kb = (int)(t % hb);
        const long long r = t / hb;
        kc = (int)(r % m[pc]);
        ka = (int)(r / m[pc]);
      }
      const int kam = ka ? n[pa] - ka : 0, kbm = kb ? n[pb] - kb : 0;
      const T wgt = (T)((ka == kam ? 0.5 : 1.0) * (kb == kbm ? 0.5 : 1.0));
      long long node[4], mode[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int k[3];
        k[pa] = (q & 1) ? kam : ka;
        k[pb] = (q & 2) ? kbm : kb;
        k[pc] = kc;
        mode[q] = ((long long)k[0] * g.m2 + k[1]) * g.m3 + k[2];
        node[q] = ((long long)(k[0] + g.o[0]) * g.n2 + k[1] + g.o[1]) * g.n3 + k[2] + g.o[2];
      }
      const long long fb = (long long)bl * CC * g.ne;
      T h[4][CC], y[4][CC];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < CC; ++i) h[q][i] = a.hat[fb + i * g.ne + node[q]];
      // T = B H
      T tt[4][CC];
#pragma unroll
      for (int i = 0; i < CC; ++i) {
        tt[0][i] = (T)0.5 * (h[0][i] + h[1][i] + h[2][i] - h[3][i]);
        tt[1][i] = (T)0.5 * (h[0][i] + h[1][i] - h[2][i] + h[3][i]);
        tt[2][i] = (T)0.5 * (h[0][i] - h[1][i] + h[2][i] + h[3][i]);
        tt[3][i] = (T)0.5 * (-h[0][i] + h[1][i] + h[2][i] + h[3][i]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        qmul<T, CC>(Qb + mode[q] * (CC == 1 ? 1 : 6), tt[q], y[q]);
#pragma unroll
        for (int i = 0; i < CC; ++i) acc.add_prod(tt[q][i], wgt * y[q][i]);
      }
      // s_hat = B Y (coinciding modes receive identical values)
#pragma unroll
      for (int i = 0; i < CC; ++i) {
        const T s0 = (T)0.5 * (y[0][i] + y[1][i] + y[2][i] - y[3][i]);
        const T s1 = (T)0.5 * (y[0][i] + y[1][i] - y[2][i] + y[3][i]);
        const T s2 = (T)0.5 * (y[0][i] - y[1][i] + y[2][i] + y[3][i]);
        const T s3 = (T)0.5 * (-y[0][i] + y[1][i] + y[2][i] + y[3][i]);
        a.hat[fb + i * g.ne + node[0]] = s0;
        a.hat[fb + i * g.ne + node[1]] = s1;
        a.hat[fb + i * g.ne + node[2]] = s2;
        a.hat[fb + i * g.ne + node[3]] = s3;
      }
    }
  }
  if (a.standalone) return;
  const double bs = block_sum_acc(acc, red_sh);
  if (threadIdx.x == 0) a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bs;
  if (last_block(a.red.ticket)) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < a.BL; q += blockDim.x / 32) {
      if (a.sc[q].done) continue;
      const double gam = warp_sum_partials(a.red.part + (long long)q * gridDim.x, gridDim.x, 1);
      if (lane == 0) direction_update(a.sc[q], gam, 0.0, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// ============================================================================ f - K u (FP64)
// r = f - K u on the free nodes (replacement into r), or max |f - K u| into tmax (report)
template <typename T, int CC>
__global__ void __launch_bounds__(kDThreads) k_dres(DResArgs<T> a) {
  __shared__ double mt[2 * 256];
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int b = bl / a.L;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  if (a.only_pending && !a.sc[bl].need_replace) return;
  const uint8_t* ph = a.phase + (long long)b * g.ne;
  const double* u = a.u64 + (long long)bl * CC * g.ne;
  const double* f = a.f64 + (long long)bl * CC * g.ne;
  double lmax = 0.0;
  for (long long fi = (long long)blockIdx.x * blockDim.x + threadIdx.x; fi < g.nf;
       fi += (long long)gridDim.x * blockDim.x) {
    int i1, i2, i3;
    const long long node = dnode_of_free(g, fi, i1, i2, i3);
    double ku[CC];
    node_Ku<double, CC>(u, ph, mt, g.pg, i1, i2, i3, ku);
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      const double rr = f[i * g.ne + node] - ku[i];
      lmax = fmax(lmax, fabs(rr));
      if (a.r) a.r[(long long)bl * CC * g.ne + i * g.ne + node] = (T)rr;
    }
  }
  const double bm = block_max(lmax, red_sh);
  if (threadIdx.x == 0 && !a.r) atomic_max_nonneg(&a.sc[bl].tmax_bits, bm);
}

// ============================================================================ replacement (mixed)
// rref <- rref - K u32 on the free nodes (rref = f - K u64 before, the FP32 increment u32 since
// the last fold), every product and sum in float pairs (df64.cuh): u32 is exact, the stencil
// coefficients are integers (12 x the unit-cube Laplacian, 72 x Klam / Kmu) times the phase
// constants as pairs, and the result is rounded to FP64 once per node.  Writes r = rref (FP32)
// and max |rref| into rmax (replacement) or tmax (report).  The fold u64 += u32 follows.
template <int CC>
__global__ void __launch_bounds__(kDThreads) k_dreplace(DResArgs<float> a, const float* u32all, int into_rmax) {
  __shared__ float2 mp[2 * 256];
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int b = bl / a.L;
  const int np2 = 2 * a.mat.n_phases;
  for (int i = threadIdx.x; i < np2; i += blockDim.x) {
    const df32 v = df_from_double(a.mat.m64[(long long)b * np2 + i]);
    mp[i] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  if (a.only_pending && !a.sc[bl].need_replace) return;
  const long long n = g.ne;
  const uint8_t* ph = a.phase + (long long)b * n;
  const float* u32 = u32all + (long long)bl * CC * n;
  double* rref = const_cast<double*>(a.f64) + (long long)bl * CC * n;
  double lmax = 0.0;
  for (long long fi = (long long)blockIdx.x * blockDim.x + threadIdx.x; fi < g.nf;
       fi += (long long)gridDim.x * blockDim.x) {
    int i1, i2, i3;
    const long long node = dnode_of_free(g, fi, i1, i2, i3);
    Nbr nb;
    neighbours(g.pg, i1, i2, i3, nb);
    double kw[CC];
    if (CC == 1) {
      df32 w[3][3][3];
#pragma unroll
      for (int s1 = 0; s1 < 3; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < 3; ++s2)
#pragma unroll
          for (int s3 = 0; s3 < 3; ++s3) w[s1][s2][s3] = df_make(__ldg(u32 + nidx(nb, s1, s2, s3)));
      df32 acc = df_make(0.0f);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
        df32 t = df_make(0.0f);
        df_add_mul(t, 4.0f, w[1][1][1]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int c1 = (c >> 2) & 1, c2 = (c >> 1) & 1, c3 = c & 1;
          const int diff = (c1 != o1) + (c2 != o2) + (c3 != o3);
          if (diff >= 2) df_add_mul(t, -1.0f, w[c1 - o1 + 1][c2 - o2 + 1][c3 - o3 + 1]);
        }
        const float2 kp = mp[2 * ph[eidx(nb, o1, o2, o3)]];
        acc = df_add(acc, df_mul({kp.x, kp.y}, t));
      }
      kw[0] = df_to_double(acc) * (g.pg.h / 12.0);
    } else {
      df32 out[3] = {df_make(0.0f), df_make(0.0f), df_make(0.0f)};
#pragma unroll 1
      for (int o = 0; o < 8; ++o) {
        const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
        df32 aL[3] = {df_make(0.0f), df_make(0.0f), df_make(0.0f)};
        df32 aM[3] = {df_make(0.0f), df_make(0.0f), df_make(0.0f)};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int c1 = (c >> 2) & 1, c2 = (c >> 1) & 1, c3 = c & 1;
          const long long q = nidx(nb, c1 - o1 + 1, c2 - o2 + 1, c3 - o3 + 1);
          const df32 wk[3] = {df_make(__ldg(u32 + q)), df_make(__ldg(u32 + n + q)), df_make(__ldg(u32 + 2 * n + q))};
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              df_add_mul(aL[i], kElastic72.lam[o][i][c][k], wk[k]);
              df_add_mul(aM[i], kElastic72.mu[o][i][c][k], wk[k]);
            }
        }
        const int p = ph[eidx(nb, o1, o2, o3)];
        const float2 lp = mp[2 * p], mu = mp[2 * p + 1];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          out[i] = df_add(out[i], df_add(df_mul({lp.x, lp.y}, aL[i]), df_mul({mu.x, mu.y}, aM[i])));
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) kw[i] = df_to_double(out[i]) * (g.pg.h / 72.0);
    }
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      const double rr = rref[i * n + node] - kw[i];
      rref[i * n + node] = rr;
      if (a.r) a.r[(long long)bl * CC * n + i * n + node] = (float)rr;
      lmax = fmax(lmax, fabs(rr));
    }
  }
  const double bm = block_max(lmax, red_sh);
  if (threadIdx.x == 0) atomic_max_nonneg(into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
}

// Elastic replacement element by element in float pairs (the periodic element scheme on the
// embedding grid: u32 is zero on the Dirichlet nodes, so the forces at the free nodes are the
// Dirichlet ones); only free nodes are updated.
__global__ void __launch_bounds__(KE_THREADS) k_dreplace_el(DResArgs<float> a, const float* u32all, int into_rmax) {
  extern __shared__ __align__(16) unsigned char re_raw[];
  __shared__ float2 kc[6 * 256];
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  replace_elastic_consts(a.mat, bl / a.L, g.pg.h, kc);
  __syncthreads();
  if (a.only_pending && !a.sc[bl].need_replace) return;
  const long long off = (long long)bl * 3 * g.ne;
  const double bm = replace_elastic_tile(
      g.pg, a.phase + (long long)(bl / a.L) * g.ne, u32all + off, nullptr, df32{0.0f, 0.0f},
      const_cast<double*>(a.f64) + off, a.r ? a.r + off : nullptr, kc, blockIdx.x, red_sh,
      reinterpret_cast<float2*>(re_raw), [&](int i1, int i2, int i3) { return dfree_node(g, i1, i2, i3); });
  if (threadIdx.x == 0) atomic_max_nonneg(into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
}

// ============================================================================ Jacobi / plain CG
// part 0: r -= alpha q, u += alpha p, ||r||_inf, stopping test
// part 1: gamma = r . z with z = D^-1 r (or r), beta
// part 2: p = z + beta p
// (free nodes only; the boundary entries stay zero)
template <typename T, int PART>
__global__ void __launch_bounds__(kDThreads) k_djac(DJacArgs<T> a) {
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const CgScal& s = a.sc[bl];
  const bool active = !s.done && (PART != 0 || !a.after_replace || s.need_replace);
  const long long n = (long long)a.c * g.ne;
  const long long off = (long long)bl * n;
  const T* idg = a.invdiag ? a.invdiag + (long long)(bl / a.L) * n : nullptr;
  DotAcc<T> acc;
  T rm = (T)0;
  if (active) {
    const T alpha = (T)s.alpha, beta = (T)s.beta;
    const bool upd = !a.after_replace && s.started;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      if (!dinterior(g, i % g.ne)) continue;
      if (PART == 0) {
        T x = a.r[off + i];
        if (upd) {
          x -= alpha * a.q[off + i];
          a.r[off + i] = x;
          a.u[off + i] += alpha * a.p[off + i];
        }
        rm = rm > dabs(x) ? rm : dabs(x);
      } else {
        const T x = a.r[off + i];
        const T z = idg ? idg[i] * x : x;
        if (PART == 1) acc.add_prod(x, z);
        else a.p[off + i] = z + beta * a.p[off + i];
      }
    }
  }
  if (PART == 0) {
    const double bm = block_max(active ? (double)rm : 0.0, red_sh);
    if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bm);
    if (last_block(a.red.ticket)) {
      residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
      if (threadIdx.x == 0) *a.red.ticket = 0u;
    }
  } else if (PART == 1) {
    const double bval = block_sum_acc(acc, red_sh);
    if (threadIdx.x == 0) a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bval;
    if (last_block(a.red.ticket)) {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int q = warp; q < a.BL; q += blockDim.x / 32) {
        if (a.sc[q].done) continue;
        const double gam = warp_sum_partials(a.red.part + (long long)q * gridDim.x, gridDim.x, 1);
        if (lane == 0) direction_update(a.sc[q], gam, 0.0, 0);
      }
      __syncthreads();
      if (threadIdx.x == 0) *a.red.ticket = 0u;
    }
  }
}

// f at free node i (the element loads of Sec. 6.1 / 6.2, as node_rhs of the periodic path) with
// exact cancellation made exact: a component whose eight element terms cancel to within
// 64 ulp of their absolute sum is the zero of a homogeneous neighbourhood and is set to 0, so
// that a homogeneous cell has a zero right-hand side instead of rounding noise (which the
// relative stopping test would otherwise iterate on, and which FP32 fields cannot resolve).
template <int CC>
__device__ __forceinline__ void dnode_rhs(const uint8_t* __restrict__ ph, const double* mt, const Grid& g,
                                          int i1, int i2, int i3, const double* load, double* f) {
  Nbr nb;
  neighbours(g, i1, i2, i3, nb);
  const double q = 0.25 * g.h * g.h;
  double acc[3] = {0.0, 0.0, 0.0}, mag[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
    const int p = ph[eidx(nb, o1, o2, o3)];
    const double g1 = 2 * o1 - 1, g2 = 2 * o2 - 1, g3 = 2 * o3 - 1;
    if (CC == 1) {
      const double t = mt[2 * p] * (g1 * load[0] + g2 * load[1] + g3 * load[2]);
      acc[0] += t;
      mag[0] += fabs(t);
    } else {
      const double is2 = 0.70710678118654752440;
      const double e11 = load[0], e22 = load[1], e33 = load[2];
      const double e12 = load[3] * is2, e13 = load[4] * is2, e23 = load[5] * is2;
      const double tr = e11 + e22 + e33;
      const double la = mt[2 * p], m2 = 2.0 * mt[2 * p + 1];
      const double s11 = la * tr + m2 * e11, s22 = la * tr + m2 * e22, s33 = la * tr + m2 * e33;
      const double s12 = m2 * e12, s13 = m2 * e13, s23 = m2 * e23;
      const double t0 = s11 * g1 + s12 * g2 + s13 * g3;
      const double t1 = s12 * g1 + s22 * g2 + s23 * g3;
      const double t2 = s13 * g1 + s23 * g2 + s33 * g3;
      acc[0] += t0; acc[1] += t1; acc[2] += t2;
      mag[0] += fabs(t0); mag[1] += fabs(t1); mag[2] += fabs(t2);
    }
  }
#pragma unroll
  for (int i = 0; i < CC; ++i) f[i] = fabs(acc[i]) <= 64.0 * 2.220446049250313e-16 * mag[i] ? 0.0 : -q * acc[i];
}

// ============================================================================ set-up, post
// f (FP64) on the free nodes, zero on the boundary; r = f, u = p = q = 0 everywhere
template <int CC>
__global__ void __launch_bounds__(kDThreads) k_dinit(DInitArgs a) {
  __shared__ double mt[2 * 256];
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int b = bl / a.L, l = bl % a.L;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  const uint8_t* ph = a.phase + (long long)b * g.ne;
  for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < g.ne;
       node += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(node % g.n3);
    const long long r = node / g.n3;
    const int i2 = (int)(r % g.n2), i1 = (int)(r / g.n2);
    double f[CC];
    if (dfree_node(g, i1, i2, i3)) {
      dnode_rhs<CC>(ph, mt, g.pg, i1, i2, i3, a.loads + l * (CC == 1 ? 3 : 6), f);
    } else {
#pragma unroll
      for (int i = 0; i < CC; ++i) f[i] = 0.0;
    }
    const long long o = (long long)bl * CC * g.ne + node;
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      const long long k = o + i * g.ne;
      a.f64[k] = f[i];
      a.u64[k] = 0.0;
      if (a.u32) ((float*)a.u32)[k] = 0.f;
      if (a.fp64) {
        ((double*)a.r)[k] = f[i];
        ((double*)a.p)[k] = 0.0;
        ((double*)a.q)[k] = 0.0;
      } else {
        ((float*)a.r)[k] = (float)f[i];
        ((float*)a.p)[k] = 0.f;
        ((float*)a.q)[k] = 0.f;
      }
    }
  }
}

// D^-1 on the free nodes, zero on the boundary
template <int CC>
__global__ void __launch_bounds__(kDThreads) k_ddiag(DDiagArgs a) {
  __shared__ double mt[2 * 256];
  const DGrid& g = a.g;
  const int b = blockIdx.y;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  const uint8_t* ph = a.phase + (long long)b * g.ne;
  for (long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x; node < g.ne;
       node += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(node % g.n3);
    const long long r = node / g.n3;
    const int i2 = (int)(r % g.n2), i1 = (int)(r / g.n2);
    double dg[CC];
    const bool in = dfree_node(g, i1, i2, i3);
    if (in) node_diag<CC>(ph, mt, g.pg, i1, i2, i3, dg);
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      const long long k = (long long)b * CC * g.ne + i * g.ne + node;
      const double v = in ? 1.0 / dg[i] : 0.0;
      if (a.fp64) ((double*)a.invdiag)[k] = v;
      else ((float*)a.invdiag)[k] = (float)v;
    }
  }
}

// averaged flux / stress: out[b][i][l] += sum over voxels / n_voxels (the corner nodes on the
// far faces wrap to the zero boundary nodes)
template <int CC>
__global__ void __launch_bounds__(kDThreads) k_davg(DAvgArgs a) {
  constexpr int DIM = CC == 1 ? 3 : 6;
  __shared__ double mt[2 * 256];
  __shared__ double red_sh[32];
  const DGrid& g = a.g;
  const int b = blockIdx.y / a.L, l = blockIdx.y % a.L;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  const uint8_t* ph = a.phase + (long long)b * g.ne;
  const double* u = a.u64 + (long long)(b * a.L + l) * CC * g.ne;
  double acc[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) acc[i] = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.ne; e += (long long)gridDim.x * blockDim.x) {
    const int e3 = (int)(e % g.n3);
    const long long r = e / g.n3;
    const int e2 = (int)(r % g.n2), e1 = (int)(r / g.n2);
    double sig[DIM];
    element_mean_flux<CC>(u, mt, ph[e], g.pg, e1, e2, e3, a.loads + l * DIM, sig);
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc[i] += sig[i];
  }
  for (int i = 0; i < DIM; ++i) {
    const double s = block_sum(acc[i], red_sh);
    if (threadIdx.x == 0) atomicAdd(a.out + ((long long)b * DIM + i) * a.L + l, s / (double)g.ne);
  }
}

// u64 += u32, u32 = 0 (mixed precision, before a replacement and at the end)
__global__ void __launch_bounds__(kDThreads) k_dfold(DGrid g, int c, double* u64, float* u32, const CgScal* sc,
                                                     int only_pending) {
  const int bl = blockIdx.y;
  if (only_pending && !sc[bl].need_replace) return;
  const long long n = (long long)c * g.ne, off = (long long)bl * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    u64[off + i] += (double)u32[off + i];
    u32[off + i] = 0.f;
  }
}

// free-node fields [cnt][M1][M2][M3] <-> embedding-grid fields [cnt][N1][N2][N3] (zero boundary)
__global__ void __launch_bounds__(kDThreads) k_dscatter(DGrid g, int cnt, const double* src, double* dst) {
  const long long total = (long long)cnt * g.ne;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long comp = i / g.ne, node = i - comp * g.ne;
    const int i3 = (int)(node % g.n3);
    const long long r = node / g.n3;
    const int i2 = (int)(r % g.n2), i1 = (int)(r / g.n2);
    double v = 0.0;
    if (dfree_node(g, i1, i2, i3))
      v = src[comp * g.nf + (((long long)(i1 - g.o[0]) * g.m2 + (i2 - g.o[1])) * g.m3 + (i3 - g.o[2]))];
    dst[i] = v;
  }
}
__global__ void __launch_bounds__(kDThreads) k_dgather(DGrid g, int cnt, const double* src, double* dst) {
  const long long total = (long long)cnt * g.nf;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long comp = i / g.nf, f = i - comp * g.nf;
    int i1, i2, i3;
    const long long node = dnode_of_free(g, f, i1, i2, i3);
    dst[i] = src[comp * g.ne + node];
  }
}

// ============================================================================ launchers
size_t dst_smem_bytes(int N, int lines, int elem_bytes) {
  // two pair buffers of 2N x lines/2 complex values and the twiddle table
  return (size_t)elem_bytes * 2 * ((size_t)2 * 2 * N * (lines / 2) + 2 * N);
}

// largest even line count <= cap whose buffers fit 96 KB (at least 2)
int dst_lines_for(int N, int elem_bytes, int cap) {
  int l = cap & ~1;
  while (l > 2 && dst_smem_bytes(N, l, elem_bytes) > 96 * 1024) l -= 2;
  return l < 2 ? 2 : l;
}

int dpass_blocks(const DGrid& g, int c, int mode, int lines) {
  const int nb3 = (g.m3 + lines - 1) / lines;
  if (mode == DP_FIRST || mode == DP_LAST) {
    const long long rows = (long long)c * g.m1 * g.m2;
    return (int)((rows + lines - 1) / lines);
  }
  if (mode == DP_MID) return c * g.m1 * nb3;
  return g.m2 * nb3;  // DP_QMUL, DP_MID1
}

static int dgrid_blocks(long long m) {
  const long long b = (m + kDThreads - 1) / kDThreads;
  return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}
int dku_blocks(const DGrid& g, int c) { return ku_blocks_x(g.pg, c); }
int djac_blocks(const DGrid& g) { return dgrid_blocks(g.ne); }

template <typename T, int MODE, int CC>
static cudaError_t dpass_go(const DPassArgs<T>& a, cudaStream_t s) {
  const int ax = (MODE == DP_FIRST || MODE == DP_LAST) ? 3 : (MODE == DP_MID ? 2 : 1);
  const int N = ax == 3 ? a.g.n3 : (ax == 2 ? a.g.n2 : a.g.n1);
  const int lines = ax == 1 ? CC * a.lines : a.lines;
  const size_t smem = dst_smem_bytes(N, lines, sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(k_dpass<T, MODE, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(dpass_blocks(a.g, CC, MODE, a.lines), a.BL);
  k_dpass<T, MODE, CC><<<grid, kDThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dpass(const DPassArgs<T>& a, int mode, cudaStream_t s) {
  if (a.c == 1) {
    switch (mode) {
      case DP_FIRST: return dpass_go<T, DP_FIRST, 1>(a, s);
      case DP_MID: return dpass_go<T, DP_MID, 1>(a, s);
      case DP_QMUL: return dpass_go<T, DP_QMUL, 1>(a, s);
      case DP_MID1: return dpass_go<T, DP_MID1, 1>(a, s);
      default: return dpass_go<T, DP_LAST, 1>(a, s);
    }
  }
  switch (mode) {
    case DP_FIRST: return dpass_go<T, DP_FIRST, 3>(a, s);
    case DP_MID: return dpass_go<T, DP_MID, 3>(a, s);
    case DP_QMUL: return dpass_go<T, DP_QMUL, 3>(a, s);
    case DP_MID1: return dpass_go<T, DP_MID1, 3>(a, s);
    default: return dpass_go<T, DP_LAST, 3>(a, s);
  }
}

template <typename T>
cudaError_t launch_dku(const DKuArgs<T>& a, cudaStream_t s) {
  StencilArgs<T> ka{};
  ka.g = a.g.pg; ka.c = a.c; ka.BL = a.BL; ka.L = a.L; ka.phase = a.phase; ka.mat = a.mat;
  ka.d = a.p; ka.p = a.q; ka.sc = a.sc; ka.red = a.red; ka.standalone = a.standalone;
  return launch_ku<T>(ka, s);
}

template <typename T>
cudaError_t launch_dres(const DResArgs<T>& a, cudaStream_t s) {
  dim3 grid(dgrid_blocks(a.g.nf), a.BL);
  if (a.c == 1) k_dres<T, 1><<<grid, kDThreads, 0, s>>>(a);
  else k_dres<T, 3><<<grid, kDThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_djac(const DJacArgs<T>& a, int part, cudaStream_t s) {
  dim3 grid(djac_blocks(a.g), a.BL);
  if (part == 0) k_djac<T, 0><<<grid, kDThreads, 0, s>>>(a);
  else if (part == 1) k_djac<T, 1><<<grid, kDThreads, 0, s>>>(a);
  else k_djac<T, 2><<<grid, kDThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dinit(const DInitArgs& a, int BL, cudaStream_t s) {
  dim3 grid(dgrid_blocks(a.g.ne), BL);
  if (a.c == 1) k_dinit<1><<<grid, kDThreads, 0, s>>>(a);
  else k_dinit<3><<<grid, kDThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ddiag(const DDiagArgs& a, int B, cudaStream_t s) {
  dim3 grid(dgrid_blocks(a.g.ne), B);
  if (a.c == 1) k_ddiag<1><<<grid, kDThreads, 0, s>>>(a);
  else k_ddiag<3><<<grid, kDThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_davg(const DAvgArgs& a, int B, cudaStream_t s) {
  const long long nb = (a.g.ne + kDThreads - 1) / kDThreads;
  dim3 grid((int)(nb < 512 ? nb : 512), B * a.L);
  if (a.c == 1) k_davg<1><<<grid, kDThreads, 0, s>>>(a);
  else k_davg<3><<<grid, kDThreads, 0, s>>>(a);
  return cudaGetLastError();
}

size_t dplane_smem_bytes(const DGrid& g, int elem_bytes) {
  const long long Pr = (g.m2 + 1) / 2, Pc = (g.m3 + 1) / 2;
  const long long half = std::max(2LL * g.n3 * Pr, 2LL * g.n2 * Pc);
  return (size_t)elem_bytes * 2 * (2 * half + 2LL * g.n3 + 2LL * g.n2);
}

template <typename T>
cudaError_t launch_dplane(const DPassArgs<T>& a, int fwd, cudaStream_t s) {
  const size_t smem = dplane_smem_bytes(a.g, sizeof(T));
  auto kern = fwd ? k_dplane<T, 1> : k_dplane<T, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.c * a.g.m1, a.BL);
  kern<<<grid, kDPlaneThreads, smem, s>>>(a);
  return cudaGetLastError();
}

int dmixq_blocks(const DGrid& g, int pa, int pb) {
  const int n[3] = {g.n1, g.n2, g.n3}, m[3] = {g.m1, g.m2, g.m3};
  return dgrid_blocks((long long)(n[pa] / 2 + 1) * (n[pb] / 2 + 1) * m[3 - pa - pb]);
}

template <typename T>
cudaError_t launch_dmixq(const DPassArgs<T>& a, int pa, int pb, cudaStream_t s) {
  dim3 grid(dmixq_blocks(a.g, pa, pb), a.BL);
  if (a.c == 1) k_dmixq<T, 1><<<grid, kDThreads, 0, s>>>(a, pa, pb);
  else k_dmixq<T, 3><<<grid, kDThreads, 0, s>>>(a, pa, pb);
  return cudaGetLastError();
}
template cudaError_t launch_dmixq<double>(const DPassArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_dmixq<float>(const DPassArgs<float>&, int, int, cudaStream_t);

cudaError_t launch_dreplace(const DResArgs<float>& a, const float* u32, int into_rmax, cudaStream_t s) {
  if (a.c == 1) {
    k_dreplace<1><<<dim3(dgrid_blocks(a.g.nf), a.BL), kDThreads, 0, s>>>(a, u32, into_rmax);
    return cudaGetLastError();
  }
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_dreplace_el, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReplaceElSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_dreplace_el<<<dim3(ke_tiles(a.g.pg), a.BL), KE_THREADS, kReplaceElSmem, s>>>(a, u32, into_rmax);
  return cudaGetLastError();
}

cudaError_t launch_dfold(const DGrid& g, int c, int BL, double* u64, float* u32, const CgScal* sc, int only_pending,
                         cudaStream_t s) {
  k_dfold<<<dim3(dgrid_blocks((long long)c * g.ne), BL), kDThreads, 0, s>>>(g, c, u64, u32, sc, only_pending);
  return cudaGetLastError();
}

cudaError_t launch_dscatter(const DGrid& g, int cnt, const double* src, double* dst, cudaStream_t s) {
  k_dscatter<<<dgrid_blocks((long long)cnt * g.ne), kDThreads, 0, s>>>(g, cnt, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_dgather(const DGrid& g, int cnt, const double* src, double* dst, cudaStream_t s) {
  k_dgather<<<dgrid_blocks((long long)cnt * g.nf), kDThreads, 0, s>>>(g, cnt, src, dst);
  return cudaGetLastError();
}

template cudaError_t launch_dplane<double>(const DPassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_dplane<float>(const DPassArgs<float>&, int, cudaStream_t);
template cudaError_t launch_dpass<double>(const DPassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_dpass<float>(const DPassArgs<float>&, int, cudaStream_t);
template cudaError_t launch_dku<double>(const DKuArgs<double>&, cudaStream_t);
template cudaError_t launch_dku<float>(const DKuArgs<float>&, cudaStream_t);
template cudaError_t launch_dres<double>(const DResArgs<double>&, cudaStream_t);
template cudaError_t launch_dres<float>(const DResArgs<float>&, cudaStream_t);
template cudaError_t launch_djac<double>(const DJacArgs<double>&, int, cudaStream_t);
template cudaError_t launch_djac<float>(const DJacArgs<float>&, int, cudaStream_t);

}  // namespace unocg
