// Transform passes of the UNO preconditioner (Algorithm 2: forward unitary transform, block
// multiply with Q, inverse transform), fused with the CG vector updates around them.
//
//   pass A  (k_plane_fwd): per (field, i1) plane: r <- r - alpha p, ||r||_inf, real-to-complex
//           FFT along axis 3 and complex FFT along axis 2, all in shared memory.  The last block
//           performs the stopping test of Algorithm 1 for every (instance, load).
//   pass B  (k_line):      per tile of (k2, k3) positions: FFT along axis 1, s_hat = Q r_hat / n
//           with the c x c symmetric block Q(k) (Eq. (prec-sparse-def)), r . s by Parseval,
//           inverse FFT along axis 1.  The last block forms gamma and beta.
//   pass C  (k_plane_inv): inverse axis-2 FFT and complex-to-real axis-3 FFT, then
//           u <- u + alpha d_old and d <- s + beta d_old.
#pragma once
#include "kargs.h"
#include "fft.cuh"
#include <cstdlib>
#include <type_traits>

namespace unocg {

static __host__ __device__ inline int pitch_of(int n3h) { return (n3h % 2 == 0) ? n3h + 1 : n3h; }

// ============================================================================ shared-memory layout
// Plane tasks: two buffers of nrows x P complex (nrows = n2 for whole planes, the chunk height in
// row mode), then twiddles W_{N3/2}, W_{N2}, W_{N3}.
template <typename T> struct PlaneSmem {
  cplx<T>* buf;
  cplx<T>* alt;
  cplx<T>* tw3h;
  cplx<T>* tw2;
  cplx<T>* tw3;
};
template <typename T>
__device__ __forceinline__ PlaneSmem<T> plane_smem_layout(void* raw, const Grid& g, int nrows) {
  PlaneSmem<T> s;
  const int P = pitch_of(g.n3h);
  s.buf = reinterpret_cast<cplx<T>*>(raw);
  s.alt = s.buf + nrows * P;
  s.tw3h = s.alt + nrows * P;
  s.tw2 = s.tw3h + g.n3 / 2;
  s.tw3 = s.tw2 + g.n2;
  return s;
}
template <typename T>
__device__ __forceinline__ void plane_load_twiddles(const PlaneSmem<T>& s, const Grid& g, const FftTables& ft) {
  load_tw<T>(s.tw3h, ft.tw3h, g.n3 / 2);
  load_tw<T>(s.tw2, ft.tw2, g.n2);
  load_tw<T>(s.tw3, ft.tw3, g.n3);
}

// ============================================================================ pass A task
// One (field, i1) plane: CG mode r <- r - alpha p (alpha != 0), |r| max; standalone mode reads
// src.  Forward r2c FFT along axis 3 and FFT along axis 2; writes the plane of `hat`.
// Returns max |r| over the plane (valid in every thread).  Call with the whole block.
template <typename T>
__device__ double plane_fwd_task(const PlaneFwdArgs<T>& a, const PlaneSmem<T>& sm, int bl, int plane,
                                 double alpha, double* red_sh, int row0 = 0, int nrows = 0) {
  using C = cplx<T>;
  const Grid& g = a.g;
  const int n3h = g.n3h, Nh = g.n3 / 2, P = pitch_of(n3h);
  const UDiv rNh = udiv_of(Nh), rn3h = udiv_of(n3h);
  const int comp = plane / g.n1, i1 = plane - comp * g.n1;
  const long long field = (long long)bl * a.c + comp;
  const bool whole = nrows == 0;
  if (whole) nrows = g.n2;
  const long long base = (field * g.n1 + i1) * (long long)g.n2 * g.n3 + (long long)row0 * g.n3;
  const int npair = nrows * Nh;
  C* buf = sm.buf;
  T lmax = (T)0;
  constexpr int U = 8;  // loads in flight per thread
  if (a.standalone) {
    const C* __restrict__ src = reinterpret_cast<const C*>(a.src + base);
    for (int i0 = threadIdx.x; i0 < npair; i0 += U * blockDim.x) {
      C v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * blockDim.x;
        if (idx < npair) v[u] = src[idx];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * blockDim.x;
        if (idx < npair) {
          int i2 = udiv(idx, rNh), m = idx - i2 * Nh;
          buf[i2 * P + m] = v[u];
        }
      }
    }
  } else {
    C* __restrict__ r = reinterpret_cast<C*>(a.r + base);
    const C* __restrict__ p = reinterpret_cast<const C*>(a.p + base);
    const T al = (T)alpha;
    const bool upd = alpha != 0.0;
    for (int i0 = threadIdx.x; i0 < npair; i0 += U * blockDim.x) {
      C v[U], q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * blockDim.x;
        if (idx < npair) {
          v[u] = r[idx];
          if (upd) q[u] = p[idx];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = i0 + u * blockDim.x;
        if (idx < npair) {
          int i2 = udiv(idx, rNh), m = idx - i2 * Nh;
          C w = v[u];
          if (upd) {
            w.x -= al * q[u].x;
            w.y -= al * q[u].y;
            r[idx] = w;
          }
          lmax = fmax(lmax, fmax(fabs(w.x), fabs(w.y)));
          buf[i2 * P + m] = w;
        }
      }
    }
  }
  __syncthreads();
  C* res = fft_lines<T, -1>(buf, sm.alt, nrows, P, 1, a.ft.p3h, sm.tw3h);
  r2c_post<T>(res, nrows, P, Nh, sm.tw3);
  if (whole) res = fft_lines<T, -1>(res, res == buf ? sm.alt : buf, n3h, 1, P, a.ft.p2, sm.tw2);
  C* out = a.hat + (field * g.n1 + i1) * (long long)g.n2 * n3h + (long long)row0 * n3h;
  const int nout = nrows * n3h;
  for (int idx = threadIdx.x; idx < nout; idx += blockDim.x) {
    int k2 = udiv(idx, rn3h), k3 = idx - k2 * n3h;
    out[idx] = res[k2 * P + k3];
  }
  if (a.standalone) {
    __syncthreads();
    return 0.0;
  }
  return block_max_t(lmax, red_sh);  // contains the barrier that protects the buffers
}

template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_plane_fwd(PlaneFwdArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  PlaneSmem<T> sm = plane_smem_layout<T>(smem_raw, a.g, a.rows ? a.rows : a.g.n2);
  plane_load_twiddles<T>(sm, a.g, a.ft);
  const int bl = blockIdx.y;
  bool active = true;
  double alpha = 0.0;
  if (!a.standalone) {
    active = !a.sc[bl].done && (!a.after_replace || a.sc[bl].need_replace);
    alpha = a.after_replace ? 0.0 : a.sc[bl].alpha;
  }
  double bmax = 0.0;
  if (active) {
    if (a.rows) {
      const int chunks = a.g.n2 / a.rows;
      const int plane = blockIdx.x / chunks, ch = blockIdx.x - plane * chunks;
      bmax = plane_fwd_task<T>(a, sm, bl, plane, alpha, red_sh, ch * a.rows, a.rows);
    } else {
      bmax = plane_fwd_task<T>(a, sm, bl, blockIdx.x, alpha, red_sh);
    }
  }
  if (a.standalone) return;
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bmax);
  if (last_block(a.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.ticket = 0u;
  }
}

// ============================================================================ pass B task
template <typename T, typename QT> struct QLoad;
template <typename T> struct QLoad<T, double> {
  static __device__ __forceinline__ T get(const double* q, long long i) { return (T)__ldg(q + i); }
};
template <typename T> struct QLoad<T, float> {
  static __device__ __forceinline__ T get(const float* q, long long i) { return (T)__ldg(q + i); }
};
template <typename T> struct QLoad<T, __nv_bfloat16> {
  static __device__ __forceinline__ T get(const __nv_bfloat16* q, long long i) {
    return (T)__bfloat162float(__ldg(q + i));
  }
};

template <typename T> struct LineSmem {
  cplx<T>* buf;
  cplx<T>* alt;
  cplx<T>* gbuf;
  cplx<T>* galt;
  cplx<T>* tw1;
};
template <typename T, int CC, int MODE>
__device__ __forceinline__ LineSmem<T> line_smem_layout(void* raw, const Grid& g, int tb) {
  LineSmem<T> s;
  const size_t SZ = (size_t)g.n1 * CC * tb;
  s.buf = reinterpret_cast<cplx<T>*>(raw);
  s.alt = s.buf + SZ;
  s.gbuf = s.buf + 2 * SZ;
  s.galt = s.buf + 3 * SZ;
  s.tw1 = s.buf + (MODE == 2 ? 4 : 2) * SZ;
  return s;
}

// One tile of TB consecutive (k2, k3) positions of one (instance, load), all c components:
// FFT along axis 1, s_hat = Q r_hat / n, Parseval partial of r . s (and of r . s_old for the
// flexible variant), inverse FFT along axis 1.  mode 0: CG, 1: apply, 2: backward.
// Returns (gamma, rs_old) partial sums of the tile, valid in thread 0.
template <typename T, typename QT, int CC, int MODE>
__device__ double2 line_task(const LineArgs<T, QT>& a, const LineSmem<T>& sm, int bl, int tile, double* red_sh) {
  using C = cplx<T>;
  const int TB = a.tb;
  const UDiv rTB = udiv_of(TB), rn3h = udiv_of(a.g.n3h);
  const Grid& g = a.g;
  const int n1 = g.n1;
  const int M = g.n2 * g.n3h;
  const int pos0 = tile * TB;
  const int nt = min(TB, M - pos0);
  const int LW = CC * TB;
  DotAcc<T> gam, rso;
  const long long fbase = (long long)bl * CC * n1 * M;
  constexpr int U = 8;
  for (int i0 = threadIdx.x; i0 < n1 * LW; i0 += U * blockDim.x) {
    C v[U], gv[U], so[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      v[u] = mk<T>((T)0, (T)0);
      gv[u] = v[u];
      so[u] = v[u];
      if (idx < n1 * LW) {
        int rest = udiv(idx, rTB), t = idx - rest * TB;
        int comp = rest % CC, k1 = rest / CC;
        if (t < nt) {
          long long gi = fbase + ((long long)comp * n1 + k1) * M + pos0 + t;
          v[u] = a.hat[gi];
          if (MODE == 2) gv[u] = a.ghat[gi];
          if (MODE == 0 && a.flexible) so[u] = a.shat[gi];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < n1 * LW) {
        int rest = udiv(idx, rTB), t = idx - rest * TB;
        int comp = rest % CC, k1 = rest / CC;
        if (MODE == 0 && a.flexible && t < nt) {
          int k3 = (pos0 + t) - udiv(pos0 + t, rn3h) * g.n3h;
          const T w = (k3 == 0 || 2 * k3 == g.n3) ? (T)1 : (T)2;
          rso.add_prod(w * v[u].x, so[u].x);
          rso.add_prod(w * v[u].y, so[u].y);
        }
        sm.buf[k1 * LW + comp * TB + t] = v[u];
        if (MODE == 2) sm.gbuf[k1 * LW + comp * TB + t] = gv[u];
      }
    }
  }
  __syncthreads();
  C* res = fft_lines<T, -1>(sm.buf, sm.alt, LW, 1, LW, a.ft.p1, sm.tw1);
  C* gres = sm.gbuf;
  if (MODE == 2) gres = fft_lines<T, -1>(sm.gbuf, sm.galt, LW, 1, LW, a.ft.p1, sm.tw1);
  const long long qb = (long long)(bl / a.L) * a.q_inst_stride;
  const T sc = (T)a.scale;
  for (int idx = threadIdx.x; idx < n1 * TB; idx += blockDim.x) {
    int k1 = udiv(idx, rTB), t = idx - k1 * TB;
    if (t >= nt) continue;
    int pos = pos0 + t;
    int k3 = pos - udiv(pos, rn3h) * g.n3h;
    const T w = (k3 == 0 || 2 * k3 == g.n3) ? (T)1 : (T)2;
    const long long qi = qb + ((long long)k1 * M + pos) * (CC == 1 ? 1 : 6);
    C* bp = res + k1 * LW + t;
    if (MODE == 2) {
      // dL/dQ_ij(k) = w Re(conj(G_i) R_j) / n with G, R unnormalized spectra
      C* gp = gres + k1 * LW + t;
      float* out = a.gq + ((long long)k1 * M + pos) * (CC == 1 ? 1 : 6);
      if (CC == 1) {
        C R = bp[0], Gv = gp[0];
        const T gr = w * (Gv.x * R.x + Gv.y * R.y) * sc;
        atomicAdd(out, (float)gr);
      } else {
        C R0 = bp[0], R1 = bp[TB], R2 = bp[2 * TB];
        C G0 = gp[0], G1 = gp[TB], G2 = gp[2 * TB];
        auto re = [](C x, C y) { return x.x * y.x + x.y * y.y; };
        const T s = w * sc;
        atomicAdd(out + 0, (float)(s * re(G0, R0)));
        atomicAdd(out + 1, (float)(s * re(G1, R1)));
        atomicAdd(out + 2, (float)(s * (re(G0, R1) + re(G1, R0))));
        atomicAdd(out + 3, (float)(s * re(G2, R2)));
        atomicAdd(out + 4, (float)(s * (re(G1, R2) + re(G2, R1))));
        atomicAdd(out + 5, (float)(s * (re(G0, R2) + re(G2, R0))));
      }
      // the gradient w.r.t. the input is P applied to the upstream gradient
      bp = gp;
    }
    if (CC == 1) {
      T q = QLoad<T, QT>::get(a.Q, qi) * sc;
      C R = bp[0];
      C S = mk<T>(q * R.x, q * R.y);
      if (MODE == 0) {
        gam.add_prod(w * R.x, S.x);
        gam.add_prod(w * R.y, S.y);
      }
      bp[0] = S;
    } else {
      T v1 = QLoad<T, QT>::get(a.Q, qi + 0) * sc, v2 = QLoad<T, QT>::get(a.Q, qi + 1) * sc;
      T v3 = QLoad<T, QT>::get(a.Q, qi + 2) * sc, v4 = QLoad<T, QT>::get(a.Q, qi + 3) * sc;
      T v5 = QLoad<T, QT>::get(a.Q, qi + 4) * sc, v6 = QLoad<T, QT>::get(a.Q, qi + 5) * sc;
      C R0 = bp[0], R1 = bp[TB], R2 = bp[2 * TB];
      C S0 = mk<T>(v1 * R0.x + v3 * R1.x + v6 * R2.x, v1 * R0.y + v3 * R1.y + v6 * R2.y);
      C S1 = mk<T>(v3 * R0.x + v2 * R1.x + v5 * R2.x, v3 * R0.y + v2 * R1.y + v5 * R2.y);
      C S2 = mk<T>(v6 * R0.x + v5 * R1.x + v4 * R2.x, v6 * R0.y + v5 * R1.y + v4 * R2.y);
      if (MODE == 0) {
        gam.add_prod(w * R0.x, S0.x);
        gam.add_prod(w * R0.y, S0.y);
        gam.add_prod(w * R1.x, S1.x);
        gam.add_prod(w * R1.y, S1.y);
        gam.add_prod(w * R2.x, S2.x);
        gam.add_prod(w * R2.y, S2.y);
      }
      bp[0] = S0;
      bp[TB] = S1;
      bp[2 * TB] = S2;
    }
  }
  __syncthreads();
  C* ob = (MODE == 2) ? gres : res;
  C* oalt = (MODE == 2) ? (gres == sm.gbuf ? sm.galt : sm.gbuf) : (res == sm.buf ? sm.alt : sm.buf);
  ob = fft_lines<T, +1>(ob, oalt, LW, 1, LW, a.ft.p1, sm.tw1);
  for (int idx = threadIdx.x; idx < n1 * LW; idx += blockDim.x) {
    int rest = udiv(idx, rTB), t = idx - rest * TB;
    int comp = rest % CC, k1 = rest / CC;
    if (t < nt) {
      long long gi = fbase + ((long long)comp * n1 + k1) * M + pos0 + t;
      a.shat[gi] = ob[k1 * LW + comp * TB + t];
    }
  }
  double2 r;
  r.x = 0.0;
  r.y = 0.0;
  if (MODE != 0) {
    __syncthreads();
    return r;
  }
  r.x = block_sum_acc(gam, red_sh);
  r.y = block_sum_acc(rso, red_sh);
  return r;
}

template <typename T, typename QT, int CC, int NTH, int MODE>
__global__ void __launch_bounds__(NTH) k_line(LineArgs<T, QT> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  LineSmem<T> sm = line_smem_layout<T, CC, MODE>(smem_raw, a.g, a.tb);
  load_tw<T>(sm.tw1, a.ft.tw1, a.g.n1);
  const int bl = blockIdx.y;
  bool active = (MODE != 0) || !a.sc[bl].done;
  double2 pr;
  pr.x = 0.0;
  pr.y = 0.0;
  if (active) pr = line_task<T, QT, CC, MODE>(a, sm, bl, blockIdx.x, red_sh);
  if (MODE != 0) return;
  if (threadIdx.x == 0) {
    double* pp = a.red.part + ((long long)bl * gridDim.x + blockIdx.x) * 2;
    pp[0] = pr.x;
    pp[1] = pr.y;
  }
  if (last_block(a.red.ticket)) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = warp; b < a.BL; b += NTH / 32) {
      const double* pp = a.red.part + (long long)b * gridDim.x * 2;
      double sg = warp_sum_partials(pp, gridDim.x, 2);
      double sr = warp_sum_partials(pp + 1, gridDim.x, 2);
      if (lane == 0 && !a.sc[b].done) direction_update(a.sc[b], sg, sr, a.flexible);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// ============================================================================ pass C task
// Inverse FFT along axis 2 and c2r along axis 3 of one plane; CG mode: u += alpha d_old,
// d = s + beta d_old; standalone: dst = s.  Call with the whole block.
template <typename T>
__device__ void plane_inv_task(const PlaneInvArgs<T>& a, const PlaneSmem<T>& sm, int bl, int plane,
                               double alpha_d, double beta_d, int row0 = 0, int nrows = 0) {
  using C = cplx<T>;
  const Grid& g = a.g;
  const int n3h = g.n3h, Nh = g.n3 / 2, P = pitch_of(n3h);
  const UDiv rNh = udiv_of(Nh), rn3h = udiv_of(n3h);
  const int comp = plane / g.n1, i1 = plane - comp * g.n1;
  const long long field = (long long)bl * a.c + comp;
  const bool whole = nrows == 0;
  if (whole) nrows = g.n2;
  C* buf = sm.buf;
  const C* __restrict__ in = a.shat + (field * g.n1 + i1) * (long long)g.n2 * n3h + (long long)row0 * n3h;
  const int nin = nrows * n3h;
  constexpr int U = 8;
  for (int i0 = threadIdx.x; i0 < nin; i0 += U * blockDim.x) {
    C v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < nin) v[u] = in[idx];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < nin) {
        int k2 = udiv(idx, rn3h), k3 = idx - k2 * n3h;
        buf[k2 * P + k3] = v[u];
      }
    }
  }
  __syncthreads();
  C* res = buf;
  if (whole) res = fft_lines<T, +1>(buf, sm.alt, n3h, 1, P, a.ft.p2, sm.tw2);
  c2r_pre<T>(res, nrows, P, Nh, sm.tw3);
  res = fft_lines<T, +1>(res, res == buf ? sm.alt : buf, nrows, P, 1, a.ft.p3h, sm.tw3h);
  const long long base = (field * g.n1 + i1) * (long long)g.n2 * g.n3 + (long long)row0 * g.n3;
  const int npair = nrows * Nh;
  if (a.standalone) {
    C* dst = reinterpret_cast<C*>(a.dst + base);
    for (int idx = threadIdx.x; idx < npair; idx += blockDim.x) {
      int i2 = udiv(idx, rNh), m = idx - i2 * Nh;
      dst[idx] = res[i2 * P + m];
    }
  } else {
    const T alpha = (T)alpha_d, beta = (T)beta_d;
    C* __restrict__ d = reinterpret_cast<C*>(a.d + base);
    C* __restrict__ u = reinterpret_cast<C*>(a.u + base);
    for (int i0 = threadIdx.x; i0 < npair; i0 += U * blockDim.x) {
      C dv[U], uv[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int idx = i0 + q * blockDim.x;
        if (idx < npair) {
          dv[q] = d[idx];
          uv[q] = u[idx];
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int idx = i0 + q * blockDim.x;
        if (idx < npair) {
          int i2 = udiv(idx, rNh), m = idx - i2 * Nh;
          C s = res[i2 * P + m];
          C uu = uv[q];
          uu.x += alpha * dv[q].x;
          uu.y += alpha * dv[q].y;
          u[idx] = uu;
          d[idx] = mk<T>(s.x + beta * dv[q].x, s.y + beta * dv[q].y);
        }
      }
    }
  }
  __syncthreads();  // buffers are reused by the next task of this block
}

template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_plane_inv(PlaneInvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PlaneSmem<T> sm = plane_smem_layout<T>(smem_raw, a.g, a.rows ? a.rows : a.g.n2);
  const int bl = blockIdx.y;
  if (!a.standalone && a.sc[bl].done) return;
  plane_load_twiddles<T>(sm, a.g, a.ft);
  double al = a.standalone ? 0.0 : a.sc[bl].alpha, be = a.standalone ? 0.0 : a.sc[bl].beta;
  if (a.rows) {
    const int chunks = a.g.n2 / a.rows;
    const int plane = blockIdx.x / chunks, ch = blockIdx.x - plane * chunks;
    plane_inv_task<T>(a, sm, bl, plane, al, be, ch * a.rows, a.rows);
  } else {
    plane_inv_task<T>(a, sm, bl, blockIdx.x, al, be);
  }
}

// ============================================================================ axis-2 pass
// FFT along axis 2 of (field, i1) planes, in place or into a.out: a block takes a tile of TB
// consecutive k3 of one plane, all n2 rows (lines at stride n3h).
template <typename T, int DIR, int NTH>
__global__ void __launch_bounds__(NTH) k_cols(ColArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TB = 16;
  const Grid& g = a.g;
  const int n2 = g.n2, n3h = g.n3h;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* alt = buf + (size_t)n2 * TB;
  C* tw = alt + (size_t)n2 * TB;
  const long long plane = blockIdx.y;  // (bl * c + comp) * n1 + i1
  const int bl = (int)(plane / ((long long)a.c * g.n1));
  if (a.sc && (a.sc[bl].done || (a.only_pending && !a.sc[bl].just_replaced))) return;
  load_tw<T>(tw, a.ft.tw2, n2);
  const int k0 = blockIdx.x * TB;
  const int nt = min(TB, n3h - k0);
  C* base = a.data + plane * (long long)n2 * n3h + k0;
  C* obase = (a.out ? a.out : a.data) + plane * (long long)n2 * n3h + k0;
  for (int idx = threadIdx.x; idx < n2 * TB; idx += NTH) {
    const int row = idx / TB, t = idx - row * TB;
    buf[idx] = t < nt ? base[(long long)row * n3h + t] : mk<T>((T)0, (T)0);
  }
  __syncthreads();
  C* res = fft_lines<T, DIR>(buf, alt, TB, 1, TB, a.ft.p2, tw);
  for (int idx = threadIdx.x; idx < n2 * TB; idx += NTH) {
    const int row = idx / TB, t = idx - row * TB;
    if (t < nt) obase[(long long)row * n3h + t] = res[idx];
  }
}

// ============================================================================ launchers
// threads per plane block: enough warps per plane to hide shared-memory and L2 latency
#ifndef UNOCG_PLANE_NTH
#define UNOCG_PLANE_NTH 0  // 0: by plane size
#endif
#ifndef UNOCG_LINE_NTH
#define UNOCG_LINE_NTH 0
#endif
static inline int plane_threads(const Grid& g) {
  if (UNOCG_PLANE_NTH) return UNOCG_PLANE_NTH;
  const long long e = (long long)g.n2 * g.n3h;
  return e >= 1024 ? 512 : 256;  // measured: 512 beats 1024 threads on 64^2 planes
}
static inline size_t plane_smem(const Grid& g, int elem_bytes) {
  // two plane buffers + the twiddle tables of N3/2, N2 and N3
  return (2 * (size_t)g.n2 * pitch_of(g.n3h) + g.n3 / 2 + g.n2 + g.n3) * elem_bytes;
}

template <typename K, typename A>
static cudaError_t launch_k(K kern, dim3 grid, int nth, size_t smem, const A& a, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, nth, smem, s>>>(a);
  return cudaGetLastError();
}

static inline size_t rows_smem(const Grid& g, int rows, int elem_bytes) {
  return (2 * (size_t)rows * pitch_of(g.n3h) + g.n3 / 2 + g.n2 + g.n3) * elem_bytes;
}

#ifdef UNOCG_FFT_HOST_DEFS
bool plane_fits(const Grid& g, int elem_bytes) { return plane_smem(g, elem_bytes) <= 220 * 1024; }
int plane_rows(const Grid& g, int elem_bytes) {
  if (plane_reg_ok(g, elem_bytes) || plane_fits(g, elem_bytes)) return 0;
  for (int rows = g.n2 / 2; rows >= 1; --rows)
    if (g.n2 % rows == 0 && rows_smem(g, rows, elem_bytes) <= 200 * 1024) return rows;
  return -1;
}
bool grid_supported(const Grid& g, int elem_bytes) {
  if (plane_rows(g, elem_bytes) < 0) return false;
  const size_t cols = (2 * (size_t)g.n2 * 16 + g.n2) * elem_bytes;  // axis-2 pass
  return cols <= 220 * 1024 && line_smem_bytes(g, 3, elem_bytes, 0) <= 220 * 1024;
}
template <typename T> cudaError_t launch_cols(const ColArgs<T>& a, int dir, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    // 256^2 planes: the register column pass (UNOCG_COLS_REG=0, read at every launch, selects
    // the shared-memory pass below; 256^3 x 3 loads: inverse transform 302 against 333 us)
    const char* e = std::getenv("UNOCG_COLS_REG");
    if (!(e && std::atoi(e) == 0) && rows_inv256_ok(a.g)) return launch_cols_reg256(a, dir, s);
  }
  const int eb = sizeof(cplx<T>);
  size_t smem = (2 * (size_t)a.g.n2 * 16 + a.g.n2) * eb;
  dim3 grid((a.g.n3h + 15) / 16, (unsigned)((long long)a.BL * a.c * a.g.n1));
  if (dir < 0) return launch_k(k_cols<T, -1, 256>, grid, 256, smem, a, s);
  return launch_k(k_cols<T, +1, 256>, grid, 256, smem, a, s);
}
template cudaError_t launch_cols<double>(const ColArgs<double>&, int, cudaStream_t);
template cudaError_t launch_cols<float>(const ColArgs<float>&, int, cudaStream_t);
#endif

template <typename T> cudaError_t launch_plane_fwd(const PlaneFwdArgs<T>& a, cudaStream_t s) {
  const int eb = sizeof(cplx<T>);
  if (!a.rows && plane_reg_ok(a.g, eb)) return launch_plane_fwd_reg<T>(a, s);
  if (a.rows) {
    if constexpr (sizeof(T) == 4)
      if (rows_inv256_ok(a.g)) return launch_rows_fwd256(a, s);
    size_t smem = rows_smem(a.g, a.rows, eb);
    dim3 grid(a.c * a.g.n1 * (a.g.n2 / a.rows), a.BL);
    return launch_k(k_plane_fwd<T, 512>, grid, 512, smem, a, s);
  }
  if (!plane_fits(a.g, eb)) return cudaErrorInvalidValue;
  size_t smem = plane_smem(a.g, eb);
  dim3 grid(a.c * a.g.n1, a.BL);
  const int nth = plane_threads(a.g);
  if (nth == 256) return launch_k(k_plane_fwd<T, 256>, grid, 256, smem, a, s);
  if (nth == 512) return launch_k(k_plane_fwd<T, 512>, grid, 512, smem, a, s);
  return launch_k(k_plane_fwd<T, 1024>, grid, 1024, smem, a, s);
}

template <typename T> cudaError_t launch_plane_inv(const PlaneInvArgs<T>& a, cudaStream_t s) {
  const int eb = sizeof(cplx<T>);
  if (!a.rows && plane_reg_ok(a.g, eb)) return launch_plane_inv_reg<T>(a, s);
  if (a.rows) {
    if constexpr (sizeof(T) == 4)
      if (rows_inv256_ok(a.g)) return launch_rows_inv256(a, s);
    size_t smem = rows_smem(a.g, a.rows, eb);
    dim3 grid(a.c * a.g.n1 * (a.g.n2 / a.rows), a.BL);
    return launch_k(k_plane_inv<T, 512>, grid, 512, smem, a, s);
  }
  if (!plane_fits(a.g, eb)) return cudaErrorInvalidValue;
  size_t smem = plane_smem(a.g, eb);
  dim3 grid(a.c * a.g.n1, a.BL);
  const int nth = plane_threads(a.g);
  if (nth == 256) return launch_k(k_plane_inv<T, 256>, grid, 256, smem, a, s);
  if (nth == 512) return launch_k(k_plane_inv<T, 512>, grid, 512, smem, a, s);
  return launch_k(k_plane_inv<T, 1024>, grid, 1024, smem, a, s);
}

static int line_tb(int c, int elem_bytes) {
  int tb = elem_bytes == 8 ? 16 : 8;  // one 128-byte segment per (k1, comp) row
  if (c == 1) tb *= 2;
  return tb;
}

#ifdef UNOCG_FFT_HOST_DEFS
size_t line_smem_bytes(const Grid& g, int c, int elem_bytes, int mode) {
  return ((size_t)g.n1 * c * line_tb(c, elem_bytes) * (mode == 2 ? 4 : 2) + g.n1) * elem_bytes;
}
int line_blocks_x(const Grid& g, int c, int elem_bytes) {
  int tb = line_tb(c, elem_bytes);
  int M = g.n2 * g.n3h;
  return (M + tb - 1) / tb;
}
#endif

template <typename T, typename QT, int CC, int MODE>
static cudaError_t launch_line_cc(LineArgs<T, QT> a, cudaStream_t s) {
  const int eb = sizeof(cplx<T>);
  a.tb = line_tb(CC, eb);
  const size_t smem = line_smem_bytes(a.g, CC, eb, MODE);
  dim3 grid(line_blocks_x(a.g, CC, eb), a.BL);
  long long e = (long long)a.g.n1 * CC * a.tb;
  if (UNOCG_LINE_NTH) e = UNOCG_LINE_NTH * 2;
  if (e >= 2048 && UNOCG_LINE_NTH >= 1024) return launch_k(k_line<T, QT, CC, 1024, MODE>, grid, 1024, smem, a, s);
  if (e >= 1024) return launch_k(k_line<T, QT, CC, 512, MODE>, grid, 512, smem, a, s);
  return launch_k(k_line<T, QT, CC, 256, MODE>, grid, 256, smem, a, s);
}

template <typename T, typename QT>
cudaError_t launch_line(const LineArgs<T, QT>& a, int backward, cudaStream_t s) {
  // instantiated combinations: (double, double) CG + apply; (float, bf16) CG;
  // (float, float) apply + backward (training operator)
  constexpr bool cg = !(std::is_same<T, float>::value && std::is_same<QT, float>::value);
  constexpr bool apply = !std::is_same<QT, __nv_bfloat16>::value;
  constexpr bool bwd = std::is_same<T, float>::value && std::is_same<QT, float>::value;
  if (!backward && line_reg_ok(a.g, a.c, sizeof(cplx<T>))) return launch_line_reg<T, QT>(a, s);
  if (backward) {
    if constexpr (bwd) {
      if (a.c == 1) return launch_line_cc<T, QT, 1, 2>(a, s);
      return launch_line_cc<T, QT, 3, 2>(a, s);
    }
    return cudaErrorInvalidValue;
  }
  if (a.standalone) {
    if constexpr (apply) {
      if (a.c == 1) return launch_line_cc<T, QT, 1, 1>(a, s);
      return launch_line_cc<T, QT, 3, 1>(a, s);
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (cg) {
    if (a.c == 1) return launch_line_cc<T, QT, 1, 0>(a, s);
    return launch_line_cc<T, QT, 3, 0>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace unocg
