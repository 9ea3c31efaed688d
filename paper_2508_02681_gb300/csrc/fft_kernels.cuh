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
#include <type_traits>

namespace unocg {

static __host__ __device__ inline int pitch_of(int n3h) { return (n3h % 2 == 0) ? n3h + 1 : n3h; }

// ============================================================================ pass A
template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_plane_fwd(PlaneFwdArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  __shared__ double red_sh[32];
  const Grid& g = a.g;
  const int n3h = g.n3h, Nh = g.n3 / 2, P = pitch_of(n3h);
  const float rNh = 1.0f / (float)Nh, rn3h = 1.0f / (float)n3h;
  const int plane = blockIdx.x;  // comp * n1 + i1
  const int bl = blockIdx.y;
  const int comp = plane / g.n1, i1 = plane % g.n1;
  const long long field = (long long)bl * a.c + comp;
  C* tw3h = buf + 2 * g.n2 * P;
  C* tw2 = tw3h + Nh;
  C* tw3 = tw2 + g.n2;
  load_tw<T>(tw3h, a.ft.tw3h, Nh);
  load_tw<T>(tw2, a.ft.tw2, g.n2);
  load_tw<T>(tw3, a.ft.tw3, g.n3);
  bool active = true;
  double alpha = 0.0;
  if (!a.standalone) {
    active = !a.sc[bl].done;
    alpha = a.after_replace ? 0.0 : a.sc[bl].alpha;
  }
  double lmax = 0.0;
  if (active) {
    const long long base = (field * g.n1 + i1) * (long long)g.n2 * g.n3;
    const int npair = g.n2 * Nh;
    if (a.standalone) {
      const C* src = reinterpret_cast<const C*>(a.src + base);
      for (int idx = threadIdx.x; idx < npair; idx += NTH) {
        int i2 = fdiv(idx, rNh), m = idx - i2 * Nh;
        buf[i2 * P + m] = src[idx];
      }
    } else {
      C* r = reinterpret_cast<C*>(a.r + base);
      const C* p = reinterpret_cast<const C*>(a.p + base);
      const T al = (T)alpha;
      for (int idx = threadIdx.x; idx < npair; idx += NTH) {
        int i2 = fdiv(idx, rNh), m = idx - i2 * Nh;
        C v = r[idx];
        if (alpha != 0.0) {
          C q = p[idx];
          v.x -= al * q.x;
          v.y -= al * q.y;
          r[idx] = v;
        }
        lmax = fmax(lmax, fmax(fabs((double)v.x), fabs((double)v.y)));
        buf[i2 * P + m] = v;
      }
    }
    __syncthreads();
    // rows: half-length complex FFT, then split into the half spectrum of the real row
    C* alt = buf + g.n2 * P;
    C* res = fft_lines<T, -1>(buf, alt, g.n2, P, 1, a.ft.p3h, tw3h);
    r2c_post<T>(res, g.n2, P, Nh, tw3);
    // columns (axis 2)
    res = fft_lines<T, -1>(res, res == buf ? alt : buf, n3h, 1, P, a.ft.p2, tw2);
    C* out = a.hat + (field * g.n1 + i1) * (long long)g.n2 * n3h;
    const int nout = g.n2 * n3h;
    for (int idx = threadIdx.x; idx < nout; idx += NTH) {
      int k2 = fdiv(idx, rn3h), k3 = idx - k2 * n3h;
      out[idx] = res[k2 * P + k3];
    }
  }
  if (a.standalone) return;
  double bmax = block_max(lmax, red_sh);
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bmax);
  if (last_block(a.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.ticket = 0u;
  }
}

// ============================================================================ pass B
template <typename T, typename QT> struct QLoad;
template <typename T> struct QLoad<T, double> {
  static __device__ __forceinline__ T get(const double* q, long long i) { return (T)__ldg(q + i); }
};
template <typename T> struct QLoad<T, float> {
  static __device__ __forceinline__ T get(const float* q, long long i) { return (T)__ldg(q + i); }
};
template <typename T> struct QLoad<T, __nv_bfloat16> {
  static __device__ __forceinline__ T get(const __nv_bfloat16* q, long long i) {
    return (T)__bfloat162float(q[i]);
  }
};

// mode: 0 = CG (Parseval dots, scalars), 1 = standalone apply, 2 = backward (weight gradient)
template <typename T, typename QT, int CC, int NTH, int MODE>
__global__ void __launch_bounds__(NTH) k_line(LineArgs<T, QT> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int TB = a.tb;
  const float rTB = 1.0f / (float)TB, rn3h = 1.0f / (float)a.g.n3h;
  const size_t SZ = (size_t)a.g.n1 * CC * TB;
  C* alt = buf + SZ;
  C* gbuf = buf + 2 * SZ;  // backward: spectra of the gradient
  C* galt = buf + 3 * SZ;
  C* tw1 = buf + (MODE == 2 ? 4 : 2) * SZ;
  load_tw<T>(tw1, a.ft.tw1, a.g.n1);
  __shared__ double red_sh[32];
  const Grid& g = a.g;
  const int n1 = g.n1;
  const int M = g.n2 * g.n3h;
  const int bl = blockIdx.y;
  const int pos0 = blockIdx.x * TB;
  const int nt = min(TB, M - pos0);
  const int LW = CC * TB;  // lines per block
  bool active = (MODE != 0) || !a.sc[bl].done;
  double gam = 0.0, rso = 0.0;
  if (active) {
    const long long fbase = (long long)bl * CC * n1 * M;
    for (int idx = threadIdx.x; idx < n1 * LW; idx += NTH) {
      int rest = fdiv(idx, rTB), t = idx - rest * TB;
      int comp = rest % CC, k1 = rest / CC;
      C v = mk<T>((T)0, (T)0), gv = v;
      if (t < nt) {
        long long gi = fbase + ((long long)comp * n1 + k1) * M + pos0 + t;
        v = a.hat[gi];
        if (MODE == 2) gv = a.ghat[gi];
        if (MODE == 0 && a.flexible) {
          C so = a.shat[gi];
          int k3 = (pos0 + t) - fdiv(pos0 + t, rn3h) * g.n3h;
          double w = (k3 == 0 || 2 * k3 == g.n3) ? 1.0 : 2.0;
          rso += w * ((double)v.x * (double)so.x + (double)v.y * (double)so.y);
        }
      }
      buf[k1 * LW + comp * TB + t] = v;
      if (MODE == 2) gbuf[k1 * LW + comp * TB + t] = gv;
    }
    __syncthreads();
    C* res = fft_lines<T, -1>(buf, alt, LW, 1, LW, a.ft.p1, tw1);
    C* gres = gbuf;
    if (MODE == 2) gres = fft_lines<T, -1>(gbuf, galt, LW, 1, LW, a.ft.p1, tw1);
    const long long qb = (long long)(bl / a.L) * a.q_inst_stride;
    const T sc = (T)a.scale;
    for (int idx = threadIdx.x; idx < n1 * TB; idx += NTH) {
      int k1 = fdiv(idx, rTB), t = idx - k1 * TB;
      if (t >= nt) continue;
      int pos = pos0 + t;
      int k3 = pos - fdiv(pos, rn3h) * g.n3h;
      double w = (k3 == 0 || 2 * k3 == g.n3) ? 1.0 : 2.0;
      const long long qi = qb + ((long long)k1 * M + pos) * (CC == 1 ? 1 : 6);
      C* bp = res + k1 * LW + t;
      if (MODE == 2) {
        // dL/dQ_ij(k) = w Re(conj(G_i) R_j) / n with G, R unnormalized spectra
        C* gp = gres + k1 * LW + t;
        float* out = a.gq + ((long long)k1 * M + pos) * (CC == 1 ? 1 : 6);
        if (CC == 1) {
          C R = bp[0], Gv = gp[0];
          double gr = w * ((double)Gv.x * R.x + (double)Gv.y * R.y) * a.scale;
          atomicAdd(out, (float)gr);
        } else {
          C R0 = bp[0], R1 = bp[TB], R2 = bp[2 * TB];
          C G0 = gp[0], G1 = gp[TB], G2 = gp[2 * TB];
          auto re = [](C x, C y) { return (double)x.x * y.x + (double)x.y * y.y; };
          double s = w * a.scale;
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
        if (MODE == 0) gam += w * ((double)R.x * S.x + (double)R.y * S.y);
        bp[0] = S;
      } else {
        T v1 = QLoad<T, QT>::get(a.Q, qi + 0) * sc, v2 = QLoad<T, QT>::get(a.Q, qi + 1) * sc;
        T v3 = QLoad<T, QT>::get(a.Q, qi + 2) * sc, v4 = QLoad<T, QT>::get(a.Q, qi + 3) * sc;
        T v5 = QLoad<T, QT>::get(a.Q, qi + 4) * sc, v6 = QLoad<T, QT>::get(a.Q, qi + 5) * sc;
        C R0 = bp[0], R1 = bp[TB], R2 = bp[2 * TB];
        C S0 = mk<T>(v1 * R0.x + v3 * R1.x + v6 * R2.x, v1 * R0.y + v3 * R1.y + v6 * R2.y);
        C S1 = mk<T>(v3 * R0.x + v2 * R1.x + v5 * R2.x, v3 * R0.y + v2 * R1.y + v5 * R2.y);
        C S2 = mk<T>(v6 * R0.x + v5 * R1.x + v4 * R2.x, v6 * R0.y + v5 * R1.y + v4 * R2.y);
        if (MODE == 0)
          gam += w * ((double)R0.x * S0.x + (double)R0.y * S0.y + (double)R1.x * S1.x +
                      (double)R1.y * S1.y + (double)R2.x * S2.x + (double)R2.y * S2.y);
        bp[0] = S0;
        bp[TB] = S1;
        bp[2 * TB] = S2;
      }
    }
    __syncthreads();
    C* ob = (MODE == 2) ? gres : res;
    C* oalt = (MODE == 2) ? (gres == gbuf ? galt : gbuf) : (res == buf ? alt : buf);
    ob = fft_lines<T, +1>(ob, oalt, LW, 1, LW, a.ft.p1, tw1);
    for (int idx = threadIdx.x; idx < n1 * LW; idx += NTH) {
      int rest = fdiv(idx, rTB), t = idx - rest * TB;
      int comp = rest % CC, k1 = rest / CC;
      if (t < nt) {
        long long gi = fbase + ((long long)comp * n1 + k1) * M + pos0 + t;
        a.shat[gi] = ob[k1 * LW + comp * TB + t];
      }
    }
  }
  if (MODE != 0) return;
  double bg = block_sum(gam, red_sh);
  double br = block_sum(rso, red_sh);
  if (threadIdx.x == 0) {
    double* pp = a.red.part + ((long long)bl * gridDim.x + blockIdx.x) * 2;
    pp[0] = bg;
    pp[1] = br;
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

// ============================================================================ pass C
template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_plane_inv(PlaneInvArgs<T> a) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const Grid& g = a.g;
  const int n3h = g.n3h, Nh = g.n3 / 2, P = pitch_of(n3h);
  const float rNh = 1.0f / (float)Nh, rn3h = 1.0f / (float)n3h;
  const int plane = blockIdx.x;
  const int bl = blockIdx.y;
  const int comp = plane / g.n1, i1 = plane % g.n1;
  const long long field = (long long)bl * a.c + comp;
  if (!a.standalone && a.sc[bl].done) return;
  C* tw3h = buf + 2 * g.n2 * P;
  C* tw2 = tw3h + Nh;
  C* tw3 = tw2 + g.n2;
  load_tw<T>(tw3h, a.ft.tw3h, Nh);
  load_tw<T>(tw2, a.ft.tw2, g.n2);
  load_tw<T>(tw3, a.ft.tw3, g.n3);
  const C* in = a.shat + (field * g.n1 + i1) * (long long)g.n2 * n3h;
  const int nin = g.n2 * n3h;
  for (int idx = threadIdx.x; idx < nin; idx += NTH) {
    int k2 = fdiv(idx, rn3h), k3 = idx - k2 * n3h;
    buf[k2 * P + k3] = in[idx];
  }
  __syncthreads();
  C* alt = buf + g.n2 * P;
  C* res = fft_lines<T, +1>(buf, alt, n3h, 1, P, a.ft.p2, tw2);
  c2r_pre<T>(res, g.n2, P, Nh, tw3);
  res = fft_lines<T, +1>(res, res == buf ? alt : buf, g.n2, P, 1, a.ft.p3h, tw3h);
  const long long base = (field * g.n1 + i1) * (long long)g.n2 * g.n3;
  const int npair = g.n2 * Nh;
  if (a.standalone) {
    C* dst = reinterpret_cast<C*>(a.dst + base);
    for (int idx = threadIdx.x; idx < npair; idx += NTH) {
      int i2 = fdiv(idx, rNh), m = idx - i2 * Nh;
      dst[idx] = res[i2 * P + m];
    }
    return;
  }
  const T alpha = (T)a.sc[bl].alpha, beta = (T)a.sc[bl].beta;
  C* d = reinterpret_cast<C*>(a.d + base);
  C* u = reinterpret_cast<C*>(a.u + base);
  for (int idx = threadIdx.x; idx < npair; idx += NTH) {
    int i2 = fdiv(idx, rNh), m = idx - i2 * Nh;
    C s = res[i2 * P + m];
    C dold = d[idx];
    C uu = u[idx];
    uu.x += alpha * dold.x;
    uu.y += alpha * dold.y;
    u[idx] = uu;
    d[idx] = mk<T>(s.x + beta * dold.x, s.y + beta * dold.y);
  }
}

// ============================================================================ launchers
static inline int plane_threads(const Grid& g) { return (long long)g.n2 * g.n3h > 4096 ? 512 : 256; }
static inline size_t plane_smem(const Grid& g, int elem_bytes) {
  // two plane buffers + the twiddle tables of N3/2, N2 and N3
  return (2 * (size_t)g.n2 * pitch_of(g.n3h) + g.n3 / 2 + g.n2 + g.n3) * elem_bytes;
}

#ifdef UNOCG_FFT_HOST_DEFS
bool plane_fits(const Grid& g, int elem_bytes) { return plane_smem(g, elem_bytes) <= 220 * 1024; }
#endif

template <typename K, typename A>
static cudaError_t launch_k(K kern, dim3 grid, int nth, size_t smem, const A& a, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, nth, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_plane_fwd(const PlaneFwdArgs<T>& a, cudaStream_t s) {
  const int eb = sizeof(cplx<T>);
  if (!plane_fits(a.g, eb)) return cudaErrorInvalidValue;
  size_t smem = plane_smem(a.g, eb);
  dim3 grid(a.c * a.g.n1, a.BL);
  if (plane_threads(a.g) == 256) return launch_k(k_plane_fwd<T, 256>, grid, 256, smem, a, s);
  return launch_k(k_plane_fwd<T, 512>, grid, 512, smem, a, s);
}

template <typename T> cudaError_t launch_plane_inv(const PlaneInvArgs<T>& a, cudaStream_t s) {
  const int eb = sizeof(cplx<T>);
  if (!plane_fits(a.g, eb)) return cudaErrorInvalidValue;
  size_t smem = plane_smem(a.g, eb);
  dim3 grid(a.c * a.g.n1, a.BL);
  if (plane_threads(a.g) == 256) return launch_k(k_plane_inv<T, 256>, grid, 256, smem, a, s);
  return launch_k(k_plane_inv<T, 512>, grid, 512, smem, a, s);
}

static int line_tb(int c, int elem_bytes) {
  int tb = elem_bytes == 8 ? 16 : 8;  // one 128-byte segment per (k1, comp) row
  if (c == 1) tb *= 2;
  return tb;
}

#ifdef UNOCG_FFT_HOST_DEFS
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
  size_t smem = ((size_t)a.g.n1 * CC * a.tb * (MODE == 2 ? 4 : 2) + a.g.n1) * eb;
  dim3 grid(line_blocks_x(a.g, CC, eb), a.BL);
  return launch_k(k_line<T, QT, CC, 256, MODE>, grid, 256, smem, a, s);
}

template <typename T, typename QT>
cudaError_t launch_line(const LineArgs<T, QT>& a, int backward, cudaStream_t s) {
  // instantiated combinations: (double, double) CG + apply; (float, bf16) CG;
  // (float, float) apply + backward (training operator)
  constexpr bool cg = !(std::is_same<T, float>::value && std::is_same<QT, float>::value);
  constexpr bool apply = !std::is_same<QT, __nv_bfloat16>::value;
  constexpr bool bwd = std::is_same<T, float>::value && std::is_same<QT, float>::value;
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
