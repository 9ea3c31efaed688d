// Register-FFT versions of the three transform passes of UNO-CG (Algorithm 2), for grids whose
// axes are 2^k or 3 x 2^k points (planes N2 = N3 in {32, 48, 64, 96, 128, 192}, axis 1 in
// {16, ..., 256}).  Same
// arguments, data layouts and CG bookkeeping as the shared-memory Stockham passes in
// fft_kernels.cuh, which remain the path for every other grid.
//
//   k_plane_fwd_reg: one (field, i1) plane per block.  Row phase: every row of N3 reals is the
//     half-length complex line z[m] = x[2m] + i x[2m+1], loaded straight from global memory
//     into the registers of G3 threads (fused r <- r - alpha p and ||r||_inf), transformed
//     (fft_dist_a), split into the half spectrum X(k), k <= N3/2, in the plane buffer.  One
//     block barrier.  Column phase: every k3 column transformed along axis 2 by G2 threads and
//     written to the spectrum buffer.
//   k_plane_inv_reg: the mirror image, fused with u <- u + alpha d_old, d <- s + beta d_old.
//   k_line_reg: W positions (k2, k3) per warp, all c components: axis-1 transform, s = Q r / n,
//     Parseval partials, inverse axis-1 transform; no block barrier until the reductions.
#include "kargs.h"
#include "cg.cuh"
#include "fft_reg.cuh"

namespace unocg {

namespace {

constexpr int pitch_reg(int n3h, int cols) {
  int p = n3h > cols ? n3h : cols;
  while (p % 16 != 4) ++p;
  return p;
}

template <typename T, int N2, int N3> struct PlaneReg {
  static constexpr int Nh = N3 / 2, n3h = N3 / 2 + 1;
  static constexpr int G3 = RegSplit<Nh>::G, V3 = RegSplit<Nh>::V;
  static constexpr int G2 = RegSplit<N2>::G, V2 = RegSplit<N2>::V;
  static constexpr int RPW = 32 / G3;                  // rows per warp
  static constexpr int CW = 32 / G2;                   // columns per warp
  static constexpr int NCG = (n3h + CW - 1) / CW;      // column groups
  static constexpr int NRG = N2 / RPW;                 // row groups
  static constexpr int P = pitch_reg(n3h, NCG * CW);   // plane pitch (complex), = 4 mod 16
  // 24 values per thread (axes of 3 x 2^k points): at most 16 warps, the row and column groups
  // spread evenly over them (192^2: 25 column groups on 13 warps)
  static constexpr bool wide = V2 > 16 || V3 > 16;
  static constexpr int WORK = NCG > NRG ? NCG : NRG, ROUNDS = (WORK + 15) / 16;
  static constexpr int NW = wide ? (WORK + ROUNDS - 1) / ROUNDS
                                 : (NCG > (NRG < 16 ? NRG : 16) ? NCG : (NRG < 16 ? NRG : 16));
  static constexpr size_t smem = ((size_t)N2 * P + Nh + N2 + N3) * sizeof(cplx<T>);
  static constexpr bool fits = smem <= 220 * 1024;
  // first-group data requested with the loop state; off where it would exceed the registers
  static constexpr bool prefetch = !(sizeof(T) == 8 && N2 >= 128) && !wide;
};

}  // namespace

// ============================================================================ forward planes
template <typename T, int N2, int N3>
__global__ void __launch_bounds__(PlaneReg<T, N2, N3>::NW * 32) k_plane_fwd_reg(PlaneFwdArgs<T> a) {
  using C = cplx<T>;
  using PR = PlaneReg<T, N2, N3>;
  constexpr int Nh = PR::Nh, n3h = PR::n3h, G3 = PR::G3, V3 = PR::V3, G2 = PR::G2, V2 = PR::V2, P = PR::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  C* plane = reinterpret_cast<C*>(smem_raw);
  C* tw3h = plane + N2 * P;
  C* tw2 = tw3h + Nh;
  C* tw3 = tw2 + N2;
  load_tw_reg<T>(tw3h, a.ft.tw3h, Nh);
  load_tw_reg<T>(tw2, a.ft.tw2, N2);
  load_tw_reg<T>(tw3, a.ft.tw3, N3);
  pdl_wait();
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plane_id = blockIdx.x;
  const int comp = plane_id / a.g.n1, i1 = plane_id - comp * a.g.n1;
  const long long field = (long long)bl * a.c + comp;
  const long long base = (field * a.g.n1 + i1) * (long long)(N2 * N3);
  // row data of one row group: z[g + G3 n1] of r (or src) and of p
  auto load_rows = [&](int rg, C* v, C* q) {
    const int row = rg * PR::RPW + lane / G3, g = lane % G3;
    if (a.standalone) {
      const C* src = reinterpret_cast<const C*>(a.src + base) + row * Nh;
#pragma unroll
      for (int n1 = 0; n1 < V3; ++n1) v[n1] = src[g + G3 * n1];
    } else {
      const C* r = reinterpret_cast<const C*>(a.r + base) + row * Nh;
      const C* p = reinterpret_cast<const C*>(a.p + base) + row * Nh;
#pragma unroll
      for (int n1 = 0; n1 < V3; ++n1) v[n1] = r[g + G3 * n1];
#pragma unroll
      for (int n1 = 0; n1 < V3; ++n1) q[n1] = p[g + G3 * n1];
    }
  };
  // the first row group's data is requested together with the loop state (one memory latency)
  C v0[V3], q0[V3];
  if (PR::prefetch && warp < PR::NRG) load_rows(warp, v0, q0);
  bool active = true;
  double alpha = 0.0;
  if (!a.standalone) {
    const CgScal& st = a.sc[bl];
    active = !st.done && (!a.after_replace || st.need_replace);
    alpha = a.after_replace ? 0.0 : st.alpha;
  }
  __syncthreads();
  T lmax = (T)0;
  if (active) {
    const T al = (T)alpha;
    const bool upd = alpha != 0.0;
    // ---- rows: axis 3
    for (int rg = warp; rg < PR::NRG; rg += PR::NW) {
      const int row = rg * PR::RPW + lane / G3, g = lane % G3;
      C v[V3], q[V3];
      if (PR::prefetch && rg == warp) {
#pragma unroll
        for (int n1 = 0; n1 < V3; ++n1) {
          v[n1] = v0[n1];
          q[n1] = q0[n1];
        }
      } else {
        load_rows(rg, v, q);
      }
      if (!a.standalone) {
        if (upd) {
          C* r = reinterpret_cast<C*>(a.r + base) + row * Nh;
#pragma unroll
          for (int n1 = 0; n1 < V3; ++n1) {
            v[n1].x -= al * q[n1].x;
            v[n1].y -= al * q[n1].y;
            r[g + G3 * n1] = v[n1];
          }
        }
#pragma unroll
        for (int n1 = 0; n1 < V3; ++n1) lmax = fmax(lmax, fmax(fabs(v[n1].x), fabs(v[n1].y)));
      }
      C* rs = plane + row * P;
      fft_dist_a<Nh, -1>(v, g, rs, 1, tw3h);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < V3 / G3; ++j)
#pragma unroll
        for (int k2 = 0; k2 < G3; ++k2) rs[scat_index<Nh>(g, j, k2)] = v[j * G3 + k2];
      __syncwarp();
      for (int k = g; k <= Nh / 2; k += G3) r2c_pair<T>(rs, k, Nh, tw3);
    }
    __syncthreads();
    // ---- columns: axis 2
    C* out = a.hat + (field * a.g.n1 + i1) * (long long)(N2 * n3h);
    for (int cg = warp; cg < PR::NCG; cg += PR::NW) {
      const int col = cg * PR::CW + lane % PR::CW, g = lane / PR::CW;
      const bool on = col < n3h;
      C v[V2];
#pragma unroll
      for (int n1 = 0; n1 < V2; ++n1) v[n1] = plane[(g + G2 * n1) * P + col];
      fft_dist_a<N2, -1>(v, g, plane + col, P, tw2);
      if (on) {
#pragma unroll
        for (int j = 0; j < V2 / G2; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G2; ++k2) out[scat_index<N2>(g, j, k2) * n3h + col] = v[j * G2 + k2];
      }
      __syncwarp();
    }
  }
  pdl_trigger();
  if (a.standalone) return;
  const double bmax = block_max_t(lmax, red_sh);
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bmax);
  if (last_block(a.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.ticket = 0u;
  }
}

// ============================================================================ inverse planes
template <typename T, int N2, int N3>
__global__ void __launch_bounds__(PlaneReg<T, N2, N3>::NW * 32) k_plane_inv_reg(PlaneInvArgs<T> a) {
  using C = cplx<T>;
  using PR = PlaneReg<T, N2, N3>;
  constexpr int Nh = PR::Nh, n3h = PR::n3h, G3 = PR::G3, V3 = PR::V3, G2 = PR::G2, V2 = PR::V2, P = PR::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* plane = reinterpret_cast<C*>(smem_raw);
  C* tw3h = plane + N2 * P;
  C* tw2 = tw3h + Nh;
  C* tw3 = tw2 + N2;
  load_tw_reg<T>(tw3h, a.ft.tw3h, Nh);
  load_tw_reg<T>(tw2, a.ft.tw2, N2);
  load_tw_reg<T>(tw3, a.ft.tw3, N3);
  pdl_wait();
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plane_id = blockIdx.x;
  const int comp = plane_id / a.g.n1, i1 = plane_id - comp * a.g.n1;
  const long long field = (long long)bl * a.c + comp;
  const C* in = a.shat + (field * a.g.n1 + i1) * (long long)(N2 * n3h);
  const long long base = (field * a.g.n1 + i1) * (long long)(N2 * N3);
  auto load_cols = [&](int cg, C* v) {
    const int col = cg * PR::CW + lane % PR::CW, g = lane / PR::CW;
    const bool on = col < n3h;
#pragma unroll
    for (int j = 0; j < V2 / G2; ++j)
#pragma unroll
      for (int k2 = 0; k2 < G2; ++k2)
        v[j * G2 + k2] = on ? in[scat_index<N2>(g, j, k2) * n3h + col] : mk<T>((T)0, (T)0);
  };
  auto load_du = [&](int rg, C* dv, C* uv) {
    const int row = rg * PR::RPW + lane / G3, g = lane % G3;
    const C* d = reinterpret_cast<const C*>(a.d + base) + row * Nh;
    const C* u = reinterpret_cast<const C*>(a.u + base) + row * Nh;
#pragma unroll
    for (int n1 = 0; n1 < V3; ++n1) {
      dv[n1] = d[g + G3 * n1];
      uv[n1] = u[g + G3 * n1];
    }
  };
  // the first column group's spectrum and the first row group's d and u are requested together
  // with the loop state (one memory latency)
  C cv0[V2], dv0[V3], uv0[V3];
  if (PR::prefetch && warp < PR::NCG) load_cols(warp, cv0);
  if (PR::prefetch && !a.standalone && warp < PR::NRG) load_du(warp, dv0, uv0);
  if (!a.standalone && a.sc[bl].done) return;
  const double al_d = a.standalone ? 0.0 : a.sc[bl].alpha, be_d = a.standalone ? 0.0 : a.sc[bl].beta;
  __syncthreads();
  // ---- columns: inverse axis 2
  for (int cg = warp; cg < PR::NCG; cg += PR::NW) {
    const int col = cg * PR::CW + lane % PR::CW, g = lane / PR::CW;
    C v[V2];
    if (PR::prefetch && cg == warp) {
#pragma unroll
      for (int i = 0; i < V2; ++i) v[i] = cv0[i];
    } else {
      load_cols(cg, v);
    }
    fft_dist_b<N2, +1>(v, g, plane + col, P, tw2);
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < V2; ++n1) plane[(g + G2 * n1) * P + col] = v[n1];
    __syncwarp();
  }
  __syncthreads();
  // ---- rows: inverse axis 3 (half spectrum -> real row)
  const T alpha = (T)al_d, beta = (T)be_d;
  for (int rg = warp; rg < PR::NRG; rg += PR::NW) {
    const int row = rg * PR::RPW + lane / G3, g = lane % G3;
    C* rs = plane + row * P;
    for (int k = g; k <= Nh / 2; k += G3) c2r_pair<T>(rs, k, Nh, tw3);
    __syncwarp();
    C v[V3];
#pragma unroll
    for (int j = 0; j < V3 / G3; ++j)
#pragma unroll
      for (int k2 = 0; k2 < G3; ++k2) v[j * G3 + k2] = rs[scat_index<Nh>(g, j, k2)];
    fft_dist_b<Nh, +1>(v, g, rs, 1, tw3h);
    if (a.standalone) {
      C* dst = reinterpret_cast<C*>(a.dst + base) + row * Nh;
#pragma unroll
      for (int n1 = 0; n1 < V3; ++n1) dst[g + G3 * n1] = v[n1];
    } else {
      C* d = reinterpret_cast<C*>(a.d + base) + row * Nh;
      C* u = reinterpret_cast<C*>(a.u + base) + row * Nh;
      C dv[V3], uv[V3];
      if (PR::prefetch && rg == warp) {
#pragma unroll
        for (int n1 = 0; n1 < V3; ++n1) {
          dv[n1] = dv0[n1];
          uv[n1] = uv0[n1];
        }
      } else {
        load_du(rg, dv, uv);
      }
#pragma unroll
      for (int n1 = 0; n1 < V3; ++n1) {
        C uu = uv[n1];
        uu.x += alpha * dv[n1].x;
        uu.y += alpha * dv[n1].y;
        u[g + G3 * n1] = uu;
        d[g + G3 * n1] = mk<T>(v[n1].x + beta * dv[n1].x, v[n1].y + beta * dv[n1].y);
      }
    }
    __syncwarp();
  }
}

// ============================================================================ axis 1 + multiply
template <typename T, typename QT> struct QRead;
template <typename T> struct QRead<T, double> {
  static __device__ __forceinline__ T get(const double* q, long long i) { return (T)__ldg(q + i); }
};
template <typename T> struct QRead<T, float> {
  static __device__ __forceinline__ T get(const float* q, long long i) { return (T)__ldg(q + i); }
};
template <typename T> struct QRead<T, __nv_bfloat16> {
  static __device__ __forceinline__ T get(const __nv_bfloat16* q, long long i) {
    return (T)__bfloat162float(__ldg(q + i));
  }
};

constexpr int kLineRegWarps = 8;

template <typename T, typename QT, int CC, int N1, int MODE>
__global__ void __launch_bounds__(kLineRegWarps * 32) k_line_reg(LineArgs<T, QT> a) {
  using C = cplx<T>;
  constexpr int G = RegSplit<N1>::G, V = RegSplit<N1>::V, VG = V / G, W = 32 / G;
  constexpr int NW = kLineRegWarps;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  C* tw1 = reinterpret_cast<C*>(smem_raw);
  C* scr_all = tw1 + N1;
  load_tw_reg<T>(tw1, a.ft.tw1, N1);
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / W, w = lane % W;
  const int M = a.g.n2 * a.g.n3h;
  const int pos = (blockIdx.x * NW + warp) * W + w;
  const bool on = pos < M;
  const long long fbase = (long long)bl * CC * N1 * M;
  const long long qb = (long long)(bl / a.L) * a.q_inst_stride;
  const T sc = (T)a.scale;
  // the weights do not change during a solve: thermal ones are fetched before the wait
  T qpre[CC == 1 ? V : 1];
  if constexpr (CC == 1) {
#pragma unroll
    for (int j = 0; j < VG; ++j)
#pragma unroll
      for (int k2 = 0; k2 < G; ++k2)
        qpre[j * G + k2] = on ? QRead<T, QT>::get(a.Q, qb + (long long)scat_index<N1>(g, j, k2) * M + pos) : (T)0;
  }
  pdl_wait();
  // the spectra are requested together with the loop state (one memory latency); with one
  // component the previous s_hat comes in the same batch, with three it is read one component
  // at a time below (all six lines at once would not fit the register file)
  constexpr bool CS = CC == 1;
  C v[CC][V], so[CS ? V : 1];
#pragma unroll
  for (int cc = 0; cc < CC; ++cc)
#pragma unroll
    for (int n1 = 0; n1 < V; ++n1) {
      const long long gi = fbase + ((long long)(cc * N1 + g + G * n1)) * M + pos;
      v[cc][n1] = on ? a.hat[gi] : mk<T>((T)0, (T)0);
      if constexpr (CS)
        if (MODE == 0) so[n1] = (on && a.flexible) ? a.shat[gi] : mk<T>((T)0, (T)0);
    }
  const bool active = (MODE != 0) || !a.sc[bl].done;
  __syncthreads();
  DotAcc<T> gam, rso;
  if (active) {
    const int k3 = on ? pos % a.g.n3h : 0;
    const T wt = (k3 == 0 || 2 * k3 == a.g.n3) ? (T)1 : (T)2;
    C* scr = scr_all + (size_t)warp * W * N1 + w;
    if (MODE == 0 && a.flexible && on) {
#pragma unroll
      for (int cc = 0; cc < CC; ++cc) {
        C sl[V];
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) {
          if constexpr (CS) {
            sl[n1] = so[n1];
          } else {
            sl[n1] = a.shat[fbase + ((long long)(cc * N1 + g + G * n1)) * M + pos];
          }
        }
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) {
          rso.add_prod(wt * v[cc][n1].x, sl[n1].x);
          rso.add_prod(wt * v[cc][n1].y, sl[n1].y);
        }
      }
    }
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) fft_dist_a<N1, -1>(v[cc], g, scr, W, tw1);
    // s_hat = Q(k) r_hat(k) / n and the Parseval partial of r . s
    if (on) {
#pragma unroll
      for (int j = 0; j < VG; ++j)
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) {
          const int k1 = scat_index<N1>(g, j, k2), e = j * G + k2;
          const long long qi = qb + ((long long)k1 * M + pos) * (CC == 1 ? 1 : 6);
          if constexpr (CC == 1) {
            const T q = qpre[e] * sc;
            const C R = v[0][e];
            const C S = mk<T>(q * R.x, q * R.y);
            if (MODE == 0) {
              gam.add_prod(wt * R.x, S.x);
              gam.add_prod(wt * R.y, S.y);
            }
            v[0][e] = S;
          } else {
            const T q1 = QRead<T, QT>::get(a.Q, qi + 0) * sc, q2 = QRead<T, QT>::get(a.Q, qi + 1) * sc;
            const T q3 = QRead<T, QT>::get(a.Q, qi + 2) * sc, q4 = QRead<T, QT>::get(a.Q, qi + 3) * sc;
            const T q5 = QRead<T, QT>::get(a.Q, qi + 4) * sc, q6 = QRead<T, QT>::get(a.Q, qi + 5) * sc;
            const C R0 = v[0][e], R1 = v[1][e], R2 = v[2][e];
            const C S0 = mk<T>(q1 * R0.x + q3 * R1.x + q6 * R2.x, q1 * R0.y + q3 * R1.y + q6 * R2.y);
            const C S1 = mk<T>(q3 * R0.x + q2 * R1.x + q5 * R2.x, q3 * R0.y + q2 * R1.y + q5 * R2.y);
            const C S2 = mk<T>(q6 * R0.x + q5 * R1.x + q4 * R2.x, q6 * R0.y + q5 * R1.y + q4 * R2.y);
            if (MODE == 0) {
              gam.add_prod(wt * R0.x, S0.x);
              gam.add_prod(wt * R0.y, S0.y);
              gam.add_prod(wt * R1.x, S1.x);
              gam.add_prod(wt * R1.y, S1.y);
              gam.add_prod(wt * R2.x, S2.x);
              gam.add_prod(wt * R2.y, S2.y);
            }
            v[0][e] = S0;
            v[1][e] = S1;
            v[2][e] = S2;
          }
        }
    }
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) fft_dist_b<N1, +1>(v[cc], g, scr, W, tw1);
    if (on) {
#pragma unroll
      for (int cc = 0; cc < CC; ++cc)
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) {
          const long long gi = fbase + ((long long)(cc * N1 + g + G * n1)) * M + pos;
          a.shat[gi] = v[cc][n1];
        }
    }
  }
  pdl_trigger();
  if (MODE != 0) return;
  double2 pr;
  pr.x = block_sum_acc(gam, red_sh);
  pr.y = block_sum_acc(rso, red_sh);
  if (threadIdx.x == 0) {
    double* pp = a.red.part + ((long long)bl * gridDim.x + blockIdx.x) * 2;
    pp[0] = pr.x;
    pp[1] = pr.y;
  }
  if (last_block(a.red.ticket)) {
    for (int b = warp; b < a.BL; b += NW) {
      const double* pp = a.red.part + (long long)b * gridDim.x * 2;
      double sg = warp_sum_partials(pp, gridDim.x, 2);
      double sr = warp_sum_partials(pp + 1, gridDim.x, 2);
      if (lane == 0 && !a.sc[b].done) direction_update(a.sc[b], sg, sr, a.flexible);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// ============================================================================ host side
namespace {

template <typename K, typename A>
cudaError_t launch_reg(K kern, dim3 grid, int nth, size_t smem, const A& a, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(kern, grid, dim3(nth), smem, s, a);
}

constexpr bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

template <typename T> size_t plane_reg_smem(int n) {
  switch (n) {
    case 32: return PlaneReg<T, 32, 32>::smem;
    case 48: return PlaneReg<T, 48, 48>::smem;
    case 64: return PlaneReg<T, 64, 64>::smem;
    case 96: return PlaneReg<T, 96, 96>::smem;
    case 128: return PlaneReg<T, 128, 128>::smem;
    case 192: return PlaneReg<T, 192, 192>::smem;
    default: return 0;
  }
}

template <typename T, int N, typename Args, bool FWD>
cudaError_t plane_reg_launch(const Args& a, cudaStream_t s) {
  using PR = PlaneReg<T, N, N>;
  if constexpr (!PR::fits) {
    return cudaErrorInvalidValue;  // plane_reg_ok refuses it
  } else {
    dim3 grid(a.c * a.g.n1, a.BL);
    if constexpr (FWD) return launch_reg(k_plane_fwd_reg<T, N, N>, grid, PR::NW * 32, PR::smem, a, s);
    else return launch_reg(k_plane_inv_reg<T, N, N>, grid, PR::NW * 32, PR::smem, a, s);
  }
}

template <typename T, typename Args, bool FWD> cudaError_t plane_reg_dispatch(const Args& a, cudaStream_t s) {
  switch (a.g.n2) {
    case 32: return plane_reg_launch<T, 32, Args, FWD>(a, s);
    case 48: return plane_reg_launch<T, 48, Args, FWD>(a, s);
    case 64: return plane_reg_launch<T, 64, Args, FWD>(a, s);
    case 96: return plane_reg_launch<T, 96, Args, FWD>(a, s);
    case 128: return plane_reg_launch<T, 128, Args, FWD>(a, s);
    case 192: return plane_reg_launch<T, 192, Args, FWD>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool plane_reg_ok(const Grid& g, int elem_bytes) {
#ifdef UNOCG_NO_REG_FFT
  return false;
#endif
  if (g.n2 != g.n3) return false;
  if (!(pow2_in(g.n2, 32, 128) || g.n2 == 48 || g.n2 == 96 || g.n2 == 192)) return false;
  const size_t smem = elem_bytes == 16 ? plane_reg_smem<double>(g.n2) : plane_reg_smem<float>(g.n2);
  return smem > 0 && smem <= 220 * 1024;
}

template <typename T> cudaError_t launch_plane_fwd_reg(const PlaneFwdArgs<T>& a, cudaStream_t s) {
  return plane_reg_dispatch<T, PlaneFwdArgs<T>, true>(a, s);
}
template <typename T> cudaError_t launch_plane_inv_reg(const PlaneInvArgs<T>& a, cudaStream_t s) {
  return plane_reg_dispatch<T, PlaneInvArgs<T>, false>(a, s);
}
template cudaError_t launch_plane_fwd_reg<float>(const PlaneFwdArgs<float>&, cudaStream_t);
template cudaError_t launch_plane_fwd_reg<double>(const PlaneFwdArgs<double>&, cudaStream_t);
template cudaError_t launch_plane_inv_reg<float>(const PlaneInvArgs<float>&, cudaStream_t);
template cudaError_t launch_plane_inv_reg<double>(const PlaneInvArgs<double>&, cudaStream_t);

// axis 1: N1 in 16..256 (2^k, and 48, 96, 192) for c = 1; 2^k up to 64 for c = 3 (three
// components of V values each stay in registers, beyond that they would spill); the 24-value
// splits (96, 192) in FP32 only
bool line_reg_ok(const Grid& g, int c, int elem_bytes) {
#ifdef UNOCG_NO_REG_FFT
  return false;
#endif
  const int n = g.n1;
  if (!(pow2_in(n, 16, 256) || n == 48 || n == 96 || n == 192)) return false;
  if ((n == 96 || n == 192) && elem_bytes == 16) return false;
  return c == 1 || (n <= 64 && n != 48);
}

int line_reg_blocks_x(const Grid& g) {
  const int G = reg_split_g(g.n1);
  if (G == 0) return 0;
  const int per_block = kLineRegWarps * (32 / G);
  const int M = g.n2 * g.n3h;
  return (M + per_block - 1) / per_block;
}

namespace {
template <typename T, typename QT, int CC, int N1, int MODE>
cudaError_t line_reg_n(const LineArgs<T, QT>& a, cudaStream_t s) {
  constexpr int G = RegSplit<N1>::G, W = 32 / G;
  const size_t smem = ((size_t)N1 + (size_t)kLineRegWarps * W * N1) * sizeof(cplx<T>);
  dim3 grid(line_reg_blocks_x(a.g), a.BL);
  return launch_reg(k_line_reg<T, QT, CC, N1, MODE>, grid, kLineRegWarps * 32, smem, a, s);
}
template <typename T, typename QT, int CC, int MODE>
cudaError_t line_reg_cc(const LineArgs<T, QT>& a, cudaStream_t s) {
  switch (a.g.n1) {
    case 16: return line_reg_n<T, QT, CC, 16, MODE>(a, s);
    case 32: return line_reg_n<T, QT, CC, 32, MODE>(a, s);
    case 48:
      if constexpr (CC == 3) return cudaErrorInvalidValue;
      else return line_reg_n<T, QT, CC, 48, MODE>(a, s);
    case 64: return line_reg_n<T, QT, CC, 64, MODE>(a, s);
    case 96:
      if constexpr (CC == 3 || sizeof(T) == 8) return cudaErrorInvalidValue;
      else return line_reg_n<T, QT, CC, 96, MODE>(a, s);
    case 192:
      if constexpr (CC == 3 || sizeof(T) == 8) return cudaErrorInvalidValue;
      else return line_reg_n<T, QT, CC, 192, MODE>(a, s);
    case 128:
      if constexpr (CC == 3) return cudaErrorInvalidValue;
      else return line_reg_n<T, QT, CC, 128, MODE>(a, s);
    case 256:
      if constexpr (CC == 3) return cudaErrorInvalidValue;
      else return line_reg_n<T, QT, CC, 256, MODE>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

template <typename T, typename QT> cudaError_t launch_line_reg(const LineArgs<T, QT>& a, cudaStream_t s) {
  // instantiated: (double, double) CG + apply; (float, bf16) CG; (float, float) apply
  constexpr bool cg = !(std::is_same<T, float>::value && std::is_same<QT, float>::value);
  constexpr bool apply = !std::is_same<QT, __nv_bfloat16>::value;
  if (a.standalone) {
    if constexpr (apply) return a.c == 1 ? line_reg_cc<T, QT, 1, 1>(a, s) : line_reg_cc<T, QT, 3, 1>(a, s);
    return cudaErrorInvalidValue;
  }
  if constexpr (cg) return a.c == 1 ? line_reg_cc<T, QT, 1, 0>(a, s) : line_reg_cc<T, QT, 3, 0>(a, s);
  return cudaErrorInvalidValue;
}
template cudaError_t launch_line_reg<double, double>(const LineArgs<double, double>&, cudaStream_t);
template cudaError_t launch_line_reg<float, __nv_bfloat16>(const LineArgs<float, __nv_bfloat16>&, cudaStream_t);
template cudaError_t launch_line_reg<float, float>(const LineArgs<float, float>&, cudaStream_t);

}  // namespace unocg
