// Matrix-free operator and pointwise kernels of the UNO-CG hot path.
//
//  * K d on the periodic voxel grid (Sec. 4.1, "matrix-free implementations" of Sec. 5.5),
//    gathered per node from the 8 elements around it (27-point node stencil).  Thermal:
//      p_a = (h/12) [ 4 (sum_e kappa_e) d_a - sum_{12 edge-diagonal b} (kappa_e1 + kappa_e2) d_b
//                     - sum_{8 corner b} kappa_e d_b ]
//    (face neighbours do not couple for trilinear bricks).  Elastic: the 3x3 blocks of
//    h (lambda_e Klam + mu_e Kmu) from element.cuh.
//  * right-hand side f = -sum_e A_e^T int_e B^T C_e eps_bar (Sec. 6), r_0 = f for u_0 = 0
//  * Jacobi preconditioner (Sec. 4.2) and the pointwise CG updates of Algorithm 1
//  * true residual f - K u in FP64, post-processing (averaged flux/stress, sensitivities)
#include "kargs.h"
#include "element.cuh"
#include "df64.cuh"
#include "stencil.cuh"
#include "ku_task.cuh"
#include "ku_elastic.cuh"
#include "replace_elastic.cuh"
#include <cstdlib>
#include <cstring>

namespace unocg {

// ============================================================================ K d
// Block partial of d . p; the last block of the grid forms alpha = gamma / (d . p) per pair.
template <typename T>
__device__ __forceinline__ void ku_finish(const StencilArgs<T>& a, int bl, double bs) {
  if (a.standalone) return;
  if (threadIdx.x == 0) a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bs;
  if (last_block(a.red.ticket)) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < a.BL; q += blockDim.x / 32) {
      double sum = warp_sum_partials(a.red.part + (long long)q * gridDim.x, gridDim.x, 1);
      if (lane == 0 && !a.sc[q].done) step_update(a.sc[q], sum);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

template <typename T, int CC>
__global__ void __launch_bounds__(256) k_ku(StencilArgs<T> a) {
  __shared__ T mt[2 * 256];
  __shared__ double red_sh[32];
  __shared__ T tile_smem[CC == 1 ? KU_DN + KU_KN : 1];
  const int bl = blockIdx.y;
  load_material<T>(mt, a.mat, bl / a.L);
  __syncthreads();
  pdl_wait();
  const double bs = ku_task<T, CC, false>(a, mt, bl, blockIdx.x, red_sh, tile_smem,
                                          a.standalone ? nullptr : &a.sc[bl].done);
  pdl_trigger();
  ku_finish<T>(a, bl, bs);
}

// K d element by element in the Walsh basis (ku_elastic.cuh)
template <typename T, int CC>
__global__ void __launch_bounds__(KE_THREADS) k_ku_el(StencilArgs<T> a) {
  extern __shared__ __align__(16) unsigned char ke_raw[];
  __shared__ T mt[2 * 256];
  __shared__ double red_sh[32];
  const int bl = blockIdx.y;
  load_material<T>(mt, a.mat, bl / a.L);
  __syncthreads();
  pdl_wait();
  const double bs = ku_element_tile<T, CC, false>(a, mt, bl, blockIdx.x, red_sh, reinterpret_cast<T*>(ke_raw),
                                              a.standalone ? nullptr : &a.sc[bl].done);
  pdl_trigger();
  ku_finish<T>(a, bl, bs);
}

// ============================================================================ init: r = f, u = d = 0
// f = -sum_e A_e^T int_e B^T C_e eps_bar (Sec. 6) node by node: with the element-mean gradient of
// the shape function of corner o, sg(o) / (4h) (sg = 2 o - 1 per axis), the integral over the
// element is (h^2 / 4) sg(o), so f(node) = -(h^2 / 4) sum_o sigma_e(o) sg(o) over the 8 elements
// e(o) = node - o.  The phase constants enter only through w_m(node) = sum_o c_m(e(o)) sg(o)
// (c_0 = kappa or lambda, c_1 = mu), formed once for all loads of the instance:
//   thermal  f = -(h^2/4) w_0 . eps_bar
//   elastic  f_i = -(h^2/4) (tr(eps) w_0,i + 2 sum_k eps_ik w_1,k)   (eps from the Mandel load)
template <typename T, int CC>
__global__ void __launch_bounds__(256) k_init(InitArgs<T> a) {
  constexpr int NM = CC == 1 ? 1 : 2;
  __shared__ double mt[2 * 256];
  const Grid& g = a.g;
  const int b = blockIdx.y;  // instance; the thread covers every load
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  int i1, i2, i3;
  if (!tile_node(g, i1, i2, i3)) return;
  const long long n = g.n;
  const uint8_t* ph = a.phase + (long long)b * n;
  const long long node = ((long long)i1 * g.n2 + i2) * g.n3 + i3;
  Nbr nb;
  neighbours(g, i1, i2, i3, nb);
  double w[NM][3];
#pragma unroll
  for (int m = 0; m < NM; ++m) w[m][0] = w[m][1] = w[m][2] = 0.0;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
    const int p = ph[eidx(nb, o1, o2, o3)];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const double v = mt[2 * p + m];
      w[m][0] += o1 ? v : -v;
      w[m][1] += o2 ? v : -v;
      w[m][2] += o3 ? v : -v;
    }
  }
  const double q = 0.25 * g.h * g.h;
  for (int l = 0; l < a.L; ++l) {
    const double* load = a.loads + l * (CC == 1 ? 3 : 6);
    double f[CC];
    if constexpr (CC == 1) {
      f[0] = -q * (w[0][0] * load[0] + w[0][1] * load[1] + w[0][2] * load[2]);
    } else {
      const double is2 = 0.70710678118654752440;
      const double e12 = load[3] * is2, e13 = load[4] * is2, e23 = load[5] * is2;
      const double tr = load[0] + load[1] + load[2];
      const double e[3][3] = {{load[0], e12, e13}, {e12, load[1], e23}, {e13, e23, load[2]}};
#pragma unroll
      for (int i = 0; i < 3; ++i)
        f[i] = -q * (tr * w[0][i] + 2.0 * (e[i][0] * w[1][0] + e[i][1] * w[1][1] + e[i][2] * w[1][2]));
    }
    const long long o = ((long long)b * a.L + l) * CC * n + node;
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      if (a.r) a.r[o + i * n] = (T)f[i];
      if (a.u) a.u[o + i * n] = (T)0;
      if (a.d) a.d[o + i * n] = (T)0;
      if (a.p) a.p[o + i * n] = (T)0;
      if (a.u64) a.u64[o + i * n] = 0.0;
      if (a.f64) a.f64[o + i * n] = f[i];
    }
  }
}

// ============================================================================ true residual
// r_true = f - K u (FP64).  u = u64 (+ u32 + alpha d when folding a mixed-precision increment,
// which is done by k_fold beforehand).  Optionally stores r_true into r (type T).
template <typename T, int CC>
__global__ void __launch_bounds__(256) k_true_res(TrueResArgs<T> a) {
  __shared__ double mt[2 * 256];
  const Grid& g = a.g;
  const int bl = blockIdx.y;
  const int b = bl / a.L, l = bl % a.L;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  if (a.only_pending && !a.sc[bl].need_replace) return;
  if (!a.only_pending && a.sc[bl].started == 0 && a.require_started) return;
  int i1, i2, i3;
  double lmax = 0.0;
  if (tile_node(g, i1, i2, i3)) {
    const long long n = g.n;
    const uint8_t* ph = a.phase + (long long)b * n;
    const double* u = a.u64 + (long long)bl * CC * n;
    const long long node = ((long long)i1 * g.n2 + i2) * g.n3 + i3;
    double f[CC], ku[CC];
    if (a.f64) {
#pragma unroll
      for (int i = 0; i < CC; ++i) f[i] = a.f64[(long long)bl * CC * n + i * n + node];
    } else {
      node_rhs<CC>(ph, mt, g, i1, i2, i3, a.loads + l * (CC == 1 ? 3 : 6), f);
    }
    node_Ku<double, CC>(u, ph, mt, g, i1, i2, i3, ku);
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      double rr = f[i] - ku[i];
      lmax = fmax(lmax, fabs(rr));
      if (a.r) a.r[(long long)bl * CC * n + i * n + node] = (T)rr;
    }
  }
  __shared__ double red_sh[32];
  double bm = block_max(lmax, red_sh);
  if (threadIdx.x == 0) atomic_max_nonneg(a.into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
}

// ============================================================================ residual replacement
// rref <- rref - K w with w = u32 + alpha d, all products and sums in float pairs (df64.cuh):
// the FP32 inputs are exact, the stencil coefficients are integers (thermal: 12 x the unit-cube
// Laplacian, elastic: 72 x Klam / Kmu) times the phase constants as pairs, and the result is
// rounded to FP64 once per node.
// After the loop, a pair whose last residual check followed a replacement has had no step since
// (the replacement folded u32 + alpha d into u64 and cleared both): K w = 0, and the final report
// needs only max |rref|, taken here over the pair's field by all blocks of its row of the grid.
__device__ __forceinline__ bool replace_w_zero(const ReplaceArgs& a, int bl) {
  return !a.only_pending && a.sc[bl].just_replaced && a.sc[bl].done;
}
__device__ __forceinline__ double rref_max_share(const ReplaceArgs& a, int bl, double* red_sh) {
  const long long m = (long long)a.c * a.g.n;
  const double* x = a.rref + (long long)bl * m;
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    v = fmax(v, fabs(x[i]));
  return block_max(v, red_sh);
}

// Thermal replacement as a march along axis 1 (each w formed once per node): a thread walks
// KR_CZ nodes of one (i2, i3) column with the 3 x 3 neighbourhoods of w = u32 + alpha d on the planes z - 1, z, z + 1 and the
// conductivities of the element planes z - 1, z in registers, all as float pairs.  For the
// element at corner offset o of the node, 12 t_o = 4 w(node) - (the 3 face-diagonal and the
// body-diagonal corners of the element, seen from the node).
constexpr int KR_CZ = 8;
__global__ void __launch_bounds__(256) k_replace_col(ReplaceArgs a) {
  __shared__ float2 mp[2 * 256];
  __shared__ double red_sh[32];
  const Grid& g = a.g;
  const int bl = blockIdx.y;
  const int b = bl / a.L;
  const int np2 = 2 * a.mat.n_phases;
  for (int i = threadIdx.x; i < np2; i += blockDim.x) {
    const df32 v = df_from_double(a.mat.m64[(long long)b * np2 + i]);
    mp[i] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  if (a.only_pending && !a.sc[bl].need_replace) return;
  if (replace_w_zero(a, bl)) {
    const double bm = rref_max_share(a, bl, red_sh);
    if (threadIdx.x == 0) atomic_max_nonneg(a.into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
    return;
  }
  const df32 al = df_from_double(a.sc[bl].alpha);
  int i1, i2, i3;
  double lmax = 0.0;
  if (tile_column_at(g, blockIdx.x, KR_CZ, i1, i2, i3)) {
    const long long n = g.n, S = (long long)g.n2 * g.n3;
    const uint8_t* ph = a.phase + (long long)b * n;
    const float* u32 = a.u32 + (long long)bl * n;
    const float* dd = a.d + (long long)bl * n;
    const int c2[3] = {i2 ? i2 - 1 : g.n2 - 1, i2, (i2 + 1 == g.n2) ? 0 : i2 + 1};
    const int c3[3] = {i3 ? i3 - 1 : g.n3 - 1, i3, (i3 + 1 == g.n3) ? 0 : i3 + 1};
    long long off[3][3];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) off[x][y] = (long long)c2[x] * g.n3 + c3[y];
    auto W = [&](long long q) { return df_axpy(al, __ldg(dd + q), __ldg(u32 + q)); };
    auto K = [&](long long q) {
      const float2 v = mp[2 * ph[q]];
      return df32{v.x, v.y};
    };
    // w[plane: 0 = z - 1, 1 = z, 2 = z + 1][row][column], kap[element plane: 0 = z - 1, 1 = z][o2][o3]
    df32 w[3][3][3], kap[2][2][2];
    const long long zm = (long long)(i1 ? i1 - 1 : g.n1 - 1) * S;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) {
        w[0][x][y] = W(zm + off[x][y]);
        w[1][x][y] = W((long long)i1 * S + off[x][y]);
      }
#pragma unroll
    for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
      for (int o3 = 0; o3 < 2; ++o3) kap[0][o2][o3] = K(zm + off[1 - o2][1 - o3]);
    const int zend = min(i1 + KR_CZ, g.n1);
    const double h12 = g.h / 12.0;
    for (int z = i1; z < zend; ++z) {
      const long long zc = (long long)z * S, zn = (long long)((z + 1 == g.n1) ? 0 : z + 1) * S;
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) w[2][x][y] = W(zn + off[x][y]);
#pragma unroll
      for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
        for (int o3 = 0; o3 < 2; ++o3) kap[1][o2][o3] = K(zc + off[1 - o2][1 - o3]);
      df32 w4 = w[1][1][1];
      w4.hi *= 4.0f;
      w4.lo *= 4.0f;
      df32 acc = df_make(0.0f);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
        // the coordinate of the corners away from the node: 2 for o = 0, 0 for o = 1
        const int d1 = 2 - 2 * o1, d2 = 2 - 2 * o2, d3 = 2 - 2 * o3;
        const df32 sd = df_add(df_add(w[d1][d2][1], w[d1][1][d3]), df_add(w[1][d2][d3], w[d1][d2][d3]));
        const df32 t = df_add(w4, df_neg(sd));
        acc = df_add(acc, df_mul(kap[1 - o1][o2][o3], t));
      }
      const long long x = (long long)bl * n + zc + off[1][1];
      const double rr = a.rref[x] - df_to_double(acc) * h12;
      a.rref[x] = rr;
      if (a.r) a.r[x] = (float)rr;
      lmax = fmax(lmax, fabs(rr));
#pragma unroll
      for (int x2 = 0; x2 < 3; ++x2)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
          w[0][x2][y] = w[1][x2][y];
          w[1][x2][y] = w[2][x2][y];
        }
#pragma unroll
      for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
        for (int o3 = 0; o3 < 2; ++o3) kap[0][o2][o3] = kap[1][o2][o3];
    }
  }
  const double bm = block_max(lmax, red_sh);
  if (threadIdx.x == 0) atomic_max_nonneg(a.into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
}

// Elastic replacement element by element in float pairs (replace_elastic.cuh)
__global__ void __launch_bounds__(KE_THREADS) k_replace_el(ReplaceArgs a) {
  extern __shared__ __align__(16) unsigned char re_raw[];
  __shared__ float2 kc[6 * 256];  // element constants of every phase as pairs
  __shared__ double red_sh[32];
  const int bl = blockIdx.y;
  replace_elastic_consts(a.mat, bl / a.L, a.g.h, kc);
  __syncthreads();
  if (a.only_pending && !a.sc[bl].need_replace) return;
  if (replace_w_zero(a, bl)) {
    const double bm = rref_max_share(a, bl, red_sh);
    if (threadIdx.x == 0) atomic_max_nonneg(a.into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
    return;
  }
  const long long off = (long long)bl * 3 * a.g.n;
  const double bm = replace_elastic_tile(a.g, a.phase + (long long)(bl / a.L) * a.g.n, a.u32 + off, a.d + off,
                                         df_from_double(a.sc[bl].alpha), a.rref + off, a.r ? a.r + off : nullptr, kc,
                                         blockIdx.x, red_sh, reinterpret_cast<float2*>(re_raw),
                                         [](int, int, int) { return true; });
  if (threadIdx.x == 0) atomic_max_nonneg(a.into_rmax ? &a.sc[bl].rmax_bits : &a.sc[bl].tmax_bits, bm);
}

// ============================================================================ pointwise kernels
// Four consecutive elements as vector accesses (16-byte aligned addresses)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// u64[i] <- u64[i] + u32[i] + alpha d[i] (u32[i] <- 0) for the elements [4 q, 4 q + 4); returns
// their sum (left to right)
template <typename T>
__device__ __forceinline__ double fold4(double* u64, T* u32, const T* d, long long q, double al) {
  const long long i = 4 * q;
  double v[4];
  T dd[4];
  ld4(u64 + i, v);
  ld4(d + i, dd);
  if (u32) {
    T uu[4];
    ld4(u32 + i, uu);
    const T z[4] = {(T)0, (T)0, (T)0, (T)0};
    st4(u32 + i, z);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += (double)uu[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] += al * (double)dd[k];
  st4(u64 + i, v);
  return ((v[0] + v[1]) + v[2]) + v[3];
}

// Mixed-precision fold before a residual replacement: u64 += u32 + alpha d; u32 = 0; alpha = 0.
// Four elements per thread and step where the slab length is a multiple of four.
template <typename T>
__global__ void k_fold(FoldArgs<T> a) {
  const int bl = blockIdx.y;
  CgScal& s = a.sc[bl];
  if (a.only_pending && !s.need_replace) return;
  const double al = s.alpha;
  const long long m = (long long)a.c * a.n;
  const long long base = (long long)bl * m;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if ((m & 3) == 0) {
    for (long long q = t0; q < (m >> 2); q += st)
      (void)fold4<T>(a.u64 + base, a.u32 ? a.u32 + base : nullptr, a.d + base, q, al);
    return;
  }
  for (long long i = t0; i < m; i += st) {
    double v = a.u64[base + i];
    if (a.u32) {
      v += (double)a.u32[base + i];
      a.u32[base + i] = (T)0;
    }
    v += al * (double)a.d[base + i];
    a.u64[base + i] = v;
  }
}
// alpha = 0 after a fold (run after k_fold has finished everywhere)
__global__ void k_clear_alpha(CgScal* sc, int BL, int only_pending) {
  int bl = blockIdx.x * blockDim.x + threadIdx.x;
  if (bl >= BL) return;
  if (only_pending && !sc[bl].need_replace) return;
  sc[bl].alpha = 0.0;
}

// Jacobi / no preconditioner, first half: r <- r - alpha p, ||r||_inf, s = r / diag(K),
// gamma = r . s; last block: stopping test and search-direction coefficient.
template <typename T>
__global__ void __launch_bounds__(256) k_jac_a(JacArgs<T> a) {
  __shared__ double red_sh[32];
  const int bl = blockIdx.y;
  CgScal& s = a.sc[bl];
  const bool active = !s.done && (!a.after_replace || s.need_replace);
  const double al = a.after_replace ? 0.0 : s.alpha;
  const T alt = (T)al;
  const bool upd = al != 0.0;
  T lmax = (T)0;
  DotAcc<T> gam;
  if (active) {
    const long long m = (long long)a.c * a.n;
    const long long base = (long long)bl * m;
    const long long ib = (long long)(bl / a.L) * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
      T r = a.r[base + i];
      if (upd) {
        r -= alt * a.p[base + i];
        a.r[base + i] = r;
      }
      T sv = a.invdiag ? r * a.invdiag[ib + i] : r;
      lmax = fmax(lmax, fabs(r));
      gam.add_prod(r, sv);
    }
  }
  double bm = block_max_t(lmax, red_sh);
  double bg = block_sum_acc(gam, red_sh);
  if (threadIdx.x == 0) {
    if (active) atomic_max_nonneg(&s.rmax_bits, bm);
    a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bg;
  }
  if (last_block(a.red.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < a.BL; q += blockDim.x / 32) {
      double sum = warp_sum_partials(a.red.part + (long long)q * gridDim.x, gridDim.x, 1);
      CgScal& t = a.sc[q];
      if (lane == 0 && !t.done && !t.need_replace && (!a.after_replace || t.just_replaced))
        direction_update(t, sum, 0.0, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// second half: u <- u + alpha d_old; d <- s + beta d_old
template <typename T>
__global__ void __launch_bounds__(256) k_jac_b(JacArgs<T> a) {
  const int bl = blockIdx.y;
  const CgScal& s = a.sc[bl];
  if (s.done) return;
  const T al = (T)s.alpha, be = (T)s.beta;
  const long long m = (long long)a.c * a.n;
  const long long base = (long long)bl * m;
  const long long ib = (long long)(bl / a.L) * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    T r = a.r[base + i];
    T sv = a.invdiag ? r * a.invdiag[ib + i] : r;
    T dold = a.d[base + i];
    a.u[base + i] += al * dold;
    a.d[base + i] = sv + be * dold;
  }
}

// inverse of the diagonal of K per instance: [B][c][n]
template <typename T, int CC>
__global__ void __launch_bounds__(256) k_invdiag(DiagArgs<T> a) {
  __shared__ double mt[2 * 256];
  const Grid& g = a.g;
  const int b = blockIdx.y;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  int i1, i2, i3;
  if (!tile_node(g, i1, i2, i3)) return;
  const long long n = g.n;
  const uint8_t* ph = a.phase + (long long)b * n;
  const long long node = ((long long)i1 * g.n2 + i2) * g.n3 + i3;
  double dg[CC];
  node_diag<CC>(ph, mt, g, i1, i2, i3, dg);
#pragma unroll
  for (int i = 0; i < CC; ++i) a.invdiag[(long long)b * CC * n + i * n + node] = (T)(1.0 / dg[i]);
}

// ============================================================================ post-processing
// Final pending update (u += alpha d, or the mixed fold) and per-(field) sums for the mean.
template <typename T>
__global__ void __launch_bounds__(256) k_final(FoldArgs<T> a) {
  __shared__ double red_sh[32];
  const int bl = blockIdx.y;
  const int comp = blockIdx.z;
  const double al = a.sc[bl].alpha;
  const long long base = ((long long)bl * a.c + comp) * a.n;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  double sum = 0.0;
  if ((a.n & 3) == 0) {
    for (long long q = t0; q < (a.n >> 2); q += st)
      sum += fold4<T>(a.u64 + base, a.u32 ? a.u32 + base : nullptr, a.d + base, q, al);
  } else {
    for (long long i = t0; i < a.n; i += st) {
      double v = a.u64[base + i];
      if (a.u32) {
        v += (double)a.u32[base + i];
        a.u32[base + i] = (T)0;
      }
      v += al * (double)a.d[base + i];
      a.u64[base + i] = v;
      sum += v;
    }
  }
  double bs = block_sum(sum, red_sh);
  if (threadIdx.x == 0)
    a.part[(((long long)bl * a.c + comp) * gridDim.x) + blockIdx.x] = bs;
}

__global__ void k_zero_mean(double* u, const double* part, int nparts, int c, long long n) {
  const int bl = blockIdx.y, comp = blockIdx.z;
  const long long f = (long long)bl * c + comp;
  __shared__ double mean;
  if (threadIdx.x < 32) {
    double s = warp_sum_partials(part + f * nparts, nparts, 1);
    if (threadIdx.x == 0) mean = s / (double)n;
  }
  __syncthreads();
  double* uf = u + f * n;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if ((n & 1) == 0) {
    double2* u2 = reinterpret_cast<double2*>(uf);
    for (long long i = t0; i < (n >> 1); i += st) {
      double2 v = u2[i];
      v.x -= mean;
      v.y -= mean;
      u2[i] = v;
    }
    return;
  }
  for (long long i = t0; i < n; i += st) uf[i] -= mean;
}

// Averaged flux / stress per (instance, load): sum over elements of C_e (eps_bar + the element-mean
// strain of u), per block, finished by k_average_finish.
// The sums are regrouped by node (the element-mean gradient is linear in the corner values).
// With s = 1 / (4h) and sg(o) = 2 o - 1 per axis, the element-mean gradient of element e is
// s sum_o sg(o) u(e + o), so sum_e kappa_e grad_e = s sum_nodes u(node) w(node) with
// w(node) = sum_o kappa(node - o) sg(o) over the 8 elements around the node (o: the node's corner
// in element node - o).  Elastic: w_lambda and w_mu likewise, and for the Mandel components
//   sum_e sigma_kk(u)  = s sum_nodes (u . w_lambda + 2 u_k w_mu,k)            (k < 3)
//   sum_e sigma_kl(u)  = s sqrt(2) sum_nodes (u_k w_mu,l + u_l w_mu,k)       (kl = 12, 13, 23).
// The loads add (sum_e C_e) eps_bar, with sum_e kappa_e = sum_nodes (sum_o kappa(node - o)) / 8.
// A thread walks KA_CZ nodes along axis 1 (the element planes z - 1 and z in registers), all
// loads of the instance in chunks of LC; fixed-order warp and block reductions (deterministic).
constexpr int KA_CZ = 8;
template <int CC, int LC>
__global__ void __launch_bounds__(256) k_average_nodes(AvgArgs a) {
  constexpr int DIM = CC == 1 ? 3 : 6, NM = CC == 1 ? 1 : 2;
  __shared__ double mt[2 * 256];
  __shared__ double wsum[8][48 + NM];  // [warp][load * DIM + i], then the material sums
  const Grid& g = a.g;
  const int b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_material<double>(mt, a.mat, b);
  __syncthreads();
  int i1, i2, i3;
  const bool valid = tile_column_at(g, blockIdx.x, KA_CZ, i1, i2, i3);
  const long long n = g.n, S = (long long)g.n2 * g.n3;
  const uint8_t* ph = a.phase + (long long)b * n;
  // element (z - o1, i2 - o2, i3 - o3) sits at plane offset eo[o2][o3] of element plane z - o1
  long long eo[2][2] = {{0, 0}, {0, 0}};
  if (valid) {
    const int m2 = i2 ? i2 - 1 : g.n2 - 1, m3 = i3 ? i3 - 1 : g.n3 - 1;
    eo[0][0] = (long long)i2 * g.n3 + i3;
    eo[0][1] = (long long)i2 * g.n3 + m3;
    eo[1][0] = (long long)m2 * g.n3 + i3;
    eo[1][1] = (long long)m2 * g.n3 + m3;
  }
  const int zend = valid ? min(i1 + KA_CZ, g.n1) : 0;
  double msum[NM];
#pragma unroll
  for (int m = 0; m < NM; ++m) msum[m] = 0.0;
  for (int l0 = 0; l0 < a.L; l0 += LC) {
    double acc[LC][DIM];
#pragma unroll
    for (int lc = 0; lc < LC; ++lc)
#pragma unroll
      for (int i = 0; i < DIM; ++i) acc[lc][i] = 0.0;
    if (valid) {
      double pm[NM][2][2], pc[NM][2][2];
      const long long zm = (long long)(i1 ? i1 - 1 : g.n1 - 1) * S;
#pragma unroll
      for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
        for (int o3 = 0; o3 < 2; ++o3) {
          const int p = ph[zm + eo[o2][o3]];
#pragma unroll
          for (int m = 0; m < NM; ++m) pm[m][o2][o3] = mt[2 * p + m];
        }
      for (int z = i1; z < zend; ++z) {
        const long long zc = (long long)z * S;
#pragma unroll
        for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
          for (int o3 = 0; o3 < 2; ++o3) {
            const int p = ph[zc + eo[o2][o3]];
#pragma unroll
            for (int m = 0; m < NM; ++m) pc[m][o2][o3] = mt[2 * p + m];
          }
        double w[NM][3];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const double sm = (pm[m][0][0] + pm[m][0][1]) + (pm[m][1][0] + pm[m][1][1]);  // o1 = 1
          const double sc = (pc[m][0][0] + pc[m][0][1]) + (pc[m][1][0] + pc[m][1][1]);  // o1 = 0
          const double tot = sm + sc;
          const double s2 = (pm[m][1][0] + pm[m][1][1]) + (pc[m][1][0] + pc[m][1][1]);  // o2 = 1
          const double s3 = (pm[m][0][1] + pm[m][1][1]) + (pc[m][0][1] + pc[m][1][1]);  // o3 = 1
          w[m][0] = sm - sc;
          w[m][1] = 2.0 * s2 - tot;
          w[m][2] = 2.0 * s3 - tot;
          if (l0 == 0) msum[m] += tot;
        }
        const long long node = zc + eo[0][0];
#pragma unroll
        for (int lc = 0; lc < LC; ++lc) {
          if (l0 + lc >= a.L) break;
          const double* u = a.u64 + ((long long)b * a.L + l0 + lc) * CC * n + node;
          if constexpr (CC == 1) {
            const double v = u[0];
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[lc][k] = fma(v, w[0][k], acc[lc][k]);
          } else {
            const double v0 = u[0], v1 = u[n], v2 = u[2 * n];
            const double tr = fma(v0, w[0][0], fma(v1, w[0][1], v2 * w[0][2]));
            acc[lc][0] += fma(2.0 * v0, w[1][0], tr);
            acc[lc][1] += fma(2.0 * v1, w[1][1], tr);
            acc[lc][2] += fma(2.0 * v2, w[1][2], tr);
            acc[lc][3] += fma(v0, w[1][1], v1 * w[1][0]);
            acc[lc][4] += fma(v0, w[1][2], v2 * w[1][0]);
            acc[lc][5] += fma(v1, w[1][2], v2 * w[1][1]);
          }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
          for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
            for (int o3 = 0; o3 < 2; ++o3) pm[m][o2][o3] = pc[m][o2][o3];
      }
    }
#pragma unroll
    for (int lc = 0; lc < LC; ++lc) {
      if (l0 + lc >= a.L) break;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        double v = acc[lc][i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) wsum[warp][(l0 + lc) * DIM + i] = v;
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    double v = msum[m];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp][48 + m] = v;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  double mb[NM];  // block sums of kappa (lambda, mu) over elements
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    double t = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) t += wsum[w2][48 + m];
    mb[m] = 0.125 * t;
  }
  const double sc = 0.25 / g.h;
  const double sq2 = 1.41421356237309504880;
  for (int q = threadIdx.x; q < a.L * DIM; q += blockDim.x) {
    double t = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) t += wsum[w2][q];
    const int l = q / DIM, i = q % DIM;
    const double* ld = a.loads + l * DIM;
    double v;
    if constexpr (CC == 1) {
      v = sc * t + mb[0] * ld[i];
    } else {
      const double tr = ld[0] + ld[1] + ld[2];
      v = i < 3 ? sc * t + mb[0] * tr + 2.0 * mb[1] * ld[i] : sq2 * sc * t + 2.0 * mb[1] * ld[i];
    }
    a.part[((long long)b * gridDim.x + blockIdx.x) * (8 * 6) + q] = v;
  }
}

__global__ void k_average_finish(double* out, const double* part, int nparts, int B, int L, int dim, double inv_n) {
  int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = warp; q < L * dim; q += blockDim.x / 32) {
    int l = q / dim, i = q % dim;
    double s = warp_sum_partials(part + (long long)b * nparts * 48 + q, nparts, 48);
    if (lane == 0) out[((long long)b * dim + i) * L + l] = s * inv_n;
  }
}

// Sensitivities: for every element, Gauss-point strains of all loads, products per phase.
template <int CC>
__global__ void __launch_bounds__(128) k_sens(AvgArgs a) {
  __shared__ double mt[2 * 256];
  extern __shared__ double sacc[];  // [n_phases][nq][L][L]
  const Grid& g = a.g;
  const int b = blockIdx.y;
  const int L = a.L;
  const int nq = CC == 1 ? 1 : 2;
  const int tot = a.mat.n_phases * nq * L * L;
  load_material<double>(mt, a.mat, b);
  for (int i = threadIdx.x; i < tot; i += blockDim.x) sacc[i] = 0.0;
  __syncthreads();
  int i1, i2, i3;
  if (tile_node(g, i1, i2, i3)) {
    const long long n = g.n;
    const long long e = ((long long)i1 * g.n2 + i2) * g.n3 + i3;
    const int p = a.phase[(long long)b * n + e];
    element_sensitivity<CC>(a.u64 + (long long)b * L * CC * n, L, g, i1, i2, i3, a.loads,
                            sacc + (long long)p * nq * L * L);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tot; i += blockDim.x)
    a.part[((long long)b * gridDim.x + blockIdx.x) * tot + i] = sacc[i];
}

__global__ void k_sens_finish(double* out, const double* part, int nparts, int tot, double inv_n) {
  int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = warp; q < tot; q += blockDim.x / 32) {
    double s = warp_sum_partials(part + (long long)b * nparts * tot + q, nparts, tot);
    if (lane == 0) out[(long long)b * tot + q] = s * inv_n;
  }
}

// [c][n] (double) -> interleaved [n][c]
__global__ void k_interleave(const double* src, double* dst, int c, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int j = 0; j < c; ++j) dst[i * c + j] = src[j * n + i];
}

__global__ void k_copy_d2f(const double* src, float* dst, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// ============================================================================ launchers
static dim3 node_grid(const Grid& g, int y) {
  int tx = (g.n3 + 31) / 32, ty = (g.n2 + 3) / 4, tz = (g.n1 + 1) / 2;
  return dim3(tx * ty * tz, y);
}
int node_blocks_x(const Grid& g) { return node_grid(g, 1).x; }

// Node tiles of the per-node K d tasks (persistent kernel): thermal 32 x 8 x KU_CZ columns,
// elastic 32 x 4 x 2 node blocks
static dim3 ku_task_grid(const Grid& g, int c, int y) {
  if (c != 1) return node_grid(g, y);
#if UNOCG_KU_MODE == 0
  int tx = (g.n3 + 31) / 32, ty = (g.n2 + 7) / 8, tz = (g.n1 + KU_TZ - 1) / KU_TZ;
#else
  int tx = (g.n3 + 31) / 32, ty = (g.n2 + 7) / 8, tz = (g.n1 + KU_CZ - 1) / KU_CZ;
#endif
  return dim3(tx * ty * tz, y);
}
int ku_tasks_x(const Grid& g, int c) { return ku_task_grid(g, c, 1).x; }

// Thermal K d: register column march (k_ku) below kThermalElementNodes nodes per field, element
// scheme (k_ku_el) from there; elastic: element scheme.  Measured per launch, 3 loads, FP32:
// 64^3 16.4 (column) vs 17.4 us (element), 128^3 73.6 vs 65.3 us, 256^3 596 vs 491 us.
// UNOCG_THERMAL_KU=element|column overrides the size rule.
constexpr long long kThermalElementNodes = 1000000;
static int thermal_override() {
  static int v = -2;
  if (v == -2) {
    const char* e = std::getenv("UNOCG_THERMAL_KU");
    v = !e ? -1 : std::strcmp(e, "element") == 0 ? 1 : std::strcmp(e, "column") == 0 ? 0 : -1;
  }
  return v;
}
static bool thermal_element(const Grid& g) {
  const int o = thermal_override();
  return o >= 0 ? o == 1 : g.n >= kThermalElementNodes;
}
// blocks of one K d launch per (instance, load)
int ku_blocks_x(const Grid& g, int c) { return (c == 1 && !thermal_element(g)) ? ku_tasks_x(g, c) : ke_tiles(g); }

template <typename T, int CC> static cudaError_t launch_ku_el(const StencilArgs<T>& a, cudaStream_t s) {
  const size_t smem = ke_smem_bytes<T, CC>();
  if (smem > 48 * 1024) {
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k_ku_el<T, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
  }
  return launch_pdl(k_ku_el<T, CC>, dim3(ke_tiles(a.g), a.BL), dim3(KE_THREADS), smem, s, a);
}

template <typename T> cudaError_t launch_ku(const StencilArgs<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    // tiles 9..16: the vector march with shape kKuTmaShapes[tile - 9]
    if (a.c == 1 && a.ku_tma > kKuTmaNumShapes && a.ku_tma <= 2 * kKuTmaNumShapes &&
        ku_vec_supported(a.g, 1, kKuTmaShapes[a.ku_tma - 1 - kKuTmaNumShapes]))
      return launch_ku_vec(a, kKuTmaShapes[a.ku_tma - 1 - kKuTmaNumShapes], s);
    if (a.c == 1 && a.ku_tma > 0 && a.ku_tma <= kKuTmaNumShapes &&
        ku_tma_supported(a.g, 1, kKuTmaShapes[a.ku_tma - 1]))
      return launch_ku_tma(a, kKuTmaShapes[a.ku_tma - 1], a.err, a.spin_limit, s);
  }
  if constexpr (sizeof(T) == 4) {
    // elastic K d with packed element pairs (k_ku_el2.cu; UNOCG_KU_EL2=0, read at every launch,
    // selects the scalar element kernel): 256^3 x 6 loads 1720 against 2336 us per launch
    const char* e = std::getenv("UNOCG_KU_EL2");
    if (a.c == 3 && !(e && std::atoi(e) == 0) && ku_el2_supported(a.g)) return launch_ku_el2(a, s);
  }
  if (a.c != 1) return launch_ku_el<T, 3>(a, s);
  if (thermal_element(a.g)) return launch_ku_el<T, 1>(a, s);
  return launch_pdl(k_ku<T, 1>, ku_task_grid(a.g, 1, a.BL), dim3(256), 0, s, a);
}
template <typename T> cudaError_t launch_init(const InitArgs<T>& a, int BL, cudaStream_t s) {
  dim3 grid = node_grid(a.g, BL / a.L);
  if (a.c == 1) k_init<T, 1><<<grid, 256, 0, s>>>(a);
  else k_init<T, 3><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_true_res(const TrueResArgs<T>& a, int BL, cudaStream_t s) {
  dim3 grid = node_grid(a.g, BL);
  if (a.c == 1) k_true_res<T, 1><<<grid, 256, 0, s>>>(a);
  else k_true_res<T, 3><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
static int pw_blocks(long long m) {
  long long b = (m + 255) / 256;
  if (b > 1184) b = 1184;  // 8 blocks per SM on 148+ SMs, grid-stride beyond
  return (int)(b < 1 ? 1 : b);
}
cudaError_t launch_replace(const ReplaceArgs& a, int BL, cudaStream_t s) {
  if (a.c == 1) {
    const dim3 grid(((a.g.n3 + 31) / 32) * ((a.g.n2 + 7) / 8) * ((a.g.n1 + KR_CZ - 1) / KR_CZ), BL);
    k_replace_col<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
  }
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_replace_el, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kReplaceElSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_replace_el<<<dim3(ke_tiles(a.g), BL), KE_THREADS, kReplaceElSmem, s>>>(a);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_fold(const FoldArgs<T>& a, int BL, cudaStream_t s) {
  k_fold<T><<<dim3(pw_blocks((long long)a.c * a.n), BL), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_clear_alpha<<<(BL + 127) / 128, 128, 0, s>>>(a.sc, BL, a.only_pending);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_final(const FoldArgs<T>& a, int BL, int nparts, cudaStream_t s) {
  k_final<T><<<dim3(nparts, BL, a.c), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_zero_mean(double* u, const double* part, int nparts, int c, long long n, int BL, cudaStream_t s) {
  k_zero_mean<<<dim3(nparts, BL, c), 256, 0, s>>>(u, part, nparts, c, n);
  return cudaGetLastError();
}
template <typename T> cudaError_t launch_jac(const JacArgs<T>& a, int which, cudaStream_t s) {
  dim3 grid(pw_blocks((long long)a.c * a.n) / (a.BL > 8 ? 4 : 1) + 1, a.BL);
  if (which == 0) k_jac_a<T><<<grid, 256, 0, s>>>(a);
  else k_jac_b<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
int jac_blocks_x(long long m, int BL) { return pw_blocks(m) / (BL > 8 ? 4 : 1) + 1; }
template <typename T> cudaError_t launch_invdiag(const DiagArgs<T>& a, int B, cudaStream_t s) {
  dim3 grid = node_grid(a.g, B);
  if (a.c == 1) k_invdiag<T, 1><<<grid, 256, 0, s>>>(a);
  else k_invdiag<T, 3><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_average(const AvgArgs& a, int B, double* out, cudaStream_t s) {
  const dim3 grid(((a.g.n3 + 31) / 32) * ((a.g.n2 + 7) / 8) * ((a.g.n1 + KA_CZ - 1) / KA_CZ), B);
  if (a.c == 1) k_average_nodes<1, 3><<<grid, 256, 0, s>>>(a);
  else k_average_nodes<3, 6><<<grid, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_average_finish<<<B, 256, 0, s>>>(out, a.part, grid.x, B, a.L, a.c == 1 ? 3 : 6, 1.0 / (double)a.g.n);
  return cudaGetLastError();
}
cudaError_t launch_sens(const AvgArgs& a, int B, double* out, cudaStream_t s) {
  dim3 grid = node_grid(a.g, B);
  int nq = a.c == 1 ? 1 : 2;
  int tot = a.mat.n_phases * nq * a.L * a.L;
  size_t smem = (size_t)tot * sizeof(double);
  if (a.c == 1) k_sens<1><<<dim3(grid.x * 2, B), 128, smem, s>>>(a);
  else k_sens<3><<<dim3(grid.x * 2, B), 128, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sens_finish<<<B, 256, 0, s>>>(out, a.part, grid.x * 2, tot, 1.0 / (double)a.g.n);
  return cudaGetLastError();
}
int sens_blocks_x(const Grid& g) { return node_grid(g, 1).x * 2; }
cudaError_t launch_interleave(const double* src, double* dst, int c, long long n, cudaStream_t s) {
  k_interleave<<<pw_blocks(n), 256, 0, s>>>(src, dst, c, n);
  return cudaGetLastError();
}

template cudaError_t launch_ku<double>(const StencilArgs<double>&, cudaStream_t);
template cudaError_t launch_ku<float>(const StencilArgs<float>&, cudaStream_t);
template cudaError_t launch_init<double>(const InitArgs<double>&, int, cudaStream_t);
template cudaError_t launch_init<float>(const InitArgs<float>&, int, cudaStream_t);
template cudaError_t launch_true_res<double>(const TrueResArgs<double>&, int, cudaStream_t);
template cudaError_t launch_true_res<float>(const TrueResArgs<float>&, int, cudaStream_t);
template cudaError_t launch_fold<double>(const FoldArgs<double>&, int, cudaStream_t);
template cudaError_t launch_fold<float>(const FoldArgs<float>&, int, cudaStream_t);
template cudaError_t launch_final<double>(const FoldArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_final<float>(const FoldArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_jac<double>(const JacArgs<double>&, int, cudaStream_t);
template cudaError_t launch_jac<float>(const JacArgs<float>&, int, cudaStream_t);
template cudaError_t launch_invdiag<double>(const DiagArgs<double>&, int, cudaStream_t);
template cudaError_t launch_invdiag<float>(const DiagArgs<float>&, int, cudaStream_t);

}  // namespace unocg
