// Thermal K d (Sec. 4.1, "matrix-free implementations" of Sec. 5.5), FP32, as a vectorised
// register march: the stencil of ku_tma.cuh with the node planes read straight from global
// memory instead of staged by the TMA.
//
// A block owns TY node rows (i2) over the whole N3 extent and marches along i1 over CZ node
// planes; a thread holds 4 consecutive nodes of one row (one 16-byte load per row and plane).
// Along axis 1 every thread keeps the 3 x 3 rows of the planes z - 1, z, z + 1 and the
// conductivities of the element planes z - 1 and z in registers, so each step reads the three
// rows i2 - 1, i2, i2 + 1 of one new node plane (the neighbouring rows are served from L1 /
// L2 to the threads of the adjacent rows) and two rows of phase labels of one new element
// plane, converted by a table lookup per element.  The axis-3 neighbours come from the adjacent
// threads of the row by warp shuffle, or from global memory where that thread is in another warp
// or across the periodic seam.  There is no block-wide synchronisation inside the march and no
// shared-memory staging, so a block is small and an SM holds several.
#include <type_traits>
#include "kargs.h"
#include "stencil.cuh"

namespace unocg {

namespace {
constexpr unsigned kFullV = 0xffffffffu;
constexpr int KV_NV = 4;      // nodes per thread along i3
constexpr int KV_UNROLL = 6;  // the register window rotates with period 6 (3 node planes, 2 element planes)

struct KuVecArgs {
  StencilArgs<float> a;
  int ty, cz, tiles;
};

// Per-thread layout constants.
struct KvGeom {
  int x0, xl, xr;      // first node column; axis-3 neighbour columns (periodic)
  bool fix_l, fix_r;   // neighbour outside this warp or across the seam: read it from memory
  long long rm, rc, rp;  // row offsets (row start) of i2 - 1, i2, i2 + 1 in a plane
};

// node values of one row: v[0] = column x0 - 1, v[1..4] = x0 .. x0 + 3, v[5] = x0 + 4
__device__ __forceinline__ void kv_row(const float* __restrict__ row, const KvGeom& G, float (&v)[KV_NV + 2]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(row + G.x0));
  float l = __shfl_up_sync(kFullV, q.w, 1);
  float r = __shfl_down_sync(kFullV, q.x, 1);
  if (G.fix_l) l = __ldg(row + G.xl);
  if (G.fix_r) r = __ldg(row + G.xr);
  v[0] = l; v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w; v[5] = r;
}

// conductivities of one element row: k[0] = element column x0 - 1, k[1..4] = x0 .. x0 + 3
__device__ __forceinline__ void kv_krow(const uint8_t* __restrict__ row, const KvGeom& G, const float* mt,
                                        float (&k)[KV_NV + 1]) {
  const unsigned w = __ldg(reinterpret_cast<const unsigned*>(row + G.x0));
  unsigned lb = __shfl_up_sync(kFullV, w, 1) >> 24;
  if (G.fix_l) lb = __ldg(row + G.xl);
  k[0] = mt[lb];
  k[1] = mt[w & 255u];
  k[2] = mt[(w >> 8) & 255u];
  k[3] = mt[(w >> 16) & 255u];
  k[4] = mt[w >> 24];
}
}  // namespace

__global__ void __launch_bounds__(512) k_ku_vec(const KuVecArgs ka) {
  __shared__ float mt[256];
  __shared__ double red_sh[32];
  const StencilArgs<float>& a = ka.a;
  const Grid& g = a.g;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int BL = a.BL;
  const int bl = blockIdx.x % BL;
  const int tile = blockIdx.x / BL;
  const int ntile2 = n2 / ka.ty;
  const int i2 = (tile % ntile2) * ka.ty + (int)threadIdx.x / (n3 / KV_NV);
  const int z0 = (tile / ntile2) * ka.cz;
  const int nsteps = min(ka.cz, n1 - z0);
  const int b = bl / a.L;
  const int tid = threadIdx.x, lane = tid & 31;
  {
    const float* src = a.mat.m32 + (long long)b * a.mat.n_phases * 2;
    for (int i = tid; i < a.mat.n_phases; i += blockDim.x) mt[i] = src[2 * i] * g.h12f;
  }
  KvGeom G;
  {
    const int TPR = n3 / KV_NV, xr_ = tid % TPR;
    G.x0 = xr_ * KV_NV;
    G.xl = (G.x0 == 0 ? n3 : G.x0) - 1;
    G.xr = (G.x0 + KV_NV == n3) ? 0 : G.x0 + KV_NV;
    G.fix_l = xr_ == 0 || lane == 0;
    G.fix_r = xr_ == TPR - 1 || lane == 31;
    G.rm = (long long)(i2 ? i2 - 1 : n2 - 1) * n3;
    G.rc = (long long)i2 * n3;
    G.rp = (long long)(i2 + 1 == n2 ? 0 : i2 + 1) * n3;
  }
  __syncthreads();
  pdl_wait();  // d and the loop state come from the kernels before this one
  const bool skip = !a.standalone && a.sc[bl].done;
  DotAcc<float> dot;
  if (!skip) {
    const long long S = (long long)n2 * n3;
    const float* __restrict__ d = a.d + (long long)bl * g.n;
    const uint8_t* __restrict__ ph = a.phase + (long long)b * g.n;
    float* __restrict__ p = a.p + (long long)bl * g.n;
    auto plane_d = [&](int z) { return d + (long long)(z < 0 ? z + n1 : (z >= n1 ? z - n1 : z)) * S; };
    auto plane_e = [&](int z) { return ph + (long long)(z < 0 ? z + n1 : (z >= n1 ? z - n1 : z)) * S; };
    // window: D[node plane mod 3][row: i2 - 1, i2, i2 + 1][column], K[element plane mod 2][o2][column]
    // (o2 = 0: element row i2, o2 = 1: element row i2 - 1)
    float D[3][3][KV_NV + 2], K[2][2][KV_NV + 1];
    {
      const float* dm = plane_d(z0 - 1);
      const float* dc = plane_d(z0);
      kv_row(dm + G.rm, G, D[0][0]); kv_row(dm + G.rc, G, D[0][1]); kv_row(dm + G.rp, G, D[0][2]);
      kv_row(dc + G.rm, G, D[1][0]); kv_row(dc + G.rc, G, D[1][1]); kv_row(dc + G.rp, G, D[1][2]);
      const uint8_t* em = plane_e(z0 - 1);
      kv_krow(em + G.rc, G, mt, K[0][0]);
      kv_krow(em + G.rm, G, mt, K[0][1]);
    }
    const long long obase = (long long)z0 * S + G.rc + G.x0;
    auto step = [&](auto S_, int j) {
      constexpr int SS = decltype(S_)::value;
      constexpr int PM = SS % 3, PC = (SS + 1) % 3, PN = (SS + 2) % 3;
      constexpr int KM = SS % 2, KC = (SS + 1) % 2;
      const int z = z0 + j;
      const float* dn = plane_d(z + 1);
      kv_row(dn + G.rm, G, D[PN][0]); kv_row(dn + G.rc, G, D[PN][1]); kv_row(dn + G.rp, G, D[PN][2]);
      const uint8_t* ec = plane_e(z);
      kv_krow(ec + G.rc, G, mt, K[KC][0]);
      kv_krow(ec + G.rm, G, mt, K[KC][1]);
      const float(&dm)[3][KV_NV + 2] = D[PM];
      const float(&dc)[3][KV_NV + 2] = D[PC];
      const float(&dnr)[3][KV_NV + 2] = D[PN];
      const float(&km)[2][KV_NV + 1] = K[KM];
      const float(&kcr)[2][KV_NV + 1] = K[KC];
      float out[KV_NV];
      float sp = 0.f;
      float q0l = kcr[0][0] + kcr[1][0], q1l = km[0][0] + km[1][0];
      float e0l = kcr[0][0] + km[0][0], e1l = kcr[1][0] + km[1][0];
#pragma unroll
      for (int i = 0; i < KV_NV; ++i) {
        const float q0r = kcr[0][i + 1] + kcr[1][i + 1], q1r = km[0][i + 1] + km[1][i + 1];
        const float e0r = kcr[0][i + 1] + km[0][i + 1], e1r = kcr[1][i + 1] + km[1][i + 1];
        const float sk = (q0l + q0r) + (q1l + q1r);
        float acc = 4.f * sk * dc[1][i + 1];
        acc = fmaf(-e1l, dc[0][i], acc);
        acc = fmaf(-e1r, dc[0][i + 2], acc);
        acc = fmaf(-e0l, dc[2][i], acc);
        acc = fmaf(-e0r, dc[2][i + 2], acc);
        acc = fmaf(-q0l, dnr[1][i], acc);
        acc = fmaf(-q0r, dnr[1][i + 2], acc);
        acc = fmaf(-q1l, dm[1][i], acc);
        acc = fmaf(-q1r, dm[1][i + 2], acc);
        acc = fmaf(-(kcr[1][i] + kcr[1][i + 1]), dnr[0][i + 1], acc);
        acc = fmaf(-(kcr[0][i] + kcr[0][i + 1]), dnr[2][i + 1], acc);
        acc = fmaf(-(km[1][i] + km[1][i + 1]), dm[0][i + 1], acc);
        acc = fmaf(-(km[0][i] + km[0][i + 1]), dm[2][i + 1], acc);
        acc = fmaf(-kcr[1][i], dnr[0][i], acc);
        acc = fmaf(-kcr[1][i + 1], dnr[0][i + 2], acc);
        acc = fmaf(-kcr[0][i], dnr[2][i], acc);
        acc = fmaf(-kcr[0][i + 1], dnr[2][i + 2], acc);
        acc = fmaf(-km[1][i], dm[0][i], acc);
        acc = fmaf(-km[1][i + 1], dm[0][i + 2], acc);
        acc = fmaf(-km[0][i], dm[2][i], acc);
        acc = fmaf(-km[0][i + 1], dm[2][i + 2], acc);
        out[i] = acc;
        sp = fmaf(acc, dc[1][i + 1], sp);
        q0l = q0r; q1l = q1r; e0l = e0r; e1l = e1r;
      }
      // the products d p of one step are summed in FP32 (four terms) and accumulated across
      // steps in the float-float pair
      dot.add(sp);
      *reinterpret_cast<float4*>(p + obase + (long long)j * S) = make_float4(out[0], out[1], out[2], out[3]);
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    using I5 = std::integral_constant<int, 5>;
    for (int j = 0; j < nsteps; j += KV_UNROLL) {
      step(I0{}, j);
      if (j + 1 >= nsteps) break;
      step(I1{}, j + 1);
      if (j + 2 >= nsteps) break;
      step(I2{}, j + 2);
      if (j + 3 >= nsteps) break;
      step(I3{}, j + 3);
      if (j + 4 >= nsteps) break;
      step(I4{}, j + 4);
      if (j + 5 >= nsteps) break;
      step(I5{}, j + 5);
    }
  }
  const double bs = block_sum_acc(dot, red_sh);
  pdl_trigger();
  if (a.standalone) return;
  if (tid == 0) a.red.part[(long long)bl * ka.tiles + tile] = bs;
  if (last_block(a.red.ticket)) {
    const int warp = tid >> 5;
    for (int q = warp; q < BL; q += blockDim.x / 32) {
      const double sum = warp_sum_partials(a.red.part + (long long)q * ka.tiles, ka.tiles, 1);
      if (lane == 0 && !a.sc[q].done) step_update(a.sc[q], sum);
    }
    __syncthreads();
    if (tid == 0) *a.red.ticket = 0u;
  }
}

// ---------------------------------------------------------------- host side
bool ku_vec_supported(const Grid& g, int c, KuTmaShape s) {
  if (c != 1 || g.n3 % 32 != 0 || g.n3 > 512) return false;
  const int th = s.rows * (g.n3 / KV_NV);
  if (th % 32 != 0 || th < 64 || th > 512) return false;
  return s.rows >= 1 && g.n2 % s.rows == 0;
}

int ku_vec_blocks_x(const Grid& g, KuTmaShape s) { return (g.n2 / s.rows) * ((g.n1 + s.planes - 1) / s.planes); }

cudaError_t launch_ku_vec(const StencilArgs<float>& a, KuTmaShape s, cudaStream_t st) {
  if (!ku_vec_supported(a.g, a.c, s)) return cudaErrorInvalidValue;
  KuVecArgs ka{};
  ka.a = a;
  ka.ty = s.rows;
  ka.cz = s.planes;
  ka.tiles = ku_vec_blocks_x(a.g, s);
  return launch_pdl(k_ku_vec, dim3(ka.tiles * a.BL), dim3(s.rows * (a.g.n3 / KV_NV)), 0, st, ka);
}

}  // namespace unocg
