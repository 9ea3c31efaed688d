// K d task functions shared by the per-phase kernel and the persistent kernel.
#pragma once
#include "stencil.cuh"

namespace unocg {

// Thermal: every thread marches along i1 over KU_CZ consecutive nodes of one (i2, i3) column,
// keeping the 3x3 neighbourhoods of the planes i1-1, i1, i1+1 and the conductivities of the
// element planes i1-1, i1 in registers: 9 loads of d and 4 phase labels per node.
#ifndef UNOCG_KU_CZ
#define UNOCG_KU_CZ 8
#endif
constexpr int KU_CZ = UNOCG_KU_CZ;

__device__ __forceinline__ bool tile_column_at(const Grid& g, int tile, int cz, int& i1, int& i2, int& i3) {
  const int nt3 = (g.n3 + 31) >> 5, nt2 = (g.n2 + 7) >> 3;
  int bx = tile;
  const int b3 = bx % nt3;
  bx /= nt3;
  const int b2 = bx % nt2;
  const int b1 = bx / nt2;
  i3 = b3 * 32 + (threadIdx.x & 31);
  i2 = b2 * 8 + (threadIdx.x >> 5);
  i1 = b1 * cz;
  return i3 < g.n3 && i2 < g.n2 && i1 < g.n1;
}

template <typename T, bool COH = false>
__device__ __forceinline__ void ku_thermal_column(const T* __restrict__ d, T* __restrict__ p,
                                                  const uint8_t* __restrict__ ph, const T* mt,
                                                  const Grid& g, int i1, int i2, int i3, int cz,
                                                  DotAcc<T>& dp, const int* skip = nullptr) {
  const int S = g.n2 * g.n3;
  const int c2[3] = {i2 ? i2 - 1 : g.n2 - 1, i2, (i2 + 1 == g.n2) ? 0 : i2 + 1};
  const int c3[3] = {i3 ? i3 - 1 : g.n3 - 1, i3, (i3 + 1 == g.n3) ? 0 : i3 + 1};
  int off[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) off[a][b] = c2[a] * g.n3 + c3[b];
  // d planes: dm (i1-1), dc (i1), dn (i1+1); element conductivities km (plane i1-1), kc (plane i1)
  T dm[3][3], dc[3][3], dn[3][3], km[2][2], kc[2][2];
  int zm = (i1 ? i1 - 1 : g.n1 - 1) * S, zc = i1 * S;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      dm[a][b] = ldf<COH>(d + zm + off[a][b]);
      dc[a][b] = ldf<COH>(d + zc + off[a][b]);
    }
  // element (e1, i2 - o2, i3 - o3) sits at off[1 - o2][1 - o3] of element plane e1
#pragma unroll
  for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
    for (int o3 = 0; o3 < 2; ++o3) km[o2][o3] = mt[2 * __ldg(ph + zm + off[1 - o2][1 - o3])];
  // a finished (instance, load) is skipped; the flag is read after the first loads are issued
  if (skip && *skip) return;
  const T hf = grid_h12<T>(g);
  const int zend = min(i1 + cz, g.n1);
  auto step = [&](int z) {
    const int zn = ((z + 1 == g.n1) ? 0 : z + 1) * S;
    zc = z * S;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) dn[a][b] = ldf<COH>(d + zn + off[a][b]);
#pragma unroll
    for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
      for (int o3 = 0; o3 < 2; ++o3) kc[o2][o3] = mt[2 * __ldg(ph + zc + off[1 - o2][1 - o3])];
    // k[o1][o2][o3]: o1 = 0 -> element plane z (kc), o1 = 1 -> plane z-1 (km)
    T sk = (kc[0][0] + kc[0][1]) + (kc[1][0] + kc[1][1]) + (km[0][0] + km[0][1]) + (km[1][0] + km[1][1]);
    T acc = (T)4 * sk * dc[1][1];
    // edge-diagonal neighbours in the plane (delta1 = 0): elements o1 in {0,1}
#pragma unroll
    for (int s2 = 0; s2 < 3; s2 += 2)
#pragma unroll
      for (int s3 = 0; s3 < 3; s3 += 2) {
        const int o2 = s2 == 0, o3 = s3 == 0;
        acc -= (kc[o2][o3] + km[o2][o3]) * dc[s2][s3];
      }
    // delta2 = 0: elements o2 in {0,1}, fixed o1, o3
#pragma unroll
    for (int s3 = 0; s3 < 3; s3 += 2) {
      const int o3 = s3 == 0;
      acc -= (kc[0][o3] + kc[1][o3]) * dn[1][s3];
      acc -= (km[0][o3] + km[1][o3]) * dm[1][s3];
    }
    // delta3 = 0: elements o3 in {0,1}, fixed o1, o2
#pragma unroll
    for (int s2 = 0; s2 < 3; s2 += 2) {
      const int o2 = s2 == 0;
      acc -= (kc[o2][0] + kc[o2][1]) * dn[s2][1];
      acc -= (km[o2][0] + km[o2][1]) * dm[s2][1];
    }
    // corners: one element each
#pragma unroll
    for (int s2 = 0; s2 < 3; s2 += 2)
#pragma unroll
      for (int s3 = 0; s3 < 3; s3 += 2) {
        const int o2 = s2 == 0, o3 = s3 == 0;
        acc -= kc[o2][o3] * dn[s2][s3];
        acc -= km[o2][o3] * dm[s2][s3];
      }
    const T out = acc * hf;
    p[zc + off[1][1]] = out;
    dp.add_prod(out, dc[1][1]);
    // shift the window
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        dm[a][b] = dc[a][b];
        dc[a][b] = dn[a][b];
      }
#pragma unroll
    for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
      for (int o3 = 0; o3 < 2; ++o3) km[o2][o3] = kc[o2][o3];
  };
  if (zend - i1 == KU_CZ) {
    // full column: unrolled, so that the loads of later planes are issued ahead
#pragma unroll
    for (int zz = 0; zz < KU_CZ; ++zz) step(i1 + zz);
  } else {
    for (int z = i1; z < zend; ++z) step(z);
  }
}


// Thermal K d on a shared-memory tile: a block of 32 (i3) x 8 (i2) threads computes a
// 32 x 8 x KU_TZ node tile.  All threads first load the node halo of d
// ((KU_TZ+2) x 10 x 34) and the element conductivities ((KU_TZ+1) x 9 x 33) with independent
// loads (one memory latency per tile), then evaluate the 21-term node stencil from shared memory.
#ifndef UNOCG_KU_TZ
#define UNOCG_KU_TZ 4
#endif
#ifndef UNOCG_KU_MODE
#define UNOCG_KU_MODE 1  // 0: shared-memory tile, 1: register column march (measured faster)
#endif
constexpr int KU_TZ = UNOCG_KU_TZ;
constexpr int KU_DN = (KU_TZ + 2) * 10 * 34;
constexpr int KU_KN = (KU_TZ + 1) * 9 * 33;

__device__ __forceinline__ int wrap_idx(int v, int n) {
  if (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

template <typename T, bool COH>
__device__ __forceinline__ void ku_thermal_tile(const T* __restrict__ d, T* __restrict__ p,
                                                  const uint8_t* __restrict__ ph, const T* mt,
                                                  const Grid& g, int tile, T* ds, T* ks, DotAcc<T>& dp) {
  const int nt3 = (g.n3 + 31) >> 5, nt2 = (g.n2 + 7) >> 3;
  const int b3 = tile % nt3;
  const int rest = tile / nt3;
  const int b2 = rest % nt2;
  const int b1 = rest / nt2;
  const int o3 = b3 * 32 - 1, o2 = b2 * 8 - 1, o1 = b1 * KU_TZ - 1;
  const int S = g.n2 * g.n3;
  constexpr int U = 8;
  // node halo of d
  for (int i0 = threadIdx.x; i0 < KU_DN; i0 += U * blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < KU_DN) {
        const int z = idx / 340, rem = idx - z * 340, y = rem / 34, x = rem - y * 34;
        const int gz = wrap_idx(o1 + z, g.n1), gy = wrap_idx(o2 + y, g.n2), gx = wrap_idx(o3 + x, g.n3);
        v[u] = ldf<COH>(d + gz * S + gy * g.n3 + gx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < KU_DN) ds[idx] = v[u];
    }
  }
  // element conductivities (element (e1, e2, e3) owns nodes e .. e+1)
  for (int i0 = threadIdx.x; i0 < KU_KN; i0 += U * blockDim.x) {
    uint8_t pv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < KU_KN) {
        const int z = idx / 297, rem = idx - z * 297, y = rem / 33, x = rem - y * 33;
        const int gz = wrap_idx(o1 + z, g.n1), gy = wrap_idx(o2 + y, g.n2), gx = wrap_idx(o3 + x, g.n3);
        pv[u] = __ldg(ph + gz * S + gy * g.n3 + gx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = i0 + u * blockDim.x;
      if (idx < KU_KN) ks[idx] = mt[2 * pv[u]];
    }
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i3 = o3 + 1 + tx, i2 = o2 + 1 + ty;
  if (i3 < g.n3 && i2 < g.n2) {
    const T hf = grid_h12<T>(g);
#pragma unroll
    for (int z = 0; z < KU_TZ; ++z) {
      const int i1 = o1 + 1 + z;
      if (i1 >= g.n1) break;
      // d at node-tile offset (z+1+a, ty+1+b, tx+1+c), a,b,c in {-1,0,1}
      auto D = [&](int a, int b, int c) { return ds[((z + 1 + a) * 10 + (ty + 1 + b)) * 34 + tx + 1 + c]; };
      // kappa of element (node - o): element-tile offset (z+1-o1, ty+1-o2, tx+1-o3)
      auto K = [&](int q1, int q2, int q3) { return ks[((z + 1 - q1) * 9 + (ty + 1 - q2)) * 33 + tx + 1 - q3]; };
      T k[2][2][2];
#pragma unroll
      for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2)
#pragma unroll
          for (int q3 = 0; q3 < 2; ++q3) k[q1][q2][q3] = K(q1, q2, q3);
      T sk = (k[0][0][0] + k[0][0][1]) + (k[0][1][0] + k[0][1][1]) + (k[1][0][0] + k[1][0][1]) +
             (k[1][1][0] + k[1][1][1]);
      const T dcen = D(0, 0, 0);
      T acc = (T)4 * sk * dcen;
#pragma unroll
      for (int s2 = -1; s2 <= 1; s2 += 2)
#pragma unroll
        for (int s3 = -1; s3 <= 1; s3 += 2) {
          const int q2 = s2 < 0, q3 = s3 < 0;
          acc -= (k[0][q2][q3] + k[1][q2][q3]) * D(0, s2, s3);
        }
#pragma unroll
      for (int s1 = -1; s1 <= 1; s1 += 2)
#pragma unroll
        for (int s3 = -1; s3 <= 1; s3 += 2) {
          const int q1 = s1 < 0, q3 = s3 < 0;
          acc -= (k[q1][0][q3] + k[q1][1][q3]) * D(s1, 0, s3);
        }
#pragma unroll
      for (int s1 = -1; s1 <= 1; s1 += 2)
#pragma unroll
        for (int s2 = -1; s2 <= 1; s2 += 2) {
          const int q1 = s1 < 0, q2 = s2 < 0;
          acc -= (k[q1][q2][0] + k[q1][q2][1]) * D(s1, s2, 0);
        }
#pragma unroll
      for (int s1 = -1; s1 <= 1; s1 += 2)
#pragma unroll
        for (int s2 = -1; s2 <= 1; s2 += 2)
#pragma unroll
          for (int s3 = -1; s3 <= 1; s3 += 2) acc -= k[s1 < 0][s2 < 0][s3 < 0] * D(s1, s2, s3);
      const T out = acc * hf;
      p[i1 * S + i2 * g.n3 + i3] = out;
      dp.add_prod(out, dcen);
    }
  }
}

// K d of one tile of (instance, load) bl: thermal = one 32 x 8 x KU_CZ column block, elastic =
// one 32 x 4 x 2 node block.  Returns the block sum of d . p (valid in thread 0).
// skip: optional flag of the pair (nonzero = finished, no work), read as late as possible.
template <typename T, int CC, bool COH>
__device__ double ku_task(const StencilArgs<T>& a, const T* mt, int bl, int tile, double* red_sh, T* tile_smem,
                          const int* skip = nullptr) {
  const Grid& g = a.g;
  const int b = bl / a.L;
  const long long n = g.n;
  const uint8_t* ph = a.phase + (long long)b * n;
  const T* d = a.d + (long long)bl * CC * n;
  T* p = a.p + (long long)bl * CC * n;
  DotAcc<T> dp;
  if (CC == 1) {
#if UNOCG_KU_MODE == 0
    ku_thermal_tile<T, COH>(d, p, ph, mt, g, tile, tile_smem, tile_smem + KU_DN, dp);
#else
    int i1, i2, i3;
    if (tile_column_at(g, tile, KU_CZ, i1, i2, i3))
      ku_thermal_column<T, COH>(d, p, ph, mt, g, i1, i2, i3, KU_CZ, dp, skip);
#endif
  } else {
    int i1, i2, i3;
    if (tile_node_at(g, tile, i1, i2, i3) && !(skip && *skip)) {
      const long long node = ((long long)i1 * g.n2 + i2) * g.n3 + i3;
      T out[CC];
      node_Ku<T, CC, COH>(d, ph, mt, g, i1, i2, i3, out);
#pragma unroll
      for (int i = 0; i < CC; ++i) {
        p[i * n + node] = out[i];
        dp.add_prod(out[i], ldf<COH>(d + i * n + node));
      }
    }
  }
  if (a.standalone) {
    __syncthreads();  // the tile buffers are reused by the next task
    return 0.0;
  }
  return block_sum_acc(dp, red_sh);  // contains the barrier that protects the tile buffers
}

}  // namespace unocg
