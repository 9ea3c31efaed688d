// K d element by element (Sec. 4.1, "matrix-free implementations" of Sec. 5.5).
//
// The force of one brick on its corners, K_e u_e = h int_unit B^T C B u dxi, is evaluated in the
// Walsh basis of the trilinear field instead of as a 24 x 24 product.  With centred unit-cube
// coordinates xi in [-1/2, 1/2]^3 and corner signs s_k = 2 a_k - 1, every component u_i is
//   u_i = sum_M c_M(u_i) prod_{k in M} xi_k,   c_M = (raw Walsh sum  sum_a prod_{k in M} s_k u_a)
//                                                   / 2^(3 - |M|)
// over the subsets M of the three axes.  The gradient of such a field and the test functions'
// gradients are again of this form, and int xi_k dxi = 0, int xi_k^2 dxi = 1/12 make the element
// integral diagonal in M: with raw Walsh sums c[M][i] of the corner values,
//   f_{a,i} = sum_{M != {}} (prod_{k in M} s_k(a)) G[M][i],
//   G[{j}][j]   = h (2 mu c[j][j] + lam T0) / 16,                T0 = c[1][1] + c[2][2] + c[3][3]
//   G[{j}][i]   = h mu (c[j][i] + c[i][j]) / 16                  (i != j)
//   G[{j,k}][j] = h ((3 mu + lam) c[jk][j] + lam c[km][m]) / 48  (m the third axis)
//   G[{j,k}][m] = h mu (2 c[jk][m] + c[km][j] + c[jm][k]) / 48
//   G[{1,2,3}][i] = h (4 mu + lam) c[123][i] / 144.
// (Isotropic C = lam tr(eps) I + 2 mu eps; the constant mode M = {} carries no force.)  About 190
// additions and multiplications per element instead of 1,152 multiply-adds per node.  Thermal
// conduction (c = 1, K_e = h kappa int grad N . grad N) in the same basis is diagonal:
//   G[M] = h kappa c[M] / 16, / 24, / 48 for |M| = 1, 2, 3.
//
// Work layout: a block of KE_THREADS threads computes a node tile of 32 (i3) x 8 (i2) nodes over
// KE_CZ consecutive node planes.  Its first 33 x 9 threads each own one element column (the tile's
// elements plus the lower halo row and column) and march along i1: per element layer they load
// the 4 corner nodes of the new node plane, reuse the 2D Walsh sums of the previous plane, form
// the 8 corner forces, keep the upper four (a1 = 1) for the next layer and publish the lower four
// plus the kept ones in shared memory; the first 256 threads then sum the four element columns
// around their node and store p = K d.
#pragma once
#include "stencil.cuh"

namespace unocg {

constexpr int KE_T3 = 32, KE_T2 = 8;                 // node tile (i3 x i2)
constexpr int KE_S3 = KE_T3 + 1, KE_S2 = KE_T2 + 1;   // element columns with the lower halo
constexpr int KE_SLOTS = KE_S3 * KE_S2;               // 297
constexpr int KE_THREADS = 320;
#ifndef UNOCG_KE_CZ
#define UNOCG_KE_CZ 8
#endif
constexpr int KE_CZ = UNOCG_KE_CZ;                    // node planes per block

// two buffers of 4 corners x CC components per element column
template <typename T, int CC> constexpr size_t ke_smem_bytes() { return 2 * 4 * CC * KE_SLOTS * sizeof(T); }

__host__ __device__ inline int ke_tiles(const Grid& g) {
  return ((g.n3 + KE_T3 - 1) / KE_T3) * ((g.n2 + KE_T2 - 1) / KE_T2) * ((g.n1 + KE_CZ - 1) / KE_CZ);
}

// 2D Walsh sums of the four corner values of one node plane (index a2 * 2 + a3):
// e = sum, k3 = sum s3 u, k2 = sum s2 u, k23 = sum s2 s3 u
template <typename T> struct KeW2 {
  T e, k3, k2, k23;
};
template <typename T>
__device__ __forceinline__ KeW2<T> ke_walsh2(T u00, T u01, T u10, T u11) {
  const T s0 = u00 + u01, d0 = u01 - u00, s1 = u10 + u11, d1 = u11 - u10;
  return {s0 + s1, d0 + d1, s1 - s0, d1 - d0};
}

// Corner forces of one element from the Walsh sums of its lower (a1 = 0) and upper (a1 = 1)
// node planes: flo[a2 * 2 + a3][i] at a1 = 0, fhi at a1 = 1.  k = (h mu / 8, h lam / 16,
// h mu / 48, h lam / 48, h (3 mu + lam) / 48, h (4 mu + lam) / 144), see the header comment.
template <typename T>
__device__ __forceinline__ void ke_element(const KeW2<T> (&L)[1], const KeW2<T> (&H)[1], const T (&k)[6],
                                           T (&flo)[4][1], T (&fhi)[4][1]) {
  // thermal: k = (h kappa / 16, h kappa / 24, h kappa / 48)
  const T G1 = k[0] * (H[0].e - L[0].e), G2 = k[0] * (L[0].k2 + H[0].k2), G3 = k[0] * (L[0].k3 + H[0].k3);
  const T G12 = k[1] * (H[0].k2 - L[0].k2), G13 = k[1] * (H[0].k3 - L[0].k3), G23 = k[1] * (L[0].k23 + H[0].k23);
  const T G123 = k[2] * (H[0].k23 - L[0].k23);
  const T ex0 = -G2, ey0 = G3 - G23, ex1 = G2, ey1 = G3 + G23;
  const T E00 = ex0 - ey0, E01 = ex0 + ey0, E10 = ex1 - ey1, E11 = ex1 + ey1;
  const T fx0 = G1 - G12, fy0 = G13 - G123, fx1 = G1 + G12, fy1 = G13 + G123;
  const T F00 = fx0 - fy0, F01 = fx0 + fy0, F10 = fx1 - fy1, F11 = fx1 + fy1;
  flo[0][0] = E00 - F00; fhi[0][0] = E00 + F00;
  flo[1][0] = E01 - F01; fhi[1][0] = E01 + F01;
  flo[2][0] = E10 - F10; fhi[2][0] = E10 + F10;
  flo[3][0] = E11 - F11; fhi[3][0] = E11 + F11;
}

template <typename T>
__device__ __forceinline__ void ke_element(const KeW2<T> (&L)[3], const KeW2<T> (&H)[3], const T (&k)[6],
                                           T (&flo)[4][3], T (&fhi)[4][3]) {
  const T A1 = k[0], b1 = k[1], a2 = k[2], b2 = k[3], A2 = k[4], g3 = k[5];
  T c1[3], c2[3], c3[3], c12[3], c13[3], c23[3], c123[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c1[i] = H[i].e - L[i].e;
    c2[i] = L[i].k2 + H[i].k2;
    c3[i] = L[i].k3 + H[i].k3;
    c12[i] = H[i].k2 - L[i].k2;
    c13[i] = H[i].k3 - L[i].k3;
    c23[i] = L[i].k23 + H[i].k23;
    c123[i] = H[i].k23 - L[i].k23;
  }
  T G1[3], G2[3], G3[3], G12[3], G13[3], G23[3], G123[3];
  // single axes: normal parts and the symmetric shear pairs
  const T t0 = b1 * ((c1[0] + c2[1]) + c3[2]);
  G1[0] = A1 * c1[0] + t0;
  G2[1] = A1 * c2[1] + t0;
  G3[2] = A1 * c3[2] + t0;
  const T a1 = (T)0.5 * A1;
  const T s01 = a1 * (c2[0] + c1[1]), s02 = a1 * (c3[0] + c1[2]), s12 = a1 * (c3[1] + c2[2]);
  G2[0] = s01; G1[1] = s01;
  G3[0] = s02; G1[2] = s02;
  G3[1] = s12; G2[2] = s12;
  // axis pairs (0-based axes: {0,1} -> c12, {0,2} -> c13, {1,2} -> c23)
  G12[0] = A2 * c12[0] + b2 * c23[2];
  G12[1] = A2 * c12[1] + b2 * c13[2];
  G12[2] = a2 * (((T)2 * c12[2] + c23[0]) + c13[1]);
  G13[0] = A2 * c13[0] + b2 * c23[1];
  G13[2] = A2 * c13[2] + b2 * c12[1];
  G13[1] = a2 * (((T)2 * c13[1] + c23[0]) + c12[2]);
  G23[1] = A2 * c23[1] + b2 * c13[0];
  G23[2] = A2 * c23[2] + b2 * c12[0];
  G23[0] = a2 * (((T)2 * c23[0] + c13[1]) + c12[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i) G123[i] = g3 * c123[i];
  // inverse Walsh: f(a1, a2, a3) = E(a2, a3) + s1 F(a2, a3)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T ex0 = -G2[i], ey0 = G3[i] - G23[i], ex1 = G2[i], ey1 = G3[i] + G23[i];
    const T E00 = ex0 - ey0, E01 = ex0 + ey0, E10 = ex1 - ey1, E11 = ex1 + ey1;
    const T fx0 = G1[i] - G12[i], fy0 = G13[i] - G123[i], fx1 = G1[i] + G12[i], fy1 = G13[i] + G123[i];
    const T F00 = fx0 - fy0, F01 = fx0 + fy0, F10 = fx1 - fy1, F11 = fx1 + fy1;
    flo[0][i] = E00 - F00; fhi[0][i] = E00 + F00;
    flo[1][i] = E01 - F01; fhi[1][i] = E01 + F01;
    flo[2][i] = E10 - F10; fhi[2][i] = E10 + F10;
    flo[3][i] = E11 - F11; fhi[3][i] = E11 + F11;
  }
}

__device__ __forceinline__ int ke_wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Element constants of phase p (see ke_element)
template <typename T, int CC>
__device__ __forceinline__ void ke_consts(const T* mt, int p, T h, T (&k)[6]) {
  if (CC == 1) {
    const T hk = h * mt[2 * p];
    k[0] = hk * (T)0.0625;
    k[1] = hk * (T)(1.0 / 24.0);
    k[2] = hk * (T)(1.0 / 48.0);
    k[3] = k[4] = k[5] = (T)0;
    return;
  }
  const T lam = mt[2 * p], mu = mt[2 * p + 1];
  k[0] = h * mu * (T)0.125;
  k[1] = h * lam * (T)0.0625;
  k[2] = h * mu * (T)(1.0 / 48.0);
  k[3] = h * lam * (T)(1.0 / 48.0);
  k[4] = h * ((T)3 * mu + lam) * (T)(1.0 / 48.0);
  k[5] = h * ((T)4 * mu + lam) * (T)(1.0 / 144.0);
}

// p = K d on node tile `tile` of (instance, load) bl; block of KE_THREADS threads, `sm` holds
// ke_smem_bytes<T, CC>().  Returns the block sum of d . p (thread 0) unless a.standalone.
// skip: optional flag of the pair (nonzero = finished), uniform over the block.
template <typename T, int CC, bool COH>
__device__ double ku_element_tile(const StencilArgs<T>& a, const T* mt, int bl, int tile, double* red_sh, T* sm,
                                  const int* skip) {
  const Grid& g = a.g;
  const long long n = g.n;
  const uint8_t* ph = a.phase + (long long)(bl / a.L) * n;
  const T* d = a.d + (long long)bl * CC * n;
  T* p = a.p + (long long)bl * CC * n;
  const int nt3 = (g.n3 + KE_T3 - 1) / KE_T3, nt2 = (g.n2 + KE_T2 - 1) / KE_T2;
  int bx = tile;
  const int b3 = bx % nt3;
  bx /= nt3;
  const int b2 = bx % nt2;
  const int b1 = bx / nt2;
  const int t3 = b3 * KE_T3, t2 = b2 * KE_T2, z0 = b1 * KE_CZ;
  const int zend = min(z0 + KE_CZ, g.n1);
  const int S = g.n2 * g.n3;
  const int tid = threadIdx.x;
  // element column of this thread (element e occupies nodes e .. e + 1, periodic)
  const bool is_el = tid < KE_SLOTS;
  const int s2 = tid / KE_S3, s3 = tid - s2 * KE_S3;
  int o00 = 0, o01 = 0, o10 = 0, o11 = 0;
  if (is_el) {
    const int e2 = ke_wrap(t2 - 1 + s2, g.n2), e3 = ke_wrap(t3 - 1 + s3, g.n3);
    const int e2p = (e2 + 1 == g.n2) ? 0 : e2 + 1, e3p = (e3 + 1 == g.n3) ? 0 : e3 + 1;
    o00 = e2 * g.n3 + e3;
    o01 = e2 * g.n3 + e3p;
    o10 = e2p * g.n3 + e3;
    o11 = e2p * g.n3 + e3p;
  }
  // output node of this thread
  const int r2 = tid >> 5, r3 = tid & 31;
  const bool is_node = tid < KE_T3 * KE_T2 && t2 + r2 < g.n2 && t3 + r3 < g.n3;
  const int noff = (t2 + r2) * g.n3 + t3 + r3;
  const T h = grid_h<T>(g);
  DotAcc<T> dp;
  KeW2<T> L[CC], H[CC];
  T carry[4][CC];
  auto load_plane = [&](int z, KeW2<T>(&W)[CC]) {
    const T* dz = d + (long long)z * S;
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      const T* di = dz + (long long)i * n;
      W[i] = ke_walsh2<T>(ldf<COH>(di + o00), ldf<COH>(di + o01), ldf<COH>(di + o10), ldf<COH>(di + o11));
    }
  };
  if (is_el) {
    // the element layer below the first node plane only contributes its upper corners
    const int zm = z0 ? z0 - 1 : g.n1 - 1;
    load_plane(zm, L);
    load_plane(z0, H);
    T k[6], flo[4][CC];
    ke_consts<T, CC>(mt, __ldg(ph + (long long)zm * S + o00), h, k);
    ke_element<T>(L, H, k, flo, carry);
  }
  if (skip && *skip) return 0.0;
  for (int z = z0; z < zend; ++z) {
    T* buf = sm + ((z - z0) & 1) * (4 * CC * KE_SLOTS);
    if (is_el) {
#pragma unroll
      for (int i = 0; i < CC; ++i) L[i] = H[i];
      load_plane(z + 1 == g.n1 ? 0 : z + 1, H);
      T k[6], flo[4][CC], fhi[4][CC];
      ke_consts<T, CC>(mt, __ldg(ph + (long long)z * S + o00), h, k);
      ke_element<T>(L, H, k, flo, fhi);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < CC; ++i) {
          buf[(i * 4 + c) * KE_SLOTS + tid] = flo[c][i] + carry[c][i];
          carry[c][i] = fhi[c][i];
        }
    }
    __syncthreads();
    if (is_node) {
      // node (r2, r3) collects corner (a2, a3) of element column (r2 + 1 - a2, r3 + 1 - a3)
      const int sA = (r2 + 1) * KE_S3 + r3 + 1, sB = r2 * KE_S3 + r3;
      const long long q = (long long)z * S + noff;
#pragma unroll
      for (int i = 0; i < CC; ++i) {
        const T* bi = buf + i * 4 * KE_SLOTS;
        const T v = (bi[sA] + bi[KE_SLOTS + sA - 1]) + (bi[2 * KE_SLOTS + sB + 1] + bi[3 * KE_SLOTS + sB]);
        p[(long long)i * n + q] = v;
        dp.add_prod(v, ldf<COH>(d + (long long)i * n + q));
      }
    }
    // the next layer writes the other buffer: one barrier per layer suffices
  }
  if (a.standalone) {
    __syncthreads();
    return 0.0;
  }
  return block_sum_acc(dp, red_sh);
}

}  // namespace unocg
