// Dirichlet boundary conditions on the voxel grid (Sec. 4.1, Sec. 6): N1 x N2 x N3 voxels,
// (N1+1)(N2+1)(N3+1) nodes, the fluctuation fixed to zero on every boundary node, so only the
// M_a = N_a - 1 interior nodes per axis carry unknowns.  Free node (j1, j2, j3) is full-grid
// node j + 1; it is corner o of the voxel e = j + 1 - o (all eight exist), and its neighbour
// j + s - 1 (s in {0,1,2}^3) is a free node when it lies in [0, M_a), else a fixed zero.
#pragma once
#include "../common.cuh"
#include "../element.cuh"

namespace unocg {

struct DGrid {
  int n1, n2, n3;   // voxels per axis
  int m1, m2, m3;   // free nodes per axis
  long long ne;     // voxels
  long long nf;     // free nodes per field
  double h, h12;    // voxel edge, h / 12
  float hf, h12f;
};

template <typename T> __device__ __forceinline__ T dgrid_h(const DGrid& g);
template <> __device__ __forceinline__ float dgrid_h<float>(const DGrid& g) { return g.hf; }
template <> __device__ __forceinline__ double dgrid_h<double>(const DGrid& g) { return g.h; }
template <typename T> __device__ __forceinline__ T dgrid_h12(const DGrid& g);
template <> __device__ __forceinline__ float dgrid_h12<float>(const DGrid& g) { return g.h12f; }
template <> __device__ __forceinline__ double dgrid_h12<double>(const DGrid& g) { return g.h12; }

// Neighbourhood of free node j: free-node offsets of the 27 neighbours (-1 when fixed) and
// voxel indices of the 8 voxels around it.
struct DNbr {
  long long row[3][3];  // (j1 + s1 - 1) m2 + (j2 + s2 - 1), times m3; -1 when outside
  int c3[3];            // j3 + s3 - 1, or -1
  long long vox[8];     // voxel of local corner o (index 4 o1 + 2 o2 + o3)
};
__device__ __forceinline__ void dneighbours(const DGrid& g, int j1, int j2, int j3, DNbr& nb) {
  int a1[3], a2[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int x1 = j1 + s - 1, x2 = j2 + s - 1, x3 = j3 + s - 1;
    a1[s] = (x1 >= 0 && x1 < g.m1) ? x1 : -1;
    a2[s] = (x2 >= 0 && x2 < g.m2) ? x2 : -1;
    nb.c3[s] = (x3 >= 0 && x3 < g.m3) ? x3 : -1;
  }
#pragma unroll
  for (int s1 = 0; s1 < 3; ++s1)
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2)
      nb.row[s1][s2] = (a1[s1] < 0 || a2[s2] < 0) ? -1LL : ((long long)a1[s1] * g.m2 + a2[s2]) * g.m3;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int e1 = j1 + 1 - ((o >> 2) & 1), e2 = j2 + 1 - ((o >> 1) & 1), e3 = j3 + 1 - (o & 1);
    nb.vox[o] = ((long long)e1 * g.n2 + e2) * g.n3 + e3;
  }
}
// value of neighbour s of field d (zero on fixed nodes)
template <typename T>
__device__ __forceinline__ T dld(const T* __restrict__ d, const DNbr& nb, int s1, int s2, int s3) {
  const long long r = nb.row[s1][s2];
  const int c = nb.c3[s3];
  return (r < 0 || c < 0) ? (T)0 : __ldg(d + r + c);
}

// (K d) at free node j, components [0, CC); d holds CC fields of nf values (stride nf).
template <typename T, int CC>
__device__ __forceinline__ void dnode_Ku(const T* __restrict__ d, const uint8_t* __restrict__ ph, const T* mt,
                                         const DGrid& g, int j1, int j2, int j3, T* out) {
  DNbr nb;
  dneighbours(g, j1, j2, j3, nb);
  if (CC == 1) {
    // trilinear Laplacian, 12 h^-1 K_e: 4 on the diagonal, 0 to edge neighbours, -1 across
    // face diagonals and the body diagonal
    T k[2][2][2];
#pragma unroll
    for (int o = 0; o < 8; ++o) k[(o >> 2) & 1][(o >> 1) & 1][o & 1] = mt[2 * __ldg(ph + nb.vox[o])];
    const T sk = (k[0][0][0] + k[0][0][1]) + (k[0][1][0] + k[0][1][1]) + (k[1][0][0] + k[1][0][1]) +
                 (k[1][1][0] + k[1][1][1]);
    T acc = (T)4 * sk * dld(d, nb, 1, 1, 1);
#pragma unroll
    for (int s2 = 0; s2 < 3; s2 += 2)
#pragma unroll
      for (int s3 = 0; s3 < 3; s3 += 2) {
        const int o2 = s2 == 0, o3 = s3 == 0;
        acc -= (k[0][o2][o3] + k[1][o2][o3]) * dld(d, nb, 1, s2, s3);
      }
#pragma unroll
    for (int s1 = 0; s1 < 3; s1 += 2)
#pragma unroll
      for (int s3 = 0; s3 < 3; s3 += 2) {
        const int o1 = s1 == 0, o3 = s3 == 0;
        acc -= (k[o1][0][o3] + k[o1][1][o3]) * dld(d, nb, s1, 1, s3);
      }
#pragma unroll
    for (int s1 = 0; s1 < 3; s1 += 2)
#pragma unroll
      for (int s2 = 0; s2 < 3; s2 += 2) {
        const int o1 = s1 == 0, o2 = s2 == 0;
        acc -= (k[o1][o2][0] + k[o1][o2][1]) * dld(d, nb, s1, s2, 1);
      }
#pragma unroll
    for (int s1 = 0; s1 < 3; s1 += 2)
#pragma unroll
      for (int s2 = 0; s2 < 3; s2 += 2)
#pragma unroll
        for (int s3 = 0; s3 < 3; s3 += 2) acc -= k[s1 == 0][s2 == 0][s3 == 0] * dld(d, nb, s1, s2, s3);
    out[0] = acc * dgrid_h12<T>(g);
  } else {
    const long long n = g.nf;
    T lam[8], mu[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int p = __ldg(ph + nb.vox[o]);
      lam[o] = mt[2 * p];
      mu[o] = mt[2 * p + 1];
    }
    T aL[8][3], aM[8][3];
#pragma unroll
    for (int o = 0; o < 8; ++o)
#pragma unroll
      for (int i = 0; i < 3; ++i) aL[o][i] = aM[o][i] = (T)0;
#pragma unroll
    for (int s = 0; s < 27; ++s) {
      const int s1 = s / 9, s2 = (s / 3) % 3, s3 = s % 3;
      T dv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dv[k] = dld(d + k * n, nb, s1, s2, s3);
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
        const int b1 = o1 + s1 - 1, b2 = o2 + s2 - 1, b3 = o3 + s3 - 1;
        if (b1 < 0 || b1 > 1 || b2 < 0 || b2 > 1 || b3 < 0 || b3 > 1) continue;
        const int bc = 4 * b1 + 2 * b2 + b3;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            aL[o][i] += elastic_table<T>().lam[o][i][bc][k] * dv[k];
            aM[o][i] += elastic_table<T>().mu[o][i][bc][k] * dv[k];
          }
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T acc = (T)0;
#pragma unroll
      for (int o = 0; o < 8; ++o) acc += lam[o] * aL[o][i] + mu[o] * aM[o][i];
      out[i] = acc * dgrid_h<T>(g);
    }
  }
}

// f at free node j: f_a = - sum_e int_e B_a^T C_e eps_bar, int_e dN_a/dx_k = (2 o_k - 1) h^2 / 4
template <int CC>
__device__ __forceinline__ void dnode_rhs(const uint8_t* __restrict__ ph, const double* mt, const DGrid& g,
                                          int j1, int j2, int j3, const double* load, double* f) {
  DNbr nb;
  dneighbours(g, j1, j2, j3, nb);
  const double q = 0.25 * g.h * g.h;
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
    const int p = ph[nb.vox[o]];
    const double g1 = 2 * o1 - 1, g2 = 2 * o2 - 1, g3 = 2 * o3 - 1;
    if (CC == 1) {
      acc[0] += mt[2 * p] * (g1 * load[0] + g2 * load[1] + g3 * load[2]);
    } else {
      const double is2 = 0.70710678118654752440;
      const double e11 = load[0], e22 = load[1], e33 = load[2];
      const double e12 = load[3] * is2, e13 = load[4] * is2, e23 = load[5] * is2;
      const double tr = e11 + e22 + e33;
      const double la = mt[2 * p], m2 = 2.0 * mt[2 * p + 1];
      const double s11 = la * tr + m2 * e11, s22 = la * tr + m2 * e22, s33 = la * tr + m2 * e33;
      const double s12 = m2 * e12, s13 = m2 * e13, s23 = m2 * e23;
      acc[0] += s11 * g1 + s12 * g2 + s13 * g3;
      acc[1] += s12 * g1 + s22 * g2 + s23 * g3;
      acc[2] += s13 * g1 + s23 * g2 + s33 * g3;
    }
  }
  for (int i = 0; i < CC; ++i) f[i] = -q * acc[i];
}

// diagonal of K at free node j (Jacobi)
template <int CC>
__device__ __forceinline__ void dnode_diag(const uint8_t* __restrict__ ph, const double* mt, const DGrid& g,
                                           int j1, int j2, int j3, double* dg) {
  DNbr nb;
  dneighbours(g, j1, j2, j3, nb);
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int p = ph[nb.vox[o]];
    if (CC == 1) {
      acc[0] += mt[2 * p] * Klap(o, o);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) acc[i] += mt[2 * p] * Klam(o, i, o, i) + mt[2 * p + 1] * Kmu(o, i, o, i);
    }
  }
  for (int i = 0; i < CC; ++i) dg[i] = acc[i] * g.h;
}

// Element-mean flux (thermal) or Mandel stress (elastic) of voxel (e1, e2, e3) for the
// fluctuation u (free-node fields, FP64, stride nf) plus the macroscopic load.
template <int CC>
__device__ __forceinline__ void delement_mean_flux(const double* __restrict__ u, const double* mt, int p,
                                                   const DGrid& g, int e1, int e2, int e3,
                                                   const double* load, double* sig) {
  const double s = 0.25 / g.h;
  double grad[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int c1 = (c >> 2) & 1, c2 = (c >> 1) & 1, c3 = c & 1;
    // corner node e + c is free node e + c - 1 when inside
    const int x1 = e1 + c1 - 1, x2 = e2 + c2 - 1, x3 = e3 + c3 - 1;
    if (x1 < 0 || x1 >= g.m1 || x2 < 0 || x2 >= g.m2 || x3 < 0 || x3 >= g.m3) continue;
    const long long node = ((long long)x1 * g.m2 + x2) * g.m3 + x3;
    const double sg[3] = {(double)(2 * c1 - 1), (double)(2 * c2 - 1), (double)(2 * c3 - 1)};
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      const double v = u[i * g.nf + node];
#pragma unroll
      for (int k = 0; k < 3; ++k) grad[i][k] += v * sg[k];
    }
  }
  if (CC == 1) {
    const double kap = mt[2 * p];
    for (int k = 0; k < 3; ++k) sig[k] = kap * (load[k] + s * grad[0][k]);
  } else {
    const double is2 = 0.70710678118654752440, sq2 = 1.41421356237309504880;
    const double e11 = load[0] + s * grad[0][0], e22 = load[1] + s * grad[1][1], e33 = load[2] + s * grad[2][2];
    const double e12 = load[3] * is2 + 0.5 * s * (grad[0][1] + grad[1][0]);
    const double e13 = load[4] * is2 + 0.5 * s * (grad[0][2] + grad[2][0]);
    const double e23 = load[5] * is2 + 0.5 * s * (grad[1][2] + grad[2][1]);
    const double la = mt[2 * p], m2 = 2.0 * mt[2 * p + 1];
    const double tr = e11 + e22 + e33;
    sig[0] = la * tr + m2 * e11;
    sig[1] = la * tr + m2 * e22;
    sig[2] = la * tr + m2 * e33;
    sig[3] = sq2 * m2 * e12;
    sig[4] = sq2 * m2 * e13;
    sig[5] = sq2 * m2 * e23;
  }
}

}  // namespace unocg
