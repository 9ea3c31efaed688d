// Per-node and per-element device functions of the periodic trilinear-brick discretization
// (Sec. 4.1): matrix-free K d, right-hand side, diagonal, element-mean flux/stress and
// Gauss-point energy products.  Node (i1, i2, i3) touches the elements e = node - o,
// o in {0,1}^3, and is their local corner o (corner index 4 o1 + 2 o2 + o3).
#pragma once
#include "common.cuh"
#include "element.cuh"

namespace unocg {

// Node handled by this thread: blocks of 32 (i3) x 4 (i2) x blockDim/128 (i1).
__device__ __forceinline__ bool tile_node_at(const Grid& g, int tile, int& i1, int& i2, int& i3) {
  const int tz_n = blockDim.x >> 7;
  const int nt3 = (g.n3 + 31) >> 5, nt2 = (g.n2 + 3) >> 2;
  int bx = tile;
  int b3 = bx % nt3;
  bx /= nt3;
  int b2 = bx % nt2;
  int b1 = bx / nt2;
  i3 = b3 * 32 + (threadIdx.x & 31);
  i2 = b2 * 4 + ((threadIdx.x >> 5) & 3);
  i1 = b1 * tz_n + (threadIdx.x >> 7);
  return i1 < g.n1 && i2 < g.n2 && i3 < g.n3;
}
__device__ __forceinline__ bool tile_node(const Grid& g, int& i1, int& i2, int& i3) {
  return tile_node_at(g, blockIdx.x, i1, i2, i3);
}

struct Nbr {
  long long row[3][3];  // (c1[a]*n2 + c2[b])*n3
  int c3[3];
  int c1[3], c2[3];
};
__device__ __forceinline__ void neighbours(const Grid& g, int i1, int i2, int i3, Nbr& nb) {
  nb.c1[0] = i1 ? i1 - 1 : g.n1 - 1; nb.c1[1] = i1; nb.c1[2] = (i1 + 1 == g.n1) ? 0 : i1 + 1;
  nb.c2[0] = i2 ? i2 - 1 : g.n2 - 1; nb.c2[1] = i2; nb.c2[2] = (i2 + 1 == g.n2) ? 0 : i2 + 1;
  nb.c3[0] = i3 ? i3 - 1 : g.n3 - 1; nb.c3[1] = i3; nb.c3[2] = (i3 + 1 == g.n3) ? 0 : i3 + 1;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) nb.row[a][b] = ((long long)nb.c1[a] * g.n2 + nb.c2[b]) * g.n3;
}
// index of neighbour s = delta + 1 in {0,1,2}^3
__device__ __forceinline__ long long nidx(const Nbr& nb, int s1, int s2, int s3) {
  return nb.row[s1][s2] + nb.c3[s3];
}
// element e = node - o  ->  the element's own (lower-corner) index
__device__ __forceinline__ long long eidx(const Nbr& nb, int o1, int o2, int o3) {
  return nb.row[1 - o1][1 - o2] + nb.c3[1 - o3];
}

// Loads of fields that other blocks of the same launch may have written (persistent kernel)
// bypass L1 (ld.global.cg); otherwise the read-only path is used.
template <bool COH, typename T> __device__ __forceinline__ T ldf(const T* p) {
  if (COH) return __ldcg(p);
  return __ldg(p);
}

template <typename T, int CC, bool COH = false>
__device__ __forceinline__ void node_Ku(const T* __restrict__ d, const uint8_t* __restrict__ ph,
                                        const T* mt, const Grid& g, int i1, int i2, int i3, T* out) {
  Nbr nb;
  neighbours(g, i1, i2, i3, nb);
  const long long n = g.n;
  if (CC == 1) {
    T k[2][2][2];
#pragma unroll
    for (int o1 = 0; o1 < 2; ++o1)
#pragma unroll
      for (int o2 = 0; o2 < 2; ++o2)
#pragma unroll
        for (int o3 = 0; o3 < 2; ++o3) k[o1][o2][o3] = mt[2 * __ldg(ph + eidx(nb, o1, o2, o3))];
    T sk = (k[0][0][0] + k[0][0][1]) + (k[0][1][0] + k[0][1][1]) + (k[1][0][0] + k[1][0][1]) +
           (k[1][1][0] + k[1][1][1]);
    T acc = (T)4 * sk * ldf<COH>(d + nidx(nb, 1, 1, 1));
#pragma unroll
    for (int s2 = 0; s2 < 3; s2 += 2)
#pragma unroll
      for (int s3 = 0; s3 < 3; s3 += 2) {
        const int o2 = s2 == 0, o3 = s3 == 0;
        acc -= (k[0][o2][o3] + k[1][o2][o3]) * ldf<COH>(d + nidx(nb, 1, s2, s3));
      }
#pragma unroll
    for (int s1 = 0; s1 < 3; s1 += 2)
#pragma unroll
      for (int s3 = 0; s3 < 3; s3 += 2) {
        const int o1 = s1 == 0, o3 = s3 == 0;
        acc -= (k[o1][0][o3] + k[o1][1][o3]) * ldf<COH>(d + nidx(nb, s1, 1, s3));
      }
#pragma unroll
    for (int s1 = 0; s1 < 3; s1 += 2)
#pragma unroll
      for (int s2 = 0; s2 < 3; s2 += 2) {
        const int o1 = s1 == 0, o2 = s2 == 0;
        acc -= (k[o1][o2][0] + k[o1][o2][1]) * ldf<COH>(d + nidx(nb, s1, s2, 1));
      }
#pragma unroll
    for (int s1 = 0; s1 < 3; s1 += 2)
#pragma unroll
      for (int s2 = 0; s2 < 3; s2 += 2)
#pragma unroll
        for (int s3 = 0; s3 < 3; s3 += 2)
          acc -= k[s1 == 0][s2 == 0][s3 == 0] * ldf<COH>(d + nidx(nb, s1, s2, s3));
    out[0] = acc * grid_h12<T>(g);
  } else {
    T lam[8], mu[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      int p = __ldg(ph + eidx(nb, (o >> 2) & 1, (o >> 1) & 1, o & 1));
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
      const long long q = nidx(nb, s1, s2, s3);
      T dv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dv[k] = ldf<COH>(d + k * n + q);
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
      out[i] = acc * grid_h<T>(g);
    }
  }
}

// f_a = - sum_e int_e B_a^T C_e eps_bar, with int_e dN_a/dx_j = (2 o_j - 1) h^2 / 4.
template <int CC>
__device__ __forceinline__ void node_rhs(const uint8_t* __restrict__ ph, const double* mt, const Grid& g,
                                         int i1, int i2, int i3, const double* load, double* f) {
  Nbr nb;
  neighbours(g, i1, i2, i3, nb);
  const double q = 0.25 * g.h * g.h;
  if (CC == 1) {
    double acc = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
      double kap = mt[2 * ph[eidx(nb, o1, o2, o3)]];
      acc += kap * ((2 * o1 - 1) * load[0] + (2 * o2 - 1) * load[1] + (2 * o3 - 1) * load[2]);
    }
    f[0] = -q * acc;
  } else {
    const double is2 = 0.70710678118654752440;
    const double e11 = load[0], e22 = load[1], e33 = load[2];
    const double e12 = load[3] * is2, e13 = load[4] * is2, e23 = load[5] * is2;
    const double tr = e11 + e22 + e33;
    double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int o1 = (o >> 2) & 1, o2 = (o >> 1) & 1, o3 = o & 1;
      int p = ph[eidx(nb, o1, o2, o3)];
      double la = mt[2 * p], m2 = 2.0 * mt[2 * p + 1];
      double s11 = la * tr + m2 * e11, s22 = la * tr + m2 * e22, s33 = la * tr + m2 * e33;
      double s12 = m2 * e12, s13 = m2 * e13, s23 = m2 * e23;
      double g1 = 2 * o1 - 1, g2 = 2 * o2 - 1, g3 = 2 * o3 - 1;
      acc[0] += s11 * g1 + s12 * g2 + s13 * g3;
      acc[1] += s12 * g1 + s22 * g2 + s23 * g3;
      acc[2] += s13 * g1 + s23 * g2 + s33 * g3;
    }
    f[0] = -q * acc[0];
    f[1] = -q * acc[1];
    f[2] = -q * acc[2];
  }
}

template <int CC>
__device__ __forceinline__ void node_diag(const uint8_t* __restrict__ ph, const double* mt, const Grid& g,
                                          int i1, int i2, int i3, double* dg) {
  Nbr nb;
  neighbours(g, i1, i2, i3, nb);
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    int p = ph[eidx(nb, (o >> 2) & 1, (o >> 1) & 1, o & 1)];
    if (CC == 1) {
      acc[0] += mt[2 * p] * Klap(o, o);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) acc[i] += mt[2 * p] * Klam(o, i, o, i) + mt[2 * p + 1] * Kmu(o, i, o, i);
    }
  }
  for (int i = 0; i < CC; ++i) dg[i] = acc[i] * g.h;
}

// Element-mean flux (thermal, kappa (g_bar + grad u)) or stress (elastic, Mandel) of the
// element at (i1, i2, i3); the element-mean gradient is sum_c u_c (2 c_k - 1) / (4 h).
template <int CC>
__device__ __forceinline__ void element_mean_flux(const double* __restrict__ u, const double* mt, int p,
                                                  const Grid& g, int i1, int i2, int i3,
                                                  const double* load, double* sig) {
  const int j1 = (i1 + 1 == g.n1) ? 0 : i1 + 1, j2 = (i2 + 1 == g.n2) ? 0 : i2 + 1,
            j3 = (i3 + 1 == g.n3) ? 0 : i3 + 1;
  const int a1[2] = {i1, j1}, a2[2] = {i2, j2}, a3[2] = {i3, j3};
  const long long n = g.n;
  const double s = 0.25 / g.h;
  double grad[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // grad[comp][dir]
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int c1 = (c >> 2) & 1, c2 = (c >> 1) & 1, c3 = c & 1;
    const long long node = ((long long)a1[c1] * g.n2 + a2[c2]) * g.n3 + a3[c3];
    const double sg[3] = {(double)(2 * c1 - 1), (double)(2 * c2 - 1), (double)(2 * c3 - 1)};
#pragma unroll
    for (int i = 0; i < CC; ++i) {
      double v = u[i * n + node];
#pragma unroll
      for (int k = 0; k < 3; ++k) grad[i][k] += v * sg[k];
    }
  }
  if (CC == 1) {
    double kap = mt[2 * p];
    for (int k = 0; k < 3; ++k) sig[k] = kap * (load[k] + s * grad[0][k]);
  } else {
    const double is2 = 0.70710678118654752440, sq2 = 1.41421356237309504880;
    double e11 = load[0] + s * grad[0][0], e22 = load[1] + s * grad[1][1], e33 = load[2] + s * grad[2][2];
    double e12 = load[3] * is2 + 0.5 * s * (grad[0][1] + grad[1][0]);
    double e13 = load[4] * is2 + 0.5 * s * (grad[0][2] + grad[2][0]);
    double e23 = load[5] * is2 + 0.5 * s * (grad[1][2] + grad[2][1]);
    double la = mt[2 * p], m2 = 2.0 * mt[2 * p + 1];
    double tr = e11 + e22 + e33;
    sig[0] = la * tr + m2 * e11;
    sig[1] = la * tr + m2 * e22;
    sig[2] = la * tr + m2 * e33;
    sig[3] = sq2 * m2 * e12;
    sig[4] = sq2 * m2 * e13;
    sig[5] = sq2 * m2 * e23;
  }
}

// Energy products at the 2x2x2 Gauss points of one element, all load pairs, added to acc
// ([nq][L][L]: thermal nq = 1 (e_l . e_m); elastic nq = 2 (tr e_l tr e_m, 2 e_l : e_m)).
template <int CC>
__device__ __forceinline__ void element_sensitivity(const double* __restrict__ ub, int L, const Grid& g,
                                                    int i1, int i2, int i3, const double* loads,
                                                    double* acc) {
  const int j1 = (i1 + 1 == g.n1) ? 0 : i1 + 1, j2 = (i2 + 1 == g.n2) ? 0 : i2 + 1,
            j3 = (i3 + 1 == g.n3) ? 0 : i3 + 1;
  const int a1[2] = {i1, j1}, a2[2] = {i2, j2}, a3[2] = {i3, j3};
  const long long n = g.n;
  long long nodes[8];
#pragma unroll
  for (int c = 0; c < 8; ++c)
    nodes[c] = ((long long)a1[(c >> 2) & 1] * g.n2 + a2[(c >> 1) & 1]) * g.n3 + a3[c & 1];
  const double gp[2] = {0.5 - 0.28867513459481288225, 0.5 + 0.28867513459481288225};
  const double ih = 1.0 / g.h;
  const int DIM = CC == 1 ? 3 : 6;
  const double is2 = 0.70710678118654752440;
  for (int q = 0; q < 8; ++q) {
    const double x[3] = {gp[(q >> 2) & 1], gp[(q >> 1) & 1], gp[q & 1]};
    double dN[8][3];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cb[3] = {(c >> 2) & 1, (c >> 1) & 1, c & 1};
      double f[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) f[j] = cb[j] ? x[j] : 1.0 - x[j];
      dN[c][0] = (2 * cb[0] - 1) * f[1] * f[2] * ih;
      dN[c][1] = (2 * cb[1] - 1) * f[0] * f[2] * ih;
      dN[c][2] = (2 * cb[2] - 1) * f[0] * f[1] * ih;
    }
    double e[8][6];
    for (int l = 0; l < L; ++l) {
      const double* u = ub + (long long)l * CC * n;
      const double* ld = loads + l * DIM;
      double gr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < CC; ++i) {
          double v = u[i * n + nodes[c]];
#pragma unroll
          for (int k = 0; k < 3; ++k) gr[i][k] += v * dN[c][k];
        }
      if (CC == 1) {
        for (int k = 0; k < 3; ++k) e[l][k] = ld[k] + gr[0][k];
      } else {
        // Mandel strain
        e[l][0] = ld[0] + gr[0][0];
        e[l][1] = ld[1] + gr[1][1];
        e[l][2] = ld[2] + gr[2][2];
        e[l][3] = ld[3] + is2 * (gr[0][1] + gr[1][0]);
        e[l][4] = ld[4] + is2 * (gr[0][2] + gr[2][0]);
        e[l][5] = ld[5] + is2 * (gr[1][2] + gr[2][1]);
      }
    }
    for (int l = 0; l < L; ++l)
      for (int m = 0; m < L; ++m) {
        if (CC == 1) {
          double s = e[l][0] * e[m][0] + e[l][1] * e[m][1] + e[l][2] * e[m][2];
          atomicAdd(acc + l * L + m, 0.125 * s);
        } else {
          double tl = e[l][0] + e[l][1] + e[l][2], tm = e[m][0] + e[m][1] + e[m][2];
          double dd = 0.0;
          for (int k = 0; k < 6; ++k) dd += e[l][k] * e[m][k];
          atomicAdd(acc + l * L + m, 0.125 * tl * tm);
          atomicAdd(acc + L * L + l * L + m, 0.125 * 2.0 * dd);
        }
      }
  }
}

}  // namespace unocg
