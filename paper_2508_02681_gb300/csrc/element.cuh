// Trilinear brick element integrals on the unit cube, as compile-time constants.
//
// For corners a, b in {0,1}^3 and derivative directions p, q the integral
//   G^{pq}_{ab} = int_{[0,1]^3} d_p N_a d_q N_b
// factorizes over the three axes into 1D integrals of the linear shape functions
// phi_0 = 1 - x, phi_1 = x:
//   int phi'_s phi'_t = (s == t ? 1 : -1),     int phi_s phi_t = (s == t ? 1/3 : 1/6),
//   int phi'_s phi_t = (s == 1 ? 1/2 : -1/2),  int phi_s phi'_t = (t == 1 ? 1/2 : -1/2).
// With them (voxel edge h; the element stiffness scales with h in 3D):
//   thermal      K_e[a,b]         = kappa h sum_j G^{jj}_{ab}
//   elastic      K_e[(a,i),(b,k)] = h ( lambda G^{ik}_{ab} + mu (delta_ik sum_j G^{jj}_{ab} + G^{ki}_{ab}) )
// which is the Galerkin form of div(3 lambda P1 + 2 mu I^s) eps(u) (Sec. 6.2), i.e.
// lambda div(u) div(v) + 2 mu eps(u):eps(v).
#pragma once

namespace unocg {

__host__ __device__ constexpr int cbit(int corner, int axis) { return (corner >> (2 - axis)) & 1; }

__host__ __device__ constexpr double g1d(int s, int t, bool ds, bool dt) {
  return (ds && dt) ? (s == t ? 1.0 : -1.0)
       : ds ? (s == 1 ? 0.5 : -0.5)
       : dt ? (t == 1 ? 0.5 : -0.5)
       : (s == t ? 1.0 / 3.0 : 1.0 / 6.0);
}

__host__ __device__ constexpr double Gpq(int p, int q, int a, int b) {
  return g1d(cbit(a, 0), cbit(b, 0), p == 0, q == 0) *
         g1d(cbit(a, 1), cbit(b, 1), p == 1, q == 1) *
         g1d(cbit(a, 2), cbit(b, 2), p == 2, q == 2);
}

__host__ __device__ constexpr double Klap(int a, int b) {
  return Gpq(0, 0, a, b) + Gpq(1, 1, a, b) + Gpq(2, 2, a, b);
}

// unit-cube lambda- and mu-parts of the elastic element matrix
__host__ __device__ constexpr double Klam(int a, int i, int b, int k) { return Gpq(i, k, a, b); }
__host__ __device__ constexpr double Kmu(int a, int i, int b, int k) {
  return (i == k ? Klap(a, b) : 0.0) + Gpq(k, i, a, b);
}

// The same entries as tables evaluated at compile time, in the arithmetic type of the kernel:
// the stencil loops index them with unrolled constants, so no coefficient is computed at run
// time (an evaluation of Klam / Kmu in device code would run in FP64).
template <typename T> struct ElasticTable {
  T lam[8][3][8][3];
  T mu[8][3][8][3];
};
template <typename T> constexpr ElasticTable<T> make_elastic_table() {
  ElasticTable<T> t{};
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 8; ++b)
        for (int k = 0; k < 3; ++k) {
          t.lam[a][i][b][k] = (T)Klam(a, i, b, k);
          t.mu[a][i][b][k] = (T)Kmu(a, i, b, k);
        }
  return t;
}
__constant__ constexpr ElasticTable<float> kElastic32 = make_elastic_table<float>();
// 72 Klam and 72 Kmu are integers (denominators of the 1D integrals: 3, 6, 2), exact in FP32
template <int S> constexpr ElasticTable<float> make_scaled_table() {
  ElasticTable<float> t{};
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 8; ++b)
        for (int k = 0; k < 3; ++k) {
          t.lam[a][i][b][k] = (float)(S * Klam(a, i, b, k));
          t.mu[a][i][b][k] = (float)(S * Kmu(a, i, b, k));
        }
  return t;
}
__constant__ constexpr ElasticTable<float> kElastic72 = make_scaled_table<72>();
__constant__ constexpr ElasticTable<double> kElastic64 = make_elastic_table<double>();
template <typename T> __device__ __forceinline__ const ElasticTable<T>& elastic_table();
template <> __device__ __forceinline__ const ElasticTable<float>& elastic_table<float>() { return kElastic32; }
template <> __device__ __forceinline__ const ElasticTable<double>& elastic_table<double>() { return kElastic64; }

}  // namespace unocg
