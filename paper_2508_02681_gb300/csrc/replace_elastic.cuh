// Residual replacement of the mixed-precision path for elasticity, element by element:
// rref <- rref - K (u32 + alpha d) with the element forces of ku_elastic.cuh (Walsh basis of the
// trilinear brick, Sec. 4.1) evaluated in float-pair arithmetic (about 44 significant bits on
// the FP32 pipes), and r <- (float) rref.  Same tiling and element-column march as
// ku_element_tile; each element costs about 190 float-pair operations instead of the 1,152
// float-pair multiply-adds per node of the node-centred stencil.
#pragma once
#include "df64.cuh"
#include "ku_elastic.cuh"

namespace unocg {

// float pair with the arithmetic operators ke_walsh2 / ke_element use
struct dfv {
  df32 v;
  __device__ __forceinline__ dfv() {}
  __device__ __forceinline__ dfv(float x) : v{x, 0.0f} {}
  __device__ __forceinline__ dfv(df32 x) : v(x) {}
};
__device__ __forceinline__ dfv operator+(dfv a, dfv b) { return df_add(a.v, b.v); }
__device__ __forceinline__ dfv operator-(dfv a, dfv b) { return df_add(a.v, df_neg(b.v)); }
__device__ __forceinline__ dfv operator-(dfv a) { return df_neg(a.v); }
__device__ __forceinline__ dfv operator*(dfv a, dfv b) { return df_mul(a.v, b.v); }

constexpr size_t kReplaceElSmem = 2 * 4 * 3 * KE_SLOTS * sizeof(float2);  // double buffer, c = 3

// Six element constants of every phase as pairs (see ke_element), for instance b.
__device__ __forceinline__ void replace_elastic_consts(const Material& mat, int b, double h, float2* kc) {
  const int np = mat.n_phases;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double lam = mat.m64[(long long)b * 2 * np + 2 * p], mu = mat.m64[(long long)b * 2 * np + 2 * p + 1];
    const double k[6] = {h * mu / 8.0, h * lam / 16.0, h * mu / 48.0, h * lam / 48.0, h * (3.0 * mu + lam) / 48.0,
                         h * (4.0 * mu + lam) / 144.0};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const df32 v = df_from_double(k[j]);
      kc[6 * p + j] = make_float2(v.hi, v.lo);
    }
  }
}

// One node tile of one (instance, load) on the periodic node grid g: rref -= K w with
// w = u32 + alpha d (dd null: w = u32), r = (float) rref, at the nodes where is_free(i1, i2, i3)
// holds (the others are left as they are).  ph, u32, dd, rref, r point at this pair's fields;
// block of KE_THREADS threads; `kc` from replace_elastic_consts, `sm` kReplaceElSmem bytes.
// Returns the max |rref| over the tile's free nodes (thread 0).
template <class FreeFn>
__device__ double replace_elastic_tile(const Grid& g, const uint8_t* ph, const float* u32, const float* dd, df32 al,
                                       double* rref, float* r, const float2* kc, int tile, double* red_sh,
                                       float2* sm, FreeFn is_free) {
  const long long n = g.n;
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
  const int r2 = tid >> 5, r3 = tid & 31;
  const bool is_node = tid < KE_T3 * KE_T2 && t2 + r2 < g.n2 && t3 + r3 < g.n3;
  const int noff = (t2 + r2) * g.n3 + t3 + r3;
  double lmax = 0.0;
  KeW2<dfv> L[3], H[3];
  dfv carry[4][3];
  auto w_at = [&](int i, long long q) {
    return dd ? dfv(df_axpy(al, __ldg(dd + i * n + q), __ldg(u32 + i * n + q))) : dfv(__ldg(u32 + i * n + q));
  };
  auto load_plane = [&](int z, KeW2<dfv>(&W)[3]) {
    const long long zq = (long long)z * S;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      W[i] = ke_walsh2<dfv>(w_at(i, zq + o00), w_at(i, zq + o01), w_at(i, zq + o10), w_at(i, zq + o11));
  };
  auto consts = [&](long long e, dfv(&k)[6]) {
    const float2* c = kc + 6 * ph[e];
#pragma unroll
    for (int j = 0; j < 6; ++j) k[j] = dfv(df32{c[j].x, c[j].y});
  };
  if (is_el) {
    const int zm = z0 ? z0 - 1 : g.n1 - 1;
    load_plane(zm, L);
    load_plane(z0, H);
    dfv k[6], flo[4][3];
    consts((long long)zm * S + o00, k);
    ke_element<dfv>(L, H, k, flo, carry);
  }
  for (int z = z0; z < zend; ++z) {
    float2* buf = sm + ((z - z0) & 1) * (12 * KE_SLOTS);
    if (is_el) {
#pragma unroll
      for (int i = 0; i < 3; ++i) L[i] = H[i];
      load_plane(z + 1 == g.n1 ? 0 : z + 1, H);
      dfv k[6], flo[4][3], fhi[4][3];
      consts((long long)z * S + o00, k);
      ke_element<dfv>(L, H, k, flo, fhi);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const dfv v = flo[c][i] + carry[c][i];
          buf[(i * 4 + c) * KE_SLOTS + tid] = make_float2(v.v.hi, v.v.lo);
          carry[c][i] = fhi[c][i];
        }
    }
    __syncthreads();
    if (is_node && is_free(z, t2 + r2, t3 + r3)) {
      const int sA = (r2 + 1) * KE_S3 + r3 + 1, sB = r2 * KE_S3 + r3;
      const long long q = (long long)z * S + noff;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float2* bi = buf + i * 4 * KE_SLOTS;
        auto at = [&](int j) { return dfv(df32{bi[j].x, bi[j].y}); };
        const dfv v = (at(sA) + at(KE_SLOTS + sA - 1)) + (at(2 * KE_SLOTS + sB + 1) + at(3 * KE_SLOTS + sB));
        const long long x = i * n + q;
        const double rr = rref[x] - df_to_double(v.v);
        rref[x] = rr;
        if (r) r[x] = (float)rr;
        lmax = fmax(lmax, fabs(rr));
      }
    }
  }
  return block_max(lmax, red_sh);
}

}  // namespace unocg
