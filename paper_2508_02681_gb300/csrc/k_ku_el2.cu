// Elastic K d (Sec. 4.1, "matrix-free implementations" of Sec. 5.5) in FP32, element by element
// in the Walsh basis of ku_elastic.cuh, with two neighbouring elements of a row computed together
// in packed FP32x2 arithmetic (one instruction for both elements of every add, multiply and fma).
//
// Work layout: a block computes the same 32 (i3) x 8 (i2) node tile as k_ku_el, over 16 or 32
// node planes.  Its first 17 x 9 threads each own one element pair (e, e + 1), e even, of one element
// row (the tile's elements plus the lower halo row and the pair holding the lower halo column)
// and march along i1: per element layer a thread loads its two node rows of the new node plane
// (one 8-byte load of nodes e, e + 1 and one 4-byte load of node e + 2 per row and component),
// forms the 2D Walsh sums of both elements, combines them with those of the previous plane, and
// gets the 8 corner forces of both elements.  Within the pair the forces on node e + 1 are summed
// at once; the thread publishes, per component and lower/upper node row, (force on node e, force
// on node e + 1) and the force on node e + 2 in a double-buffered shared array (one barrier per
// layer), keeping the upper-plane corners for the next layer.  The first 16 x 8 threads then own
// two nodes each and add the four contributions of the neighbouring pairs and rows, taking d for
// the dot product d . p from the element threads' loads.  Measured at 256^3 x 6 loads: 1433 us
// per launch against 2336 us for the scalar element kernel.
#include <cstdlib>
#include "kargs.h"
#include "stencil.cuh"
#include "ku_elastic.cuh"

namespace unocg {

namespace {
constexpr int K2_PAIRS = KE_T3 / 2 + 1;          // 17 element pairs a row
constexpr int K2_ROWS = KE_T2 + 1;               // 9 element rows
constexpr int K2_SLOTS = K2_PAIRS * K2_ROWS;     // 153
constexpr int K2_THREADS = 160;
// one layer: [a2][component][slot] float2 (forces on nodes e, e + 1) and float (node e + 2); then
// the carried upper-plane corners [4 corners][component][slot] float2
constexpr int K2_LAYER_F2 = 2 * 3 * K2_SLOTS;
constexpr size_t kKuEl2Smem = 2 * (size_t)K2_LAYER_F2 * (sizeof(float2) + sizeof(float)) + 12 * K2_SLOTS * sizeof(float2) +
                               3 * 3 * K2_SLOTS * sizeof(float2);

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_set(float v) { return make_float2(v, v); }

// 2D Walsh sums of one node plane for both elements of the pair (see ke_walsh2): lo = node row
// a2 = 0, hi = a2 = 1; lo.x/lo.y = nodes (e, e + 1), lo2 = node e + 2
struct W2p {
  float2 e, k3, k2, k23;
};
__device__ __forceinline__ W2p walsh_pair(float2 lo, float lo2, float2 hi, float hi2) {
  const float2 u01 = make_float2(lo.y, lo2), u11 = make_float2(hi.y, hi2);
  const float2 s0 = p_add(lo, u01), d0 = p_sub(u01, lo), s1 = p_add(hi, u11), d1 = p_sub(u11, hi);
  return {p_add(s0, s1), p_add(d0, d1), p_sub(s1, s0), p_sub(d1, d0)};
}

// element constants of the two phases (ke_consts, with a1 = A1 / 2 added): k[7]
__device__ __forceinline__ void consts_pair(const float* mt, unsigned pe, unsigned pe1, float h, float2 (&k)[7]) {
  const float2 lm0 = *reinterpret_cast<const float2*>(mt + 2 * pe);
  const float2 lm1 = *reinterpret_cast<const float2*>(mt + 2 * pe1);
  const float2 lam = make_float2(lm0.x, lm1.x), mu = make_float2(lm0.y, lm1.y);
  const float2 l48 = p_mul(lam, p_set(h * (1.f / 48.f)));
  k[0] = p_mul(mu, p_set(h * 0.125f));
  k[1] = p_mul(lam, p_set(h * 0.0625f));
  k[2] = p_mul(mu, p_set(h * (1.f / 48.f)));
  k[3] = l48;
  k[4] = p_fma(mu, p_set(h * (3.f / 48.f)), l48);
  k[5] = p_fma(mu, p_set(h * (4.f / 144.f)), p_mul(lam, p_set(h * (1.f / 144.f))));
  k[6] = p_mul(mu, p_set(h * 0.0625f));
}

// corner forces of the two elements (ke_element for c = 3): flo[a2 * 2 + a3][i] at a1 = 0, fhi at
// a1 = 1
__device__ __forceinline__ void element_pair(const W2p (&L)[3], const W2p (&H)[3], const float2 (&k)[7],
                                             float2 (&flo)[4][3], float2 (&fhi)[4][3]) {
  const float2 A1 = k[0], b1 = k[1], a2 = k[2], b2 = k[3], A2 = k[4], g3 = k[5], a1 = k[6];
  float2 c1[3], c2[3], c3[3], c12[3], c13[3], c23[3], c123[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c1[i] = p_sub(H[i].e, L[i].e);
    c2[i] = p_add(L[i].k2, H[i].k2);
    c3[i] = p_add(L[i].k3, H[i].k3);
    c12[i] = p_sub(H[i].k2, L[i].k2);
    c13[i] = p_sub(H[i].k3, L[i].k3);
    c23[i] = p_add(L[i].k23, H[i].k23);
    c123[i] = p_sub(H[i].k23, L[i].k23);
  }
  float2 G1[3], G2[3], G3[3], G12[3], G13[3], G23[3], G123[3];
  const float2 t0 = p_mul(b1, p_add(p_add(c1[0], c2[1]), c3[2]));
  G1[0] = p_fma(A1, c1[0], t0);
  G2[1] = p_fma(A1, c2[1], t0);
  G3[2] = p_fma(A1, c3[2], t0);
  const float2 s01 = p_mul(a1, p_add(c2[0], c1[1])), s02 = p_mul(a1, p_add(c3[0], c1[2])),
               s12 = p_mul(a1, p_add(c3[1], c2[2]));
  G2[0] = s01; G1[1] = s01;
  G3[0] = s02; G1[2] = s02;
  G3[1] = s12; G2[2] = s12;
  const float2 two = p_set(2.f);
  G12[0] = p_fma(A2, c12[0], p_mul(b2, c23[2]));
  G12[1] = p_fma(A2, c12[1], p_mul(b2, c13[2]));
  G12[2] = p_mul(a2, p_add(p_fma(two, c12[2], c23[0]), c13[1]));
  G13[0] = p_fma(A2, c13[0], p_mul(b2, c23[1]));
  G13[2] = p_fma(A2, c13[2], p_mul(b2, c12[1]));
  G13[1] = p_mul(a2, p_add(p_fma(two, c13[1], c23[0]), c12[2]));
  G23[1] = p_fma(A2, c23[1], p_mul(b2, c13[0]));
  G23[2] = p_fma(A2, c23[2], p_mul(b2, c12[0]));
  G23[0] = p_mul(a2, p_add(p_fma(two, c23[0], c13[1]), c12[2]));
#pragma unroll
  for (int i = 0; i < 3; ++i) G123[i] = p_mul(g3, c123[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 ey0 = p_sub(G3[i], G23[i]), ey1 = p_add(G3[i], G23[i]);
    // E(a2, a3) = ex(a2) -/+ ey(a2) with ex0 = -G2, ex1 = G2
    const float2 E00 = p_sub(p_set(0.f), p_add(G2[i], ey0)), E01 = p_sub(ey0, G2[i]);
    const float2 E10 = p_sub(G2[i], ey1), E11 = p_add(G2[i], ey1);
    const float2 fx0 = p_sub(G1[i], G12[i]), fy0 = p_sub(G13[i], G123[i]);
    const float2 fx1 = p_add(G1[i], G12[i]), fy1 = p_add(G13[i], G123[i]);
    const float2 F00 = p_sub(fx0, fy0), F01 = p_add(fx0, fy0), F10 = p_sub(fx1, fy1), F11 = p_add(fx1, fy1);
    flo[0][i] = p_sub(E00, F00); fhi[0][i] = p_add(E00, F00);
    flo[1][i] = p_sub(E01, F01); fhi[1][i] = p_add(E01, F01);
    flo[2][i] = p_sub(E10, F10); fhi[2][i] = p_add(E10, F10);
    flo[3][i] = p_sub(E11, F11); fhi[3][i] = p_add(E11, F11);
  }
}
}  // namespace

__global__ void __launch_bounds__(K2_THREADS, 4) k_ku_el2(StencilArgs<float> a, int cz) {
  extern __shared__ __align__(16) unsigned char k2_raw[];
  __shared__ __align__(16) float mt[2 * 256];
  __shared__ double red_sh[32];
  const Grid& g = a.g;
  const int bl = blockIdx.y;
  load_material<float>(mt, a.mat, bl / a.L);
  __syncthreads();
  pdl_wait();
  const long long n = g.n;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const uint8_t* __restrict__ ph = a.phase + (long long)(bl / a.L) * n;
  const float* __restrict__ d = a.d + (long long)bl * 3 * n;
  float* __restrict__ p = a.p + (long long)bl * 3 * n;
  const int nt3 = (n3 + KE_T3 - 1) / KE_T3, nt2 = (n2 + KE_T2 - 1) / KE_T2;
  int bx = blockIdx.x;
  const int b3 = bx % nt3;
  bx /= nt3;
  const int b2 = bx % nt2;
  const int b1 = bx / nt2;
  const int t3 = b3 * KE_T3, t2 = b2 * KE_T2, z0 = b1 * cz;
  const int zend = min(z0 + cz, n1);
  const long long S = (long long)n2 * n3;
  const int tid = threadIdx.x;
  float2* lf_buf = reinterpret_cast<float2*>(k2_raw);                 // [2 layers][K2_LAYER_F2]
  float* r_buf = reinterpret_cast<float*>(lf_buf + 2 * K2_LAYER_F2);  // [2 layers][K2_LAYER_F2]
  // the upper-plane corner forces of the pair wait for the next layer here, [corner][comp][slot]
  // (in shared memory rather than registers: four blocks per SM instead of three)
  float2* carry = reinterpret_cast<float2*>(r_buf + 2 * K2_LAYER_F2);
  // d at the pair's nodes (e, e + 1) of its lower node row, [plane mod 3][component][slot]: the
  // node-pair threads of the next layer take d for the dot product d . p from here.  Plane q is
  // written in the element phase of layer q - 1 and read in the node phase of layer q; three
  // buffers, because the element phase of layer q + 1 (writing plane q + 2) may already run
  // while other threads are in the node phase of layer q.
  float2* dsave = carry + 12 * K2_SLOTS;
  // element pair of this thread: elements e, e + 1 (e even) of element row e2
  const bool is_el = tid < K2_SLOTS;
  const int s2 = tid / K2_PAIRS, kp = tid - s2 * K2_PAIRS;
  int rlo = 0, rhi = 0, ce = 0, ce2 = 0;
  if (is_el) {
    const int e2 = ke_wrap(t2 - 1 + s2, n2), e = ke_wrap(t3 - 2 + 2 * kp, n3);
    rlo = e2 * n3;
    rhi = (e2 + 1 == n2 ? 0 : e2 + 1) * n3;
    ce = e;
    ce2 = e + 2 == n3 ? 0 : e + 2;
  }
  // node pair of this thread
  const int r2 = tid >> 4, kk = tid & 15;
  const bool is_node = tid < 128 && t2 + r2 < n2 && t3 + 2 * kk < n3;
  const int noff = (t2 + r2) * n3 + t3 + 2 * kk;
  const float h = g.hf;
  DotAcc<float> dp;
  W2p L[3], H[3];
  auto load_plane = [&](int z, W2p(&W)[3], float2* save) {
    const float* dz = d + (long long)z * S;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float* di = dz + (long long)i * n;
      const float2 lo = __ldg(reinterpret_cast<const float2*>(di + rlo + ce));
      if (save) save[i * K2_SLOTS + tid] = lo;
      const float2 hi = __ldg(reinterpret_cast<const float2*>(di + rhi + ce));
      W[i] = walsh_pair(lo, __ldg(di + rlo + ce2), hi, __ldg(di + rhi + ce2));
    }
  };
  auto consts_at = [&](int z, float2(&k)[7]) {
    const unsigned w = __ldg(reinterpret_cast<const unsigned short*>(ph + (long long)z * S + rlo + ce));
    consts_pair(mt, w & 255u, w >> 8, h, k);
  };
  const bool skip = !a.standalone && a.sc[bl].done;  // uniform over the block
  if (!skip) {
    if (is_el) {
      // the element layer below the first node plane only contributes its upper corners
      const int zm = z0 ? z0 - 1 : n1 - 1;
      load_plane(zm, L, nullptr);
      load_plane(z0, H, dsave);
      float2 k[7], flo[4][3], fhi[4][3];
      consts_at(zm, k);
      element_pair(L, H, k, flo, fhi);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int i = 0; i < 3; ++i) carry[(c * 3 + i) * K2_SLOTS + tid] = fhi[c][i];
    }
    for (int z = z0; z < zend; ++z) {
      float2* lf = lf_buf + ((z - z0) & 1) * K2_LAYER_F2;
      float* rr = r_buf + ((z - z0) & 1) * K2_LAYER_F2;
      if (is_el) {
#pragma unroll
        for (int i = 0; i < 3; ++i) L[i] = H[i];
        load_plane(z + 1 == n1 ? 0 : z + 1, H, dsave + ((z + 1 - z0) % 3) * 3 * K2_SLOTS);
        float2 k[7], flo[4][3], fhi[4][3];
        consts_at(z, k);
        element_pair(L, H, k, flo, fhi);
#pragma unroll
        for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            float2* c0 = carry + (2 * a2 * 3 + i) * K2_SLOTS + tid;        // corner a3 = 0: nodes e, e + 1
            float2* c1 = carry + ((2 * a2 + 1) * 3 + i) * K2_SLOTS + tid;  // corner a3 = 1: nodes e + 1, e + 2
            const float2 f0 = p_add(flo[2 * a2][i], *c0);
            const float2 f1 = p_add(flo[2 * a2 + 1][i], *c1);
            *c0 = fhi[2 * a2][i];
            *c1 = fhi[2 * a2 + 1][i];
            const int o = (a2 * 3 + i) * K2_SLOTS + tid;
            lf[o] = make_float2(f0.x, f0.y + f1.x);
            rr[o] = f1.y;
          }
      }
      __syncthreads();
      if (is_node) {
        // nodes (n, n + 1), n = t3 + 2 kk, of node row t2 + r2: element row r2 + 1 (slot row) gives
        // its lower corners (a2 = 0), element row r2 its upper corners (a2 = 1); pair kk + 1 starts
        // at element n, pair kk ends with element n - 1
        const int sA = (r2 + 1) * K2_PAIRS + kk + 1, sB = r2 * K2_PAIRS + kk + 1;
        const long long q = (long long)z * S + noff;
        float sp = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 u0 = lf[i * K2_SLOTS + sA], u1 = lf[(3 + i) * K2_SLOTS + sB];
          const float w0 = rr[i * K2_SLOTS + sA - 1], w1 = rr[(3 + i) * K2_SLOTS + sB - 1];
          const float2 v = make_float2((u0.x + w0) + (u1.x + w1), u0.y + u1.y);
          *reinterpret_cast<float2*>(p + (long long)i * n + q) = v;
          const float2 dv = dsave[((z - z0) % 3) * 3 * K2_SLOTS + i * K2_SLOTS + sA];  // nodes (n, n + 1)
          sp = fmaf(v.x, dv.x, sp);
          sp = fmaf(v.y, dv.y, sp);
        }
        dp.add(sp);  // the six products of a node pair summed in FP32, then in the float pair
      }
      // the next layer writes the other buffer: one barrier per layer suffices
    }
  }
  pdl_trigger();
  if (a.standalone) return;
  const double bs = block_sum_acc(dp, red_sh);
  if (threadIdx.x == 0) a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bs;
  if (last_block(a.red.ticket)) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int qq = warp; qq < a.BL; qq += blockDim.x / 32) {
      const double sum = warp_sum_partials(a.red.part + (long long)qq * gridDim.x, gridDim.x, 1);
      if (lane == 0 && !a.sc[qq].done) step_update(a.sc[qq], sum);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

bool ku_el2_supported(const Grid& g) { return g.n3 % 2 == 0; }

cudaError_t launch_ku_el2(const StencilArgs<float>& a, cudaStream_t s) {
  if (a.c != 3 || !ku_el2_supported(a.g)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ku_el2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKuEl2Smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // node planes per block: 16 below 10^6 nodes per field, 32 from there (one pre-loop element
  // layer per block; 256^3 x 6 loads: 1616 / 1505 / 1433 us per launch for 8 / 16 / 32 planes,
  // 64^3 elastic solve 4.20 ms with 16 against 4.53 ms with 32); UNOCG_KE2_CZ overrides
  const Grid& g = a.g;
  const char* e = std::getenv("UNOCG_KE2_CZ");
  const int cz = (e && std::atoi(e) > 0) ? std::atoi(e) : (g.n >= 1000000 ? 32 : 16);
  const int tiles = ((g.n3 + KE_T3 - 1) / KE_T3) * ((g.n2 + KE_T2 - 1) / KE_T2) * ((g.n1 + cz - 1) / cz);
  if (tiles > ke_tiles(g)) return cudaErrorInvalidValue;  // partial sums are sized for KE_CZ planes
  return launch_pdl(k_ku_el2, dim3(tiles, a.BL), dim3(K2_THREADS), kKuEl2Smem, s, a, cz);
}

}  // namespace unocg
