// Axis-1 pass of the UNO preconditioner in the mixed-precision CG loop for elasticity (c = 3;
// Algorithm 2: FFT of each displacement component along axis 1, the block multiply
// s_hat(k) = Q(k) r_hat(k) / n with the symmetric 3 x 3 block Q(k) of every frequency, the
// Parseval partials of r . s and, for the flexible variant, r . s_old, inverse FFT along axis 1)
// on tiles staged by the TMA: k_line_tma3 for axes of N1 <= 64 points (all operands staged),
// k_line_tma3w for 96..256 points (only the r_hat tiles staged; see its section below).
//
// A block owns K3_P = 16 consecutive (k2, k3) positions of one (instance, load) over all N1
// values of axis 1 and all three components.  One thread issues the tile copies: r_hat and
// s_old of each component (16 complex FP32 = 128-byte rows, 128-byte swizzle) and the BF16 block
// entries (16 positions x 6 per row); an mbarrier with a transaction count signals their arrival.
// A line (one position, one component) is transformed by G threads of one warp in registers
// (fft_reg.cuh).  The components are transformed one after the other, each spectrum written back
// into its own tile in the scattered order of the register FFT; every thread then multiplies the
// three components of its own frequencies, and the inverse transforms follow component by
// component.  So a thread holds one component's V values at a time, where the register pass
// (k_line_reg) holds all three.  The first s_old tile, once its products with r_hat are summed,
// holds the exchange slots (each line its own N1, bit 3 of the slot index flipped for every
// other line); bulk tensor stores write the three results to s_hat.
#include "kargs.h"
#include "fft_reg.cuh"
#include "tma.cuh"
#include "driver_api.h"

namespace unocg {

namespace {
constexpr int K3_P = 16;  // positions per block (one 128-byte row of complex FP32)

struct alignas(64) Line3Maps {
  CUtensorMap hat;   // r_hat  [BL * 3][N1][2M] floats, box {32, N1, 1}, 128-byte swizzle
  CUtensorMap shat;  // s_hat  same layout
  CUtensorMap q;     // Q      [Bq][N1][6M] bf16, box {96, N1, 1}
};

struct Line3Args {
  LineArgs<float, __nv_bfloat16> a;
  int tiles;            // blocks per (instance, load)
  int* err;
  long long spin_limit;
};

// shared memory: alignment slack, three r_hat and three s_old tiles, the block entries
template <int N1> constexpr size_t k3_smem_bytes() { return 1024 + 6 * (size_t)N1 * 128 + (size_t)N1 * 192; }
template <int N1> constexpr int k3_min_blocks() {
  constexpr int by_threads = 768 / (K3_P * RegSplit<N1>::G);
  constexpr int by_smem = (int)(233472 / (k3_smem_bytes<N1>() + 1024));
  return by_threads < by_smem ? by_threads : by_smem;
}

__device__ __forceinline__ float2* tile_at(unsigned char* t, int row, int p) {
  return reinterpret_cast<float2*>(t + swz128_off8(row, p));
}
}  // namespace

template <int N1>
__global__ void __launch_bounds__(K3_P * RegSplit<N1>::G, k3_min_blocks<N1>())
    k_line_tma3(const __grid_constant__ Line3Maps maps, const Line3Args la) {
  using C = float2;
  constexpr int G = RegSplit<N1>::G, V = RegSplit<N1>::V, VG = V / G, W = 32 / G;
  constexpr int NTH = K3_P * G;
  constexpr int TB = N1 * 128;  // bytes of one tile
  extern __shared__ unsigned char k3_raw[];
  __shared__ double red_sh[32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_abort;
  const LineArgs<float, __nv_bfloat16>& a = la.a;
  // tiles 1024-byte aligned for the swizzle: r_hat of components 0..2 (becoming s_hat), s_old of
  // components 0..2 (the first one the exchange scratch once read), the block entries [N1][16][6]
  unsigned char* base = k3_raw + ((1024u - (sm_addr(k3_raw) & 1023u)) & 1023u);
  unsigned char* t_hat = base;
  unsigned char* t_old = base + 3 * TB;
  const __nv_bfloat16* t_q = reinterpret_cast<const __nv_bfloat16*>(base + 6 * TB);
  const C* __restrict__ tw1 = reinterpret_cast<const C*>(a.ft.tw1);
  const int tid = threadIdx.x;
  const int bl = blockIdx.y;
  const int tile = blockIdx.x;
  const int pos0 = tile * K3_P;
  const int M = a.g.n2 * a.g.n3h;
  const int b = bl / a.L;
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();  // r_hat, s_hat and the loop state come from the kernels before this one
  const bool active = !a.sc[bl].done;
  if (active && tid == 0) {
    mbar_expect_tx(&bar, (uint32_t)(3 * TB * (a.flexible ? 2 : 1) + N1 * 192));
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      tma_load_3d(t_hat + cc * TB, &maps.hat, 2 * pos0, 0, bl * 3 + cc, &bar);
      if (a.flexible) tma_load_3d(t_old + cc * TB, &maps.shat, 2 * pos0, 0, bl * 3 + cc, &bar);
    }
    tma_load_3d(const_cast<__nv_bfloat16*>(t_q), &maps.q, 6 * pos0, 0, a.q_inst_stride ? b : 0, &bar);
  }
  DotAcc<float> gam, rso;
  if (active) {
    if (!mbar_wait(&bar, 0u, la.spin_limit)) {
      s_abort = 1;
      if (la.err) atomicExch(la.err, 1);
    }
    __syncthreads();
    // after a timeout the copies may still be in flight: wait for them (bounded) before leaving
    if (s_abort && tid == 0) (void)mbar_wait(&bar, 0u, la.spin_limit);
    if (!s_abort) {
      const int p = tid / G, g = tid % G;  // position within the tile, thread of the line
      const int pos = pos0 + p;
      const bool on = pos < M;
      const int k3 = on ? pos % a.g.n3h : 0;
      const float wt = (k3 == 0 || 2 * k3 == a.g.n3) ? 1.f : 2.f;
      const float sc = (float)a.scale;
      // Parseval partial r . s_old: the thread's products summed in FP32, then in the pair
      if (a.flexible && on) {
        float part = 0.f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int n1 = 0; n1 < V; ++n1) {
            const C rv = *tile_at(t_hat + cc * TB, g + G * n1, p);
            const C so = *tile_at(t_old + cc * TB, g + G * n1, p);
            part = fmaf(rv.x, so.x, fmaf(rv.y, so.y, part));
          }
        rso.add(wt * part);
      }
      __syncthreads();  // the s_old tiles have been read: the first one is the exchange scratch
      // exchange slots: the line's own N1 slots, odd lines with slot index bit 3 flipped
      const int warp = tid >> 5, lane = tid & 31, w = lane / G;
      const XorSlot<C> scr{reinterpret_cast<C*>(t_old) + (size_t)(warp * W + w) * N1, (w & 1) << 3};
      C v[V];
      // forward transforms; the spectrum of each component goes back into its tile, row k1 of
      // the thread's column (the line's inputs have all been read at the first warp
      // synchronisation inside fft_dist_a)
#pragma unroll 1
      for (int cc = 0; cc < 3; ++cc) {
        unsigned char* t = t_hat + cc * TB;
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) v[n1] = *tile_at(t, g + G * n1, p);
        fft_dist_a_at<N1, -1>(v, g, scr, tw1);
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) *tile_at(t, scat_index<N1>(g, j, k2), p) = v[j * G + k2];
        __syncwarp();
      }
      // s_hat = Q r_hat / n at the thread's frequencies, all components; r . s
      if (on) {
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) {
            const int k1 = scat_index<N1>(g, j, k2);
            // entries (Q00, Q11, Q01, Q22, Q12, Q02) of the block, three bf16 pairs
            const __nv_bfloat162* qp = reinterpret_cast<const __nv_bfloat162*>(t_q + (k1 * K3_P + p) * 6);
            const float2 qa = __bfloat1622float2(qp[0]), qb = __bfloat1622float2(qp[1]),
                         qc = __bfloat1622float2(qp[2]);
            const float q00 = qa.x * sc, q11 = qa.y * sc, q01 = qb.x * sc, q22 = qb.y * sc, q12 = qc.x * sc,
                        q02 = qc.y * sc;
            C* r0 = tile_at(t_hat, k1, p);
            C* r1 = tile_at(t_hat + TB, k1, p);
            C* r2 = tile_at(t_hat + 2 * TB, k1, p);
            const C R0 = *r0, R1 = *r1, R2 = *r2;
            const C S0 = make_float2(q00 * R0.x + q01 * R1.x + q02 * R2.x, q00 * R0.y + q01 * R1.y + q02 * R2.y);
            const C S1 = make_float2(q01 * R0.x + q11 * R1.x + q12 * R2.x, q01 * R0.y + q11 * R1.y + q12 * R2.y);
            const C S2 = make_float2(q02 * R0.x + q12 * R1.x + q22 * R2.x, q02 * R0.y + q12 * R1.y + q22 * R2.y);
            part = fmaf(R0.x, S0.x, fmaf(R0.y, S0.y, part));
            part = fmaf(R1.x, S1.x, fmaf(R1.y, S1.y, part));
            part = fmaf(R2.x, S2.x, fmaf(R2.y, S2.y, part));
            *r0 = S0;
            *r1 = S1;
            *r2 = S2;
          }
        gam.add(wt * part);
      }
      __syncwarp();
      // inverse transforms back to the natural order, component by component
#pragma unroll 1
      for (int cc = 0; cc < 3; ++cc) {
        unsigned char* t = t_hat + cc * TB;
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) v[j * G + k2] = *tile_at(t, scat_index<N1>(g, j, k2), p);
        fft_dist_b_at<N1, +1>(v, g, scr, tw1);
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) *tile_at(t, g + G * n1, p) = v[n1];
        __syncwarp();
      }
      fence_async_shared();
    }
    __syncthreads();
    if (!s_abort && tid == 0) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) tma_store_3d(&maps.shat, 2 * pos0, 0, bl * 3 + cc, t_hat + cc * TB);
      tma_store_commit();
    }
  }
  pdl_trigger();
  double2 pr;
  pr.x = block_sum_acc(gam, red_sh);
  pr.y = block_sum_acc(rso, red_sh);
  if (tid == 0) {
    double* pp = a.red.part + ((long long)bl * gridDim.x + blockIdx.x) * 2;
    pp[0] = pr.x;
    pp[1] = pr.y;
  }
  if (last_block(a.red.ticket)) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int q = warp; q < a.BL; q += NTH / 32) {
      const double* pp = a.red.part + (long long)q * gridDim.x * 2;
      const double sg = warp_sum_partials(pp, gridDim.x, 2);
      const double sr = warp_sum_partials(pp + 1, gridDim.x, 2);
      if (lane == 0 && !a.sc[q].done) direction_update(a.sc[q], sg, sr, a.flexible);
    }
    __syncthreads();
    if (tid == 0) *a.red.ticket = 0u;
  }
  // the tiles must stay in shared memory until the bulk stores have read them, and the stores
  // are complete before the block exits
  if (active && tid == 0) tma_store_wait_all();
}

// ---------------------------------------------------------------- axes of 96..256 points
// For longer axis-1 lines the s_old tiles and the weights do not fit next to the three r_hat
// tiles, so only the r_hat tiles are staged (TMA, 128-byte swizzle): the previous s_hat is read
// by every thread for its own elements straight from global memory (component by component,
// before that component's transform), the block entries likewise at the multiply, and each line
// uses its own column of its tile as the exchange slots (its values are in registers before the
// first exchange and go back to the same column after the last).  Lanes of the 16-thread lines
// of 256 points interleave as in k_line_tma, so that a half-warp touches eight rows of two
// positions (distinct chunks of the swizzle); the 8-thread lines of 128 and 192 points and the
// 4-thread lines of 96 points hold that by construction.
namespace {
template <int N1> constexpr size_t k3w_smem_bytes() { return 1024 + 3 * (size_t)N1 * 128; }
template <int N1> constexpr int k3w_min_blocks() {
  constexpr int by_threads = 1024 / (K3_P * RegSplit<N1>::G);
  constexpr int by_smem = (int)(233472 / (k3w_smem_bytes<N1>() + 1024 + 512));
  return by_threads < by_smem ? by_threads : by_smem;
}
struct SwzSlot {
  unsigned char* t;
  int p;
  __device__ __forceinline__ float2& operator()(int s) const { return *tile_at(t, s, p); }
};
}  // namespace

template <int N1>
__global__ void __launch_bounds__(K3_P * RegSplit<N1>::G, k3w_min_blocks<N1>())
    k_line_tma3w(const __grid_constant__ Line3Maps maps, const Line3Args la) {
  using C = float2;
  constexpr int G = RegSplit<N1>::G, V = RegSplit<N1>::V, VG = V / G, W = 32 / G;
  constexpr int NTH = K3_P * G;
  constexpr int TB = N1 * 128;  // bytes of one tile
  extern __shared__ unsigned char k3_raw[];
  __shared__ double red_sh[32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_abort;
  const LineArgs<float, __nv_bfloat16>& a = la.a;
  unsigned char* t_hat = k3_raw + ((1024u - (sm_addr(k3_raw) & 1023u)) & 1023u);  // three tiles
  const C* __restrict__ tw1 = reinterpret_cast<const C*>(a.ft.tw1);
  const int tid = threadIdx.x;
  const int bl = blockIdx.y;
  const int pos0 = blockIdx.x * K3_P;
  const int M = a.g.n2 * a.g.n3h;
  const int b = bl / a.L;
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();  // r_hat, s_hat and the loop state come from the kernels before this one
  const bool active = !a.sc[bl].done;
  if (active && tid == 0) {
    mbar_expect_tx(&bar, (uint32_t)(3 * TB));
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) tma_load_3d(t_hat + cc * TB, &maps.hat, 2 * pos0, 0, bl * 3 + cc, &bar);
  }
  DotAcc<float> gam, rso;
  // lanes: see the header of this section
  const int warp = tid >> 5, lane = tid & 31;
  const int w = G == 16 ? (lane >> 3) & 1 : lane / G;
  const int g = G == 16 ? (lane & 7) + ((lane >> 4) << 3) : lane % G;
  const int p = warp * W + w;  // position within the tile
  const int pos = pos0 + p;
  const bool on = pos < M;
  // previous s_hat of this position, component cc, row r: [(bl * 3 + cc) * N1 + r] * M + pos; the
  // values of one component are requested one step ahead (component 0 while the tiles arrive)
  const C* so_base = reinterpret_cast<const C*>(a.shat) + (long long)bl * 3 * N1 * M + (on ? pos : 0);
  const bool use_so = active && a.flexible && on;
  C so[V];
  auto load_so = [&](int cc) {
    if (use_so) {
#pragma unroll
      for (int n1 = 0; n1 < V; ++n1) so[n1] = __ldg(so_base + ((long long)cc * N1 + g + G * n1) * M);
    }
  };
  load_so(0);
  if (active) {
    if (!mbar_wait(&bar, 0u, la.spin_limit)) {
      s_abort = 1;
      if (la.err) atomicExch(la.err, 1);
    }
    __syncthreads();
    if (s_abort && tid == 0) (void)mbar_wait(&bar, 0u, la.spin_limit);
    if (!s_abort) {
      const int k3 = on ? pos % a.g.n3h : 0;
      const float wt = (k3 == 0 || 2 * k3 == a.g.n3) ? 1.f : 2.f;
      const float sc = (float)a.scale;
      C v[V];
      // forward transforms, component by component; r . s_old on the way
#pragma unroll 1
      for (int cc = 0; cc < 3; ++cc) {
        unsigned char* t = t_hat + cc * TB;
        if (use_so) {
          float part = 0.f;
#pragma unroll
          for (int n1 = 0; n1 < V; ++n1) {
            const C rv = *tile_at(t, g + G * n1, p);
            part = fmaf(rv.x, so[n1].x, fmaf(rv.y, so[n1].y, part));
          }
          rso.add(wt * part);
        }
        if (cc < 2) load_so(cc + 1);
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) v[n1] = *tile_at(t, g + G * n1, p);
        fft_dist_a_at<N1, -1>(v, g, SwzSlot{t, p}, tw1);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) *tile_at(t, scat_index<N1>(g, j, k2), p) = v[j * G + k2];
        __syncwarp();
      }
      // s_hat = Q r_hat / n at the thread's frequencies, all components; r . s
      if (on) {
        const __nv_bfloat16* qrow = a.Q + (a.q_inst_stride ? (long long)b * a.q_inst_stride : 0) + 6LL * pos;
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) {
            const int k1 = scat_index<N1>(g, j, k2);
            // entries (Q00, Q11, Q01, Q22, Q12, Q02) of the block, three bf16 pairs
            const __nv_bfloat162* qp = reinterpret_cast<const __nv_bfloat162*>(qrow + (long long)k1 * 6 * M);
            const float2 qa = __bfloat1622float2(qp[0]), qb = __bfloat1622float2(qp[1]),
                         qc = __bfloat1622float2(qp[2]);
            const float q00 = qa.x * sc, q11 = qa.y * sc, q01 = qb.x * sc, q22 = qb.y * sc, q12 = qc.x * sc,
                        q02 = qc.y * sc;
            C* r0 = tile_at(t_hat, k1, p);
            C* r1 = tile_at(t_hat + TB, k1, p);
            C* r2 = tile_at(t_hat + 2 * TB, k1, p);
            const C R0 = *r0, R1 = *r1, R2 = *r2;
            const C S0 = make_float2(q00 * R0.x + q01 * R1.x + q02 * R2.x, q00 * R0.y + q01 * R1.y + q02 * R2.y);
            const C S1 = make_float2(q01 * R0.x + q11 * R1.x + q12 * R2.x, q01 * R0.y + q11 * R1.y + q12 * R2.y);
            const C S2 = make_float2(q02 * R0.x + q12 * R1.x + q22 * R2.x, q02 * R0.y + q12 * R1.y + q22 * R2.y);
            part = fmaf(R0.x, S0.x, fmaf(R0.y, S0.y, part));
            part = fmaf(R1.x, S1.x, fmaf(R1.y, S1.y, part));
            part = fmaf(R2.x, S2.x, fmaf(R2.y, S2.y, part));
            *r0 = S0;
            *r1 = S1;
            *r2 = S2;
          }
        gam.add(wt * part);
      }
      __syncwarp();
      // inverse transforms back to the natural order, component by component
#pragma unroll 1
      for (int cc = 0; cc < 3; ++cc) {
        unsigned char* t = t_hat + cc * TB;
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) v[j * G + k2] = *tile_at(t, scat_index<N1>(g, j, k2), p);
        fft_dist_b_at<N1, +1>(v, g, SwzSlot{t, p}, tw1);
        __syncwarp();
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) *tile_at(t, g + G * n1, p) = v[n1];
        __syncwarp();
      }
      fence_async_shared();
    }
    __syncthreads();
    if (!s_abort && tid == 0) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) tma_store_3d(&maps.shat, 2 * pos0, 0, bl * 3 + cc, t_hat + cc * TB);
      tma_store_commit();
    }
  }
  pdl_trigger();
  double2 pr;
  pr.x = block_sum_acc(gam, red_sh);
  pr.y = block_sum_acc(rso, red_sh);
  if (tid == 0) {
    double* pp = a.red.part + ((long long)bl * gridDim.x + blockIdx.x) * 2;
    pp[0] = pr.x;
    pp[1] = pr.y;
  }
  if (last_block(a.red.ticket)) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int q = warp; q < a.BL; q += NTH / 32) {
      const double* pp = a.red.part + (long long)q * gridDim.x * 2;
      const double sg = warp_sum_partials(pp, gridDim.x, 2);
      const double sr = warp_sum_partials(pp + 1, gridDim.x, 2);
      if (lane == 0 && !a.sc[q].done) direction_update(a.sc[q], sg, sr, a.flexible);
    }
    __syncthreads();
    if (tid == 0) *a.red.ticket = 0u;
  }
  if (active && tid == 0) tma_store_wait_all();
}

// ---------------------------------------------------------------- host side
bool line_tma3_supported(const Grid& g) {
  if (!(g.n1 == 16 || g.n1 == 32 || g.n1 == 64 || g.n1 == 96 || g.n1 == 128 || g.n1 == 192 || g.n1 == 256))
    return false;
  const long long M = (long long)g.n2 * g.n3h;
  if (M % 8 != 0) return false;  // 16-byte row strides of the Q and spectrum tensors
  return tensor_map_encoder() != nullptr;
}

namespace {
CUresult encode3(CUtensorMap* m, CUtensorMapDataType dt, size_t esz, const void* ptr, cuuint64_t d0, cuuint64_t d1,
                 cuuint64_t d2, cuuint32_t b0, cuuint32_t b1, CUtensorMapSwizzle sw) {
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * esz, d0 * d1 * esz};
  const cuuint32_t box[3] = {b0, b1, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return tensor_map_encoder()(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int N1>
cudaError_t line_tma3w_n(const Line3Maps& maps, const Line3Args& la, cudaStream_t st) {
  constexpr int NTH = K3_P * RegSplit<N1>::G;
  const size_t smem = k3w_smem_bytes<N1>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_tma3w<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_line_tma3w<N1>, dim3(la.tiles, la.a.BL), dim3(NTH), smem, st, maps, la);
}

template <int N1>
cudaError_t line_tma3_n(const Line3Maps& maps, const Line3Args& la, cudaStream_t st) {
  constexpr int NTH = K3_P * RegSplit<N1>::G;
  const size_t smem = k3_smem_bytes<N1>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_tma3<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_line_tma3<N1>, dim3(la.tiles, la.a.BL), dim3(NTH), smem, st, maps, la);
}
}  // namespace

cudaError_t launch_line_tma3(const LineArgs<float, __nv_bfloat16>& a, int* err, long long spin_limit, cudaStream_t st) {
  const Grid& g = a.g;
  if (a.c != 3 || !line_tma3_supported(g)) return cudaErrorInvalidValue;
  const cuuint64_t M = (cuuint64_t)g.n2 * g.n3h;
  const int Bq = a.q_inst_stride ? a.BL / a.L : 1;
  Line3Maps maps;
  if (encode3(&maps.hat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.hat, 2 * M, g.n1, (cuuint64_t)a.BL * 3, 2 * K3_P, g.n1,
              CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS ||
      encode3(&maps.shat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.shat, 2 * M, g.n1, (cuuint64_t)a.BL * 3, 2 * K3_P, g.n1,
              CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS ||
      encode3(&maps.q, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.Q, 6 * M, g.n1, Bq, 6 * K3_P, g.n1,
              CU_TENSOR_MAP_SWIZZLE_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  Line3Args la{};
  la.a = a;
  la.tiles = (int)((M + K3_P - 1) / K3_P);
  la.err = err;
  la.spin_limit = spin_limit;
  switch (g.n1) {
    case 16: return line_tma3_n<16>(maps, la, st);
    case 32: return line_tma3_n<32>(maps, la, st);
    case 64: return line_tma3_n<64>(maps, la, st);
    case 96: return line_tma3w_n<96>(maps, la, st);
    case 128: return line_tma3w_n<128>(maps, la, st);
    case 192: return line_tma3w_n<192>(maps, la, st);
    case 256: return line_tma3w_n<256>(maps, la, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace unocg
