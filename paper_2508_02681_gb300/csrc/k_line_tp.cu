// Axis-1 pass of the UNO preconditioner in the mixed-precision CG loop for c = 1 (Algorithm 2: FFT
// along axis 1, block multiply s_hat = Q r_hat / n with the Parseval partials of r . s and r .
// s_old, inverse FFT along axis 1), as a persistent pipeline of TMA tiles.
//
// The tile work is that of k_line_tma (16 consecutive (k2, k3) positions of one (instance, load)
// over all N1 values: r_hat and s_old tiles of 128-byte rows with the 128-byte swizzle, the BF16
// weights, line FFTs by G threads of a warp in registers, the result in place of r_hat and one
// bulk tensor store).  Here a block stays resident and walks the tiles blockIdx.x, blockIdx.x +
// gridDim.x, ... through a ring of NS shared-memory stages: one producer thread issues the copies
// of the next tiles while the consumer warps transform the current one, and stores a finished
// tile before reloading its stage.  Each stage has a "full" mbarrier (transaction count of the
// copies) and an "empty" mbarrier (one arrival per consumer warp once its results are in the
// stage).  So the memory traffic of one tile overlaps the arithmetic of another inside the
// block, where k_line_tma relies on other blocks of the SM for that.  All waits are bounded: a
// timeout sets the error flag and every role leaves its loop; issued copies are waited for
// (bounded) before the block exits.
#include <cstdlib>
#include "kargs.h"
#include "fft_reg.cuh"
#include "tma.cuh"
#include "driver_api.h"

namespace unocg {

namespace {
constexpr int TP_P = 16;  // positions per tile

struct LineTpMaps {
  CUtensorMap hat;   // r_hat  [BL][N1][2M] floats, box {32, N1, 1}, 128-byte swizzle
  CUtensorMap shat;  // s_hat  same layout
  CUtensorMap q;     // Q      [Bq][N1][M] bf16, box {16, N1, 1}
};

struct LineTpArgs {
  LineArgs<float, __nv_bfloat16> a;
  int tiles;            // tiles per (instance, load)
  long long units;      // tiles of all pairs
  int* err;
  long long spin_limit;
};

// one stage: r_hat tile, s_old tile (N1 rows of 128 bytes each), Q tile (N1 rows of 32 bytes),
// rounded to 1024 bytes (the swizzled tiles are 1024-byte aligned)
template <int N1> __host__ __device__ constexpr size_t tp_stage_bytes() { return ((size_t)N1 * 288 + 1023) / 1024 * 1024; }
template <int N1> __host__ __device__ constexpr int tp_stages() { return 3 * tp_stage_bytes<N1>() + 1024 <= 225 * 1024 ? 3 : 2; }
template <int N1> __host__ __device__ constexpr size_t tp_smem_bytes() { return 1024 + tp_stages<N1>() * tp_stage_bytes<N1>(); }
template <int N1> __host__ __device__ constexpr int tp_consumers() { return TP_P * RegSplit<N1>::G; }
template <int N1> __host__ __device__ constexpr int tp_blocks_per_sm() {
  constexpr int by_smem = (int)(233472 / (tp_smem_bytes<N1>() + 1024 + 512));
  constexpr int by_threads = 2048 / (tp_consumers<N1>() + 32);
  return by_smem < by_threads ? by_smem : by_threads;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(b)) : "memory");
}
__device__ __forceinline__ void consumer_sync(int nth) { asm volatile("bar.sync 1, %0;" ::"r"(nth) : "memory"); }

}  // namespace

template <int N1>
__global__ void __launch_bounds__(tp_consumers<N1>() + 32, tp_blocks_per_sm<N1>())
    k_line_tp(const __grid_constant__ LineTpMaps maps, const LineTpArgs la) {
  using C = float2;
  constexpr int G = RegSplit<N1>::G, V = RegSplit<N1>::V, VG = V / G, W = 32 / G;
  constexpr int NTH = tp_consumers<N1>();
  constexpr int NS = tp_stages<N1>();
  constexpr int TB = N1 * 128;  // bytes of one spectrum tile
  constexpr size_t SB = tp_stage_bytes<N1>();
  extern __shared__ unsigned char tp_raw[];
  __shared__ __align__(8) uint64_t full[NS], empty[NS];
  __shared__ long long s_unit[NS];
  __shared__ double red_sh[2][32];
  __shared__ volatile int c_abort;  // set by consumers only, read by them after a consumer barrier
  const LineArgs<float, __nv_bfloat16>& a = la.a;
  unsigned char* base = tp_raw + ((1024u - (sm_addr(tp_raw) & 1023u)) & 1023u);
  const C* __restrict__ tw1 = reinterpret_cast<const C*>(a.ft.tw1);
  const int tid = threadIdx.x;
  const int M = a.g.n2 * a.g.n3h;
  const long long units = la.units;
  const int tiles = la.tiles;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NTH / 32);
    }
    c_abort = 0;
    mbar_fence_init();
  }
  __syncthreads();
  pdl_wait();  // r_hat, s_hat and the loop state come from the kernels before this one
  // the tiles of this block, finished pairs skipped (their flags do not change during the launch)
  auto next_unit = [&](long long u) {
    while (u < units && a.sc[u / tiles].done) u += gridDim.x;
    return u;
  };
  const bool flexible = a.flexible != 0;
  const uint32_t tx_bytes = (uint32_t)(TB * (flexible ? 2 : 1) + N1 * 2 * TP_P);
  if (tid == NTH) {
    // ------------------------------------------------------------ producer (one thread)
    int k = 0;
    bool ok = true;
    for (long long u = next_unit(blockIdx.x); u < units; u = next_unit(u + gridDim.x), ++k) {
      const int s = k % NS;
      unsigned char* st = base + s * SB;
      if (k >= NS) {
        // the consumers are done with the tile k - NS of this stage: store it, let the store read
        // the stage, then reuse it
        if (c_abort || !mbar_wait(&empty[s], (uint32_t)((k / NS - 1) & 1), la.spin_limit)) {
          ok = false;
          break;
        }
        const long long uo = s_unit[s];
        tma_store_3d(&maps.shat, 2 * (int)(uo % tiles) * TP_P, 0, (int)(uo / tiles), st);
        tma_store_commit();
        tma_store_wait_read();
      }
      s_unit[s] = u;
      const int bl = (int)(u / tiles), pos0 = (int)(u % tiles) * TP_P;
      mbar_expect_tx(&full[s], tx_bytes);
      tma_load_3d(st, &maps.hat, 2 * pos0, 0, bl, &full[s]);
      if (flexible) tma_load_3d(st + TB, &maps.shat, 2 * pos0, 0, bl, &full[s]);
      tma_load_3d(st + 2 * TB, &maps.q, pos0, 0, a.q_inst_stride ? bl / a.L : 0, &full[s]);
    }
    // the last tiles of the ring
    for (int j = k - NS < 0 ? 0 : k - NS; j < k; ++j) {
      const int s = j % NS;
      if (!ok || c_abort || !mbar_wait(&empty[s], (uint32_t)((j / NS) & 1), la.spin_limit)) {
        ok = false;
        break;
      }
      const long long uo = s_unit[s];
      tma_store_3d(&maps.shat, 2 * (int)(uo % tiles) * TP_P, 0, (int)(uo / tiles), base + s * SB);
      tma_store_commit();
    }
    if (!ok) {
      if (la.err) atomicExch(la.err, 1);
      // copies still in flight land before the block leaves (bounded)
      for (int j = k - NS < 0 ? 0 : k - NS; j < k; ++j)
        (void)mbar_wait(&full[j % NS], (uint32_t)((j / NS) & 1), la.spin_limit);
    }
    tma_store_wait_all();
  } else if (tid < NTH) {
    // ------------------------------------------------------------ consumers
    // a warp takes two positions; for the 16-thread lines of 256 points the lanes interleave
    // (lanes 0-7 and 16-23 one line, 8-15 and 24-31 the other) so that each half-warp reads eight
    // consecutive rows of both positions: eight distinct 16-byte chunks of the swizzled tile
    const int warp = tid >> 5, lane = tid & 31;
    const int w = G == 16 ? (lane >> 3) & 1 : lane / G;
    const int g = G == 16 ? (lane & 7) + ((lane >> 4) << 3) : lane % G;
    const int p = warp * W + w;  // position within the tile
    const float sc = (float)a.scale;
    int k = 0;
    for (long long u = next_unit(blockIdx.x); u < units; u = next_unit(u + gridDim.x), ++k) {
      const int s = k % NS;
      unsigned char* t_hat = base + s * SB;
      unsigned char* t_old = t_hat + TB;
      const __nv_bfloat16* t_q = reinterpret_cast<const __nv_bfloat16*>(t_hat + 2 * TB);
      // a timeout of any consumer ends the loop of all of them at the same tile (the flag is
      // written before and read after a consumer barrier); a producer that gave up stops
      // loading, so the consumers time out here too
      if (!mbar_wait(&full[s], (uint32_t)((k / NS) & 1), la.spin_limit)) {
        c_abort = 1;
        if (la.err) atomicExch(la.err, 1);
      }
      consumer_sync(NTH);
      if (c_abort) break;
      const int bl = (int)(u / tiles), tile = (int)(u % tiles);
      const int pos = tile * TP_P + p;
      const bool on = pos < M;
      const int k3 = on ? pos % a.g.n3h : 0;
      const float wt = (k3 == 0 || 2 * k3 == a.g.n3) ? 1.f : 2.f;
      DotAcc<float> gam, rso;
      C v[V];
#pragma unroll
      for (int n1 = 0; n1 < V; ++n1) v[n1] = *reinterpret_cast<const C*>(t_hat + swz128_off8(g + G * n1, p));
      if (flexible && on) {
        float part = 0.f;
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) {
          const C so = *reinterpret_cast<const C*>(t_old + swz128_off8(g + G * n1, p));
          part = fmaf(v[n1].x, so.x, fmaf(v[n1].y, so.y, part));
        }
        rso.add(wt * part);
      }
      consumer_sync(NTH);  // the s_old tile is free: exchange scratch of the line transforms
      // exchange slots: the line's own N1 slots, odd lines of the warp with slot index bit 3
      // flipped (the two lines of a half-warp then use complementary banks)
      const XorSlot<C> scr{reinterpret_cast<C*>(t_old) + (size_t)(warp * W + w) * N1, (w & 1) << 3};
      fft_dist_a_at<N1, -1>(v, g, scr, tw1);
      if (on) {
        float part = 0.f;  // r . s = sum q |r_hat|^2 over the thread's modes
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) {
            const int k1 = scat_index<N1>(g, j, k2), e = j * G + k2;
            const float q = __bfloat162float(t_q[k1 * TP_P + p]) * sc;
            const C R = v[e];
            part = fmaf(q, fmaf(R.x, R.x, R.y * R.y), part);
            v[e] = make_float2(q * R.x, q * R.y);
          }
        gam.add(wt * part);
      }
      fft_dist_b_at<N1, +1>(v, g, scr, tw1);
#pragma unroll
      for (int n1 = 0; n1 < V; ++n1) *reinterpret_cast<C*>(t_hat + swz128_off8(g + G * n1, p)) = v[n1];
      fence_async_shared();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      // the tile's partial sums, in a fixed order (warps, then the two sums)
      for (int o = 16; o > 0; o >>= 1) {
        gam.add(__shfl_xor_sync(0xffffffffu, gam.hi, o));
        gam.lo = __fadd_rn(gam.lo, __shfl_xor_sync(0xffffffffu, gam.lo, o));
        rso.add(__shfl_xor_sync(0xffffffffu, rso.hi, o));
        rso.lo = __fadd_rn(rso.lo, __shfl_xor_sync(0xffffffffu, rso.lo, o));
      }
      double* rs = red_sh[k & 1];
      if (lane == 0) {
        rs[warp] = gam.value();
        rs[16 + warp] = rso.value();
      }
      consumer_sync(NTH);
      if (tid == 0) {
        double sg = 0.0, sr = 0.0;
        for (int i = 0; i < NTH / 32; ++i) {
          sg += rs[i];
          sr += rs[16 + i];
        }
        double* pp = a.red.part + ((long long)bl * tiles + tile) * 2;
        pp[0] = sg;
        pp[1] = sr;
      }
    }
  }
  pdl_trigger();
  if (last_block(a.red.ticket)) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int q = warp; q < a.BL; q += (NTH + 32) / 32) {
      const double* pp = a.red.part + (long long)q * tiles * 2;
      const double sg = warp_sum_partials(pp, tiles, 2);
      const double sr = warp_sum_partials(pp + 1, tiles, 2);
      if (lane == 0 && !a.sc[q].done) direction_update(a.sc[q], sg, sr, a.flexible);
    }
    __syncthreads();
    if (tid == 0) *a.red.ticket = 0u;
  }
}

// ---------------------------------------------------------------- host side
namespace {
CUresult tp_encode(CUtensorMap* m, CUtensorMapDataType dt, size_t esz, const void* ptr, cuuint64_t d0, cuuint64_t d1,
                   cuuint64_t d2, cuuint32_t b0, cuuint32_t b1, CUtensorMapSwizzle sw) {
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * esz, d0 * d1 * esz};
  const cuuint32_t box[3] = {b0, b1, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return tensor_map_encoder()(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int N1>
cudaError_t line_tp_n(const LineTpMaps& maps, LineTpArgs& la, int sm_count, cudaStream_t st) {
  constexpr int NT = tp_consumers<N1>() + 32;
  const size_t smem = tp_smem_bytes<N1>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_tp<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  long long slots = (long long)sm_count * tp_blocks_per_sm<N1>();
  // UNOCG_LINE_TP_BLOCKS caps the grid (read at each launch; tests walk many tiles per block)
  const char* e = std::getenv("UNOCG_LINE_TP_BLOCKS");
  if (e && std::atoi(e) > 0 && std::atoi(e) < slots) slots = std::atoi(e);
  const unsigned grid = (unsigned)(la.units < slots ? la.units : slots);
  return launch_pdl(k_line_tp<N1>, dim3(grid), dim3(NT), smem, st, maps, la);
}
}  // namespace

// the pipeline needs 128-byte rows of 16 positions and power-of-two axis-1 lines of 64..256
bool line_tp_supported(const Grid& g) {
  if (!(g.n1 == 64 || g.n1 == 128 || g.n1 == 256)) return false;
  const long long M = (long long)g.n2 * g.n3h;
  return M % 8 == 0 && tensor_map_encoder() != nullptr;
}

cudaError_t launch_line_tp(const LineArgs<float, __nv_bfloat16>& a, int* err, long long spin_limit, int sm_count,
                           cudaStream_t st) {
  const Grid& g = a.g;
  if (a.c != 1 || !line_tp_supported(g) || a.standalone) return cudaErrorInvalidValue;
  const cuuint64_t M = (cuuint64_t)g.n2 * g.n3h;
  const int Bq = a.q_inst_stride ? a.BL / a.L : 1;
  LineTpMaps maps;
  if (tp_encode(&maps.hat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.hat, 2 * M, g.n1, a.BL, 2 * TP_P, g.n1,
                CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS ||
      tp_encode(&maps.shat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.shat, 2 * M, g.n1, a.BL, 2 * TP_P, g.n1,
                CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS ||
      tp_encode(&maps.q, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.Q, M, g.n1, Bq, TP_P, g.n1,
                CU_TENSOR_MAP_SWIZZLE_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  LineTpArgs la{};
  la.a = a;
  la.tiles = (int)((M + TP_P - 1) / TP_P);
  la.units = (long long)la.tiles * a.BL;
  la.err = err;
  la.spin_limit = spin_limit;
  switch (g.n1) {
    case 64: return line_tp_n<64>(maps, la, sm_count, st);
    case 128: return line_tp_n<128>(maps, la, sm_count, st);
    case 256: return line_tp_n<256>(maps, la, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace unocg
