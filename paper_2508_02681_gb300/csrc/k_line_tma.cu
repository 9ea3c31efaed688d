// Axis-1 pass of the UNO preconditioner in the mixed-precision CG loop (Algorithm 2: FFT along
// axis 1, block multiply s_hat = Q r_hat / n with the Parseval partials of r . s and, for the
// flexible variant, r . s_old, inverse FFT along axis 1) for c = 1 on tiles staged by the TMA.
//
// A block owns KL_P = 16 consecutive (k2, k3) positions of one (instance, load) over all N1
// values of axis 1.  One thread issues three tile copies: the axis-2/3 spectrum r_hat and the
// previous s_hat (16 complex FP32 = 128 bytes per row, N1 rows, 128-byte swizzle so that the
// column reads of the line transforms spread over the shared-memory banks) and the BF16 weights
// Q (16 positions x N1 rows); an mbarrier with a transaction count signals their arrival.  A
// line (one position) is transformed by G threads of one warp in registers (fft_reg.cuh: V
// values each, one exchange through shared memory; the s_old tile, once its products with
// r_hat are summed, holds the exchange slots, each line its own N1 with the slot index bit 3
// flipped for every other line).  The 16 threads of the two 256-point lines of a warp interleave
// their lanes so that a half-warp reads eight consecutive rows of two positions (eight distinct
// 16-byte chunks of the swizzle, no bank conflicts).  The result overwrites the r_hat tile in
// place (every thread writes the elements it read) and one bulk tensor store writes it to s_hat.
// Loads of whole 128-byte rows replace the 16-byte-per-row accesses of a warp holding two
// positions of 256-point lines.
#include <cstdlib>
#include <type_traits>
#include "kargs.h"
#include "fft_reg.cuh"
#include "tma.cuh"
#include "driver_api.h"

namespace unocg {

constexpr int KL_P = 16;  // positions per block (one 128-byte row of complex FP32), or 8 (64 bytes)

// Byte offset of element (row r, column p) of a TMA tile of P complex FP32 per row, written with
// the 128-byte swizzle (P = 16: chunk XOR r mod 8) or the 64-byte one (P = 8: the 16-byte chunk
// index XOR bits 7..8 of the row's byte address, (r / 2) mod 4)
template <int P> __device__ __forceinline__ uint32_t swz_off8(int r, int p) {
  if constexpr (P == 16) return swz128_off8(r, p);
  else return (uint32_t)(r * 64 + ((((p >> 1) ^ (r >> 1)) & 3) << 4) + ((p & 1) << 3));
}

struct alignas(64) LineTmaMaps {
  CUtensorMap hat;   // r_hat  [BL][N1][2M] floats, box {32, N1, 1}, 128-byte swizzle
  CUtensorMap shat;  // s_hat  same layout
  CUtensorMap q;     // Q      [Bq][N1][M] bf16, box {16, N1, 1}
};

struct LineTmaArgs {
  LineArgs<float, __nv_bfloat16> a;
  int tiles;            // blocks per (instance, load)
  int* err;
  long long spin_limit;
};

// shared memory of one block (1024-byte alignment slack, r_hat and s_old tiles, Q tile) and the
// blocks per SM the launch bounds ask for: at most 24 warps, and what the 228 KB of shared memory
// per SM hold (1 KB reserved per block)
template <int N1, int P> constexpr size_t kl_smem_bytes() { return 1024 + 2 * (size_t)N1 * 8 * P + (size_t)N1 * 2 * P; }
// blocks per SM the launch bounds ask for: at most 24 warps and what the 228 KB of shared memory
// hold (1 KB reserved per block); 256-point lines in 8-position tiles keep at least 96 registers
// (five blocks: no spills)
template <int N1, int P> constexpr int kl_min_blocks() {
  constexpr int by_threads = 768 / (P * RegSplit<N1>::G);
  constexpr int by_smem = (int)(233472 / (kl_smem_bytes<N1, P>() + 1024));
  constexpr int m = by_threads < by_smem ? by_threads : by_smem;
  return (N1 == 256 && P == 8 && m > 5) ? 5 : m;
}

template <int N1, int P>
__global__ void __launch_bounds__(P * RegSplit<N1>::G, kl_min_blocks<N1, P>())
    k_line_tma(const __grid_constant__ LineTmaMaps maps, const LineTmaArgs la) {
  using C = float2;
  constexpr int G = RegSplit<N1>::G, V = RegSplit<N1>::V, VG = V / G, W = 32 / G;
  constexpr int NTH = P * G;
  constexpr int TB = N1 * 8 * P;  // bytes of one spectrum tile
  extern __shared__ unsigned char kl_raw[];
  __shared__ double red_sh[32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_abort;
  const LineArgs<float, __nv_bfloat16>& a = la.a;
  // tiles: r_hat (becomes s_hat) and s_old (becomes the exchange scratch), each N1 rows of P
  // complex, 1024-byte aligned for the swizzle; Q (N1 x P bf16)
  unsigned char* base = kl_raw + ((1024u - (sm_addr(kl_raw) & 1023u)) & 1023u);
  unsigned char* t_hat = base;
  unsigned char* t_old = base + TB;
  const __nv_bfloat16* t_q = reinterpret_cast<const __nv_bfloat16*>(base + 2 * TB);
  // twiddles from the global table (L1-resident): without their shared copy three 256-thread
  // blocks fit an SM
  const C* __restrict__ tw1 = reinterpret_cast<const C*>(a.ft.tw1);
  const int tid = threadIdx.x;
  const int bl = blockIdx.y;
  const int tile = blockIdx.x;
  const int pos0 = tile * P;
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
    const uint32_t bytes = (uint32_t)(TB * (a.flexible ? 2 : 1) + N1 * 2 * P);
    mbar_expect_tx(&bar, bytes);
    tma_load_3d(t_hat, &maps.hat, 2 * pos0, 0, bl, &bar);
    if (a.flexible) tma_load_3d(t_old, &maps.shat, 2 * pos0, 0, bl, &bar);
    tma_load_3d(const_cast<__nv_bfloat16*>(t_q), &maps.q, pos0, 0, a.q_inst_stride ? b : 0, &bar);
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
      // position within the tile and thread of the line; 16-thread lines in 16-position tiles
      // interleave their lanes (0-7 and 16-23 one line, 8-15 and 24-31 the other) so that each
      // half-warp reads eight consecutive rows of two positions: distinct chunks of the swizzle
      constexpr bool ilv = G == 16 && P == 16;
      const int lane_ = tid & 31;
      const int p = ilv ? (tid >> 5) * W + ((lane_ >> 3) & 1) : tid / G;
      const int g = ilv ? (lane_ & 7) + ((lane_ >> 4) << 3) : tid % G;
      const int pos = pos0 + p;
      const bool on = pos < M;
      const int k3 = on ? pos % a.g.n3h : 0;
      const float wt = (k3 == 0 || 2 * k3 == a.g.n3) ? 1.f : 2.f;
      const float sc = (float)a.scale;
      C v[V];
#pragma unroll
      for (int n1 = 0; n1 < V; ++n1) v[n1] = *reinterpret_cast<const C*>(t_hat + swz_off8<P>(g + G * n1, p));
      // Parseval partials: the thread's V products are summed in FP32 (their rounding stays below
      // that of the FP32 spectra themselves) and accumulated in the float-float pair
      if (a.flexible && on) {
        float part = 0.f;
#pragma unroll
        for (int n1 = 0; n1 < V; ++n1) {
          const C so = *reinterpret_cast<const C*>(t_old + swz_off8<P>(g + G * n1, p));
          part = fmaf(v[n1].x, so.x, fmaf(v[n1].y, so.y, part));
        }
        rso.add(wt * part);
      }
      __syncthreads();  // the s_old tile is free: exchange scratch of the line transforms
      // exchange slots: the line's own N1 slots, odd lines with slot index bit 3 flipped
      const int w = p % W, warp = tid >> 5;
      const XorSlot<C> scr{reinterpret_cast<C*>(t_old) + (size_t)(warp * W + w) * N1, (w & 1) << 3};
      fft_dist_a_at<N1, -1>(v, g, scr, tw1);
      if (on) {
        float part = 0.f;  // r . s = sum q |r_hat|^2 over the thread's modes
#pragma unroll
        for (int j = 0; j < VG; ++j)
#pragma unroll
          for (int k2 = 0; k2 < G; ++k2) {
            const int k1 = scat_index<N1>(g, j, k2), e = j * G + k2;
            const float q = __bfloat162float(t_q[k1 * P + p]) * sc;
            const C R = v[e];
            part = fmaf(q, fmaf(R.x, R.x, R.y * R.y), part);
            v[e] = make_float2(q * R.x, q * R.y);
          }
        gam.add(wt * part);
      }
      fft_dist_b_at<N1, +1>(v, g, scr, tw1);
#pragma unroll
      for (int n1 = 0; n1 < V; ++n1) *reinterpret_cast<C*>(t_hat + swz_off8<P>(g + G * n1, p)) = v[n1];
      fence_async_shared();
    }
    __syncthreads();
    if (!s_abort && tid == 0) {
      tma_store_3d(&maps.shat, 2 * pos0, 0, bl, t_hat);
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
  // the tile must stay in shared memory until the bulk store has read it, and the store is
  // complete before the block exits
  if (active && tid == 0) tma_store_wait_all();
}

// ---------------------------------------------------------------- host side
bool line_tma_supported(const Grid& g, int c) {
  if (c == 3) return line_tma3_supported(g);
  if (c != 1) return false;
  if (!(g.n1 == 16 || g.n1 == 32 || g.n1 == 48 || g.n1 == 64 || g.n1 == 96 || g.n1 == 128 || g.n1 == 192 ||
        g.n1 == 256))
    return false;
  const long long M = (long long)g.n2 * g.n3h;
  if (M % 8 != 0) return false;  // 16-byte row strides of the Q and spectrum tensors
  return tensor_map_encoder() != nullptr;
}

// partial sums per (instance, load): one per block of the narrower tile (8 positions)
int line_tma_blocks_x(const Grid& g) { return (int)(((long long)g.n2 * g.n3h + 7) / 8); }

// positions per block: 16 (128-byte rows, 128-byte swizzle; the default) or 8 (64-byte rows,
// 64-byte swizzle: half the shared memory per block, about twice the blocks per SM), selected by
// UNOCG_LINE_P at every launch.  Measured per launch with three loads, before the conflict-free
// lane layout: 256^3 203.6 (16) against 203.4 us (8), 192^3 83.4 against 97.6 us.
static int line_tma_p(const Grid&) {
  const char* e = std::getenv("UNOCG_LINE_P");
  return (e && std::atoi(e) == 8) ? 8 : 16;
}
static CUresult encode_3d(CUtensorMap* m, CUtensorMapDataType dt, size_t esz, const void* ptr, cuuint64_t d0,
                          cuuint64_t d1, cuuint64_t d2, cuuint32_t b0, cuuint32_t b1, CUtensorMapSwizzle sw) {
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {d0 * esz, d0 * d1 * esz};
  const cuuint32_t box[3] = {b0, b1, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return tensor_map_encoder()(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int N1, int P>
static cudaError_t line_tma_n(const LineTmaMaps& maps, const LineTmaArgs& la, cudaStream_t st) {
  constexpr int NTH = P * RegSplit<N1>::G;
  const size_t smem = kl_smem_bytes<N1, P>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_line_tma<N1, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_line_tma<N1, P>, dim3(la.tiles, la.a.BL), dim3(NTH), smem, st, maps, la);
}

template <int P>
static cudaError_t line_tma_p_launch(const LineTmaMaps& maps, const LineTmaArgs& la, cudaStream_t st) {
  switch (la.a.g.n1) {
    case 16: return line_tma_n<16, P>(maps, la, st);
    case 32: return line_tma_n<32, P>(maps, la, st);
    case 48: return line_tma_n<48, P>(maps, la, st);
    case 64: return line_tma_n<64, P>(maps, la, st);
    case 96: return line_tma_n<96, P>(maps, la, st);
    case 128: return line_tma_n<128, P>(maps, la, st);
    case 192: return line_tma_n<192, P>(maps, la, st);
    case 256: return line_tma_n<256, P>(maps, la, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_line_tma(const LineArgs<float, __nv_bfloat16>& a, int* err, long long spin_limit, cudaStream_t st) {
  if (a.c == 3) return launch_line_tma3(a, err, spin_limit, st);
  const Grid& g = a.g;
  const cuuint64_t M = (cuuint64_t)g.n2 * g.n3h;
  const int Bq = a.q_inst_stride ? a.BL / a.L : 1;
  const int P = line_tma_p(g);
  const CUtensorMapSwizzle sw = P == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  LineTmaMaps maps;
  if (encode_3d(&maps.hat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.hat, 2 * M, g.n1, a.BL, 2 * P, g.n1, sw) !=
          CUDA_SUCCESS ||
      encode_3d(&maps.shat, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.shat, 2 * M, g.n1, a.BL, 2 * P, g.n1, sw) !=
          CUDA_SUCCESS ||
      encode_3d(&maps.q, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, a.Q, M, g.n1, Bq, P, g.n1, CU_TENSOR_MAP_SWIZZLE_NONE) !=
          CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  LineTmaArgs la{};
  la.a = a;
  la.tiles = (int)((M + P - 1) / P);
  la.err = err;
  la.spin_limit = spin_limit;
  return P == 16 ? line_tma_p_launch<16>(maps, la, st) : line_tma_p_launch<8>(maps, la, st);
}

}  // namespace unocg
