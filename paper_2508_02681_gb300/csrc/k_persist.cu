// Persistent UNO-CG: the whole loop of Algorithm 2 in one cooperative launch.
//
// For grids whose per-phase work is only a few hundred blocks, launch latency and per-block
// start-up dominate the per-phase kernels.  Here every block of a co-resident grid loops over
// the tasks of one phase (planes, axis-1 tiles, K d tiles), then all blocks meet at a grid
// barrier.  Each block reduces the per-task partial sums of the finished phase itself, in a
// fixed order, so all blocks hold identical CG scalars (gamma, beta, alpha, stopping test)
// without a second barrier.  Iteration: [axis-1 pass] B [inverse plane pass] B [K d] B
// [residual update + forward plane pass] B + stopping test, plus (mixed precision) the FP64
// residual replacement [fold] B [f - K u] B [forward plane pass] B when requested.
//
// The grid barrier spins at most `spin_limit` SM clock cycles; on expiry it raises a flag that
// every block observes at its next barrier, all blocks return, and the host reports
// UNOCG_ERR_DEVICE_TIMEOUT.  Fields written by other blocks of this launch are read through
// L2 (ld.global.cg); this translation unit is compiled with -dlcm=cg.
#include "fft_kernels.cuh"
#include "ku_task.cuh"
#include "persist.h"

namespace unocg {

__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* err, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 1;
    volatile int* verr = err;
    const unsigned int g0 = *gen;
    __threadfence();
    const unsigned int nb = gridDim.x;
    ok = 1;
    if (atomicAdd(bar, 1u) == nb - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (*verr || clock64() - t0 > limit) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// max / sum of `count` partials by one warp (fixed order, result in every lane)
__device__ __forceinline__ double warp_max_partials(const double* p, int count) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int x = lane; x < count; x += 32) s = fmax(s, ld_cg(p + x));
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  return s;
}

template <typename T, typename QT, int CC>
struct Persist {
  const PersistArgs<T, QT>& a;
  PlaneSmem<T> ps;
  LineSmem<T> ls;
  CgScal* S;
  T* mt;          // per-instance material tables, type T
  double* mt64;   // per-instance material tables, FP64 (true residual)
  double* red_sh;
  int* flags;     // [0] any active, [1] any replacement pending
  LoopCtl ctl;

  __device__ bool barrier() { return grid_barrier(a.bar, a.err, a.spin_limit); }

  // forward plane pass over all active pairs, then the stopping test (every block)
  __device__ bool phase_fwd(int after_replace) {
    const int np = a.pf.c * a.pf.g.n1;
    const int total = a.BL * np;
    for (int task = blockIdx.x; task < total; task += gridDim.x) {
      const int bl = task / np, plane = task - bl * np;
      if (S[bl].done || (after_replace && !S[bl].need_replace)) continue;
      const double al = after_replace ? 0.0 : S[bl].alpha;
      double m = plane_fwd_task<T>(a.pf, ps, bl, plane, al, red_sh);
      if (threadIdx.x == 0) a.part[a.off_max + (long long)bl * np + plane] = m;
    }
    if (!barrier()) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bl = warp; bl < a.BL; bl += blockDim.x / 32) {
      if (S[bl].done || (after_replace && !S[bl].need_replace)) continue;
      double m = warp_max_partials(a.part + a.off_max + (long long)bl * np, np);
      if (lane == 0) S[bl].rmax_bits = (unsigned long long)__double_as_longlong(m);
    }
    __syncthreads();
    residual_decision(S, a.BL, ctl, after_replace);
    __syncthreads();
    return true;
  }

  __device__ bool phase_line() {
    const int nt = a.n_line_tasks;
    const int total = a.BL * nt;
    for (int task = blockIdx.x; task < total; task += gridDim.x) {
      const int bl = task / nt, tile = task - bl * nt;
      if (S[bl].done) continue;
      double2 pr = line_task<T, QT, CC, 0>(a.la, ls, bl, tile, red_sh);
      if (threadIdx.x == 0) {
        double* pp = a.part + a.off_line + ((long long)bl * nt + tile) * 2;
        pp[0] = pr.x;
        pp[1] = pr.y;
      }
    }
    if (!barrier()) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bl = warp; bl < a.BL; bl += blockDim.x / 32) {
      if (S[bl].done) continue;
      const double* pp = a.part + a.off_line + (long long)bl * nt * 2;
      double sg = warp_sum_partials(pp, nt, 2);
      double sr = warp_sum_partials(pp + 1, nt, 2);
      if (lane == 0) direction_update(S[bl], sg, sr, ctl.flexible);
    }
    __syncthreads();
    return true;
  }

  __device__ bool phase_inv() {
    const int np = a.pi.c * a.pi.g.n1;
    const int total = a.BL * np;
    for (int task = blockIdx.x; task < total; task += gridDim.x) {
      const int bl = task / np, plane = task - bl * np;
      if (S[bl].done) continue;
      plane_inv_task<T>(a.pi, ps, bl, plane, S[bl].alpha, S[bl].beta);
    }
    return barrier();
  }

  __device__ bool phase_ku() {
    const int nt = a.n_ku_tasks;
    const int total = a.BL * nt;
    const int np2 = 2 * a.ka.mat.n_phases;
    for (int task = blockIdx.x; task < total; task += gridDim.x) {
      const int bl = task / nt, tile = task - bl * nt;
      if (S[bl].done) continue;
      double dp = ku_task<T, CC, true>(a.ka, mt + (bl / a.L) * np2, bl, tile, red_sh, reinterpret_cast<T*>(ps.buf));
      if (threadIdx.x == 0) a.part[a.off_ku + (long long)bl * nt + tile] = dp;
    }
    if (!barrier()) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bl = warp; bl < a.BL; bl += blockDim.x / 32) {
      if (S[bl].done) continue;
      double sum = warp_sum_partials(a.part + a.off_ku + (long long)bl * nt, nt, 1);
      if (lane == 0) step_update(S[bl], sum);
    }
    __syncthreads();
    return true;
  }

  // FP64 residual replacement of the pending pairs: u64 += u32 + alpha d, u32 = 0, alpha = 0,
  // r = f - K u64; then a forward plane pass of the new residual and its stopping test.
  __device__ bool phase_replace() {
    const long long m = (long long)CC * a.pf.g.n;
    const int chunks = a.n_fold_chunks;
    const int total = a.BL * chunks;
    const long long per = (m + chunks - 1) / chunks;
    for (int task = blockIdx.x; task < total; task += gridDim.x) {
      const int bl = task / chunks, ch = task - bl * chunks;
      if (S[bl].done || !S[bl].need_replace) continue;
      const double al = S[bl].alpha;
      const long long base = (long long)bl * m;
      const long long lo = ch * per, hi = min(m, lo + per);
      for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        double v = __ldcg(a.fo.u64 + base + i) + (double)__ldcg(a.fo.u32 + base + i) +
                   al * (double)__ldcg(a.fo.d + base + i);
        a.fo.u64[base + i] = v;
        a.fo.u32[base + i] = (T)0;
      }
    }
    if (!barrier()) return false;
    for (int bl = threadIdx.x; bl < a.BL; bl += blockDim.x)
      if (!S[bl].done && S[bl].need_replace) S[bl].alpha = 0.0;
    __syncthreads();
    // r = f - K u64 in FP64 on node tiles
    const int nt = a.n_tr_tasks;
    const int np2 = 2 * a.ka.mat.n_phases;
    const Grid& g = a.pf.g;
    for (int task = blockIdx.x; task < a.BL * nt; task += gridDim.x) {
      const int bl = task / nt, tile = task - bl * nt;
      if (S[bl].done || !S[bl].need_replace) continue;
      const int b = bl / a.L, l = bl - b * a.L;
      int i1, i2, i3;
      if (tile_node_at(g, tile, i1, i2, i3)) {
        const long long n = g.n;
        const uint8_t* ph = a.ka.phase + (long long)b * n;
        const double* u = a.fo.u64 + (long long)bl * CC * n;
        const long long node = ((long long)i1 * g.n2 + i2) * g.n3 + i3;
        double f[CC], ku[CC];
        node_rhs<CC>(ph, mt64 + b * np2, g, i1, i2, i3, a.loads + l * (CC == 1 ? 3 : 6), f);
        node_Ku<double, CC, true>(u, ph, mt64 + b * np2, g, i1, i2, i3, ku);
#pragma unroll
        for (int i = 0; i < CC; ++i) a.pf.r[(long long)bl * CC * n + i * n + node] = (T)(f[i] - ku[i]);
      }
    }
    if (!barrier()) return false;
    return phase_fwd(1);
  }
};

template <typename T, typename QT, int CC>
__global__ void __launch_bounds__(256) k_persist(PersistArgs<T, QT> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  __shared__ int flags[2];
  using C = cplx<T>;
  const Grid& g = a.pf.g;
  const int P = pitch_of(g.n3h);
  const int tb = a.la.tb;
  static_assert(kPersistKuTileValues == (size_t)(KU_DN + KU_KN), "tile size mismatch");
  const size_t nA = max(max((size_t)2 * g.n2 * P, (size_t)2 * g.n1 * CC * tb), kPersistKuTileValues / 2 + 1);
  C* A = reinterpret_cast<C*>(smem_raw);
  C* tw = A + nA;
  C* tw3h = tw;
  C* tw2 = tw3h + g.n3 / 2;
  C* tw3 = tw2 + g.n2;
  C* tw1 = tw3 + g.n3;
  CgScal* S = reinterpret_cast<CgScal*>(tw1 + g.n1);
  double* mt64 = reinterpret_cast<double*>(S + a.BL);
  const int nmat = a.B * 2 * a.ka.mat.n_phases;
  T* mt = reinterpret_cast<T*>(mt64 + nmat);
  load_tw<T>(tw3h, a.pf.ft.tw3h, g.n3 / 2);
  load_tw<T>(tw2, a.pf.ft.tw2, g.n2);
  load_tw<T>(tw3, a.pf.ft.tw3, g.n3);
  load_tw<T>(tw1, a.la.ft.tw1, g.n1);
  for (int i = threadIdx.x; i < nmat; i += blockDim.x) {
    mt64[i] = a.ka.mat.m64[i];
    mt[i] = mat_ptr<T>(a.ka.mat)[i];
  }
  {
    int* z = reinterpret_cast<int*>(S);
    const int nz = a.BL * (int)(sizeof(CgScal) / sizeof(int));
    for (int i = threadIdx.x; i < nz; i += blockDim.x) z[i] = 0;
  }
  __syncthreads();

  Persist<T, QT, CC> ps{a, PlaneSmem<T>{A, A + g.n2 * P, tw3h, tw2, tw3},
                        LineSmem<T>{A, A + (size_t)g.n1 * CC * tb, nullptr, nullptr, tw1},
                        S, mt, mt64, red_sh, flags, a.ctl};
  ps.ctl.set_while = 0;
  ps.ctl.set_if = 0;
  ps.ctl.active_flag = &flags[0];
  ps.ctl.replace_flag = &flags[1];
  ps.ctl.counters = blockIdx.x == 0 ? a.counters : nullptr;

  bool ok = ps.phase_fwd(0);
  const int guard_max = 4 * a.ctl.max_iter + 16;
  for (int guard = 0; ok && flags[0] && guard < guard_max; ++guard) {
    ok = ps.phase_line() && ps.phase_inv() && ps.phase_ku() && ps.phase_fwd(0);
    if (ok && flags[1]) ok = ps.phase_replace();
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int bl = threadIdx.x; bl < a.BL; bl += blockDim.x) a.sc[bl] = S[bl];
  }
}

template <typename T, typename QT, int CC>
static cudaError_t launch_persist_cc(PersistArgs<T, QT>& a, cudaStream_t s, int sm_count) {
  auto kern = k_persist<T, QT, CC>;
  size_t smem = persist_smem_bytes(a.pf.g, CC, a.la.tb, sizeof(cplx<T>), a.BL, a.B, a.ka.mat.n_phases, sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int want = max(max(a.BL * a.pf.c * a.pf.g.n1, a.BL * a.n_line_tasks), a.BL * a.n_ku_tasks);
  int blocks = min(per_sm * sm_count, want);
  blocks = max(blocks, 1);
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(256), args, smem, s);
}

template <typename T, typename QT>
cudaError_t launch_persist(PersistArgs<T, QT>& a, cudaStream_t s, int sm_count) {
  if (a.pf.c == 1) return launch_persist_cc<T, QT, 1>(a, s, sm_count);
  return launch_persist_cc<T, QT, 3>(a, s, sm_count);
}

template cudaError_t launch_persist<float, __nv_bfloat16>(PersistArgs<float, __nv_bfloat16>&, cudaStream_t, int);
template cudaError_t launch_persist<double, double>(PersistArgs<double, double>&, cudaStream_t, int);

}  // namespace unocg
