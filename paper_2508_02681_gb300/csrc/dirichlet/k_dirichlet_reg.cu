// Register-resident sine-transform passes of the Dirichlet-BC solver for power-of-two axes
// (N in {8, ..., 128}): the odd-extended pair lines of length 2N (dargs.h) are transformed by
// the warp-level FFT of fft_reg.cuh, G lanes per pair, with one shared-memory exchange each.
//
//   k_dplane_reg: one interior plane (instance-load, component, i1) per block, held in shared
//     memory as reals: coalesced load (with r -= alpha q, u += alpha p, ||r||_inf and the stopping
//     test in loop mode), rows (axis 3) then columns (axis 2), coalesced store to the spectrum;
//     the inverse reads the spectrum, transforms columns then rows, and writes p = s + beta p.
//   k_dline_reg (c = 1): a tile of W consecutive (k2, k3) positions per block, axis 1: forward
//     DST, s_hat = Q r_hat with the Parseval partial of r.s, second DST straight from the
//     scattered spectrum (the forward DFT read from the other side), coalesced store.
//
// Block multiply on the odd-extended spectrum: with w = (i/2) Z[m] = X_a + i X_b at the mode
// k = min(m, 2N - m) - 1 (for m > N the odd symmetry Z[2N - m] = -Z[m] gives -w), the input of
// the second transform is z'[m] = Q_a Re w + i Q_b Im w at every m (0 at m = 0, N), so no
// exchange between lanes is needed.
#include "../fft_reg.cuh"
#include "../kargs.h"
#include "dargs.h"

namespace unocg {

namespace {

template <int N> struct DReg {
  static constexpr int L = 2 * N;
  static constexpr int G = RegSplit<L>::G, V = RegSplit<L>::V, VG = V / G;
  static constexpr int PPW = 32 / G;  // pairs per warp
  static constexpr int NP = N / 2;    // pairs of the N - 1 interior lines (the last is half zero)
  static constexpr int PITCH = N + 1; // real plane / tile pitch
};

constexpr int kPlaneWarps = 8;
constexpr int kLineWarps = 4;

template <typename T>
__device__ __forceinline__ void ld_tw(cplx<T>* dst, const void* src, int n) {
  const cplx<T>* s = (const cplx<T>*)src;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = s[i];
}

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < (T)0 ? -x : x; }

// natural-order input of pair (line a = 2p, line b = 2p + 1) of a real buffer with elements
// at buf[line * ls + j * es]: z[m] = x_a[m-1] + i x_b[m-1], odd-extended
template <int N, typename T>
__device__ __forceinline__ void dst_load(cplx<T>* v, const T* buf, int la, int ls, int es, int g) {
  using R = DReg<N>;
#pragma unroll
  for (int n1 = 0; n1 < R::V; ++n1) {
    const int m = g + R::G * n1;
    cplx<T> z = mk<T>((T)0, (T)0);
    if (m != 0 && m != N) {
      const int j = m < N ? m - 1 : 2 * N - m - 1;
      const T xa = buf[la * ls + j * es], xb = buf[(la + 1) * ls + j * es];
      z = m < N ? mk<T>(xa, xb) : mk<T>(-xa, -xb);
    }
    v[n1] = z;
  }
}

// unnormalized DST coefficients of the pair from the scattered spectrum, into the buffer
template <int N, typename T>
__device__ __forceinline__ void dst_store_scattered(const cplx<T>* v, T* buf, int la, int ls, int es, int g) {
  using R = DReg<N>;
#pragma unroll
  for (int j = 0; j < R::VG; ++j)
#pragma unroll
    for (int k2 = 0; k2 < R::G; ++k2) {
      const int m = scat_index<R::L>(g, j, k2);
      if (m >= 1 && m < N) {
        const cplx<T> z = v[j * R::G + k2];
        buf[la * ls + (m - 1) * es] = (T)-0.5 * z.y;
        buf[(la + 1) * ls + (m - 1) * es] = (T)0.5 * z.x;
      }
    }
}

// y = Q x for the unique entries q in the paper's order (v1=Q11 v2=Q22 v3=Q12 v4=Q33 v5=Q23 v6=Q13)
template <typename T, int CC>
__device__ __forceinline__ void qmul_reg(const T* __restrict__ q, const T* x, T* y) {
  if (CC == 1) {
    y[0] = q[0] * x[0];
  } else {
    y[0] = q[0] * x[0] + q[2] * x[1] + q[5] * x[2];
    y[1] = q[2] * x[0] + q[1] * x[1] + q[4] * x[2];
    y[2] = q[5] * x[0] + q[4] * x[1] + q[3] * x[2];
  }
}

}  // namespace

// ============================================================================ planes
template <typename T, int N, int FWD>
__global__ void __launch_bounds__(kPlaneWarps * 32) k_dplane_reg(DPassArgs<T> a) {
  using C = cplx<T>;
  using R = DReg<N>;
  constexpr int M = N - 1, P = R::PITCH;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red_sh[32];
  T* pl = reinterpret_cast<T*>(dsm);                                    // N x P reals
  C* scr = reinterpret_cast<C*>(dsm + ((sizeof(T) * N * P + 15) / 16) * 16);  // per pair group
  C* tw = scr + kPlaneWarps * R::PPW * R::L;
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int comp = blockIdx.x / g.m1, j1 = blockIdx.x - comp * g.m1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = (long long)bl * a.c * g.ne + ((long long)comp * g.n1 + j1 + 1) * (long long)N * N;
  bool active = true;
  if (!a.standalone) {
    const CgScal& s = a.sc[bl];
    active = !s.done && (!FWD || !a.after_replace || s.need_replace);
  }
  T rm = (T)0;
  if (active) {
    ld_tw<T>(tw, a.t.tw[2], R::L);  // N2 = N3: one table serves both axes
    // coalesced load of the interior plane; row M and column M stay zero
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int j2 = idx / N, j3 = idx - j2 * N;
      T x = (T)0;
      if (j2 < M && j3 < M) {
        const long long ga = base + (long long)(j2 + 1) * N + j3 + 1;
        if (!FWD) {
          x = a.hat[ga];
        } else if (a.standalone) {
          x = a.src[ga];
        } else {
          const CgScal& s = a.sc[bl];
          x = a.r[ga];
          if (!a.after_replace && s.started) {
            const T alpha = (T)s.alpha;
            x -= alpha * a.q[ga];
            a.r[ga] = x;
            a.u[ga] += alpha * a.p[ga];
          }
          rm = rm > tabs(x) ? rm : tabs(x);
        }
      }
      pl[j2 * P + j3] = x;
    }
    __syncthreads();
    // two phases: FWD rows then columns, inverse columns then rows
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
      const bool rows = (ph == 0) == (FWD != 0);
      const int ls = rows ? P : 1, es = rows ? 1 : P;  // line stride, element stride
      for (int p0 = warp * R::PPW; p0 < R::NP; p0 += kPlaneWarps * R::PPW) {
        const int pr = p0 + lane / R::G, gl = lane % R::G;
        const int prc = pr < R::NP ? pr : R::NP - 1;  // idle lanes repeat a valid pair, no store
        C v[R::V];
        dst_load<N, T>(v, pl, 2 * prc, ls, es, gl);
        C* sp = scr + (warp * R::PPW + lane / R::G) * R::L;
        fft_dist_a<R::L, -1>(v, gl, sp, 1, tw);
        if (pr < R::NP) dst_store_scattered<N, T>(v, pl, 2 * pr, ls, es, gl);
        __syncwarp();
      }
      __syncthreads();
    }
    // coalesced store
    const T beta = (FWD || a.standalone) ? (T)0 : (T)a.sc[bl].beta;
    for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
      const int j2 = idx / M, j3 = idx - j2 * M;
      const long long ga = base + (long long)(j2 + 1) * N + j3 + 1;
      const T x = pl[j2 * P + j3];
      if (FWD) a.hat[ga] = x;
      else if (a.standalone) a.out[ga] = x;
      else a.p[ga] = x + beta * a.p[ga];
    }
  }
  if (a.standalone || !FWD) return;
  const double bm = block_max_t(rm, red_sh);
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bm);
  if (last_block(a.red.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// ============================================================================ axis 1 with Q
// Every lane group transforms the same two positions for all CC components in turn, so the
// spectral indices it holds are the same for every component and the c x c block multiply
// needs no exchange.
template <typename T, int N, int CC>
__global__ void __launch_bounds__(kLineWarps * 32) k_dline_reg(DPassArgs<T> a) {
  using C = cplx<T>;
  using R = DReg<N>;
  constexpr int M = N - 1;
  constexpr int W = kLineWarps * R::PPW * 2;  // positions per block
  constexpr int TP = W + 1;                   // tile pitch
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red_sh[32];
  T* tile = reinterpret_cast<T*>(dsm);  // CC x N x TP reals: [comp][j1][position]
  C* scr = reinterpret_cast<C*>(dsm + ((sizeof(T) * CC * N * TP + 15) / 16) * 16);
  C* tw = scr + kLineWarps * R::PPW * R::L;
  const DGrid& g = a.g;
  const int bl = blockIdx.y;
  const int nb3 = (g.m3 + W - 1) / W;
  const int k2 = blockIdx.x / nb3, k30 = (blockIdx.x - k2 * nb3) * W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long base = (long long)bl * CC * g.ne;
  const bool active = a.standalone || !a.sc[bl].done;
  DotAcc<T> acc;
  if (active) {
    ld_tw<T>(tw, a.t.tw[0], R::L);
    for (int idx = threadIdx.x; idx < CC * N * W; idx += blockDim.x) {
      const int w = idx % W, r = idx / W;
      const int j = r % N, comp = r / N;
      const int k3 = k30 + w;
      T x = (T)0;
      if (j < M && k3 < g.m3)
        x = a.hat[base + comp * g.ne + ((long long)(j + 1) * g.n2 + k2 + 1) * g.n3 + k3 + 1];
      tile[(comp * N + j) * TP + w] = x;
    }
    __syncthreads();
    {
      const int pr = warp * R::PPW + lane / R::G, gl = lane % R::G;
      const int wa = 2 * pr;
      C* sp = scr + pr * R::L;
      C v[CC][R::V];
#pragma unroll
      for (int cc = 0; cc < CC; ++cc) {
        dst_load<N, T>(v[cc], tile + cc * N * TP, wa, 1, TP, gl);
        fft_dist_a<R::L, -1>(v[cc], gl, sp, 1, tw);
      }
      // block multiply at the held spectral indices (scattered order)
      const T* Q = reinterpret_cast<const T*>(a.Q) + (long long)(bl / a.L) * a.q_inst_stride;
      const int k3a = k30 + wa, k3b = k3a + 1;
      constexpr int NQ = CC == 1 ? 1 : 6;
#pragma unroll
      for (int j = 0; j < R::VG; ++j)
#pragma unroll
        for (int t = 0; t < R::G; ++t) {
          const int m = scat_index<R::L>(gl, j, t);
          const int e = j * R::G + t;
          if (m == 0 || m == N) {
#pragma unroll
            for (int cc = 0; cc < CC; ++cc) v[cc][e] = mk<T>((T)0, (T)0);
            continue;
          }
          const int k = (m < N ? m : 2 * N - m) - 1;
          const long long row = ((long long)k * g.m2 + k2) * g.m3;
          T xa[CC], xb[CC], ya[CC], yb[CC];
#pragma unroll
          for (int cc = 0; cc < CC; ++cc) {
            xa[cc] = (T)-0.5 * v[cc][e].y;  // w = (i/2) Z
            xb[cc] = (T)0.5 * v[cc][e].x;
          }
          if (k3a < g.m3) qmul_reg<T, CC>(Q + (row + k3a) * NQ, xa, ya);
          else for (int cc = 0; cc < CC; ++cc) ya[cc] = (T)0;
          if (k3b < g.m3) qmul_reg<T, CC>(Q + (row + k3b) * NQ, xb, yb);
          else for (int cc = 0; cc < CC; ++cc) yb[cc] = (T)0;
#pragma unroll
          for (int cc = 0; cc < CC; ++cc) {
            if (m < N) {
              acc.add_prod(xa[cc], ya[cc]);
              acc.add_prod(xb[cc], yb[cc]);
            }
            v[cc][e] = mk<T>(ya[cc], yb[cc]);
          }
        }
#pragma unroll
      for (int cc = 0; cc < CC; ++cc) {
        fft_dist_b<R::L, -1>(v[cc], gl, sp, 1, tw);
        // natural order: lane gl holds Z2[gl + G n1]
#pragma unroll
        for (int n1 = 0; n1 < R::V; ++n1) {
          const int m = gl + R::G * n1;
          if (m >= 1 && m < N) {
            tile[(cc * N + m - 1) * TP + wa] = (T)-0.5 * v[cc][n1].y;
            tile[(cc * N + m - 1) * TP + wa + 1] = (T)0.5 * v[cc][n1].x;
          }
        }
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < CC * M * W; idx += blockDim.x) {
      const int w = idx % W, r = idx / W;
      const int j = r % M, comp = r / M;
      const int k3 = k30 + w;
      if (k3 < g.m3)
        a.hat[base + comp * g.ne + ((long long)(j + 1) * g.n2 + k2 + 1) * g.n3 + k3 + 1] = tile[(comp * N + j) * TP + w];
    }
  }
  if (a.standalone) return;
  const double bs = block_sum_acc(acc, red_sh);
  if (threadIdx.x == 0) a.red.part[(long long)bl * gridDim.x + blockIdx.x] = bs;
  if (last_block(a.red.ticket)) {
    const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    for (int q = wp; q < a.BL; q += blockDim.x / 32) {
      if (a.sc[q].done) continue;
      const double gam = warp_sum_partials(a.red.part + (long long)q * gridDim.x, gridDim.x, 1);
      if (ln == 0) direction_update(a.sc[q], gam, 0.0, 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.red.ticket = 0u;
  }
}

// ============================================================================ launchers
template <typename T, int N> static size_t plane_reg_smem() {
  using R = DReg<N>;
  return ((sizeof(T) * N * R::PITCH + 15) / 16) * 16 + sizeof(cplx<T>) * ((size_t)kPlaneWarps * R::PPW * R::L + R::L);
}
template <typename T, int N, int CC> static size_t line_reg_smem() {
  using R = DReg<N>;
  constexpr int W = kLineWarps * R::PPW * 2;
  return ((sizeof(T) * CC * N * (W + 1) + 15) / 16) * 16 + sizeof(cplx<T>) * ((size_t)kLineWarps * R::PPW * R::L + R::L);
}

static bool pow2_small(int n) { return n == 8 || n == 16 || n == 32 || n == 64 || n == 128; }

bool dplane_reg_ok(const DGrid& g) { return g.n2 == g.n3 && pow2_small(g.n3); }
// c = 1 only: for c = 3 the 3 x V complex values per thread (174 registers at N1 = 64, FP32)
// leave two blocks per SM, and the shared-memory pass is faster (64^3 elastic Dirichlet solve,
// six loads, mixed: 16.0 vs 17.1 ms)
bool dline_reg_ok(const DGrid& g, int c, int elem_bytes) {
  (void)elem_bytes;
  return pow2_small(g.n1) && c == 1;
}

int dline_reg_positions(int n1) {
  switch (n1) {
    case 8: return kLineWarps * DReg<8>::PPW * 2;
    case 16: return kLineWarps * DReg<16>::PPW * 2;
    case 32: return kLineWarps * DReg<32>::PPW * 2;
    case 64: return kLineWarps * DReg<64>::PPW * 2;
    default: return kLineWarps * DReg<128>::PPW * 2;
  }
}
int dline_reg_blocks(const DGrid& g) {
  const int W = dline_reg_positions(g.n1);
  return g.m2 * ((g.m3 + W - 1) / W);
}

template <typename T, int N>
static cudaError_t plane_go(const DPassArgs<T>& a, int fwd, cudaStream_t s) {
  const size_t smem = plane_reg_smem<T, N>();
  auto kern = fwd ? k_dplane_reg<T, N, 1> : k_dplane_reg<T, N, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(a.c * a.g.m1, a.BL), kPlaneWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int CC>
static cudaError_t line_go_c(const DPassArgs<T>& a, cudaStream_t s) {
  const size_t smem = line_reg_smem<T, N, CC>();
  cudaError_t e = cudaFuncSetAttribute(k_dline_reg<T, N, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_dline_reg<T, N, CC><<<dim3(dline_reg_blocks(a.g), a.BL), kLineWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int N>
static cudaError_t line_go(const DPassArgs<T>& a, cudaStream_t s) {
  if (a.c == 1) return line_go_c<T, N, 1>(a, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_dplane_reg(const DPassArgs<T>& a, int fwd, cudaStream_t s) {
  switch (a.g.n3) {
    case 8: return plane_go<T, 8>(a, fwd, s);
    case 16: return plane_go<T, 16>(a, fwd, s);
    case 32: return plane_go<T, 32>(a, fwd, s);
    case 64: return plane_go<T, 64>(a, fwd, s);
    case 128: return plane_go<T, 128>(a, fwd, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_dline_reg(const DPassArgs<T>& a, cudaStream_t s) {
  switch (a.g.n1) {
    case 8: return line_go<T, 8>(a, s);
    case 16: return line_go<T, 16>(a, s);
    case 32: return line_go<T, 32>(a, s);
    case 64: return line_go<T, 64>(a, s);
    case 128: return line_go<T, 128>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_dplane_reg<double>(const DPassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_dplane_reg<float>(const DPassArgs<float>&, int, cudaStream_t);
template cudaError_t launch_dline_reg<double>(const DPassArgs<double>&, cudaStream_t);
template cudaError_t launch_dline_reg<float>(const DPassArgs<float>&, cudaStream_t);

}  // namespace unocg
