// Shared device-side definitions of the UNO-CG kernels: complex helpers, per-solve CG
// scalars, problem descriptors and the last-block reduction pattern.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace unocg {

// ---------------------------------------------------------------- complex numbers
template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T x, T y) {
  cplx<T> r; r.x = x; r.y = y; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i (forward) / +i (inverse)
template <int DIR, typename C> __device__ __forceinline__ C cmul_mi(C a) {
  C r;
  if (DIR < 0) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; }
  return r;
}

// ---------------------------------------------------------------- CG state per (instance, load)
struct CgScal {
  double gamma;       // r . s of the current iteration
  double gamma_prev;  // r . s of the previous iteration
  double alpha;       // step width pending for the next residual / solution update
  double beta;        // search-direction coefficient
  double rs_old;      // r_{m+1} . s_m (flexible variant)
  double r0max;       // ||r_0||_inf
  double rmax;        // ||r||_inf of the latest residual
  double true_res;    // ||f - K u||_inf / ||f||_inf (FP64) at the latest check
  double rrep;        // ||r||_inf right after the latest replacement (r_0 before any)
  unsigned long long rmax_bits;  // running max of |r| as ordered bits (non-negative doubles)
  unsigned long long tmax_bits;  // running max of |f - K u| (true residual kernel)
  int iters;
  int done;
  int status;         // 0 ok, UNOCG_ERR_* when done
  int need_replace;   // residual replacement requested (mixed precision)
  int started;        // r0max recorded
  int just_replaced;  // the last residual check followed a replacement of this pair
  int rep_iter;       // iteration count at the latest replacement
  int pad;
};

// ---------------------------------------------------------------- problem descriptor
struct Grid {
  int n1, n2, n3, n3h;      // n3h = n3/2 + 1
  long long n;              // nodes per field
  long long nh;             // half-grid modes per field
  double h;                 // voxel edge
  double h12;               // h / 12 (thermal stencil scale)
  float hf, h12f;           // the same in FP32 (no FP64 arithmetic on per-node paths)
};
__host__ __device__ inline void grid_scales(Grid& g) {
  g.h12 = g.h / 12.0;
  g.hf = (float)g.h;
  g.h12f = (float)g.h12;
}
template <typename T> __device__ __forceinline__ T grid_h(const Grid& g);
template <> __device__ __forceinline__ float grid_h<float>(const Grid& g) { return g.hf; }
template <> __device__ __forceinline__ double grid_h<double>(const Grid& g) { return g.h; }
template <typename T> __device__ __forceinline__ T grid_h12(const Grid& g);
template <> __device__ __forceinline__ float grid_h12<float>(const Grid& g) { return g.h12f; }
template <> __device__ __forceinline__ double grid_h12<double>(const Grid& g) { return g.h12; }

// ---------------------------------------------------------------- dot-product accumulation
// Per-thread partial sums of the CG dot products.  FP64 fields accumulate in FP64.  FP32 fields
// accumulate in an error-free float-float pair (products split exactly by FMA, sums by TwoSum):
// about 44 significant bits on the FP32 pipes, converted to FP64 once per thread for the FP64
// block and grid reductions (GB300's FP64 pipe is far too narrow for per-element FP64 work).
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(hi, x);
    const float bp = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    hi = t;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Radix plan of one transform length.
struct FftPlan {
  int N;
  int nst;
  int radix[12];
};

struct FftTables {
  FftPlan p1, p2, p3h;          // axis 1 (N1), axis 2 (N2), half axis 3 (N3/2)
  const void* tw1;              // W_{N1}^m, m < N1    (cplx<T>)
  const void* tw2;              // W_{N2}^m
  const void* tw3h;             // W_{N3/2}^m
  const void* tw3;              // W_{N3}^m, m < N3 (real-to-complex post-processing)
};

// Per-instance phase table: m64/m32[(b * n_phases + p) * 2 + {0,1}] = (kappa, 0) or (lambda, mu).
struct Material {
  int n_phases;
  const double* m64;
  const float* m32;
};

template <typename T> __device__ __forceinline__ const T* mat_ptr(const Material& m);
template <> __device__ __forceinline__ const double* mat_ptr<double>(const Material& m) { return m.m64; }
template <> __device__ __forceinline__ const float* mat_ptr<float>(const Material& m) { return m.m32; }

// Copy the table of instance b to shared memory (n_phases <= 256).
template <typename T> __device__ __forceinline__ void load_material(T* mt, const Material& m, int b) {
  const T* src = mat_ptr<T>(m) + (long long)b * m.n_phases * 2;
  for (int i = threadIdx.x; i < 2 * m.n_phases; i += blockDim.x) mt[i] = src[i];
}

// Counters and partial sums of one kernel "site" (reductions finished by the last block).
struct Reduce {
  double* part;                 // [BL][gridDim.x][nv]
  unsigned int* ticket;         // one counter, reset by the last block
};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double bits_to_double(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// Block-wide sum of one double; result valid in thread 0.  Uses `sh` (>= 32 doubles).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}
// Block-wide sum of per-thread accumulators; result valid in thread 0.  The float-float pairs are
// combined with FP32 operations (TwoSum) and converted to FP64 by one warp only.
__device__ __forceinline__ double block_sum_acc(const DotAcc<double>& a, double* sh) { return block_sum(a.value(), sh); }
__device__ __forceinline__ double block_sum_acc(DotAcc<float> a, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, a.hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a.add(oh);
    a.lo = __fadd_rn(a.lo, ol);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = a.value();
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  }
  return s;
}

__device__ __forceinline__ double block_max_f(float v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  }
  return s;
}
__device__ __forceinline__ double block_max_t(float v, double* sh) { return block_max_f(v, sh); }
__device__ __forceinline__ double block_max_t(double v, double* sh) { return block_max(v, sh); }

// Stream order of the `_dev` entry points: they enqueue on the caller's stream (NULL: the
// legacy default stream), after the work already enqueued on the context's stream, and the
// context's later work runs after theirs.  Each direction is one event record + wait; nothing
// is added while either stream captures a graph (the capture then owns the ordering).
static inline bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    (void)cudaGetLastError();  // e.g. the legacy stream while another stream captures globally
    return true;
  }
  return st != cudaStreamCaptureStatusNone;
}
static inline cudaError_t order_after(cudaEvent_t* ev, cudaStream_t from, cudaStream_t to) {
  if (from == to || stream_capturing(from) || stream_capturing(to)) return cudaSuccess;
  if (!*ev) {
    cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaEventRecord(*ev, from);
  return e == cudaSuccess ? cudaStreamWaitEvent(to, *ev, 0) : e;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start while the kernel
// before it in the stream is still running.  pdl_wait() blocks until that kernel has completed
// and its memory is visible: call it before touching anything the previous kernels wrote.
// pdl_trigger() lets the next kernel start launching (its blocks then wait in pdl_wait()).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Returns true in every thread of the block that arrives last at `ticket` (over all blocks
// of the grid).  Callers write their partials before and read all partials after.
// Thread 0 publishes its own earlier writes (the block's partials) with a release increment
// of the ticket; the last block acquires all of them before reading.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    unsigned t;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(t) : "l"(ticket) : "memory");
    am_last = (t == total - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

// Sum of `count` partials p[0], p[stride], ... by one warp: each lane adds a fixed strided subset
// in order, then a fixed shuffle tree (deterministic).  Result in every lane.
__device__ __forceinline__ double warp_sum_partials(const double* p, int count, int stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int x = lane; x < count; x += 32) s += ld_cg(p + (long long)x * stride);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

}  // namespace unocg
