// Kernel argument blocks and host launchers shared by the kernel translation units and the
// C ABI driver.
#pragma once
#include "common.cuh"
#include "cg.cuh"

namespace unocg {
// Launch with the programmatic-stream-serialization attribute (the kernel must call pdl_wait()
// before reading what earlier kernels wrote).  UNOCG_PDL=0 at build time launches plainly.
#ifndef UNOCG_PDL
#define UNOCG_PDL 1
#endif
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                     cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = UNOCG_PDL ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace unocg

namespace unocg {

// ---------------------------------------------------------------- FFT passes
template <typename T> struct PlaneFwdArgs {
  Grid g;
  int c, BL;
  T* r;                 // CG mode: residual, updated in place r <- r - alpha p
  const T* p;           // CG mode: K d of the previous iteration
  const T* src;         // standalone mode: input fields [BL][c][n]
  cplx<T>* hat;         // output: axes-2/3 spectra [BL][c][n1][n2][n3h]
  CgScal* sc;           // CG mode
  FftTables ft;
  unsigned int* ticket;
  LoopCtl ctl;
  int after_replace;    // CG mode: residual was just replaced (no update, alpha = 0)
  int standalone;       // transform src only (no CG bookkeeping)
  int rows;             // 0: whole planes (axes 3 and 2); else chunks of `rows` rows, axis 3 only
};

template <typename T, typename QT> struct LineArgs {
  Grid g;
  int c, BL, L;         // L = loads per instance (weights may be per instance)
  const cplx<T>* hat;   // axes-2/3 spectra of r  [BL][c][n1][M], M = n2*n3h
  cplx<T>* shat;        // output: P applied, axis 1 inverted again  [BL][c][n1][M]
  const cplx<T>* ghat;  // backward mode: spectra of the upstream gradient
  const QT* Q;          // unique block entries [Bq][n1][M][C]
  long long q_inst_stride;  // entries per instance (0 = shared)
  double scale;         // 1 / n (unnormalized transform pair)
  CgScal* sc;
  Reduce red;
  FftTables ft;
  int tb;               // positions per block
  int flexible;
  int standalone;       // 1: apply only (no CG bookkeeping)
  float* gq;            // backward: dL/dv accumulated over the batch [n1][M][C] (float)
};

template <typename T> struct PlaneInvArgs {
  Grid g;
  int c, BL;
  const cplx<T>* shat;  // [BL][c][n1][n2][n3h]
  T* d;                 // CG mode: search direction, d <- s + beta d
  T* u;                 // CG mode: solution, u <- u + alpha d_old
  T* dst;               // standalone: output s
  CgScal* sc;
  FftTables ft;
  int standalone;
  int rows;             // 0: whole planes; else chunks of `rows` rows, axis 3 only (axis 2 done)
  cplx<T>* cols_out;    // rows mode: the axis-2 pass writes here (null: in place over shat), so
                        // that shat keeps s_hat for the r . s_old term of the flexible variant
};

// In-place FFT along axis 2 of every (field, i1) plane, for planes too large for one block.
template <typename T> struct ColArgs {
  Grid g;
  int c, BL;
  cplx<T>* data;        // [BL][c][n1][n2][n3h]
  const CgScal* sc;     // skip finished pairs (null: all)
  FftTables ft;
  int only_pending;     // CG after a replacement: only the pairs just replaced
  cplx<T>* out;         // destination, same layout (null: in place)
};

// ---------------------------------------------------------------- material / stencil

template <typename T> struct StencilArgs {
  Grid g;
  int c, BL, L;
  const uint8_t* phase; // [B][n]
  Material mat;
  const T* d;           // [BL][c][n]
  T* p;                 // [BL][c][n]
  CgScal* sc;
  Reduce red;
  int standalone;       // no CG bookkeeping (operator apply)
  int ku_tma;           // FP32 thermal: 1 + index into kKuTmaShapes of the TMA-staged kernel,
                        // 9 + index of the vector march, 0 none
  int* err;             // bounded waits: flag raised on expiry (null: none)
  long long spin_limit; // SM clock cycles a wait may take
};

// Tile shape of the TMA-staged thermal K d (k_ku_tma.cu): node rows per tile (N3 / 4 threads
// per row) and node planes per block.
struct KuTmaShape {
  int rows, planes;
};
constexpr int kKuTmaNumShapes = 8;
extern const KuTmaShape kKuTmaShapes[kKuTmaNumShapes];
int ku_tma_threads(const Grid& g, KuTmaShape s);
bool ku_tma_supported(const Grid& g, int c, KuTmaShape s);
int ku_tma_blocks_x(const Grid& g, KuTmaShape s);
cudaError_t launch_ku_tma(const StencilArgs<float>& a, KuTmaShape s, int* err, long long spin_limit, cudaStream_t st);
// the same stencil as a register march over node planes read straight from global memory
// (k_ku_vec.cu), same tile shapes
bool ku_vec_supported(const Grid& g, int c, KuTmaShape s);
int ku_vec_blocks_x(const Grid& g, KuTmaShape s);
cudaError_t launch_ku_vec(const StencilArgs<float>& a, KuTmaShape s, cudaStream_t st);
// elastic K d element by element with element pairs in packed FP32x2 arithmetic (k_ku_el2.cu);
// N3 even, same tiles (and blocks per launch) as the scalar element kernel
bool ku_el2_supported(const Grid& g);
cudaError_t launch_ku_el2(const StencilArgs<float>& a, cudaStream_t st);

// 256 x 256 plane passes on two-CTA clusters, FP32 (k_plane_cl.cu)
bool plane_cl_ok(const Grid& g);
cudaError_t launch_plane_fwd_cl(const PlaneFwdArgs<float>& a, cudaStream_t s);
cudaError_t launch_plane_inv_cl(const PlaneInvArgs<float>& a, cudaStream_t s);
// inverse axis-3 row pass of 256 x 256 FP32 planes with the CG updates (after the column pass)
bool rows_inv256_ok(const Grid& g);
cudaError_t launch_rows_inv256(const PlaneInvArgs<float>& a, cudaStream_t s);
// forward axis-3 row pass of the same planes, fused with r <- r - alpha p (before the column pass)
cudaError_t launch_rows_fwd256(const PlaneFwdArgs<float>& a, cudaStream_t s);

// TMA-staged axis-1 pass of the mixed-precision loop, c = 1 and 3 (k_line_tma.cu)
bool line_tma_supported(const Grid& g, int c);
int line_tma_blocks_x(const Grid& g);
template <typename T, typename QT> struct LineArgs;
cudaError_t launch_line_tma(const LineArgs<float, __nv_bfloat16>& a, int* err, long long spin_limit, cudaStream_t st);
// the same for c = 3, N1 in {16, 32, 64} (k_line_tma3.cu); launch_line_tma forwards c = 3 here
bool line_tma3_supported(const Grid& g);
cudaError_t launch_line_tma3(const LineArgs<float, __nv_bfloat16>& a, int* err, long long spin_limit, cudaStream_t st);
// the same pass for c = 1 as a persistent pipeline of TMA tiles (k_line_tp.cu): N1 = 64, 128, 256
bool line_tp_supported(const Grid& g);
cudaError_t launch_line_tp(const LineArgs<float, __nv_bfloat16>& a, int* err, long long spin_limit, int sm_count,
                           cudaStream_t st);

template <typename T> struct InitArgs {
  Grid g;
  int c, L;
  const uint8_t* phase;
  Material mat;
  const double* loads;  // [L][3 or 6]
  T* r; T* u; T* d; T* p;   // any may be null
  double* u64;          // optional FP64 solution (zeroed)
  double* f64;          // optional FP64 right-hand side output
};

template <typename T> struct TrueResArgs {
  Grid g;
  int c, L;
  const uint8_t* phase;
  Material mat;
  const double* loads;
  const double* u64;    // [BL][c][n]
  const double* f64;    // optional: the FP64 right-hand side [BL][c][n] (else recomputed)
  T* r;                 // optional: store f - K u
  CgScal* sc;
  int only_pending;     // only (instance, load) with need_replace set
  int require_started;
  int into_rmax;        // accumulate into rmax_bits (replacement) instead of tmax_bits (report)
};

// Mixed-precision residual replacement: rref <- rref - K (u32 + alpha d) with FP64 accuracy
// (float-pair arithmetic from the FP32 fields), r = rref in FP32, max |rref| per pair.  rref is
// the FP64 residual f - K u64 of the FP64 solution (f before the first replacement); the fold
// u64 += u32 + alpha d follows.
struct ReplaceArgs {
  Grid g;
  int c, L;
  const uint8_t* phase;
  Material mat;
  const float* u32;     // [BL][c][n] increment since the last replacement
  const float* d;       // [BL][c][n] search direction of the pending step alpha d
  double* rref;         // [BL][c][n] FP64 residual, updated in place
  float* r;             // optional: the FP32 residual of the iteration
  CgScal* sc;
  int only_pending;     // only pairs with need_replace set
  int into_rmax;        // accumulate into rmax_bits (replacement) or tmax_bits (final report)
};
cudaError_t launch_replace(const ReplaceArgs& a, int BL, cudaStream_t s);

template <typename T> struct FoldArgs {
  int c;
  long long n;
  double* u64;
  T* u32;               // optional increment (mixed precision)
  const T* d;
  CgScal* sc;
  int only_pending;
  double* part;         // k_final: per-block sums for the mean
};

template <typename T> struct JacArgs {
  int c, BL, L;
  long long n;
  T* r; const T* p; T* d; T* u;
  const T* invdiag;     // [B][c][n] or null (no preconditioner)
  CgScal* sc;
  Reduce red;
  LoopCtl ctl;
  int after_replace;
};

template <typename T> struct DiagArgs {
  Grid g;
  int c;
  const uint8_t* phase;
  Material mat;
  T* invdiag;
};

struct AvgArgs {
  Grid g;
  int c, L;
  const uint8_t* phase;
  Material mat;
  const double* loads;
  const double* u64;    // [B][L][c][n]
  double* part;
};

// launchers (k_stencil.cu)
template <typename T> cudaError_t launch_ku(const StencilArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_init(const InitArgs<T>& a, int BL, cudaStream_t s);
template <typename T> cudaError_t launch_true_res(const TrueResArgs<T>& a, int BL, cudaStream_t s);
template <typename T> cudaError_t launch_fold(const FoldArgs<T>& a, int BL, cudaStream_t s);
template <typename T> cudaError_t launch_final(const FoldArgs<T>& a, int BL, int nparts, cudaStream_t s);
template <typename T> cudaError_t launch_jac(const JacArgs<T>& a, int which, cudaStream_t s);
template <typename T> cudaError_t launch_invdiag(const DiagArgs<T>& a, int B, cudaStream_t s);
cudaError_t launch_zero_mean(double* u, const double* part, int nparts, int c, long long n, int BL, cudaStream_t s);
cudaError_t launch_average(const AvgArgs& a, int B, double* out, cudaStream_t s);
cudaError_t launch_sens(const AvgArgs& a, int B, double* out, cudaStream_t s);
cudaError_t launch_interleave(const double* src, double* dst, int c, long long n, cudaStream_t s);
int node_blocks_x(const Grid& g);
int ku_blocks_x(const Grid& g, int c);  // blocks of one K d launch per (instance, load)
int ku_tasks_x(const Grid& g, int c);   // K d tasks of the persistent kernel per (instance, load)
int jac_blocks_x(long long m, int BL);
int sens_blocks_x(const Grid& g);

// launchers (k_fft.cu)
template <typename T> cudaError_t launch_plane_fwd(const PlaneFwdArgs<T>& a, cudaStream_t s);
template <typename T, typename QT> cudaError_t launch_line(const LineArgs<T, QT>& a, int backward, cudaStream_t s);
template <typename T> cudaError_t launch_plane_inv(const PlaneInvArgs<T>& a, cudaStream_t s);
int line_blocks_x(const Grid& g, int c, int elem_bytes);
// register-FFT passes for power-of-two axes (k_fft_reg.cu); the *_ok tests say whether they
// apply to a grid (plane: N2 = N3 in {32, 64, 128}; axis 1: 16..256)
bool plane_reg_ok(const Grid& g, int elem_bytes);
bool line_reg_ok(const Grid& g, int c, int elem_bytes);
int line_reg_blocks_x(const Grid& g);
template <typename T> cudaError_t launch_plane_fwd_reg(const PlaneFwdArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_plane_inv_reg(const PlaneInvArgs<T>& a, cudaStream_t s);
template <typename T, typename QT> cudaError_t launch_line_reg(const LineArgs<T, QT>& a, cudaStream_t s);
// dynamic shared memory of the axis-1 pass (mode 2: backward, four line buffers)
size_t line_smem_bytes(const Grid& g, int c, int elem_bytes, int mode);
bool plane_fits(const Grid& g, int elem_bytes);
int plane_rows(const Grid& g, int elem_bytes);  // 0 if whole planes fit, else rows per block
bool grid_supported(const Grid& g, int elem_bytes);
template <typename T> cudaError_t launch_cols(const ColArgs<T>& a, int dir, cudaStream_t s);
// axis-2 pass of 256 x 256 FP32 planes, two columns a warp in registers (k_plane_cl.cu)
cudaError_t launch_cols_reg256(const ColArgs<float>& a, int dir, cudaStream_t s);

}  // namespace unocg
