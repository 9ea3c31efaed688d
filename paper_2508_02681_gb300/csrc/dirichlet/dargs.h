// Kernel arguments and launchers of the Dirichlet-BC solver (sine transform, Sec. 5.2.2 and the
// Dirichlet row of Table (fnocg-mode-selection-2d)); kernels in k_dirichlet.cu.
//
// Fields: real arrays [BL][c][N1][N2][N3] on the embedding grid of dgrid.cuh (BL = instances x
// loads): the free nodes plus zero boundary nodes.
// The sine transform along one axis of N voxels (N - 1 free nodes) is computed for two lines at
// once: line a in the real and line b in the imaginary part of one complex sequence of length
// 2N, odd-extended (z[0] = z[N] = 0, z[2N - j] = -z[j]); its DFT is -2i X_a + 2 X_b with
// X[k] = sum_j x[j] sin(pi (j+1)(k+1) / N), the unnormalized DST-I.  The normalization of the
// orthonormal transform, prod_a 2 / N_a over the pair T^T Q T, is folded into the stored Q.
#pragma once
#include <cuda_runtime.h>

#include "../cg.cuh"
#include "../common.cuh"
#include "dgrid.cuh"

namespace unocg {

// radix plan and twiddles W_{2 N_a}^m (m < 2 N_a, cplx<T>) of the three axes
struct DstTables {
  FftPlan p[3];
  const void* tw[3];
};

enum DPassMode {
  DP_FIRST = 0,  // axis 3, forward: (r -= alpha q, u += alpha p, ||r||_inf, stopping test) then DST
  DP_MID = 1,    // axis 2, either direction: DST in place
  DP_QMUL = 2,   // axis 1: DST, s_hat = Q r_hat, gamma = r.s, DST, beta
  DP_LAST = 3,   // axis 3, inverse: DST, p = s + beta p (or s written out)
  DP_MID1 = 4,   // axis 1 without the block multiply (two periodic axes: see k_dmixq)
};

template <typename T> struct DPassArgs {
  DGrid g;
  int c, BL, L;
  int lines;               // lines per block (axis 3) or positions per block (axes 1, 2)
  const T* src;            // DP_FIRST standalone input
  T* hat;                  // spectrum buffer (in place for DP_MID, DP_QMUL)
  T* out;                  // DP_LAST standalone output
  // CG fields (loop mode)
  T* r;
  const T* q;
  T* p;
  T* u;                    // solution (FP64 path) or its FP32 increment since the last fold
  const void* Q;           // unique entries [Bq][M1][M2][M3][C], type T (scaled, see above)
  long long q_inst_stride; // entries between instances (0: shared)
  CgScal* sc;
  Reduce red;
  LoopCtl ctl;
  int after_replace;       // DP_FIRST: check of the replaced pairs only, no update
  int standalone;          // no CG state: plain transform / apply
  DstTables t;
};

template <typename T> struct DKuArgs {
  DGrid g;
  int c, BL, L;
  const uint8_t* phase;    // [B][N1][N2][N3]
  Material mat;
  const T* p;              // direction (zero on the boundary nodes)
  T* q;                    // K p (rows of the boundary nodes are not used)
  CgScal* sc;
  Reduce red;
  int standalone;
};

// r = f - K u (FP64) for the pending pairs (replacement; into_r), or max |f - K u| into tmax
template <typename T> struct DResArgs {
  DGrid g;
  int c, BL, L;
  const uint8_t* phase;
  Material mat;
  const double* u64;
  const double* f64;
  T* r;                    // replacement target (nullptr: report only)
  CgScal* sc;
  int only_pending;
};

// Jacobi / unpreconditioned CG: update pass and direction pass
template <typename T> struct DJacArgs {
  DGrid g;
  int c, BL;
  T* r;
  const T* q;
  T* p;
  T* u;                    // as DPassArgs::u
  const T* invdiag;        // [B][c][N1][N2][N3] (zero on the boundary) or nullptr (none)
  int L;
  CgScal* sc;
  Reduce red;
  LoopCtl ctl;
  int after_replace;
};

struct DInitArgs {
  DGrid g;
  int c, L;
  const uint8_t* phase;
  Material mat;
  const double* loads;     // [L][dim]
  double* f64;             // [BL][c][N1][N2][N3]
  double* u64;
  void* u32;               // mixed precision: FP32 increment, zeroed (nullptr for FP64)
  void* r;                 // T: r = f
  void* p;                 // T: 0
  void* q;                 // T: 0
  int fp64;
};

struct DAvgArgs {
  DGrid g;
  int c, L;
  const uint8_t* phase;
  Material mat;
  const double* loads;
  const double* u64;
  double* out;             // [B][dim][L], zeroed by the caller, accumulated
};

struct DDiagArgs {
  DGrid g;
  int c;
  const uint8_t* phase;
  Material mat;
  void* invdiag;           // T [B][c][N1][N2][N3]
  int fp64;
};

size_t dst_smem_bytes(int N, int lines, int elem_bytes);
int dst_lines_for(int N, int elem_bytes, int cap);

template <typename T> cudaError_t launch_dpass(const DPassArgs<T>& a, int mode, cudaStream_t s);
// axes 3 and 2 of whole planes in one pass (fwd: DP_FIRST + DP_MID, else DP_MID + DP_LAST) when
// dplane_smem_bytes fits a block
size_t dplane_smem_bytes(const DGrid& g, int elem_bytes);
template <typename T> cudaError_t launch_dplane(const DPassArgs<T>& a, int fwd, cudaStream_t s);
// register-resident versions (k_dirichlet_reg.cu): planes with N2 = N3 in {8, ..., 128}; axis 1
// with the block multiply for c = 1 and N1 in {8, ..., 128}
bool dplane_reg_ok(const DGrid& g);
bool dline_reg_ok(const DGrid& g, int c, int elem_bytes);
int dline_reg_blocks(const DGrid& g);
template <typename T> cudaError_t launch_dplane_reg(const DPassArgs<T>& a, int fwd, cudaStream_t s);
template <typename T> cudaError_t launch_dline_reg(const DPassArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_dku(const DKuArgs<T>& a, cudaStream_t s);
// two periodic axes pa < pb: s_hat = B Q B r_hat on the separable Hartley spectrum (k_dmixq)
int dmixq_blocks(const DGrid& g, int pa, int pb);
template <typename T> cudaError_t launch_dmixq(const DPassArgs<T>& a, int pa, int pb, cudaStream_t s);
template <typename T> cudaError_t launch_dres(const DResArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_djac(const DJacArgs<T>& a, int part, cudaStream_t s);
cudaError_t launch_dinit(const DInitArgs& a, int BL, cudaStream_t s);
// mixed precision: rref (the f64 field of DResArgs, f - K u64) -= K u32 in float pairs on the
// free nodes, r = rref when a.r is set, max |rref| into rmax (into_rmax) or tmax
cudaError_t launch_dreplace(const DResArgs<float>& a, const float* u32, int into_rmax, cudaStream_t s);
// mixed precision: u64 += u32, u32 = 0 for the pending (only_pending) or all pairs
cudaError_t launch_dfold(const DGrid& g, int c, int BL, double* u64, float* u32, const CgScal* sc, int only_pending,
                         cudaStream_t s);
cudaError_t launch_davg(const DAvgArgs& a, int B, cudaStream_t s);
cudaError_t launch_ddiag(const DDiagArgs& a, int B, cudaStream_t s);
int dku_blocks(const DGrid& g, int c);
int djac_blocks(const DGrid& g);
cudaError_t launch_dscatter(const DGrid& g, int cnt, const double* src, double* dst, cudaStream_t s);
cudaError_t launch_dgather(const DGrid& g, int cnt, const double* src, double* dst, cudaStream_t s);
int dpass_blocks(const DGrid& g, int c, int mode, int lines);

}  // namespace unocg
