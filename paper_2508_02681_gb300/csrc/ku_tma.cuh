// Thermal K d (Sec. 4.1, "matrix-free implementations" of Sec. 5.5) on node planes staged in
// shared memory by the tensor-memory accelerator (TMA), FP32 fields.
//
// Work layout.  A block owns a tile of TY node rows (i2) over the whole i3 extent of the grid
// and marches along i1 over CZ node planes.  Each thread holds NV = 4 consecutive nodes of one
// row (one 16-byte vector).  Node plane q of the tile is brought into a ring of shared-memory
// buffers by three TMA box copies: the TY rows of the tile and, as one-row boxes, the two halo
// rows i2_0 - 1 and i2_0 + TY taken modulo N2 (the periodic wrap along axis 2).  The element
// phase labels of plane e (rows i2_0 - 1 .. i2_0 + TY - 1) arrive the same way into a second
// ring and are converted once per plane into conductivities (scaled by h / 12).  Along axis 3
// the halo values come from the neighbouring threads of the row by warp shuffles (a row of
// N3 <= 128 nodes lies in one warp, where the shuffle index wraps periodically; for N3 = 256 the
// two lanes at the warp edges read their neighbour from shared memory).  Along axis 1 every
// thread keeps the 3 x 3 rows of the node planes z - 1, z, z + 1 and the conductivities of
// element planes z - 1 and z in registers, so each step reads one new node plane and one new
// element plane.  One thread issues the copies; completion is tracked by mbarriers with
// transaction counts.  Every wait is bounded: on expiry the block raises the context's timeout
// flag, waits (bounded again) for its copies still in flight and returns.
//
// Stencil.  With k_{o1 o2 o3} the scaled conductivity of the element (z - o1, i2 - o2, i3 - o3)
// around node (z, i2, i3) and d(s1, s2, s3) the neighbour at offset s:
//   p = 4 (sum_o k_o) d(0,0,0)
//       - sum_{s2,s3 = +-1} (k_{0 o2 o3} + k_{1 o2 o3}) d(0, s2, s3)
//       - sum_{s1,s3 = +-1} (k_{o1 0 o3} + k_{o1 1 o3}) d(s1, 0, s3)
//       - sum_{s1,s2 = +-1} (k_{o1 o2 0} + k_{o1 o2 1}) d(s1, s2, 0)
//       - sum_{s = +-1} k_{o1 o2 o3} d(s1, s2, s3)
// with o_a = 1 where s_a = -1 (the elements on the side of the neighbour); face neighbours do
// not couple for trilinear bricks.  The pair sums are formed once per element column and
// shared by the nodes of a thread.
#pragma once
#include <cuda.h>
#include "stencil.cuh"
#include "tma.cuh"

namespace unocg {

// ---------------------------------------------------------------- arguments
// Tensor maps of one launch: d as [BL][N1][N2][N3] FP32, the phase labels as [B][N1][N2][N3] u8,
// each with a TY-row box and a one-row box (both the whole N3 extent).
struct alignas(64) KuTmaMaps {
  CUtensorMap d_rows, d_row, ph_rows, ph_row;
};

struct KuTmaArgs {
  StencilArgs<float> a;
  int ty;            // node rows per tile (divides N2)
  int cz;            // node planes per block
  int tiles;         // blocks per (instance, load): (N2 / ty) * ceil(N1 / cz)
  int* err;          // timeout flag (null: none)
  long long spin_limit;
};

constexpr int KT_NV = 4;         // nodes per thread along i3
constexpr int KT_DS = 4;         // node-plane ring depth (a power of two: cheap slot and phase)
constexpr int KT_PS = 3;         // phase-plane ring depth
constexpr int KT_UNROLL = 6;     // steps per loop body (the register window rotates with period 6)

// Dynamic shared memory of one block: node-plane ring, two conductivity planes, phase ring
// (each buffer a multiple of 128 bytes), plus 128 bytes of alignment slack.
__host__ __device__ inline size_t kt_dslot_bytes(int ty, int n3) { return (size_t)(ty + 2) * n3 * sizeof(float); }
__host__ __device__ inline size_t kt_kslot_bytes(int ty, int n3) { return (size_t)(ty + 1) * n3 * sizeof(float); }
__host__ __device__ inline size_t kt_pslot_bytes(int ty, int n3) { return (((size_t)(ty + 1) * n3) + 127) / 128 * 128; }
__host__ __device__ inline size_t kt_smem_bytes(int ty, int n3) {
  return 128 + KT_DS * kt_dslot_bytes(ty, n3) + 2 * kt_kslot_bytes(ty, n3) + KT_PS * kt_pslot_bytes(ty, n3);
}

}  // namespace unocg
