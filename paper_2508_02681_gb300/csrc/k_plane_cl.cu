// Transform passes of 256 x 256 planes (axes 2 and 3) of the mixed-precision loop (Algorithm 2:
// forward and inverse unitary transform around the block multiply; FP32).  A half-spectrum plane
// of 256 rows x 129 complex FP32 values (264 KB) exceeds one block's shared memory, so a
// transform is either two passes through global memory or one pass over two blocks.
//
// Two passes (the default): register row passes (k_rows_fwd256 / k_rows_inv256: 4 rows a warp,
// the CG updates fused) and a register column pass (k_cols_reg256: two columns a warp, read
// straight into the line FFT's distribution, no block barrier).
//
// One pass on thread-block clusters of two CTAs (selected per transform): the two CTAs split the
// plane by rows for the axis-3 transforms and by columns for the axis-2 transforms, and move the
// values between the two splits through distributed shared memory: a CTA writes each row result
// into the shared memory of the CTA that owns its column (rank 0: columns 0..64, rank 1:
// 65..128), with one cluster barrier between the phases.
//
//   k_plane_fwd_cl: r <- r - alpha p, ||r||_inf, rows (axis 3, r2c), exchange, columns (axis 2),
//                   r_hat written; the last block performs the residual check.
//   k_plane_inv_cl: columns (inverse axis 2) from s_hat, exchange, rows (c2r),
//                   u <- u + alpha d_old, d <- s + beta d_old.
//
// Every phase uses the register-resident line FFTs of fft_reg.cuh (rows: 128-point half-length
// lines, 8 threads each; columns: 256-point lines, 16 threads each).
#include <cooperative_groups.h>
#include "kargs.h"
#include "fft_reg.cuh"

namespace cgr = cooperative_groups;

namespace unocg {

namespace {
// L2 prefetch of the 128-byte line holding p
__device__ __forceinline__ void pf_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

constexpr int PN = 256, PNh = 128, Pn3h = 129;
constexpr int PG3 = RegSplit<PNh>::G, PV3 = RegSplit<PNh>::V, PRPW = 32 / PG3;  // rows: 8 threads, 16 values
constexpr int PG2 = RegSplit<PN>::G, PV2 = RegSplit<PN>::V, PCW = 32 / PG2;     // columns: 16 threads, 16 values
constexpr int PNW = 16;                          // warps per CTA
// columns of rank r: [pcol0(r), pcol0(r) + pncol(r)) -- rank 0: 0..64, rank 1: 65..128
__host__ __device__ constexpr int pcol0(int r) { return r ? 65 : 0; }
__host__ __device__ constexpr int pncol(int r) { return r ? 64 : 65; }
constexpr int PCP = 66;                          // pitch of the column buffer (column 65: scratch of the idle lane)
constexpr int PRS = 130;                         // pitch of a row scratch (129 values)
constexpr int PRP = 132;                         // pitch of the inverse row buffer
constexpr size_t kTwBytes = (size_t)(PNh + PN + PN) * sizeof(float2);
constexpr size_t kFwdSmem = (size_t)PN * PCP * sizeof(float2) + (size_t)PNW * PRPW * PRS * sizeof(float2) + kTwBytes;
constexpr size_t kInvSmem = (size_t)PNh * PRP * sizeof(float2) + (size_t)PNW * PCW * PN * sizeof(float2) + kTwBytes;
}  // namespace

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PNW * 32) k_plane_fwd_cl(PlaneFwdArgs<float> a) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  cgr::cluster_group cluster = cgr::this_cluster();
  const int rank = (int)cluster.block_rank();
  C* colbuf = reinterpret_cast<C*>(smem_raw);                 // [256 rows][PCP] this rank's columns
  C* rowscr = colbuf + PN * PCP;                               // [warp][PRPW rows][PRS]
  C* tw3h = rowscr + PNW * PRPW * PRS;
  C* tw2 = tw3h + PNh;
  C* tw3 = tw2 + PN;
  C* colbuf_peer = cluster.map_shared_rank(colbuf, 1 - rank);
  load_tw_reg<float>(tw3h, a.ft.tw3h, PNh);
  load_tw_reg<float>(tw2, a.ft.tw2, PN);
  load_tw_reg<float>(tw3, a.ft.tw3, PN);
  pdl_wait();
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plane_id = blockIdx.x >> 1;
  const int comp = plane_id / a.g.n1, i1 = plane_id - comp * a.g.n1;
  const long long field = (long long)bl * a.c + comp;
  const long long base = (field * a.g.n1 + i1) * (long long)(PN * PN);
  bool active = true;
  double alpha = 0.0;
  if (!a.standalone) {
    const CgScal& st = a.sc[bl];
    active = !st.done && (!a.after_replace || st.need_replace);
    alpha = a.after_replace ? 0.0 : st.alpha;
  }
  __syncthreads();
  float lmax = 0.f;
  if (active) {  // the same for both CTAs of the cluster (one plane, one (instance, load))
    const float al = (float)alpha;
    const bool upd = alpha != 0.0;
    // the rows of this warp's second row group are requested into L2 now (their loads follow
    // the first group's transform)
    if (!a.standalone && warp + PNW < PNh / PRPW) {
      const int row = rank * PNh + (warp + PNW) * PRPW + lane / PG3;
      const long long o = base + (long long)row * PN + (lane % PG3) * 32;
      pf_l2(a.r + o);
      pf_l2(a.p + o);
    }
    // ---- rows of this rank: axis 3 (half-length complex lines of 128 points), r2c
    for (int rg = warp; rg < PNh / PRPW; rg += PNW) {
      const int rl = rg * PRPW + lane / PG3, g = lane % PG3;
      const int row = rank * PNh + rl;
      C v[PV3];
      if (a.standalone) {
        const C* src = reinterpret_cast<const C*>(a.src + base) + row * PNh;
#pragma unroll
        for (int n1 = 0; n1 < PV3; ++n1) v[n1] = src[g + PG3 * n1];
      } else {
        C* r = reinterpret_cast<C*>(a.r + base) + row * PNh;
        const C* p = reinterpret_cast<const C*>(a.p + base) + row * PNh;
        C q[PV3];
#pragma unroll
        for (int n1 = 0; n1 < PV3; ++n1) {
          v[n1] = r[g + PG3 * n1];
          q[n1] = p[g + PG3 * n1];
        }
        if (upd) {
#pragma unroll
          for (int n1 = 0; n1 < PV3; ++n1) {
            v[n1].x -= al * q[n1].x;
            v[n1].y -= al * q[n1].y;
            r[g + PG3 * n1] = v[n1];
          }
        }
#pragma unroll
        for (int n1 = 0; n1 < PV3; ++n1) lmax = fmaxf(lmax, fmaxf(fabsf(v[n1].x), fabsf(v[n1].y)));
      }
      C* rs = rowscr + (warp * PRPW + lane / PG3) * PRS;
      fft_dist_a<PNh, -1>(v, g, rs, 1, tw3h);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < PV3 / PG3; ++j)
#pragma unroll
        for (int k2 = 0; k2 < PG3; ++k2) rs[scat_index<PNh>(g, j, k2)] = v[j * PG3 + k2];
      __syncwarp();
      for (int k = g; k <= PNh / 2; k += PG3) r2c_pair<float>(rs, k, PNh, tw3);
      __syncwarp();
      // each value to the column owner: rank 0 columns 0..64, rank 1 columns 65..128
      for (int k3 = g; k3 < Pn3h; k3 += PG3) {
        const int own = k3 < pcol0(1) ? 0 : 1;
        C* dst = own == rank ? colbuf : colbuf_peer;
        dst[row * PCP + (k3 - pcol0(own))] = rs[k3];
      }
      __syncwarp();
    }
  }
  cluster.sync();  // both ranks' row values are in place (also orders the shared-memory writes)
  if (active) {
    // ---- columns of this rank: axis 2 (256-point lines)
    const int ncol = pncol(rank), ncg = (ncol + PCW - 1) / PCW;
    C* out = a.hat + (field * a.g.n1 + i1) * (long long)(PN * Pn3h) + pcol0(rank);
    for (int cg = warp; cg < ncg; cg += PNW) {
      const int col = cg * PCW + lane % PCW, g = lane / PCW;
      C v[PV2];
#pragma unroll
      for (int n1 = 0; n1 < PV2; ++n1) v[n1] = colbuf[(g + PG2 * n1) * PCP + col];
      fft_dist_a<PN, -1>(v, g, colbuf + col, PCP, tw2);
      // the column's spectrum back into its own slots of the column buffer (row k2 of column
      // col); the idle lane's padding column 65 is not written out
      __syncwarp();
#pragma unroll
      for (int j = 0; j < PV2 / PG2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < PG2; ++k2) colbuf[scat_index<PN>(g, j, k2) * PCP + col] = v[j * PG2 + k2];
      __syncwarp();
    }
    __syncthreads();
    // whole rows of this rank's columns: contiguous runs of ncol values in r_hat
    for (int k2 = warp; k2 < PN; k2 += PNW) {
      const C* src = colbuf + k2 * PCP;
      C* dst = out + (long long)k2 * Pn3h;
      for (int c = lane; c < ncol; c += 32) dst[c] = src[c];
    }
  }
  pdl_trigger();
  if (a.standalone) return;
  const double bmax = block_max_t(lmax, red_sh);
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bmax);
  if (last_block(a.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.ticket = 0u;
  }
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PNW * 32) k_plane_inv_cl(PlaneInvArgs<float> a) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cgr::cluster_group cluster = cgr::this_cluster();
  const int rank = (int)cluster.block_rank();
  C* rowbuf = reinterpret_cast<C*>(smem_raw);                 // [128 rows of this rank][PRP]
  C* colscr = rowbuf + PNh * PRP;                              // [warp][256 slots][PCW columns]
  C* tw3h = colscr + PNW * PCW * PN;
  C* tw2 = tw3h + PNh;
  C* tw3 = tw2 + PN;
  C* rowbuf_peer = cluster.map_shared_rank(rowbuf, 1 - rank);
  load_tw_reg<float>(tw3h, a.ft.tw3h, PNh);
  load_tw_reg<float>(tw2, a.ft.tw2, PN);
  load_tw_reg<float>(tw3, a.ft.tw3, PN);
  pdl_wait();
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plane_id = blockIdx.x >> 1;
  const int comp = plane_id / a.g.n1, i1 = plane_id - comp * a.g.n1;
  const long long field = (long long)bl * a.c + comp;
  const long long base = (field * a.g.n1 + i1) * (long long)(PN * PN);
  // a finished (instance, load): both CTAs of the cluster return (no cluster barrier is pending)
  if (!a.standalone && a.sc[bl].done) return;
  const float alpha = a.standalone ? 0.f : (float)a.sc[bl].alpha;
  const float beta = a.standalone ? 0.f : (float)a.sc[bl].beta;
  // the d and u rows of this thread's row phase are requested into L2 while the columns are
  // transformed
  if (!a.standalone) {
    for (int rg = warp; rg < PNh / PRPW; rg += PNW) {
      const int row = rank * PNh + rg * PRPW + lane / PG3;
      const long long o = base + (long long)row * PN + (lane % PG3) * 32;
      pf_l2(a.d + o);
      pf_l2(a.u + o);
    }
  }
  __syncthreads();
  // ---- columns of this rank: inverse axis 2 from s_hat, each value to the row owner.  A warp's
  // first two column groups are read before either is transformed (one memory latency).
  {
    const int ncol = pncol(rank), ncg = (ncol + PCW - 1) / PCW;
    const C* in = a.shat + (field * a.g.n1 + i1) * (long long)(PN * Pn3h) + pcol0(rank);
    C* scr = colscr + warp * PCW * PN + (lane % PCW);
    const int g = lane / PCW;
    auto load_col = [&](int cg, C (&v)[PV2]) {
      const int col = cg * PCW + lane % PCW;
      const bool on = cg < ncg && col < ncol;
#pragma unroll
      for (int j = 0; j < PV2 / PG2; ++j)
#pragma unroll
        for (int k2 = 0; k2 < PG2; ++k2)
          v[j * PG2 + k2] = on ? in[scat_index<PN>(g, j, k2) * Pn3h + col] : make_float2(0.f, 0.f);
    };
    auto transform_col = [&](int cg, C (&v)[PV2]) {
      const int col = cg * PCW + lane % PCW;
      fft_dist_b<PN, +1>(v, g, scr, PCW, tw2);
      if (col < ncol) {
        const int k3 = pcol0(rank) + col;
#pragma unroll
        for (int n1 = 0; n1 < PV2; ++n1) {
          const int row = g + PG2 * n1;       // rows 0..127 belong to rank 0, 128..255 to rank 1
          C* dst = (row >> 7) == rank ? rowbuf : rowbuf_peer;
          dst[(row & (PNh - 1)) * PRP + k3] = v[n1];
        }
      }
      __syncwarp();
    };
    for (int cg = warp; cg < ncg; cg += 2 * PNW) {
      C v0[PV2], v1[PV2];
      load_col(cg, v0);
      load_col(cg + PNW, v1);
      transform_col(cg, v0);
      if (cg + PNW < ncg) transform_col(cg + PNW, v1);
    }
  }
  cluster.sync();  // every row of this rank is complete
  // ---- rows of this rank: inverse axis 3 (half spectrum -> real row), CG updates
  for (int rg = warp; rg < PNh / PRPW; rg += PNW) {
    const int rl = rg * PRPW + lane / PG3, g = lane % PG3;
    const int row = rank * PNh + rl;
    C* rs = rowbuf + rl * PRP;
    for (int k = g; k <= PNh / 2; k += PG3) c2r_pair<float>(rs, k, PNh, tw3);
    __syncwarp();
    C v[PV3];
#pragma unroll
    for (int j = 0; j < PV3 / PG3; ++j)
#pragma unroll
      for (int k2 = 0; k2 < PG3; ++k2) v[j * PG3 + k2] = rs[scat_index<PNh>(g, j, k2)];
    fft_dist_b<PNh, +1>(v, g, rs, 1, tw3h);
    if (a.standalone) {
      C* dst = reinterpret_cast<C*>(a.dst + base) + row * PNh;
#pragma unroll
      for (int n1 = 0; n1 < PV3; ++n1) dst[g + PG3 * n1] = v[n1];
    } else {
      C* d = reinterpret_cast<C*>(a.d + base) + row * PNh;
      C* u = reinterpret_cast<C*>(a.u + base) + row * PNh;
#pragma unroll
      for (int n1 = 0; n1 < PV3; ++n1) {
        const C dv = d[g + PG3 * n1];
        C uu = u[g + PG3 * n1];
        uu.x += alpha * dv.x;
        uu.y += alpha * dv.y;
        u[g + PG3 * n1] = uu;
        d[g + PG3 * n1] = make_float2(v[n1].x + beta * dv.x, v[n1].y + beta * dv.y);
      }
    }
    __syncwarp();
  }
  pdl_trigger();
}

// ---------------------------------------------------------------- row pass of 256^2 planes
// Inverse axis 3 of 256 x 256 FP32 planes row by row, after the axis-2 column pass, fused with
// the CG updates (the second half of the two-pass inverse transform).  A warp takes 4 rows (8
// threads a row, the register line FFT of fft_reg.cuh), a block 32 rows of one plane: each warp
// copies its rows of the half spectrum into shared memory in whole-row runs, untangles the real
// spectrum pairwise (c2r_pair), transforms the 128-point half-length lines and updates u and d.
// The rows of d and u are requested into L2 at the start.
namespace {
constexpr int RI_W = 8;                      // warps per block
constexpr int RI_R = RI_W * PRPW;            // rows per block
constexpr size_t kRowsInvSmem = (size_t)RI_R * PRP * sizeof(float2) + (size_t)(PNh + PN) * sizeof(float2);
}  // namespace

__global__ void __launch_bounds__(RI_W * 32) k_rows_inv256(PlaneInvArgs<float> a) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* rowbuf = reinterpret_cast<C*>(smem_raw);  // [RI_R rows][PRP]
  C* tw3h = rowbuf + RI_R * PRP;
  C* tw3 = tw3h + PNh;
  load_tw_reg<float>(tw3h, a.ft.tw3h, PNh);
  load_tw_reg<float>(tw3, a.ft.tw3, PN);
  constexpr int chunks = PN / RI_R;
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plane_id = blockIdx.x / chunks, ch = blockIdx.x - plane_id * chunks;
  const int comp = plane_id / a.g.n1, i1 = plane_id - comp * a.g.n1;
  const long long field = (long long)bl * a.c + comp;
  const long long base = (field * a.g.n1 + i1) * (long long)(PN * PN);
  const int rl = warp * PRPW + lane / PG3, g = lane % PG3;
  const int row = ch * RI_R + rl;
  if (!a.standalone) {  // each thread one 128-byte line of its row of d and of u
    const long long o = base + (long long)row * PN + g * 32;
    pf_l2(a.d + o);
    pf_l2(a.u + o);
  }
  pdl_wait();
  if (!a.standalone && a.sc[bl].done) return;
  const float alpha = a.standalone ? 0.f : (float)a.sc[bl].alpha;
  const float beta = a.standalone ? 0.f : (float)a.sc[bl].beta;
  __syncthreads();  // twiddles
  const C* in = a.shat + (field * a.g.n1 + i1) * (long long)(PN * Pn3h);
#pragma unroll
  for (int r = 0; r < PRPW; ++r) {
    const int lr = warp * PRPW + r;
    const C* src = in + (long long)(ch * RI_R + lr) * Pn3h;
    C* dst = rowbuf + lr * PRP;
#pragma unroll
    for (int i = 0; i < (Pn3h + 31) / 32; ++i) {
      const int k = lane + 32 * i;
      if (k < Pn3h) dst[k] = src[k];
    }
  }
  __syncwarp();
  C* rs = rowbuf + rl * PRP;
  for (int k = g; k <= PNh / 2; k += PG3) c2r_pair<float>(rs, k, PNh, tw3);
  __syncwarp();
  C v[PV3];
#pragma unroll
  for (int j = 0; j < PV3 / PG3; ++j)
#pragma unroll
    for (int k2 = 0; k2 < PG3; ++k2) v[j * PG3 + k2] = rs[scat_index<PNh>(g, j, k2)];
  fft_dist_b<PNh, +1>(v, g, rs, 1, tw3h);
  if (a.standalone) {
    C* dst = reinterpret_cast<C*>(a.dst + base) + row * PNh;
#pragma unroll
    for (int n1 = 0; n1 < PV3; ++n1) dst[g + PG3 * n1] = v[n1];
  } else {
    C* d = reinterpret_cast<C*>(a.d + base) + row * PNh;
    C* u = reinterpret_cast<C*>(a.u + base) + row * PNh;
#pragma unroll
    for (int n1 = 0; n1 < PV3; ++n1) {
      const C dv = d[g + PG3 * n1];
      C uu = u[g + PG3 * n1];
      uu.x += alpha * dv.x;
      uu.y += alpha * dv.y;
      u[g + PG3 * n1] = uu;
      d[g + PG3 * n1] = make_float2(v[n1].x + beta * dv.x, v[n1].y + beta * dv.y);
    }
  }
  pdl_trigger();
}

// Forward axis 3 of 256 x 256 FP32 planes row by row, before the axis-2 column pass, fused with
// r <- r - alpha p and ||r||_inf (the first half of the two-pass forward transform; the last
// block performs the residual check).  Same layout as k_rows_inv256: 4 rows per warp, 32 per
// block; each row's half spectrum (129 values) is written in one run.
__global__ void __launch_bounds__(RI_W * 32) k_rows_fwd256(PlaneFwdArgs<float> a) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red_sh[32];
  C* rowbuf = reinterpret_cast<C*>(smem_raw);  // [RI_R rows][PRP]
  C* tw3h = rowbuf + RI_R * PRP;
  C* tw3 = tw3h + PNh;
  load_tw_reg<float>(tw3h, a.ft.tw3h, PNh);
  load_tw_reg<float>(tw3, a.ft.tw3, PN);
  constexpr int chunks = PN / RI_R;
  const int bl = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int plane_id = blockIdx.x / chunks, ch = blockIdx.x - plane_id * chunks;
  const int comp = plane_id / a.g.n1, i1 = plane_id - comp * a.g.n1;
  const long long field = (long long)bl * a.c + comp;
  const long long base = (field * a.g.n1 + i1) * (long long)(PN * PN);
  const int rl = warp * PRPW + lane / PG3, g = lane % PG3;
  const int row = ch * RI_R + rl;
  pdl_wait();
  bool active = true;
  double alpha = 0.0;
  if (!a.standalone) {
    const CgScal& st = a.sc[bl];
    active = !st.done && (!a.after_replace || st.need_replace);
    alpha = a.after_replace ? 0.0 : st.alpha;
  }
  __syncthreads();  // twiddles
  float lmax = 0.f;
  if (active) {
    C v[PV3];
    if (a.standalone) {
      const C* src = reinterpret_cast<const C*>(a.src + base) + row * PNh;
#pragma unroll
      for (int n1 = 0; n1 < PV3; ++n1) v[n1] = src[g + PG3 * n1];
    } else {
      C* r = reinterpret_cast<C*>(a.r + base) + row * PNh;
      const C* p = reinterpret_cast<const C*>(a.p + base) + row * PNh;
      const float al = (float)alpha;
      C q[PV3];
#pragma unroll
      for (int n1 = 0; n1 < PV3; ++n1) {
        v[n1] = r[g + PG3 * n1];
        q[n1] = p[g + PG3 * n1];
      }
      if (alpha != 0.0) {
#pragma unroll
        for (int n1 = 0; n1 < PV3; ++n1) {
          v[n1].x -= al * q[n1].x;
          v[n1].y -= al * q[n1].y;
          r[g + PG3 * n1] = v[n1];
        }
      }
#pragma unroll
      for (int n1 = 0; n1 < PV3; ++n1) lmax = fmaxf(lmax, fmaxf(fabsf(v[n1].x), fabsf(v[n1].y)));
    }
    C* rs = rowbuf + rl * PRP;
    fft_dist_a<PNh, -1>(v, g, rs, 1, tw3h);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < PV3 / PG3; ++j)
#pragma unroll
      for (int k2 = 0; k2 < PG3; ++k2) rs[scat_index<PNh>(g, j, k2)] = v[j * PG3 + k2];
    __syncwarp();
    for (int k = g; k <= PNh / 2; k += PG3) r2c_pair<float>(rs, k, PNh, tw3);
    __syncwarp();
    C* out = a.hat + (field * a.g.n1 + i1) * (long long)(PN * Pn3h);
#pragma unroll
    for (int r = 0; r < PRPW; ++r) {
      const int lr = warp * PRPW + r;
      const C* src = rowbuf + lr * PRP;
      C* dst = out + (long long)(ch * RI_R + lr) * Pn3h;
#pragma unroll
      for (int i = 0; i < (Pn3h + 31) / 32; ++i) {
        const int k = lane + 32 * i;
        if (k < Pn3h) dst[k] = src[k];
      }
    }
  }
  pdl_trigger();
  if (a.standalone) return;
  const double bmax = block_max_t(lmax, red_sh);
  if (threadIdx.x == 0 && active) atomic_max_nonneg(&a.sc[bl].rmax_bits, bmax);
  if (last_block(a.ticket)) {
    residual_decision(a.sc, a.BL, a.ctl, a.after_replace);
    if (threadIdx.x == 0) *a.ticket = 0u;
  }
}

// ---------------------------------------------------------------- column pass of 256^2 planes
// FFT along axis 2 of 256 x 256 FP32 half-spectrum planes (129 columns of 256 points), in place
// or into a.out.  A warp takes two adjacent columns (16 threads a column, the register line FFT
// of fft_reg.cuh) and reads them straight from global memory into the line FFT's distribution:
// thread g holds rows g + 16 j, and the scattered order of the 256-point split is the same row
// set, so results go back to global memory from the same registers.  The only shared memory is
// the warp's exchange scratch and the twiddles: no block barrier after the start, the warps of
// a block run independently and one warp's loads overlap another's arithmetic.  The (plane,
// column pair) units are numbered across the grid, 65 a plane (the last one holds the Nyquist
// column and an idle half).
namespace {
constexpr int CR_W = 8;                      // warps per block
constexpr int CR_PAIRS = (Pn3h + 1) / 2;     // 65 column pairs a plane
constexpr size_t kColsRegSmem = (size_t)CR_W * 2 * PN * sizeof(float2) + (size_t)PN * sizeof(float2);
}  // namespace

template <int DIR>
__global__ void __launch_bounds__(CR_W * 32) k_cols_reg256(ColArgs<float> a, long long units) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* scr_all = reinterpret_cast<C*>(smem_raw);  // [warp][2 lines][256]
  C* tw2 = scr_all + CR_W * 2 * PN;
  load_tw_reg<float>(tw2, a.ft.tw2, PN);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long unit = (long long)blockIdx.x * CR_W + warp;
  if (unit >= units) return;
  const long long plane = unit / CR_PAIRS;  // (bl * c + comp) * n1 + i1
  const int pair = (int)(unit - plane * CR_PAIRS);
  const int bl = (int)(plane / ((long long)a.c * a.g.n1));
  if (a.sc && (a.sc[bl].done || (a.only_pending && !a.sc[bl].just_replaced))) return;
  const int line = lane / PG2, g = lane % PG2;
  const int col = 2 * pair + line;
  const bool on = col < Pn3h;
  const C* src = a.data + plane * (long long)(PN * Pn3h) + col;
  C* dst = (a.out ? a.out : a.data) + plane * (long long)(PN * Pn3h) + col;
  C* scr = scr_all + (warp * 2 + line) * PN;
  C v[PV2];
  // natural rows g + 16 j in; the scattered index of value j * G + k2 is g + 16 k2 (V = G)
  static_assert(PV2 == PG2, "256-point split with V = G");
#pragma unroll
  for (int j = 0; j < PV2; ++j) v[j] = on ? __ldg(src + (long long)(g + PG2 * j) * Pn3h) : make_float2(0.f, 0.f);
  if (DIR < 0) fft_dist_a<PN, -1>(v, g, scr, 1, tw2);
  else fft_dist_b<PN, +1>(v, g, scr, 1, tw2);
  if (on) {
#pragma unroll
    for (int j = 0; j < PV2; ++j) dst[(long long)(g + PG2 * j) * Pn3h] = v[j];
  }
}

// ---------------------------------------------------------------- host side
bool plane_cl_ok(const Grid& g) {
#ifdef UNOCG_NO_CLUSTER_PLANES
  return false;
#endif
  return g.n2 == PN && g.n3 == PN;
}

template <typename K, typename A>
static cudaError_t launch_cl(K kern, size_t smem, const A& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * a.c * a.g.n1, a.BL);
  cfg.blockDim = dim3(PNW * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = UNOCG_PDL ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_plane_fwd_cl(const PlaneFwdArgs<float>& a, cudaStream_t s) {
  return launch_cl(k_plane_fwd_cl, kFwdSmem, a, s);
}
cudaError_t launch_plane_inv_cl(const PlaneInvArgs<float>& a, cudaStream_t s) {
  return launch_cl(k_plane_inv_cl, kInvSmem, a, s);
}

bool rows_inv256_ok(const Grid& g) {
#ifdef UNOCG_NO_CLUSTER_PLANES
  return false;
#endif
  return g.n2 == PN && g.n3 == PN;
}

cudaError_t launch_rows_inv256(const PlaneInvArgs<float>& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_rows_inv256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowsInvSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_rows_inv256, dim3(a.c * a.g.n1 * (PN / RI_R), a.BL), dim3(RI_W * 32), kRowsInvSmem, s, a);
}

cudaError_t launch_rows_fwd256(const PlaneFwdArgs<float>& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_rows_fwd256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowsInvSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(k_rows_fwd256, dim3(a.c * a.g.n1 * (PN / RI_R), a.BL), dim3(RI_W * 32), kRowsInvSmem, s, a);
}

// register column pass of 256 x 256 FP32 planes (see k_cols_reg256)
cudaError_t launch_cols_reg256(const ColArgs<float>& a, int dir, cudaStream_t s) {
  if (!rows_inv256_ok(a.g)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_cols_reg256<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kColsRegSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_cols_reg256<+1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColsRegSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long units = (long long)a.BL * a.c * a.g.n1 * CR_PAIRS;
  const dim3 grid((unsigned)((units + CR_W - 1) / CR_W));
  if (dir < 0) k_cols_reg256<-1><<<grid, CR_W * 32, kColsRegSmem, s>>>(a, units);
  else k_cols_reg256<+1><<<grid, CR_W * 32, kColsRegSmem, s>>>(a, units);
  return cudaGetLastError();
}

}  // namespace unocg
