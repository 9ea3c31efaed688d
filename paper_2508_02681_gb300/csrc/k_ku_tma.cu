// Thermal K d on TMA-staged node planes (layout and stencil in ku_tma.cuh), its launcher with
// the tensor maps, and the tile shapes the autotuner chooses from.
#include <cstdio>
#include <type_traits>
#include "kargs.h"
#include "ku_tma.cuh"
#include "driver_api.h"

namespace unocg {

namespace {
constexpr unsigned kFull = 0xffffffffu;
static_assert(KT_UNROLL % KT_PS == 0 && KT_UNROLL % 2 == 0 && (KT_DS & (KT_DS - 1)) == 0,
              "phase-ring slots repeat within the unrolled loop body; the node ring is a power of two");

// Per-thread constants of the tile layout.
struct KtGeom {
  int x0;            // first of the thread's KT_NV nodes along i3
  int src_l, src_r;  // lanes holding the axis-3 neighbours (periodic within the row)
  bool fix_l, fix_r; // neighbour in another warp: read from shared memory instead
  int xl, xr;        // axis-3 neighbour columns (periodic)
  int rm, rc, rp;    // offsets (row start + x0) of the tile rows ty - 1, ty, ty + 1 in a plane buffer
  int em, ec;        // the same for element rows ty - 1 (o2 = 1) and ty (o2 = 0)
};

// Row of node values at `p` = row start + x0: v[0] = column x0 - 1, v[1..4] = x0 .. x0 + 3,
// v[5] = x0 + 4 (periodic).
__device__ __forceinline__ void kt_row(const float* p, const KtGeom& G, float (&v)[KT_NV + 2]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  float l = __shfl_sync(kFull, q.w, G.src_l);
  float r = __shfl_sync(kFull, q.x, G.src_r);
  if (G.fix_l) l = p[G.xl - G.x0];
  if (G.fix_r) r = p[G.xr - G.x0];
  v[0] = l; v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w; v[5] = r;
}
// Row of element conductivities at `p` = row start + x0: v[0] = column x0 - 1, v[1..4] = x0 .. x0 + 3.
__device__ __forceinline__ void kt_krow(const float* p, const KtGeom& G, float (&v)[KT_NV + 1]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  float l = __shfl_sync(kFull, q.w, G.src_l);
  if (G.fix_l) l = p[G.xl - G.x0];
  v[0] = l; v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
}

__device__ __forceinline__ int wrap_n(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
}  // namespace

// One block: tile (i2_0 .. i2_0 + ty - 1) x (all i3) of one (instance, load), node planes
// z0 .. z0 + nsteps - 1.  blockIdx.x = tile * BL + bl, so the blocks of one tile for the loads
// of an instance run next to each other and share the phase planes in L2.
__global__ void __launch_bounds__(512) k_ku_tma(const __grid_constant__ KuTmaMaps maps, const KuTmaArgs ka) {
  extern __shared__ unsigned char kt_raw[];
  __shared__ float mt[256];
  __shared__ double red_sh[32];
  __shared__ __align__(8) uint64_t bar_d[KT_DS];
  __shared__ __align__(8) uint64_t bar_p[KT_PS];
  __shared__ int s_abort;

  const StencilArgs<float>& a = ka.a;
  const Grid& g = a.g;
  const int TY = ka.ty, n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int BL = a.BL;
  const int bl = blockIdx.x % BL;
  const int tile = blockIdx.x / BL;
  const int ntile2 = n2 / TY;
  const int i2_0 = (tile % ntile2) * TY;
  const int z0 = (tile / ntile2) * ka.cz;
  const int nsteps = min(ka.cz, n1 - z0);
  const int b = bl / a.L;
  const int tid = threadIdx.x;

  unsigned char* base = kt_raw + ((128u - (sm_addr(kt_raw) & 127u)) & 127u);
  const int dvals = (TY + 2) * n3, kvals = (TY + 1) * n3;
  const size_t psz = kt_pslot_bytes(TY, n3);
  float* dbuf = reinterpret_cast<float*>(base);
  float* kbuf = dbuf + KT_DS * dvals;
  unsigned char* pbuf = reinterpret_cast<unsigned char*>(kbuf + 2 * kvals);

  // conductivities scaled by h / 12 (the element matrix is (h / 12) times integers)
  {
    const float* src = a.mat.m32 + (long long)b * a.mat.n_phases * 2;
    for (int i = tid; i < a.mat.n_phases; i += blockDim.x) mt[i] = src[2 * i] * g.h12f;
  }
  if (tid == 0) {
    for (int i = 0; i < KT_DS; ++i) mbar_init(&bar_d[i], 1);
    for (int i = 0; i < KT_PS; ++i) mbar_init(&bar_p[i], 1);
    s_abort = 0;
    mbar_fence_init();
  }
  KtGeom G;
  {
    // a row of the tile is TPR = N3 / 4 consecutive threads; the axis-3 neighbours of a thread's
    // four nodes are the last value of the previous thread of the row and the first of the next
    // (periodic within the row), taken by shuffle where that thread is in the same warp
    const int TPR = n3 / KT_NV;
    const int ty = tid / TPR, xr_ = tid % TPR;
    G.x0 = xr_ * KT_NV;
    const int tl = xr_ == 0 ? tid + TPR - 1 : tid - 1;
    const int tr = xr_ == TPR - 1 ? tid - TPR + 1 : tid + 1;
    G.src_l = tl & 31;
    G.src_r = tr & 31;
    G.fix_l = (tl >> 5) != (tid >> 5);
    G.fix_r = (tr >> 5) != (tid >> 5);
    G.xl = (G.x0 == 0 ? n3 : G.x0) - 1;
    G.xr = (G.x0 + KT_NV == n3) ? 0 : G.x0 + KT_NV;
    G.rm = (ty == 0 ? TY : ty - 1) * n3 + G.x0;
    G.rc = ty * n3 + G.x0;
    G.rp = (ty + 1 == TY ? TY + 1 : ty + 1) * n3 + G.x0;
    G.em = G.rm;
    G.ec = G.rc;
  }
  __syncthreads();
  pdl_wait();  // d and the loop state come from the kernels before this one
  const bool skip = !a.standalone && a.sc[bl].done;
  DotAcc<float> dot;
  const int ndl = nsteps + 2;   // node planes z0 - 1 .. z0 + nsteps
  const int npl = nsteps + 1;   // element planes z0 - 1 .. z0 + nsteps - 1
  const long long lim = ka.spin_limit;

  auto issue_d = [&](int k) {
    const int q = wrap_n(z0 - 1 + k, n1);
    uint64_t* bar = &bar_d[k % KT_DS];
    float* dst = dbuf + (k % KT_DS) * dvals;
    mbar_expect_tx(bar, (uint32_t)(dvals * sizeof(float)));
    tma_load_4d(dst, &maps.d_rows, 0, i2_0, q, bl, bar);
    tma_load_4d(dst + TY * n3, &maps.d_row, 0, wrap_n(i2_0 - 1, n2), q, bl, bar);
    tma_load_4d(dst + (TY + 1) * n3, &maps.d_row, 0, wrap_n(i2_0 + TY, n2), q, bl, bar);
  };
  auto issue_p = [&](int k) {
    const int e = wrap_n(z0 - 1 + k, n1);
    uint64_t* bar = &bar_p[k % KT_PS];
    unsigned char* dst = pbuf + (k % KT_PS) * psz;
    mbar_expect_tx(bar, (uint32_t)kvals);
    tma_load_4d(dst, &maps.ph_rows, 0, i2_0, e, b, bar);
    tma_load_4d(dst + TY * n3, &maps.ph_row, 0, wrap_n(i2_0 - 1, n2), e, b, bar);
  };
  auto wait_d = [&](int k) -> bool { return mbar_wait(&bar_d[k % KT_DS], (uint32_t)((k / KT_DS) & 1), lim); };
  auto wait_p = [&](int k) -> bool { return mbar_wait(&bar_p[k % KT_PS], (uint32_t)((k / KT_PS) & 1), lim); };
  // phase slot ps -> conductivity slot ks
  auto convert_slot = [&](int ps, int ks) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(pbuf + ps * psz);
    float4* dst = reinterpret_cast<float4*>(kbuf + ks * kvals);
    for (int w = tid; w < kvals / 4; w += blockDim.x) {
      const uint32_t v = src[w];
      dst[w] = make_float4(mt[v & 255u], mt[(v >> 8) & 255u], mt[(v >> 16) & 255u], mt[v >> 24]);
    }
  };
  // phase plane k -> conductivity plane k % 2
  auto convert = [&](int k) { convert_slot(k % KT_PS, k & 1); };
  auto timeout = [&]() {
    s_abort = 1;
    if (ka.err) atomicExch(ka.err, 1);
  };
  int issued_d = 0, issued_p = 0;   // meaningful in thread 0

  if (!skip) {
    if (tid == 0) {
      for (; issued_p < KT_PS && issued_p < npl; ++issued_p) issue_p(issued_p);
      for (; issued_d < KT_DS && issued_d < ndl; ++issued_d) issue_d(issued_d);
    }
    // window registers: D[plane mod 3][row: 0 = i2 - 1, 1 = i2, 2 = i2 + 1][column]
    float D[3][3][KT_NV + 2];
    // Kc[element plane mod 2][o2][column j = x0 - 1 + j]
    float Kc[2][2][KT_NV + 1];
    if (!(wait_p(0) && wait_p(1))) timeout();
    else {
      convert(0);
      convert(1);
    }
    if (!(wait_d(0) && wait_d(1))) timeout();
    __syncthreads();
    bool alive = !s_abort;
    if (alive) {
      const float* d0 = dbuf;
      const float* d1 = dbuf + dvals;
      kt_row(d0 + G.rm, G, D[0][0]); kt_row(d0 + G.rc, G, D[0][1]); kt_row(d0 + G.rp, G, D[0][2]);
      kt_row(d1 + G.rm, G, D[1][0]); kt_row(d1 + G.rc, G, D[1][1]); kt_row(d1 + G.rp, G, D[1][2]);
      kt_krow(kbuf + G.ec, G, Kc[0][0]);
      kt_krow(kbuf + G.em, G, Kc[0][1]);
    }
    __syncthreads();  // loads 0, 1 and conductivity plane 0 are in registers
    if (alive && tid == 0) {
      for (; issued_d < KT_DS + 2 && issued_d < ndl; ++issued_d) issue_d(issued_d);
      for (; issued_p < KT_PS + 2 && issued_p < npl; ++issued_p) issue_p(issued_p);
    }
    const long long plane = (long long)n2 * n3;
    const int i2 = i2_0 + G.rc / n3;
    const long long obase = (long long)bl * g.n + (long long)z0 * plane + (long long)i2 * n3 + G.x0;

    // One step at node plane z = z0 + j; S = j mod 6 selects the rotating register roles.
    auto step = [&](auto S_, int j) -> bool {
      constexpr int S = decltype(S_)::value;
      constexpr int PM = S % 3, PC = (S + 1) % 3, PN = (S + 2) % 3;
      constexpr int KM = S % 2, KC = (S + 1) % 2;
      // node plane z + 1 (load j + 2); the phase-ring slot and parity are fixed by S (6 is a
      // multiple of its depth)
      constexpr int PSL = (S + 2) % KT_PS, PPAR = ((S + 2) / KT_PS) & 1;
      const int dsl = (j + 2) & (KT_DS - 1);
      if (!mbar_wait(&bar_d[dsl], (uint32_t)(((j + 2) / KT_DS) & 1), lim)) timeout();
      const float* dn = dbuf + dsl * dvals;
      kt_row(dn + G.rm, G, D[PN][0]); kt_row(dn + G.rc, G, D[PN][1]); kt_row(dn + G.rp, G, D[PN][2]);
      // element plane z (converted one step earlier)
      const float* kc = kbuf + ((S + 1) & 1) * kvals;
      kt_krow(kc + G.ec, G, Kc[KC][0]);
      kt_krow(kc + G.em, G, Kc[KC][1]);
      // element plane z + 1 for the next step
      if (j + 2 < npl) {
        if (!mbar_wait(&bar_p[PSL], (uint32_t)PPAR, lim)) {
          timeout();
        } else {
          convert_slot(PSL, S & 1);
        }
      }
      const float(&dm)[3][KT_NV + 2] = D[PM];
      const float(&dc)[3][KT_NV + 2] = D[PC];
      const float(&dnr)[3][KT_NV + 2] = D[PN];
      const float(&km)[2][KT_NV + 1] = Kc[KM];
      const float(&kcr)[2][KT_NV + 1] = Kc[KC];
      // pair sums over the two element rows (q) and over the two element planes (e), formed per
      // element column as the nodes of the thread are visited (column i shared by nodes i - 1, i)
      float out[KT_NV];
      float sp = 0.f;
      float q0l = kcr[0][0] + kcr[1][0], q1l = km[0][0] + km[1][0];
      float e0l = kcr[0][0] + km[0][0], e1l = kcr[1][0] + km[1][0];
#pragma unroll
      for (int i = 0; i < KT_NV; ++i) {
        const float q0r = kcr[0][i + 1] + kcr[1][i + 1], q1r = km[0][i + 1] + km[1][i + 1];
        const float e0r = kcr[0][i + 1] + km[0][i + 1], e1r = kcr[1][i + 1] + km[1][i + 1];
        const float sk = (q0l + q0r) + (q1l + q1r);
        float acc = 4.f * sk * dc[1][i + 1];
        // in-plane diagonal neighbours (0, s2, s3)
        acc = fmaf(-e1l, dc[0][i], acc);
        acc = fmaf(-e1r, dc[0][i + 2], acc);
        acc = fmaf(-e0l, dc[2][i], acc);
        acc = fmaf(-e0r, dc[2][i + 2], acc);
        // (s1, 0, s3)
        acc = fmaf(-q0l, dnr[1][i], acc);
        acc = fmaf(-q0r, dnr[1][i + 2], acc);
        acc = fmaf(-q1l, dm[1][i], acc);
        acc = fmaf(-q1r, dm[1][i + 2], acc);
        // (s1, s2, 0): the two elements along axis 3
        acc = fmaf(-(kcr[1][i] + kcr[1][i + 1]), dnr[0][i + 1], acc);
        acc = fmaf(-(kcr[0][i] + kcr[0][i + 1]), dnr[2][i + 1], acc);
        acc = fmaf(-(km[1][i] + km[1][i + 1]), dm[0][i + 1], acc);
        acc = fmaf(-(km[0][i] + km[0][i + 1]), dm[2][i + 1], acc);
        // corners
        acc = fmaf(-kcr[1][i], dnr[0][i], acc);
        acc = fmaf(-kcr[1][i + 1], dnr[0][i + 2], acc);
        acc = fmaf(-kcr[0][i], dnr[2][i], acc);
        acc = fmaf(-kcr[0][i + 1], dnr[2][i + 2], acc);
        acc = fmaf(-km[1][i], dm[0][i], acc);
        acc = fmaf(-km[1][i + 1], dm[0][i + 2], acc);
        acc = fmaf(-km[0][i], dm[2][i], acc);
        acc = fmaf(-km[0][i + 1], dm[2][i + 2], acc);
        out[i] = acc;
        sp = fmaf(acc, dc[1][i + 1], sp);
        q0l = q0r; q1l = q1r; e0l = e0r; e1l = e1r;
      }
      // the products d p of one step are summed in FP32 (four terms, whose rounding stays below
      // that of the FP32 p itself) and accumulated across steps in the float-float pair
      dot.add(sp);
      *reinterpret_cast<float4*>(a.p + obase + (long long)j * plane) = make_float4(out[0], out[1], out[2], out[3]);
      __syncthreads();  // every thread is done with node plane j + 2 and phase plane j + 2
      if (s_abort) return false;
      if (tid == 0) {
        if (issued_d < ndl) issue_d(issued_d++);
        if (issued_p < npl) issue_p(issued_p++);
      }
      return true;
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    using I5 = std::integral_constant<int, 5>;
    for (int j = 0; alive && j < nsteps; j += KT_UNROLL) {
      if (!step(I0{}, j)) { alive = false; break; }
      if (j + 1 >= nsteps) break;
      if (!step(I1{}, j + 1)) { alive = false; break; }
      if (j + 2 >= nsteps) break;
      if (!step(I2{}, j + 2)) { alive = false; break; }
      if (j + 3 >= nsteps) break;
      if (!step(I3{}, j + 3)) { alive = false; break; }
      if (j + 4 >= nsteps) break;
      if (!step(I4{}, j + 4)) { alive = false; break; }
      if (j + 5 >= nsteps) break;
      if (!step(I5{}, j + 5)) { alive = false; break; }
    }
    if (!alive && tid == 0) {
      // after a timeout: wait (bounded) for the copies still in flight before the block exits --
      // the last one issued into each ring slot (earlier ones of that slot have completed)
      for (int k = max(0, issued_d - KT_DS); k < issued_d; ++k)
        (void)mbar_wait(&bar_d[k % KT_DS], (uint32_t)((k / KT_DS) & 1), lim);
      for (int k = max(0, issued_p - KT_PS); k < issued_p; ++k)
        (void)mbar_wait(&bar_p[k % KT_PS], (uint32_t)((k / KT_PS) & 1), lim);
    }
  }
  const double bs = block_sum_acc(dot, red_sh);
  pdl_trigger();
  if (a.standalone) return;
  if (tid == 0) a.red.part[(long long)bl * ka.tiles + tile] = bs;
  if (last_block(a.red.ticket)) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int q = warp; q < BL; q += blockDim.x / 32) {
      const double sum = warp_sum_partials(a.red.part + (long long)q * ka.tiles, ka.tiles, 1);
      if (lane == 0 && !a.sc[q].done) step_update(a.sc[q], sum);
    }
    __syncthreads();
    if (tid == 0) *a.red.ticket = 0u;
  }
}

// ---------------------------------------------------------------- host side
// Tile shapes: node rows TY per tile (each row takes N3 / 4 threads, so a block has
// TY * N3 / 4 threads) and node planes per block.  The automatic choice and the autotuner pick
// among them.
const KuTmaShape kKuTmaShapes[kKuTmaNumShapes] = {{4, 12}, {8, 12}, {2, 12}, {8, 24}, {16, 6}, {4, 24}, {16, 12}, {8, 6}};

int ku_tma_threads(const Grid& g, KuTmaShape s) { return s.rows * (g.n3 / KT_NV); }

bool ku_tma_supported(const Grid& g, int c, KuTmaShape s) {
  if (c != 1) return false;
  // whole rows in one TMA box (at most 256 values); rows of a multiple of 128 bytes keep every
  // copy destination 128-byte aligned
  if (g.n3 % 32 != 0 || g.n3 > 256) return false;
  const int th = ku_tma_threads(g, s);
  if (th % 32 != 0 || th < 64 || th > 512) return false;
  if (s.rows < 1 || g.n2 % s.rows != 0 || (s.rows * g.n3) % 128 != 0) return false;
  if (kt_smem_bytes(s.rows, g.n3) > 200 * 1024) return false;
  return tensor_map_encoder() != nullptr;
}

int ku_tma_blocks_x(const Grid& g, KuTmaShape s) {
  return (g.n2 / s.rows) * ((g.n1 + s.planes - 1) / s.planes);
}

static CUresult encode_4d(CUtensorMap* m, CUtensorMapDataType dt, size_t esz, const void* ptr, const Grid& g,
                          int count, int box_rows) {
  const cuuint64_t dims[4] = {(cuuint64_t)g.n3, (cuuint64_t)g.n2, (cuuint64_t)g.n1, (cuuint64_t)count};
  const cuuint64_t strides[3] = {(cuuint64_t)g.n3 * esz, (cuuint64_t)g.n2 * g.n3 * esz, (cuuint64_t)g.n * esz};
  const cuuint32_t box[4] = {(cuuint32_t)g.n3, (cuuint32_t)box_rows, 1u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  return tensor_map_encoder()(m, dt, 4, const_cast<void*>(ptr), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

cudaError_t launch_ku_tma(const StencilArgs<float>& a, KuTmaShape s, int* err, long long spin_limit, cudaStream_t st) {
  const Grid& g = a.g;
  const int ty = s.rows;
  KuTmaMaps maps;
  const int B = a.BL / a.L;
  if (encode_4d(&maps.d_rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.d, g, a.BL, ty) != CUDA_SUCCESS ||
      encode_4d(&maps.d_row, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.d, g, a.BL, 1) != CUDA_SUCCESS ||
      encode_4d(&maps.ph_rows, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, a.phase, g, B, ty) != CUDA_SUCCESS ||
      encode_4d(&maps.ph_row, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, a.phase, g, B, 1) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  KuTmaArgs ka{};
  ka.a = a;
  ka.ty = ty;
  ka.cz = s.planes;
  ka.tiles = ku_tma_blocks_x(g, s);
  ka.err = err;
  ka.spin_limit = spin_limit;
  const size_t smem = kt_smem_bytes(ty, g.n3);
  static size_t smem_set = 0;
  if (smem > 48 * 1024 && smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_ku_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  return launch_pdl(k_ku_tma, dim3(ka.tiles * a.BL), dim3(ku_tma_threads(g, s)), smem, st, maps, ka);
}

}  // namespace unocg
