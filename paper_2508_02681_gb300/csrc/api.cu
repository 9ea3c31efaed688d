// C ABI of the UNO-CG solver (include/unocg.h): contexts, set-up, the device-resident CG loop
// of Algorithm 1 / Algorithm 2 in a CUDA graph with conditional nodes, post-processing.
//
// One CG iteration of UNO-CG is four kernels (see k_fft.cu / k_stencil.cu):
//   k_line      FFT axis 1, s_hat = Q r_hat / n, gamma = r.s (Parseval), inverse axis 1, beta
//   k_plane_inv inverse FFT axes 2/3, u += alpha d_old, d = s + beta d_old
//   k_ku        p = K d, d.p, alpha
//   k_plane_fwd r -= alpha p, ||r||_inf, stopping test, forward FFT axes 3/2
// Jacobi / unpreconditioned CG uses k_jac_b, k_ku, k_jac_a.  In mixed precision a conditional
// IF node runs the FP64 residual replacement (fold u, r = f - K u) when the last residual check
// requests it.
#include <algorithm>
#include <atomic>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <initializer_list>
#include <type_traits>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "driver_api.h"
#include "kargs.h"
#include "persist.h"
#include "setup.h"
#include "unocg.h"

using namespace unocg;

namespace {

// NVTX range for the duration of an entry point (visible to Nsight tools, inert otherwise)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

constexpr int kMaxTickets = 8;
enum Ticket { T_PLANE = 0, T_LINE = 1, T_KU = 2, T_JAC = 3, T_PLANE2 = 4, T_JAC2 = 5 };

// Radix plans of the shared-memory Stockham passes.  order 0: radix 8, 4, 2, then 3, 5 (fewest
// stages, the default); 1: radix 4, 2, 3, 5 (no radix 8: fewer registers per butterfly);
// 2: radix 5, 3 first, then 4, 2.  The autotuner picks one per context.
bool factor_plan(int N, FftPlan* p, int order = 0) {
  p->N = N;
  p->nst = 0;
  int m = N;
  auto take = [&](int r) {
    while (m % r == 0 && p->nst < 12) { p->radix[p->nst++] = r; m /= r; }
  };
  if (order == 2) { take(5); take(3); }
  if (order == 0) take(8);
  take(4);
  take(2);
  take(3);
  take(5);
  return m == 1 && p->nst <= 12;
}

template <typename T>
std::vector<cplx<T>> twiddles(int N) {
  std::vector<cplx<T>> w(N);
  for (int m = 0; m < N; ++m) {
    long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)N;
    w[m] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
  }
  return w;
}

struct Fields64 {
  double *r = nullptr, *d = nullptr, *p = nullptr, *u = nullptr;
  double2 *rhat = nullptr, *shat = nullptr;
};
struct Fields32 {
  float *r = nullptr, *d = nullptr, *p = nullptr, *u = nullptr;
  float2 *rhat = nullptr, *shat = nullptr;
  double* u64 = nullptr;
  double* f64 = nullptr;  // FP64 right-hand side of the true residual (written once per solve)
};

struct GraphKey {
  int precond = -1, precision = -1, flexible = -1, replace_every = -1, max_iter = -1, L = -1;
  double tol = -1.0, replace_drop = -1.0;
  bool operator==(const GraphKey& o) const {
    return precond == o.precond && precision == o.precision && flexible == o.flexible &&
           replace_every == o.replace_every && max_iter == o.max_iter && L == o.L && tol == o.tol &&
           replace_drop == o.replace_drop;
  }
};

}  // namespace

struct unocg_ctx {
  int physics = 1, c = 1, B = 1, dim = 3;
  Grid g{};
  double L0 = 1.0;
  int n_phases = 0, L = 0;
  bool have_phase = false, have_props = false, have_loads = false;
  int wkind = -1;
  bool q_dirty = true, bf16_spd_ok = true;
  double spd_eps = 0.0;
  std::vector<double> w_host;  // user weights (BLOCKS / THETA / MODES), FP64
  int modes_M = -1;            // MODES: mode-set parameter M
  cudaStream_t stream = nullptr, own_stream = nullptr;
  cudaEvent_t join_ev = nullptr;  // orders the `_dev` entry points against the context stream
  std::string err;
  // device data
  uint8_t* phase = nullptr;
  double* props_d = nullptr;  // raw properties
  double* mat64 = nullptr;
  float* mat32 = nullptr;
  double* ref = nullptr;      // [B][2]
  double* loads_d = nullptr;
  double* Q64 = nullptr;
  float* Q32 = nullptr;
  __nv_bfloat16* Q16 = nullptr;
  int Bq = 1;
  void* tw64[4] = {nullptr, nullptr, nullptr, nullptr};
  void* tw32[4] = {nullptr, nullptr, nullptr, nullptr};
  FftPlan p1{}, p2{}, p3h{};
  CgScal* sc = nullptr;
  double* part = nullptr;
  size_t part_n = 0;
  unsigned int* tickets = nullptr;
  int* flags = nullptr;  // [0] active, [1] replace, [2..3] loop counters, [4..5] grid barrier, [6] timeout
  int sm_count = 0;
  int last_path = 0;     // 0 host loop, 1 graph, 2 persistent
  long long spin_limit = 2000000000LL;  // grid-barrier wait limit (SM clock cycles)
  unsigned long long* fails = nullptr;
  Fields64 f64;
  Fields32 f32;
  double* invdiag64 = nullptr;
  float* invdiag32 = nullptr;
  double* ceff = nullptr;   // [B][dim][L]
  double* sens = nullptr;
  double* stage = nullptr;  // [c*n] interleave staging
  bool solved = false;
  int last_precision = 0;
  // graph cache
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
  unocg_solve_opts last_opts{};
  // tuning (unocg_set_tuning / unocg_autotune): radix order of the Stockham plans and the loop
  // driver taken by use_graph = 3
  int radix_order = 0, tuned_path = 1;
  // thermal FP32 K d: -1 automatic, 0 the register-march / element kernels, k = 1..8 the
  // TMA-staged kernel with tile shape kKuTmaShapes[k - 1], k = 9..16 the vector march with tile
  // shape kKuTmaShapes[k - 9] (unocg_set_ku_tile / unocg_autotune_ku)
  int ku_tile = -1;
  // changes whenever a captured graph of this context becomes invalid (and at creation): the
  // batch graphs of unocg_batch_solve that include the context compare it
  unsigned long long epoch = 0;
};

static std::atomic<unsigned long long> g_epoch{1};

struct unocg_uno {
  int c = 1;
  Grid g{};
  FftPlan p1{}, p2{}, p3h{};
  void* tw32[4] = {nullptr, nullptr, nullptr, nullptr};
  float* Q32 = nullptr;
  float* Qtmp = nullptr;
  const float* theta = nullptr;
  float2 *hat = nullptr, *shat = nullptr, *ghat = nullptr;
  size_t cap = 0;  // fields of capacity
  float* gq = nullptr;
  float* gq2 = nullptr;
  int modes_M = -1;            // >= 0: theta holds bypass + mode weights [1 + n_modes][C]
  double* mscratch = nullptr;  // partial sums of the bypass gradient
  std::string err;
};

static int n_modes_of(int M) { return (2 * M + 1) * (2 * M + 1) * (M + 1) - 1; }
static bool modes_fit(const Grid& g, int M) { return M >= 0 && 2 * M + 1 <= g.n1 && 2 * M + 1 <= g.n2 && 2 * M <= g.n3; }

// ------------------------------------------------------------------ helpers
static int fail(unocg_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}
#define CK(...)                                                                           \
  do {                                                                                    \
    cudaError_t e_ = (__VA_ARGS__);                                                       \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? UNOCG_ERR_OOM : UNOCG_ERR_CUDA,  \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));             \
  } while (0)

template <typename P>
static cudaError_t dalloc(P** p, size_t count) {
  if (*p) return cudaSuccess;
  return cudaMalloc((void**)p, count * sizeof(P));
}

static FftTables tables(unocg_ctx* ctx, bool fp64) {
  FftTables t;
  t.p1 = ctx->p1;
  t.p2 = ctx->p2;
  t.p3h = ctx->p3h;
  void* const* tw = fp64 ? ctx->tw64 : ctx->tw32;
  t.tw1 = tw[0];
  t.tw2 = tw[1];
  t.tw3h = tw[2];
  t.tw3 = tw[3];
  return t;
}

static Material material(unocg_ctx* ctx) {
  Material m;
  m.n_phases = ctx->n_phases;
  m.m64 = ctx->mat64;
  m.m32 = ctx->mat32;
  return m;
}

static bool grid_ok(int n1, int n2, int n3) {
  FftPlan p;
  if (n1 < 2 || n2 < 2 || n3 < 4 || (n3 % 2)) return false;
  return factor_plan(n1, &p) && factor_plan(n2, &p) && factor_plan(n3 / 2, &p);
}

template <typename T>
static cudaError_t upload_twiddles(void** dst, int n1, int n2, int n3) {
  int Ns[4] = {n1, n2, n3 / 2, n3};
  for (int i = 0; i < 4; ++i) {
    auto w = twiddles<T>(Ns[i]);
    cudaError_t e = cudaMalloc(&dst[i], w.size() * sizeof(cplx<T>));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(dst[i], w.data(), w.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------------ create / destroy
extern "C" int unocg_create(unocg_ctx** out, int physics, int batch, int n1, int n2, int n3, double L0) {
  unocg_ctx* ctx = nullptr;
  if (!out) return UNOCG_ERR_INVALID_ARG;
  *out = nullptr;
  if ((physics != UNOCG_THERMAL && physics != UNOCG_ELASTIC) || batch < 1 || !(L0 > 0.0))
    return UNOCG_ERR_INVALID_ARG;
  if (!grid_ok(n1, n2, n3)) return UNOCG_ERR_INVALID_ARG;
  {
    Grid tg{};
    tg.n1 = n1; tg.n2 = n2; tg.n3 = n3; tg.n3h = n3 / 2 + 1;
    if (!grid_supported(tg, 8) || !grid_supported(tg, 16)) return UNOCG_ERR_INVALID_ARG;
  }
  ctx = new unocg_ctx();
  ctx->epoch = g_epoch.fetch_add(1);
  ctx->physics = physics;
  ctx->c = physics == UNOCG_THERMAL ? 1 : 3;
  ctx->dim = physics == UNOCG_THERMAL ? 3 : 6;
  ctx->B = batch;
  ctx->L0 = L0;
  ctx->g.n1 = n1;
  ctx->g.n2 = n2;
  ctx->g.n3 = n3;
  ctx->g.n3h = n3 / 2 + 1;
  ctx->g.n = (long long)n1 * n2 * n3;
  ctx->g.nh = (long long)n1 * n2 * (n3 / 2 + 1);
  ctx->g.h = L0 / n1;
  grid_scales(ctx->g);
  factor_plan(n1, &ctx->p1);
  factor_plan(n2, &ctx->p2);
  factor_plan(n3 / 2, &ctx->p3h);
  *out = ctx;
  CK(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
  ctx->stream = ctx->own_stream;
  CK(upload_twiddles<double>(ctx->tw64, n1, n2, n3));
  CK(upload_twiddles<float>(ctx->tw32, n1, n2, n3));
  CK(cudaMalloc(&ctx->phase, (size_t)batch * ctx->g.n));
  CK(cudaMalloc(&ctx->tickets, kMaxTickets * sizeof(unsigned int)));
  CK(cudaMemset(ctx->tickets, 0, kMaxTickets * sizeof(unsigned int)));
  CK(cudaMalloc(&ctx->flags, 8 * sizeof(int)));
  CK(cudaMemset(ctx->flags, 0, 8 * sizeof(int)));
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, dev));
  }
  CK(cudaMalloc(&ctx->fails, sizeof(unsigned long long)));
  CK(cudaMalloc(&ctx->ref, 2 * batch * sizeof(double)));
  return UNOCG_OK;
}

static void free_graph(unocg_ctx* ctx) {
  if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->exec = nullptr;
  ctx->graph = nullptr;
  ctx->key = GraphKey();
  ctx->epoch = g_epoch.fetch_add(1);
}

static void forget_batches(const unocg_ctx* ctx);

extern "C" void unocg_destroy(unocg_ctx* ctx) {
  if (ctx) forget_batches(ctx);
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_graph(ctx);
  void* ptrs[] = {ctx->phase, ctx->props_d, ctx->mat64, ctx->mat32, ctx->ref, ctx->loads_d, ctx->Q64,
                  ctx->Q32, ctx->Q16, ctx->sc, ctx->part, ctx->tickets, ctx->flags, ctx->fails,
                  ctx->f64.r, ctx->f64.d, ctx->f64.p, ctx->f64.u, ctx->f64.rhat, ctx->f64.shat,
                  ctx->f32.r, ctx->f32.d, ctx->f32.p, ctx->f32.u, ctx->f32.rhat, ctx->f32.shat,
                  ctx->f32.u64, ctx->f32.f64, ctx->invdiag64, ctx->invdiag32, ctx->ceff, ctx->sens, ctx->stage,
                  ctx->tw64[0], ctx->tw64[1], ctx->tw64[2], ctx->tw64[3],
                  ctx->tw32[0], ctx->tw32[1], ctx->tw32[2], ctx->tw32[3]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  delete ctx;
}

extern "C" const char* unocg_last_error(const unocg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int unocg_set_wait_limit(unocg_ctx* ctx, double seconds) {
  if (!ctx || !(seconds >= 0.0)) return fail(ctx, UNOCG_ERR_INVALID_ARG, "wait limit must be >= 0");
  double cycles = seconds * 2.07e9;  // SM clock upper bound of the target GPU
  ctx->spin_limit = cycles < 1.0 ? 1LL : (long long)cycles;
  return UNOCG_OK;
}

extern "C" int unocg_set_stream(unocg_ctx* ctx, void* stream) {
  if (!ctx) return UNOCG_ERR_INVALID_ARG;
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return UNOCG_OK;
}

// ------------------------------------------------------------------ inputs
static int check_phase_range(unocg_ctx* ctx, int n_phases) {
  if (n_phases < 1 || n_phases > 255) return fail(ctx, UNOCG_ERR_INVALID_ARG, "n_phases must be in [1, 255]");
  if (ctx->have_props && n_phases != ctx->n_phases) {
    ctx->have_props = false;  // properties must be set again for the new phase count
  }
  ctx->n_phases = n_phases;
  return UNOCG_OK;
}

extern "C" int unocg_set_microstructure(unocg_ctx* ctx, const uint8_t* phase, int n_phases) {
  if (!ctx || !phase) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  int rc = check_phase_range(ctx, n_phases);
  if (rc) return rc;
  size_t m = (size_t)ctx->B * ctx->g.n;
  for (size_t i = 0; i < m; ++i)
    if (phase[i] >= n_phases) return fail(ctx, UNOCG_ERR_INVALID_ARG, "phase label >= n_phases");
  CK(cudaMemcpyAsync(ctx->phase, phase, m, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_phase = true;
  return UNOCG_OK;
}

extern "C" int unocg_set_microstructure_dev(unocg_ctx* ctx, const uint8_t* phase_dev, int n_phases, void* stream) {
  if (!ctx || !phase_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  int rc = check_phase_range(ctx, n_phases);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  CK(order_after(&ctx->join_ev, ctx->stream, s));
  CK(cudaMemcpyAsync(ctx->phase, phase_dev, (size_t)ctx->B * ctx->g.n, cudaMemcpyDeviceToDevice, s));
  CK(order_after(&ctx->join_ev, s, ctx->stream));
  ctx->have_phase = true;
  return UNOCG_OK;
}

extern "C" int unocg_set_phase_properties(unocg_ctx* ctx, const double* props) {
  if (!ctx || !props) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (ctx->n_phases < 1) return fail(ctx, UNOCG_ERR_STATE, "set the microstructure (phase count) first");
  const int np = ctx->physics == UNOCG_THERMAL ? 1 : 2;
  const int count = ctx->B * ctx->n_phases;
  for (int i = 0; i < count; ++i) {
    if (ctx->physics == UNOCG_THERMAL) {
      if (!(props[i] > 0.0) || !std::isfinite(props[i]))
        return fail(ctx, UNOCG_ERR_INVALID_ARG, "conductivities must be positive");
    } else {
      double E = props[2 * i], nu = props[2 * i + 1];
      if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5))
        return fail(ctx, UNOCG_ERR_INVALID_ARG, "need E > 0 and -1 < nu < 0.5");
    }
  }
  CK(dalloc(&ctx->props_d, (size_t)count * np));
  CK(dalloc(&ctx->mat64, (size_t)count * 2));
  CK(dalloc(&ctx->mat32, (size_t)count * 2));
  CK(cudaMemcpyAsync(ctx->props_d, props, (size_t)count * np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_material(ctx->props_d, ctx->mat64, ctx->mat32, count, ctx->physics, ctx->stream));
  CK(launch_ref_props(ctx->mat64, ctx->ref, ctx->B, ctx->n_phases, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_props = true;
  if (ctx->wkind == UNOCG_W_REFERENCE_MEDIUM) ctx->q_dirty = true;
  return UNOCG_OK;
}

extern "C" int unocg_set_macro_load(unocg_ctx* ctx, int n_loads, const double* loads) {
  if (!ctx || !loads || n_loads < 1 || n_loads > 8)
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "need 1 <= n_loads <= 8 and a load array");
  // a non-finite load would give a right-hand side without a finite entry, whose max-norm
  // reduction (fmax drops NaN) would read as zero: reject it here
  for (int i = 0; i < n_loads * ctx->dim; ++i)
    if (!std::isfinite(loads[i])) return fail(ctx, UNOCG_ERR_INVALID_ARG, "non-finite load");
  if (ctx->loads_d && n_loads != ctx->L) {
    cudaFree(ctx->loads_d);
    ctx->loads_d = nullptr;
  }
  if (n_loads != ctx->L) {
    // per-(instance, load) buffers depend on L
    free_graph(ctx);
    Fields64& a = ctx->f64;
    Fields32& b = ctx->f32;
    void* ptrs[] = {a.r, a.d, a.p, a.u, a.rhat, a.shat, b.r, b.d, b.p, b.u, b.rhat, b.shat, b.u64,
                    ctx->sc, ctx->ceff, ctx->sens, ctx->part};
    cudaStreamSynchronize(ctx->stream);
    for (void* p : ptrs)
      if (p) cudaFree(p);
    ctx->f64 = Fields64();
    ctx->f32 = Fields32();
    ctx->sc = nullptr;
    ctx->ceff = nullptr;
    ctx->sens = nullptr;
    ctx->part = nullptr;
    ctx->solved = false;
  }
  ctx->L = n_loads;
  CK(dalloc(&ctx->loads_d, (size_t)n_loads * ctx->dim));
  CK(cudaStreamSynchronize(ctx->stream));  // a solve in flight may still read the previous loads
  CK(cudaMemcpy(ctx->loads_d, loads, (size_t)n_loads * ctx->dim * sizeof(double), cudaMemcpyHostToDevice));
  ctx->have_loads = true;
  return UNOCG_OK;
}

// ------------------------------------------------------------------ weights
static int finish_weights(unocg_ctx* ctx) {
  // FP64 entries are in Q64 ([Bq][nh][C]); check, then make the FP32 / BF16 copies.
  const int NQ = ctx->c == 1 ? 1 : 6;
  const long long m = (long long)ctx->Bq * ctx->g.nh * NQ;
  CK(cudaMemsetAsync(ctx->fails, 0, sizeof(unsigned long long), ctx->stream));
  CK(launch_spd_check64(ctx->Q64, ctx->g.nh, ctx->Bq, ctx->c, ctx->spd_eps, ctx->fails, ctx->stream));
  unsigned long long nf = 0;
  CK(cudaMemcpyAsync(&nf, ctx->fails, sizeof(nf), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (nf) return fail(ctx, UNOCG_ERR_NOT_SPD, "UNO weights fail the safety check on " + std::to_string(nf) + " modes");
  CK(dalloc(&ctx->Q32, (size_t)m));
  CK(dalloc(&ctx->Q16, (size_t)m));
  CK(launch_convert32(ctx->Q64, ctx->Q32, m, ctx->stream));
  CK(launch_convert16(ctx->Q64, ctx->Q16, m, ctx->stream));
  CK(cudaMemsetAsync(ctx->fails, 0, sizeof(unsigned long long), ctx->stream));
  CK(launch_spd_check16(ctx->Q16, ctx->g.nh, ctx->Bq, ctx->c, ctx->spd_eps, ctx->fails, ctx->stream));
  CK(cudaMemcpyAsync(&nf, ctx->fails, sizeof(nf), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->bf16_spd_ok = (nf == 0);
  ctx->q_dirty = false;
  return UNOCG_OK;
}

static int build_weights(unocg_ctx* ctx) {
  const int NQ = ctx->c == 1 ? 1 : 6;
  if (ctx->wkind == UNOCG_W_REFERENCE_MEDIUM) {
    if (!ctx->have_props) return fail(ctx, UNOCG_ERR_STATE, "reference-medium weights need phase properties");
    if (ctx->Bq != ctx->B && ctx->Q64) {
      cudaFree(ctx->Q64); cudaFree(ctx->Q32); cudaFree(ctx->Q16);
      ctx->Q64 = nullptr; ctx->Q32 = nullptr; ctx->Q16 = nullptr;
    }
    ctx->Bq = ctx->B;
    CK(dalloc(&ctx->Q64, (size_t)ctx->B * ctx->g.nh * NQ));
    RefQArgs a{ctx->g, ctx->c, ctx->ref, ctx->Q64};
    CK(launch_ref_q(a, ctx->B, ctx->stream));
    return finish_weights(ctx);
  }
  // user weights: host FP64 copy -> device, psi (THETA) or bypass + modes (MODES), symmetrize the
  // self-conjugate planes
  if (ctx->Bq != 1 && ctx->Q64) {
    cudaFree(ctx->Q64); cudaFree(ctx->Q32); cudaFree(ctx->Q16);
    ctx->Q64 = nullptr; ctx->Q32 = nullptr; ctx->Q16 = nullptr;
  }
  ctx->Bq = 1;
  const size_t m = (size_t)ctx->g.nh * NQ;
  CK(dalloc(&ctx->Q64, m));
  double* tmp = nullptr;
  double* tmp2 = nullptr;
  const size_t mw = std::max(m, ctx->w_host.size());
  CK(cudaMalloc(&tmp, mw * sizeof(double)));
  cudaError_t e = cudaMalloc(&tmp2, m * sizeof(double));
  if (e != cudaSuccess) { cudaFree(tmp); return fail(ctx, UNOCG_ERR_OOM, "weights buffer"); }
  e = cudaMemcpyAsync(tmp, ctx->w_host.data(), ctx->w_host.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && ctx->wkind == UNOCG_W_THETA) {
    e = launch_psi64(tmp, tmp2, ctx->g.nh, ctx->c, ctx->stream);
    std::swap(tmp, tmp2);
  } else if (e == cudaSuccess && ctx->wkind == UNOCG_W_MODES) {
    e = launch_modes_expand64(tmp, ctx->modes_M, ctx->g, ctx->c, tmp2, ctx->stream);
    std::swap(tmp, tmp2);
  }
  if (e == cudaSuccess) e = launch_symmetrize64(tmp, ctx->Q64, ctx->g, NQ, 1, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(tmp);
  cudaFree(tmp2);
  if (e != cudaSuccess) return fail(ctx, UNOCG_ERR_CUDA, std::string("weights: ") + cudaGetErrorString(e));
  return finish_weights(ctx);
}

extern "C" int unocg_set_uno_modes(unocg_ctx* ctx, int M, const void* w, int dtype, double spd_eps) {
  if (!ctx) return UNOCG_ERR_INVALID_ARG;
  if (!modes_fit(ctx->g, M)) return fail(ctx, UNOCG_ERR_INVALID_ARG, "mode set [-M,M]^2 x [0,M] does not fit the grid");
  if (!w || (dtype != UNOCG_DTYPE_F64 && dtype != UNOCG_DTYPE_F32))
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "weights need a host array of dtype F64 or F32");
  if (!(spd_eps >= 0.0)) return fail(ctx, UNOCG_ERR_INVALID_ARG, "spd_eps must be >= 0");
  ctx->spd_eps = spd_eps;
  ctx->wkind = UNOCG_W_MODES;
  ctx->modes_M = M;
  ctx->q_dirty = true;
  const size_t m = (size_t)(1 + n_modes_of(M)) * (ctx->c == 1 ? 1 : 6);
  ctx->w_host.resize(m);
  for (size_t i = 0; i < m; ++i)
    ctx->w_host[i] = dtype == UNOCG_DTYPE_F64 ? ((const double*)w)[i] : (double)((const float*)w)[i];
  return build_weights(ctx);
}

extern "C" int unocg_set_uno_weights(unocg_ctx* ctx, int kind, const void* w, int dtype, double spd_eps) {
  NvtxRange nvtx_("unocg_set_uno_weights");
  if (!ctx) return UNOCG_ERR_INVALID_ARG;
  if (kind != UNOCG_W_REFERENCE_MEDIUM && kind != UNOCG_W_BLOCKS && kind != UNOCG_W_THETA)
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "unknown weight kind");
  if (!(spd_eps >= 0.0)) return fail(ctx, UNOCG_ERR_INVALID_ARG, "spd_eps must be >= 0");
  ctx->spd_eps = spd_eps;
  ctx->wkind = kind;
  ctx->q_dirty = true;
  if (kind != UNOCG_W_REFERENCE_MEDIUM) {
    if (!w || (dtype != UNOCG_DTYPE_F64 && dtype != UNOCG_DTYPE_F32))
      return fail(ctx, UNOCG_ERR_INVALID_ARG, "weights need a host array of dtype F64 or F32");
    const size_t m = (size_t)ctx->g.nh * (ctx->c == 1 ? 1 : 6);
    ctx->w_host.resize(m);
    for (size_t i = 0; i < m; ++i)
      ctx->w_host[i] = dtype == UNOCG_DTYPE_F64 ? ((const double*)w)[i] : (double)((const float*)w)[i];
    return build_weights(ctx);
  }
  if (ctx->have_props) return build_weights(ctx);
  return UNOCG_OK;
}

// ------------------------------------------------------------------ workspaces
static int ensure_workspace(unocg_ctx* ctx, int precision, int precond) {
  const long long n = ctx->g.n;
  const size_t BLc = (size_t)ctx->B * ctx->L * ctx->c;
  const size_t fld = BLc * n;
  const size_t hat = BLc * ctx->g.nh;
  const int BL = ctx->B * ctx->L;
  CK(dalloc(&ctx->sc, (size_t)BL));
  // partial sums: the largest per-kernel demand
  size_t need = 0;
  need = std::max(need, (size_t)BL * line_blocks_x(ctx->g, ctx->c, 8) * 2);
  need = std::max(need, (size_t)BL * line_blocks_x(ctx->g, ctx->c, 16) * 2);
  need = std::max(need, (size_t)BL * line_reg_blocks_x(ctx->g) * 2);
  need = std::max(need, (size_t)BL * line_tma_blocks_x(ctx->g) * 2);
  need = std::max(need, (size_t)BL * node_blocks_x(ctx->g));
  need = std::max(need, (size_t)BL * ku_blocks_x(ctx->g, ctx->c));
  need = std::max(need, (size_t)BL * ku_tasks_x(ctx->g, ctx->c));
  for (int k = 0; k < kKuTmaNumShapes; ++k) {
    if (ku_tma_supported(ctx->g, ctx->c, kKuTmaShapes[k]))
      need = std::max(need, (size_t)BL * ku_tma_blocks_x(ctx->g, kKuTmaShapes[k]));
    if (ku_vec_supported(ctx->g, ctx->c, kKuTmaShapes[k]))
      need = std::max(need, (size_t)BL * ku_vec_blocks_x(ctx->g, kKuTmaShapes[k]));
  }
  need = std::max(need, (size_t)BL * jac_blocks_x((long long)ctx->c * n, BL));
  need = std::max(need, (size_t)BL * ctx->c * 1184);
  need = std::max(need, (size_t)ctx->B * node_blocks_x(ctx->g) * 48);
  if (need > ctx->part_n) {
    if (ctx->part) cudaFree(ctx->part);
    ctx->part = nullptr;
    CK(cudaMalloc(&ctx->part, need * sizeof(double)));
    ctx->part_n = need;
  }
  CK(dalloc(&ctx->ceff, (size_t)ctx->B * ctx->dim * ctx->L));
  if (precision == UNOCG_FP64) {
    Fields64& f = ctx->f64;
    CK(dalloc(&f.r, fld)); CK(dalloc(&f.d, fld)); CK(dalloc(&f.p, fld)); CK(dalloc(&f.u, fld));
    if (precond == UNOCG_PRECOND_UNO) { CK(dalloc(&f.rhat, hat)); CK(dalloc(&f.shat, hat)); }
    if (precond == UNOCG_PRECOND_JACOBI) CK(dalloc(&ctx->invdiag64, (size_t)ctx->B * ctx->c * n));
  } else {
    Fields32& f = ctx->f32;
    CK(dalloc(&f.r, fld)); CK(dalloc(&f.d, fld)); CK(dalloc(&f.p, fld)); CK(dalloc(&f.u, fld));
    CK(dalloc(&f.u64, fld));
    CK(dalloc(&f.f64, fld));
    if (precond == UNOCG_PRECOND_UNO) { CK(dalloc(&f.rhat, hat)); CK(dalloc(&f.shat, hat)); }
    if (precond == UNOCG_PRECOND_JACOBI) CK(dalloc(&ctx->invdiag32, (size_t)ctx->B * ctx->c * n));
  }
  return UNOCG_OK;
}

// ------------------------------------------------------------------ the iteration, as launches
template <typename T> struct Sel;
template <> struct Sel<double> {
  using QT = double;
  static Fields64& f(unocg_ctx* c) { return c->f64; }
  static const double* Q(unocg_ctx* c) { return c->Q64; }
  static double* invdiag(unocg_ctx* c) { return c->invdiag64; }
  static double* u64(unocg_ctx* c) { return c->f64.u; }
  static double* u32(unocg_ctx*) { return nullptr; }
  static const double* f64(unocg_ctx*) { return nullptr; }
};
template <> struct Sel<float> {
  using QT = __nv_bfloat16;
  static Fields32& f(unocg_ctx* c) { return c->f32; }
  static const __nv_bfloat16* Q(unocg_ctx* c) { return c->Q16; }
  static float* invdiag(unocg_ctx* c) { return c->invdiag32; }
  static double* u64(unocg_ctx* c) { return c->f32.u64; }
  static const double* f64(unocg_ctx* c) { return c->f32.f64; }
  static float* u32(unocg_ctx* c) { return c->f32.u; }
};

struct Plan {
  unocg_solve_opts o;
  int mixed;
};

// Forward transform over axes 3 and 2: whole planes in one pass where a plane fits one block's
// shared memory, else the row pass (axis 3) followed by the in-place axis-2 column pass.
// 256 x 256 FP32 planes may take one pass on two-CTA clusters instead.  UNOCG_PLANE_CL selects
// the passes that take it, as a mask read at each enqueue: 1 forward, 2 inverse (default 0: on a
// 256^3 field of three loads, with the register row and column passes, the forward measured
// 281 us per launch as two passes against 310 us on clusters, the inverse 302 against 444 us).
static bool plane_cl_on(const Grid& g, int which) {
  const char* e = std::getenv("UNOCG_PLANE_CL");
  const int mask = e ? std::atoi(e) : 0;
  return (mask & which) != 0 && plane_cl_ok(g);
}

template <typename T>
static cudaError_t fwd_transform(PlaneFwdArgs<T>& a, cudaStream_t s, int only_pending) {
  if constexpr (std::is_same<T, float>::value)
    if (plane_cl_on(a.g, 1)) return launch_plane_fwd_cl(a, s);
  a.rows = plane_rows(a.g, sizeof(T) * 2);
  cudaError_t e = launch_plane_fwd<T>(a, s);
  if (e != cudaSuccess || a.rows == 0) return e;
  ColArgs<T> ca{a.g, a.c, a.BL, a.hat, a.sc, a.ft, only_pending};
  return launch_cols<T>(ca, -1, s);
}

// Inverse of fwd_transform; the column pass runs in place on a.shat, or into a.cols_out.
template <typename T>
static cudaError_t inv_transform(PlaneInvArgs<T>& a, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value)
    if (plane_cl_on(a.g, 2)) return launch_plane_inv_cl(a, s);
  a.rows = plane_rows(a.g, sizeof(T) * 2);
  if (a.rows) {
    ColArgs<T> ca{a.g, a.c, a.BL, const_cast<cplx<T>*>(a.shat), a.sc, a.ft, 0, a.cols_out};
    cudaError_t e = launch_cols<T>(ca, +1, s);
    if (e != cudaSuccess) return e;
    if (a.cols_out) a.shat = a.cols_out;
  }
  return launch_plane_inv<T>(a, s);
}

template <typename T>
static cudaError_t enq_plane_fwd(unocg_ctx* ctx, cudaStream_t s, const LoopCtl& ctl, int after_replace, int ticket) {
  auto& f = Sel<T>::f(ctx);
  PlaneFwdArgs<T> a{};
  a.g = ctx->g; a.c = ctx->c; a.BL = ctx->B * ctx->L;
  a.r = f.r; a.p = f.p; a.src = nullptr; a.hat = f.rhat; a.sc = ctx->sc;
  a.ft = tables(ctx, sizeof(T) == 8);
  a.ticket = ctx->tickets + ticket;
  a.ctl = ctl; a.after_replace = after_replace; a.standalone = 0;
  return fwd_transform<T>(a, s, after_replace);
}

template <typename T>
static cudaError_t enq_jac_a(unocg_ctx* ctx, cudaStream_t s, const LoopCtl& ctl, int after_replace, int ticket, int precond) {
  auto& f = Sel<T>::f(ctx);
  JacArgs<T> a{};
  a.c = ctx->c; a.BL = ctx->B * ctx->L; a.L = ctx->L; a.n = ctx->g.n;
  a.r = f.r; a.p = f.p; a.d = f.d; a.u = f.u;
  a.invdiag = precond == UNOCG_PRECOND_JACOBI ? Sel<T>::invdiag(ctx) : nullptr;
  a.sc = ctx->sc; a.red = Reduce{ctx->part, ctx->tickets + ticket};
  a.ctl = ctl; a.after_replace = after_replace;
  return launch_jac<T>(a, 0, s);
}

template <typename T>
static cudaError_t enq_residual_check(unocg_ctx* ctx, cudaStream_t s, const LoopCtl& ctl, int after_replace, int precond) {
  if (precond == UNOCG_PRECOND_UNO)
    return enq_plane_fwd<T>(ctx, s, ctl, after_replace, after_replace ? T_PLANE2 : T_PLANE);
  return enq_jac_a<T>(ctx, s, ctl, after_replace, after_replace ? T_JAC2 : T_JAC, precond);
}

template <typename T>
static cudaError_t enq_pre(unocg_ctx* ctx, cudaStream_t s, const Plan& pl, const LoopCtl& ctl) {
  auto& f = Sel<T>::f(ctx);
  const int BL = ctx->B * ctx->L;
  cudaError_t e = cudaMemsetAsync(ctx->sc, 0, BL * sizeof(CgScal), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->tickets, 0, kMaxTickets * sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->flags + 2, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->flags + 6, 0, sizeof(int), s);  // wait-timeout flag
  if (e != cudaSuccess) return e;
  InitArgs<T> ia{};
  ia.g = ctx->g; ia.c = ctx->c; ia.L = ctx->L; ia.phase = ctx->phase; ia.mat = material(ctx);
  ia.loads = ctx->loads_d; ia.r = f.r; ia.u = f.u; ia.d = f.d; ia.p = f.p;
  ia.u64 = pl.mixed ? ctx->f32.u64 : nullptr;
  ia.f64 = pl.mixed ? ctx->f32.f64 : nullptr;
  e = launch_init<T>(ia, BL, s);
  if (e != cudaSuccess) return e;
  if (pl.o.precond == UNOCG_PRECOND_JACOBI) {
    DiagArgs<T> da{ctx->g, ctx->c, ctx->phase, material(ctx), Sel<T>::invdiag(ctx)};
    e = launch_invdiag<T>(da, ctx->B, s);
    if (e != cudaSuccess) return e;
  }
  return enq_residual_check<T>(ctx, s, ctl, 0, pl.o.precond);
}

// TMA-staged axis-1 pass of the mixed-precision loop (c = 1: N1 of 2^k or 3 x 2^k points up to 256; c = 3: up to 64);
// UNOCG_LINE_TMA=0 at run time keeps the register-FFT pass (for comparisons)
static bool line_tma_on(const unocg_ctx* ctx) {
  const char* e = std::getenv("UNOCG_LINE_TMA");  // read at every enqueue
  return !(e && std::atoi(e) == 0) && line_tma_supported(ctx->g, ctx->c);
}

// c = 1: the persistent TMA pipeline for the axis-1 pass with UNOCG_LINE_TP=1 (read at each
// enqueue).  Off by default: with the conflict-free lane layout both passes move the same bytes
// at about the same rate (256^3 x 3 loads: 174 us per launch pipelined, 170 us one tile per
// block).
static bool line_tp_on(const unocg_ctx* ctx) {
  const char* e = std::getenv("UNOCG_LINE_TP");
  return ctx->c == 1 && e && std::atoi(e) == 1 && line_tp_supported(ctx->g);
}

template <typename T>
static cudaError_t enq_precond(unocg_ctx* ctx, cudaStream_t s, const Plan& pl, const LoopCtl& ctl, int part) {
  // part 0: transform axis 1 + block multiply (UNO) / direction update (Jacobi, none)
  // part 1: inverse plane transform with the direction update (UNO only)
  auto& f = Sel<T>::f(ctx);
  const int BL = ctx->B * ctx->L;
  if (pl.o.precond == UNOCG_PRECOND_UNO) {
    if (part == 0) {
      using QT = typename Sel<T>::QT;
      LineArgs<T, QT> la{};
      la.g = ctx->g; la.c = ctx->c; la.BL = BL; la.L = ctx->L;
      la.hat = f.rhat; la.shat = f.shat; la.ghat = nullptr;
      la.Q = Sel<T>::Q(ctx);
      la.q_inst_stride = ctx->Bq > 1 ? ctx->g.nh * (ctx->c == 1 ? 1 : 6) : 0;
      la.scale = 1.0 / (double)ctx->g.n;
      la.sc = ctx->sc; la.red = Reduce{ctx->part, ctx->tickets + T_LINE};
      la.ft = tables(ctx, sizeof(T) == 8);
      la.flexible = pl.o.flexible; la.standalone = 0; la.gq = nullptr;
      if constexpr (std::is_same<T, float>::value)
        if (line_tma_on(ctx)) {
          if (line_tp_on(ctx)) return launch_line_tp(la, ctx->flags + 6, ctx->spin_limit, ctx->sm_count, s);
          return launch_line_tma(la, ctx->flags + 6, ctx->spin_limit, s);
        }
      return launch_line<T, QT>(la, 0, s);
    }
    PlaneInvArgs<T> pa{};
    pa.g = ctx->g; pa.c = ctx->c; pa.BL = BL; pa.shat = f.shat; pa.d = f.d; pa.u = f.u; pa.dst = nullptr;
    pa.sc = ctx->sc; pa.ft = tables(ctx, sizeof(T) == 8); pa.standalone = 0;
    // r_hat is free until the next forward pass: the axis-2 pass of large planes writes there
    // and leaves s_hat for the flexible r . s_old of the next block multiply
    pa.cols_out = f.rhat;
    return inv_transform<T>(pa, s);
  }
  if (part == 1) return cudaSuccess;
  JacArgs<T> a{};
  a.c = ctx->c; a.BL = BL; a.L = ctx->L; a.n = ctx->g.n;
  a.r = f.r; a.p = f.p; a.d = f.d; a.u = f.u;
  a.invdiag = pl.o.precond == UNOCG_PRECOND_JACOBI ? Sel<T>::invdiag(ctx) : nullptr;
  a.sc = ctx->sc; a.red = Reduce{ctx->part, ctx->tickets + T_JAC};
  a.ctl = ctl;
  return launch_jac<T>(a, 1, s);
}

// K d tiles: 0 the earlier kernels, 1..8 the TMA-staged kernel with shape kKuTmaShapes[k - 1],
// 9..16 the vector march (register window over node planes read from global memory) with shape
// kKuTmaShapes[k - 9].
constexpr int kKuTiles = 2 * kKuTmaNumShapes;
static bool ku_tile_ok(const Grid& g, int c, int tile) {
  if (tile == 0) return true;
  if (tile < 0 || tile > kKuTiles) return false;
  return tile <= kKuTmaNumShapes ? ku_tma_supported(g, c, kKuTmaShapes[tile - 1])
                                 : ku_vec_supported(g, c, kKuTmaShapes[tile - 1 - kKuTmaNumShapes]);
}

// Automatic choice, the vector march in both regimes:
//  * below 10^6 nodes per field (fields in L2, latency bound): the first of the 6-plane tiles
//    (8, 6), (16, 6) with at least one block per SM over all (instance, load) fields, else the
//    register column march (64^3, 3 loads, back-to-back launches: 5.6 us for (8, 6) against 8.0
//    for the column march and 9.0 for the best TMA tile);
//  * from 10^6 nodes: of the vector shapes (4, 24), (8, 24), (4, 12), (8, 12), (2, 12) with at
//    least two blocks per SM the one that keeps the most warps resident, the earlier on a tie
//    (256^3 x 3 loads: (4, 24) 178 us against 182 for (2, 12) and 218 for the best TMA tile;
//    192^3: (2, 12) 88 us, 15 warps per SM, against 97 us for (4, 24), 12 warps), else the TMA
//    tile of most blocks.
static int ku_tma_choice(const unocg_ctx* ctx) {
  if (ctx->c != 1 || ctx->ku_tile == 0) return 0;
  if (ctx->ku_tile > 0) return ku_tile_ok(ctx->g, 1, ctx->ku_tile) ? ctx->ku_tile : 0;
  const long long BL = (long long)ctx->B * std::max(ctx->L, 1);
  const long long sms = std::max(ctx->sm_count, 1);
  auto first_vec = [&](std::initializer_list<int> pref, long long want) {
    for (int k : pref) {  // 1-based shape indices
      const KuTmaShape sh = kKuTmaShapes[k - 1];
      if (ku_vec_supported(ctx->g, 1, sh) && BL * ku_vec_blocks_x(ctx->g, sh) >= want) return kKuTmaNumShapes + k;
    }
    return 0;
  };
  if (ctx->g.n < 1000000) return first_vec({8, 5}, sms);  // (8, 6), (16, 6); else the column march
  // from 10^6 nodes: of (4, 24), (8, 24), (4, 12), (8, 12), (2, 12) with at least two blocks per
  // SM, the one with the most resident warps (128 registers a thread), the earlier on a tie
  int v = 0, v_warps = 0;
  for (int k : {6, 4, 1, 2, 3}) {
    const KuTmaShape sh = kKuTmaShapes[k - 1];
    if (!ku_vec_supported(ctx->g, 1, sh) || BL * ku_vec_blocks_x(ctx->g, sh) < 2 * sms) continue;
    const int threads = ku_tma_threads(ctx->g, sh);
    const int warps = std::min(65536 / (threads * 128), 2048 / threads) * (threads / 32);
    if (warps > v_warps) { v = kKuTmaNumShapes + k; v_warps = warps; }
  }
  if (v) return v;
  int most = 0;
  long long most_blocks = -1;
  for (int k = 0; k < kKuTmaNumShapes; ++k) {
    const KuTmaShape sh = kKuTmaShapes[k];
    if (!ku_tma_supported(ctx->g, 1, sh)) continue;
    const long long blocks = BL * ku_tma_blocks_x(ctx->g, sh);
    if (blocks > most_blocks) { most = k + 1; most_blocks = blocks; }
  }
  return most;
}

template <typename T>
static StencilArgs<T> ku_args(unocg_ctx* ctx) {
  auto& f = Sel<T>::f(ctx);
  StencilArgs<T> ka{};
  ka.g = ctx->g; ka.c = ctx->c; ka.BL = ctx->B * ctx->L; ka.L = ctx->L; ka.phase = ctx->phase;
  ka.mat = material(ctx);
  ka.d = f.d; ka.p = f.p; ka.sc = ctx->sc; ka.red = Reduce{ctx->part, ctx->tickets + T_KU}; ka.standalone = 0;
  ka.ku_tma = sizeof(T) == 4 ? ku_tma_choice(ctx) : 0;
  ka.err = ctx->flags + 6;
  ka.spin_limit = ctx->spin_limit;
  return ka;
}

template <typename T>
static cudaError_t enq_ku(unocg_ctx* ctx, cudaStream_t s) {
  return launch_ku<T>(ku_args<T>(ctx), s);
}

template <typename T>
static cudaError_t enq_body(unocg_ctx* ctx, cudaStream_t s, const Plan& pl, const LoopCtl& ctl) {
  cudaError_t e = enq_precond<T>(ctx, s, pl, ctl, 0);
  if (e == cudaSuccess) e = enq_precond<T>(ctx, s, pl, ctl, 1);
  if (e == cudaSuccess) e = enq_ku<T>(ctx, s);
  if (e == cudaSuccess) e = enq_residual_check<T>(ctx, s, ctl, 0, pl.o.precond);
  return e;
}

// Mixed precision: the FP64 residual rref = f - K u64 (f32.f64, written with f by the set-up)
// is brought up to date, rref -= K (u32 + alpha d), in float-pair arithmetic; the pending
// increment is folded into u64 afterwards.
static ReplaceArgs replace_args(unocg_ctx* ctx, int only_pending, int into_rmax) {
  ReplaceArgs ra{};
  ra.g = ctx->g; ra.c = ctx->c; ra.L = ctx->L; ra.phase = ctx->phase; ra.mat = material(ctx);
  ra.u32 = ctx->f32.u; ra.d = ctx->f32.d; ra.rref = ctx->f32.f64; ra.r = into_rmax ? ctx->f32.r : nullptr;
  ra.sc = ctx->sc; ra.only_pending = only_pending; ra.into_rmax = into_rmax;
  return ra;
}

// Residual replacement for the pending (instance, load) pairs, then a fresh residual check
template <typename T>
static cudaError_t enq_replace(unocg_ctx* ctx, cudaStream_t s, const Plan& pl, const LoopCtl& ctl) {
  auto& f = Sel<T>::f(ctx);
  const int BL = ctx->B * ctx->L;
  cudaError_t e = launch_replace(replace_args(ctx, 1, 1), BL, s);
  if (e != cudaSuccess) return e;
  FoldArgs<T> fa{};
  fa.c = ctx->c; fa.n = ctx->g.n; fa.u64 = Sel<T>::u64(ctx); fa.u32 = Sel<T>::u32(ctx); fa.d = f.d;
  fa.sc = ctx->sc; fa.only_pending = 1; fa.part = nullptr;
  e = launch_fold<T>(fa, BL, s);
  if (e != cudaSuccess) return e;
  return enq_residual_check<T>(ctx, s, ctl, 1, pl.o.precond);
}

// rref_kept: the loop maintained the FP64 residual rref (graph and host loops; the persistent
// kernel replaces residuals by FP64 evaluations of its own and does not)
template <typename T>
static cudaError_t enq_post(unocg_ctx* ctx, cudaStream_t s, const Plan& pl, bool rref_kept = true) {
  const bool inc = pl.mixed && rref_kept;
  auto& f = Sel<T>::f(ctx);
  const int BL = ctx->B * ctx->L;
  const int nparts = 256;  // blocks per field of the final fold and the mean
  // reported true residual of the final iterate: mixed precision brings rref up to date with the
  // last increment (before the final fold); FP64 evaluates f - K u directly (after it)
  cudaError_t e = cudaSuccess;
  if (inc) e = launch_replace(replace_args(ctx, 0, 0), BL, s);
  if (e != cudaSuccess) return e;
  FoldArgs<T> fa{};
  fa.c = ctx->c; fa.n = ctx->g.n; fa.u64 = Sel<T>::u64(ctx); fa.u32 = Sel<T>::u32(ctx); fa.d = f.d;
  fa.sc = ctx->sc; fa.only_pending = 0; fa.part = ctx->part;
  e = launch_final<T>(fa, BL, nparts, s);
  if (e != cudaSuccess) return e;
  if (!inc) {
    TrueResArgs<T> ta{};
    ta.g = ctx->g; ta.c = ctx->c; ta.L = ctx->L; ta.phase = ctx->phase; ta.mat = material(ctx);
    ta.loads = ctx->loads_d; ta.u64 = Sel<T>::u64(ctx); ta.f64 = Sel<T>::f64(ctx); ta.r = nullptr; ta.sc = ctx->sc;
    ta.only_pending = 0; ta.require_started = 0; ta.into_rmax = 0;
    e = launch_true_res<T>(ta, BL, s);
    if (e != cudaSuccess) return e;
  }
  e = launch_zero_mean(Sel<T>::u64(ctx), ctx->part, nparts, ctx->c, ctx->g.n, BL, s);
  if (e != cudaSuccess) return e;
  AvgArgs aa{};
  aa.g = ctx->g; aa.c = ctx->c; aa.L = ctx->L; aa.phase = ctx->phase; aa.mat = material(ctx);
  aa.loads = ctx->loads_d; aa.u64 = Sel<T>::u64(ctx); aa.part = ctx->part;
  return launch_average(aa, ctx->B, ctx->ceff, s);
}

// Captures one context's solve into the capture in progress on stream cs: set-up, the WHILE
// conditional node whose body is one CG iteration (with an IF node for the residual replacement
// of the mixed path), post-processing.  The conditional handles belong to the capture's graph.
template <typename T>
static cudaError_t capture_chain(unocg_ctx* ctx, const Plan& pl, cudaStream_t cs) {
  cudaStream_t bs = nullptr, rs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
  cudaGraph_t cg = nullptr;
  cudaStreamCaptureStatus st;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, nullptr, nullptr, nullptr);
  cudaGraphConditionalHandle hw = 0, hi = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, cg, 0, cudaGraphCondAssignDefault);
  LoopCtl ctl{};
  ctl.tol = pl.o.tol; ctl.max_iter = pl.o.max_iter; ctl.mixed = pl.mixed;
  ctl.replace_every = pl.o.replace_every; ctl.replace_drop = pl.o.replace_drop; ctl.flexible = pl.o.flexible;
  ctl.h_while = hw; ctl.set_while = 1; ctl.set_if = 0;
  ctl.counters = ctx->flags + 2;
  if (e == cudaSuccess) e = enq_pre<T>(ctx, cs, pl, ctl);
  cudaGraphNode_t wnode;
  cudaGraphNodeParams wp{};
  if (e == cudaSuccess) {
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &nd);
    if (e == cudaSuccess) {
      wp.type = cudaGraphNodeTypeConditional;
      wp.conditional.handle = hw;
      wp.conditional.type = cudaGraphCondTypeWhile;
      wp.conditional.size = 1;
      e = cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &wp);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  }
  if (e == cudaSuccess) {
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    LoopCtl bctl = ctl;
    if (e == cudaSuccess && pl.mixed) {
      e = cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault);
      bctl.h_if = hi;
      bctl.set_if = 1;
    }
    if (e == cudaSuccess) e = enq_body<T>(ctx, bs, pl, bctl);
    if (e == cudaSuccess && pl.mixed) {
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaGraph_t bg = nullptr;
      e = cudaStreamGetCaptureInfo(bs, &st, nullptr, &bg, &deps, nullptr, &nd);
      cudaGraphNode_t inode;
      cudaGraphNodeParams ip{};
      if (e == cudaSuccess) {
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hi;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        e = cudaGraphAddNode(&inode, bg, deps, nullptr, nd, &ip);
      }
      if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(bs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
      if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(rs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        LoopCtl rctl = ctl;
        rctl.set_while = 0;
        rctl.set_if = 0;
        if (e == cudaSuccess) e = enq_replace<T>(ctx, rs, pl, rctl);
        cudaGraph_t tmp;
        cudaError_t e2 = cudaStreamEndCapture(rs, &tmp);
        if (e == cudaSuccess) e = e2;
      }
    }
    cudaGraph_t tmp;
    cudaError_t e2 = cudaStreamEndCapture(bs, &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = enq_post<T>(ctx, cs, pl);
  if (bs) cudaStreamDestroy(bs);
  if (rs) cudaStreamDestroy(rs);
  return e;
}

template <typename T>
static int build_graph(unocg_ctx* ctx, const Plan& pl) {
  cudaStream_t cs = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = capture_chain<T>(ctx, pl, cs);
  cudaError_t e3 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e3;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(ctx, UNOCG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(ctx, UNOCG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  free_graph(ctx);
  ctx->graph = g;
  ctx->exec = ex;
  return UNOCG_OK;
}

// Host-driven loop (debugging): one residual check per iteration read back by the host.
template <typename T>
static int run_host_loop(unocg_ctx* ctx, const Plan& pl) {
  cudaStream_t s = ctx->stream;
  LoopCtl ctl{};
  ctl.tol = pl.o.tol; ctl.max_iter = pl.o.max_iter; ctl.mixed = pl.mixed;
  ctl.replace_every = pl.o.replace_every; ctl.replace_drop = pl.o.replace_drop; ctl.flexible = pl.o.flexible;
  ctl.active_flag = ctx->flags; ctl.replace_flag = ctx->flags + 1;
  ctl.counters = ctx->flags + 2;
  CK(enq_pre<T>(ctx, s, pl, ctl));
  int hf[2] = {0, 0};
  const long long cap = 4LL * pl.o.max_iter + 16;
  for (long long it = 0; it < cap; ++it) {
    CK(cudaMemcpyAsync(hf, ctx->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!hf[0]) break;
    CK(enq_body<T>(ctx, s, pl, ctl));
    if (pl.mixed) {
      CK(cudaMemcpyAsync(hf, ctx->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hf[1]) {
        LoopCtl rctl = ctl;
        rctl.active_flag = nullptr;  // keep the loop running; the next check decides
        CK(enq_replace<T>(ctx, s, pl, rctl));
      }
    }
  }
  CK(enq_post<T>(ctx, s, pl));
  return UNOCG_OK;
}

// Whole loop in one cooperative launch (k_persist.cu), between the set-up and post kernels.
static bool persistent_fits(unocg_ctx* ctx, const unocg_solve_opts* o) {
  if (o->precond != UNOCG_PRECOND_UNO) return false;
  const int BL = ctx->B * ctx->L;
  if (BL > 128 || ctx->B * ctx->n_phases * 2 > 4096) return false;
  const int eb = o->precision == UNOCG_FP64 ? 16 : 8;
  const int tb = (eb == 8 ? 16 : 8) * (ctx->c == 1 ? 2 : 1);
  size_t smem = persist_smem_bytes(ctx->g, ctx->c, tb, eb, BL, ctx->B, ctx->n_phases, eb / 2);
  return smem <= 200 * 1024;
}

template <typename T>
static int run_persistent(unocg_ctx* ctx, const Plan& pl) {
  using QT = typename Sel<T>::QT;
  cudaStream_t s = ctx->stream;
  auto& f = Sel<T>::f(ctx);
  const int BL = ctx->B * ctx->L;
  CK(cudaMemsetAsync(ctx->sc, 0, BL * sizeof(CgScal), s));
  CK(cudaMemsetAsync(ctx->flags, 0, 8 * sizeof(int), s));
  InitArgs<T> ia{};
  ia.g = ctx->g; ia.c = ctx->c; ia.L = ctx->L; ia.phase = ctx->phase; ia.mat = material(ctx);
  ia.loads = ctx->loads_d; ia.r = f.r; ia.u = f.u; ia.d = f.d; ia.p = f.p;
  ia.u64 = pl.mixed ? ctx->f32.u64 : nullptr;
  ia.f64 = pl.mixed ? ctx->f32.f64 : nullptr;
  CK(launch_init<T>(ia, BL, s));
  PersistArgs<T, QT> a{};
  a.pf.g = ctx->g; a.pf.c = ctx->c; a.pf.BL = BL; a.pf.r = f.r; a.pf.p = f.p; a.pf.hat = f.rhat;
  a.pf.ft = tables(ctx, sizeof(T) == 8); a.pf.standalone = 0;
  a.la.g = ctx->g; a.la.c = ctx->c; a.la.BL = BL; a.la.L = ctx->L; a.la.hat = f.rhat; a.la.shat = f.shat;
  a.la.Q = Sel<T>::Q(ctx);
  a.la.q_inst_stride = ctx->Bq > 1 ? ctx->g.nh * (ctx->c == 1 ? 1 : 6) : 0;
  a.la.scale = 1.0 / (double)ctx->g.n; a.la.ft = tables(ctx, sizeof(T) == 8);
  a.la.flexible = pl.o.flexible; a.la.standalone = 0;
  a.la.tb = (sizeof(T) == 4 ? 16 : 8) * (ctx->c == 1 ? 2 : 1);
  a.pi.g = ctx->g; a.pi.c = ctx->c; a.pi.BL = BL; a.pi.shat = f.shat; a.pi.d = f.d; a.pi.u = f.u;
  a.pi.ft = tables(ctx, sizeof(T) == 8); a.pi.standalone = 0;
  a.ka.g = ctx->g; a.ka.c = ctx->c; a.ka.BL = BL; a.ka.L = ctx->L; a.ka.phase = ctx->phase;
  a.ka.mat = material(ctx); a.ka.d = f.d; a.ka.p = f.p; a.ka.standalone = 0;
  a.fo.c = ctx->c; a.fo.n = ctx->g.n; a.fo.u64 = Sel<T>::u64(ctx); a.fo.u32 = Sel<T>::u32(ctx); a.fo.d = f.d;
  a.loads = ctx->loads_d;
  a.sc = ctx->sc;
  a.B = ctx->B; a.L = ctx->L; a.BL = BL;
  a.n_line_tasks = line_blocks_x(ctx->g, ctx->c, sizeof(T) * 2);
  a.n_ku_tasks = ku_tasks_x(ctx->g, ctx->c);
  a.n_tr_tasks = node_blocks_x(ctx->g);
  a.n_fold_chunks = 64;
  const long long np = (long long)ctx->c * ctx->g.n1;
  a.off_max = 0;
  a.off_line = (long long)BL * np;
  a.off_ku = a.off_line + (long long)BL * a.n_line_tasks * 2;
  const size_t need = (size_t)(a.off_ku + (long long)BL * a.n_ku_tasks);
  if (need > ctx->part_n) {
    if (ctx->part) cudaFree(ctx->part);
    ctx->part = nullptr;
    CK(cudaMalloc(&ctx->part, need * sizeof(double)));
    ctx->part_n = need;
  }
  a.part = ctx->part;
  a.counters = ctx->flags + 2;
  a.bar = reinterpret_cast<unsigned int*>(ctx->flags + 4);
  a.err = ctx->flags + 6;
  a.ctl.tol = pl.o.tol; a.ctl.max_iter = pl.o.max_iter; a.ctl.mixed = pl.mixed;
  a.ctl.replace_every = pl.o.replace_every; a.ctl.replace_drop = pl.o.replace_drop; a.ctl.flexible = pl.o.flexible;
  a.spin_limit = ctx->spin_limit;
  CK(launch_persist<T, QT>(a, s, ctx->sm_count));
  CK(enq_post<T>(ctx, s, pl, false));
  return UNOCG_OK;
}

static int prepare_solve(unocg_ctx* ctx, const unocg_solve_opts* o, Plan* pl) {
  if (!ctx || !o) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->have_phase || !ctx->have_props || !ctx->have_loads)
    return fail(ctx, UNOCG_ERR_STATE, "set microstructure, phase properties and loads first");
  if (o->precond < 0 || o->precond > 2 || (o->precision != UNOCG_FP64 && o->precision != UNOCG_MIXED) ||
      !(o->tol > 0.0) || o->max_iter < 1 || o->replace_every < 0 || !(o->replace_drop >= 0.0) ||
      !(o->replace_drop < 1.0))
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "invalid solve options");
  if (o->precond == UNOCG_PRECOND_UNO) {
    if (ctx->wkind < 0) return fail(ctx, UNOCG_ERR_STATE, "set UNO weights first");
    if (ctx->q_dirty) {
      int rc = build_weights(ctx);
      if (rc) return rc;
    }
    if (o->precision == UNOCG_MIXED && !ctx->bf16_spd_ok)
      return fail(ctx, UNOCG_ERR_NOT_SPD, "UNO weights fail the safety check after rounding to BF16");
  }
  pl->o = *o;
  pl->mixed = o->precision == UNOCG_MIXED;
  if (!pl->mixed) {
    pl->o.replace_every = 0;
    pl->o.replace_drop = 0.0;
  }
  return ensure_workspace(ctx, o->precision, o->precond);
}

extern "C" int unocg_get_uno_weights(unocg_ctx* ctx, int instance, double* out) {
  if (!ctx || !out) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (ctx->wkind < 0) return fail(ctx, UNOCG_ERR_STATE, "set UNO weights first");
  if (instance < 0 || instance >= ctx->B) return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance out of range");
  if (ctx->q_dirty) {
    int rc = build_weights(ctx);
    if (rc) return rc;
  }
  const size_t m = (size_t)ctx->g.nh * (ctx->c == 1 ? 1 : 6);
  const double* src = ctx->Q64 + (ctx->Bq > 1 ? instance * m : 0);
  // the weights are built on the context stream (non-blocking: a plain cudaMemcpy would not wait)
  CK(cudaMemcpyAsync(out, src, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return UNOCG_OK;
}

extern "C" int unocg_solve_async(unocg_ctx* ctx, const unocg_solve_opts* o) {
  NvtxRange nvtx_("unocg_solve_async");
  Plan pl;
  int rc = prepare_solve(ctx, o, &pl);
  if (rc) return rc;
  ctx->last_opts = *o;
  ctx->last_precision = o->precision;
  ctx->solved = false;
  int path = o->use_graph;
  // automatic: the driver chosen by the autotuner, else the graph loop (a kernel boundary in a
  // graph costs less than a grid barrier)
  if (path == 3) path = (ctx->tuned_path == 2 && persistent_fits(ctx, o)) ? 2 : 1;
  if (path == 2 && !persistent_fits(ctx, o)) return fail(ctx, UNOCG_ERR_INVALID_ARG, "problem too large for the persistent kernel");
  ctx->last_path = path;
  if (path == 0) {
    rc = pl.mixed ? run_host_loop<float>(ctx, pl) : run_host_loop<double>(ctx, pl);
    if (rc) return rc;
  } else if (path == 2) {
    rc = pl.mixed ? run_persistent<float>(ctx, pl) : run_persistent<double>(ctx, pl);
    if (rc) return rc;
  } else {
    GraphKey k;
    k.precond = o->precond; k.precision = o->precision; k.flexible = o->flexible;
    k.replace_every = pl.o.replace_every; k.replace_drop = pl.o.replace_drop; k.max_iter = o->max_iter; k.L = ctx->L; k.tol = o->tol;
    if (!ctx->exec || !(k == ctx->key)) {
      rc = pl.mixed ? build_graph<float>(ctx, pl) : build_graph<double>(ctx, pl);
      if (rc) return rc;
      ctx->key = k;
    }
    CK(cudaGraphLaunch(ctx->exec, ctx->stream));
  }
  ctx->solved = true;
  return UNOCG_OK;
}

extern "C" int unocg_solve_wait(unocg_ctx* ctx, unocg_solve_info* info) {
  if (!ctx) return UNOCG_ERR_INVALID_ARG;
  if (!ctx->solved) return fail(ctx, UNOCG_ERR_STATE, "no solve in flight");
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  const int BL = ctx->B * ctx->L;
  std::vector<CgScal> hs(BL);
  CK(cudaMemcpy(hs.data(), ctx->sc, BL * sizeof(CgScal), cudaMemcpyDeviceToHost));
  int status = UNOCG_OK, mx = 0;
  for (int i = 0; i < BL; ++i) {
    const CgScal& s = hs[i];
    int st = s.done ? s.status : UNOCG_ERR_NOT_CONVERGED;
    if (status == UNOCG_OK && st != UNOCG_OK) status = st;
    mx = std::max(mx, s.iters);
    if (info) {
      double f0 = s.r0max;
      if (info->iters) info->iters[i] = s.iters;
      if (info->rel_res) info->rel_res[i] = f0 > 0 ? s.rmax / f0 : 0.0;
      if (info->true_rel_res) {
        double tm;
        std::memcpy(&tm, &s.tmax_bits, sizeof(tm));
        info->true_rel_res[i] = f0 > 0 ? tm / f0 : 0.0;
      }
      if (info->load_status) info->load_status[i] = st;
    }
  }
  int ctl[8];
  CK(cudaMemcpy(ctl, ctx->flags, 8 * sizeof(int), cudaMemcpyDeviceToHost));
  if (ctl[6]) {
    status = UNOCG_ERR_DEVICE_TIMEOUT;
  }
  if (info) {
    int cnt[2] = {ctl[2], ctl[3]};
    info->status = status;
    info->max_iters = mx;
    info->checks = cnt[0];
    info->replacements = cnt[1];
  }
  if (status != UNOCG_OK) {
    ctx->err = status == UNOCG_ERR_NOT_CONVERGED ? "not converged within max_iter"
             : status == UNOCG_ERR_DEVICE_TIMEOUT ? "grid barrier wait expired" : "CG breakdown";
  }
  return status;
}

extern "C" int unocg_solve(unocg_ctx* ctx, const unocg_solve_opts* o, unocg_solve_info* info) {
  int rc = unocg_solve_async(ctx, o);
  if (rc) return rc;
  return unocg_solve_wait(ctx, info);
}

// ------------------------------------------------------------------ outputs
static const double* final_u(unocg_ctx* ctx) {
  return ctx->last_precision == UNOCG_FP64 ? ctx->f64.u : ctx->f32.u64;
}

extern "C" int unocg_get_fluctuation(unocg_ctx* ctx, int instance, int load, double* out) {
  if (!ctx || !out) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->solved) return fail(ctx, UNOCG_ERR_STATE, "no solution");
  if (instance < 0 || instance >= ctx->B || load < 0 || load >= ctx->L)
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance/load out of range");
  const long long n = ctx->g.n;
  CK(dalloc(&ctx->stage, (size_t)ctx->c * n));
  const double* src = final_u(ctx) + ((long long)instance * ctx->L + load) * ctx->c * n;
  CK(launch_interleave(src, ctx->stage, ctx->c, n, ctx->stream));
  CK(cudaMemcpyAsync(out, ctx->stage, (size_t)ctx->c * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return UNOCG_OK;
}

extern "C" int unocg_get_fluctuation_dev(unocg_ctx* ctx, int instance, int load, double* out_dev, void* stream) {
  if (!ctx || !out_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->solved) return fail(ctx, UNOCG_ERR_STATE, "no solution");
  if (instance < 0 || instance >= ctx->B || load < 0 || load >= ctx->L)
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance/load out of range");
  const long long n = ctx->g.n;
  const double* src = final_u(ctx) + ((long long)instance * ctx->L + load) * ctx->c * n;
  cudaStream_t s = (cudaStream_t)stream;
  CK(order_after(&ctx->join_ev, ctx->stream, s));
  CK(cudaMemcpyAsync(out_dev, src, (size_t)ctx->c * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(order_after(&ctx->join_ev, s, ctx->stream));
  return UNOCG_OK;
}

extern "C" int unocg_get_effective_tensor(unocg_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->solved) return fail(ctx, UNOCG_ERR_STATE, "no solution");
  CK(cudaMemcpyAsync(out, ctx->ceff, (size_t)ctx->B * ctx->dim * ctx->L * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return UNOCG_OK;
}

extern "C" int unocg_get_sensitivity(unocg_ctx* ctx, double* out) {
  if (!ctx || !out) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->solved) return fail(ctx, UNOCG_ERR_STATE, "no solution");
  const int L = ctx->L, np = ctx->n_phases, nq = ctx->c == 1 ? 1 : 2;
  const int tot = np * nq * L * L;
  if (tot > 6000) return fail(ctx, UNOCG_ERR_INVALID_ARG, "too many phases x loads for the sensitivity kernel");
  CK(dalloc(&ctx->sens, (size_t)ctx->B * tot));
  double* spart = nullptr;
  CK(cudaMallocAsync(&spart, (size_t)ctx->B * sens_blocks_x(ctx->g) * tot * sizeof(double), ctx->stream));
  AvgArgs aa{};
  aa.g = ctx->g; aa.c = ctx->c; aa.L = L; aa.phase = ctx->phase; aa.mat = material(ctx);
  aa.loads = ctx->loads_d; aa.u64 = final_u(ctx); aa.part = spart;
  cudaError_t se = launch_sens(aa, ctx->B, ctx->sens, ctx->stream);
  cudaFreeAsync(spart, ctx->stream);
  CK(se);
  std::vector<double> raw((size_t)ctx->B * tot);
  CK(cudaMemcpyAsync(raw.data(), ctx->sens, raw.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->c == 1) {
    std::memcpy(out, raw.data(), raw.size() * sizeof(double));
    return UNOCG_OK;
  }
  // elastic: chain (dW/dlambda, dW/dmu) to (dW/dE, dW/dnu) per phase
  std::vector<double> props((size_t)ctx->B * np * 2);
  CK(cudaMemcpy(props.data(), ctx->props_d, props.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int b = 0; b < ctx->B; ++b)
    for (int p = 0; p < np; ++p) {
      double E = props[(b * np + p) * 2], nu = props[(b * np + p) * 2 + 1];
      double dlE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), dmE = 1.0 / (2.0 * (1.0 + nu));
      double dln = E * (1.0 + 2.0 * nu * nu) / ((1.0 + nu) * (1.0 + nu) * (1.0 - 2.0 * nu) * (1.0 - 2.0 * nu));
      double dmn = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
      const double* wl = raw.data() + (size_t)b * tot + (size_t)p * 2 * L * L;
      const double* wm = wl + L * L;
      double* oE = out + ((size_t)b * 2 * np + 2 * p) * L * L;
      double* on = oE + L * L;
      for (int q = 0; q < L * L; ++q) {
        oE[q] = wl[q] * dlE + wm[q] * dmE;
        on[q] = wl[q] * dln + wm[q] * dmn;
      }
    }
  return UNOCG_OK;
}

// Per-kernel CUDA-event timing of the first `reps` CG iterations of a fresh solve (same
// kernels and launch shapes as the graph); leaves the context without a valid solution.
template <typename T>
static int profile_iters(unocg_ctx* ctx, const Plan& pl, int reps, double* ms_out, int n_out) {
  cudaStream_t s = ctx->stream;
  LoopCtl ctl{};
  ctl.tol = pl.o.tol; ctl.max_iter = pl.o.max_iter; ctl.mixed = 0;
  ctl.replace_every = 0; ctl.replace_drop = 0.0; ctl.flexible = pl.o.flexible;
  Plan p2 = pl;
  p2.mixed = 0;
  CK(enq_pre<T>(ctx, s, p2, ctl));
  const int nk = 4;
  std::vector<cudaEvent_t> ev(2 * nk * reps);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  for (int r = 0; r < reps; ++r) {
    for (int k = 0; k < nk; ++k) {
      CK(cudaEventRecord(ev[2 * (r * nk + k)], s));
      if (k < 2) CK(enq_precond<T>(ctx, s, p2, ctl, k));
      else if (k == 2) CK(enq_ku<T>(ctx, s));
      else CK(enq_residual_check<T>(ctx, s, ctl, 0, pl.o.precond));
      CK(cudaEventRecord(ev[2 * (r * nk + k) + 1], s));
    }
  }
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nk && k < n_out; ++k) {
    double tot = 0.0;
    for (int r = 0; r < reps; ++r) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[2 * (r * nk + k)], ev[2 * (r * nk + k) + 1]));
      tot += ms;
    }
    ms_out[k] = tot / reps;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  ctx->solved = false;
  return UNOCG_OK;
}

extern "C" int unocg_profile_iteration(unocg_ctx* ctx, const unocg_solve_opts* o, int reps, double* ms_out, int n_out) {
  if (!ctx || !o || reps < 1 || !ms_out || n_out < 1) return fail(ctx, UNOCG_ERR_INVALID_ARG, "bad arguments");
  Plan pl;
  int rc = prepare_solve(ctx, o, &pl);
  if (rc) return rc;
  return pl.mixed ? profile_iters<float>(ctx, pl, reps, ms_out, n_out)
                  : profile_iters<double>(ctx, pl, reps, ms_out, n_out);
}

// ------------------------------------------------------------------ batch graph
// unocg_batch_solve with the graph driver captures the solves of all its contexts (of any grid
// sizes) as parallel branches of one CUDA graph -- each branch the context's set-up, its WHILE
// loop of CG iterations over all its (instance, load) pairs with their convergence flags, and
// its post-processing -- and launches it once.  Captured graphs are kept for reuse, keyed by
// the contexts, their epochs and the solve options.
namespace {
struct BatchGraph {
  std::vector<unocg_ctx*> ctxs;
  std::vector<unsigned long long> epochs;
  std::vector<GraphKey> keys;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchGraph*> g_batches;  // most recently built last
constexpr size_t kMaxBatchGraphs = 4;

void destroy_batch(BatchGraph* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}
}  // namespace

// drop the cached batch graphs that include `ctx` (called when it is destroyed)
static void forget_batches(const unocg_ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (size_t i = 0; i < g_batches.size();) {
    BatchGraph* b = g_batches[i];
    if (std::find(b->ctxs.begin(), b->ctxs.end(), ctx) != b->ctxs.end()) {
      cudaStreamSynchronize(b->stream);
      destroy_batch(b);
      g_batches.erase(g_batches.begin() + i);
    } else {
      ++i;
    }
  }
}

static GraphKey graph_key(const unocg_ctx* ctx, const Plan& pl) {
  GraphKey k;
  k.precond = pl.o.precond; k.precision = pl.o.precision; k.flexible = pl.o.flexible;
  k.replace_every = pl.o.replace_every; k.replace_drop = pl.o.replace_drop; k.max_iter = pl.o.max_iter;
  k.L = ctx->L; k.tol = pl.o.tol;
  return k;
}

template <typename T>
static int build_batch(const std::vector<unocg_ctx*>& cx, const std::vector<Plan>& pls, BatchGraph* b) {
  unocg_ctx* ctx = cx[0];
  CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  const size_t n = cx.size();
  std::vector<cudaStream_t> ss(n, nullptr);
  std::vector<cudaEvent_t> joins(n, nullptr);
  cudaEvent_t fork = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaEventRecord(fork, b->stream);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(ss[i], fork, 0);  // the branch joins the capture
    if (e == cudaSuccess) e = capture_chain<T>(cx[i], pls[i], ss[i]);
    if (e == cudaSuccess) e = cudaEventRecord(joins[i], ss[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, joins[i], 0);
  }
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(b->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
    cudaError_t e3 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e3;
  }
  for (size_t i = 0; i < n; ++i) {
    if (ss[i]) cudaStreamDestroy(ss[i]);
    if (joins[i]) cudaEventDestroy(joins[i]);
  }
  if (fork) cudaEventDestroy(fork);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  b->graph = g;
  if (e != cudaSuccess) return fail(ctx, UNOCG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  return UNOCG_OK;
}

extern "C" int unocg_batch_solve(int n_ctx, unocg_ctx* const* ctxs, const unocg_solve_opts* opts,
                                 unocg_solve_info* infos) {
  NvtxRange nvtx_("unocg_batch_solve");
  if (n_ctx < 1 || !ctxs || !opts) return UNOCG_ERR_INVALID_ARG;
  std::vector<unocg_ctx*> cx(ctxs, ctxs + n_ctx);
  for (int i = 0; i < n_ctx; ++i) {
    if (!cx[i]) return UNOCG_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (cx[j] == cx[i]) return fail(cx[i], UNOCG_ERR_INVALID_ARG, "a context appears twice in the batch");
  }
  const bool one_graph = n_ctx > 1 && (opts->use_graph == 1 || opts->use_graph == 3);
  if (!one_graph) {
    // host-driven or persistent drivers: each context's solve on its own stream, concurrently
    for (int i = 0; i < n_ctx; ++i) {
      int rc = unocg_solve_async(cx[i], opts);
      if (rc) return rc;
    }
  } else {
    std::vector<Plan> pls(n_ctx);
    std::vector<GraphKey> keys(n_ctx);
    std::vector<unsigned long long> epochs(n_ctx);
    for (int i = 0; i < n_ctx; ++i) {
      int rc = prepare_solve(cx[i], opts, &pls[i]);
      if (rc) return rc;
      keys[i] = graph_key(cx[i], pls[i]);
      epochs[i] = cx[i]->epoch;
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchGraph* b = nullptr;
    for (size_t i = 0; i < g_batches.size() && !b; ++i) {
      BatchGraph* c = g_batches[i];
      if (c->ctxs == cx && c->epochs == epochs && c->keys.size() == keys.size() &&
          std::equal(keys.begin(), keys.end(), c->keys.begin()))
        b = c;
    }
    if (!b) {
      b = new BatchGraph();
      b->ctxs = cx;
      b->epochs = epochs;
      b->keys = keys;
      int rc = pls[0].mixed ? build_batch<float>(cx, pls, b) : build_batch<double>(cx, pls, b);
      if (rc) {
        destroy_batch(b);
        return rc;
      }
      if (g_batches.size() >= kMaxBatchGraphs) {
        cudaStreamSynchronize(g_batches.front()->stream);
        destroy_batch(g_batches.front());
        g_batches.erase(g_batches.begin());
      }
      g_batches.push_back(b);
    }
    // stream order: each context's earlier work, then the batch graph, then its later work
    for (unocg_ctx* c : cx) {
      cudaError_t e = order_after(&c->join_ev, c->stream, b->stream);
      if (e != cudaSuccess) return fail(c, UNOCG_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return fail(cx[0], UNOCG_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    for (unocg_ctx* c : cx) {
      e = order_after(&c->join_ev, b->stream, c->stream);
      if (e != cudaSuccess) return fail(c, UNOCG_ERR_CUDA, cudaGetErrorString(e));
      c->last_opts = *opts;
      c->last_precision = opts->precision;
      c->last_path = 1;
      c->solved = true;
    }
  }
  int status = UNOCG_OK;
  for (int i = 0; i < n_ctx; ++i) {
    int rc = unocg_solve_wait(cx[i], infos ? infos + i : nullptr);
    if (status == UNOCG_OK && rc != UNOCG_OK) status = rc;
  }
  return status;
}

// ------------------------------------------------------------------ operator-level entry points
extern "C" int unocg_apply_K_dev(unocg_ctx* ctx, int instance, const double* d_dev, double* p_dev, void* stream) {
  NvtxRange nvtx_("unocg_apply_K_dev");
  if (!ctx || !d_dev || !p_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->have_phase || !ctx->have_props) return fail(ctx, UNOCG_ERR_STATE, "microstructure/properties missing");
  if (instance < 0 || instance >= ctx->B) return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance out of range");
  StencilArgs<double> a{};
  a.g = ctx->g; a.c = ctx->c; a.BL = 1; a.L = 1;
  a.phase = ctx->phase + (long long)instance * ctx->g.n;
  a.mat = material(ctx);
  a.mat.m64 += (long long)instance * ctx->n_phases * 2;
  a.mat.m32 += (long long)instance * ctx->n_phases * 2;
  a.d = d_dev; a.p = p_dev; a.sc = nullptr; a.standalone = 1;
  cudaStream_t s = (cudaStream_t)stream;
  CK(order_after(&ctx->join_ev, ctx->stream, s));
  CK(launch_ku<double>(a, s));
  CK(order_after(&ctx->join_ev, s, ctx->stream));
  return UNOCG_OK;
}

extern "C" int unocg_apply_K32_dev(unocg_ctx* ctx, int instance, const float* d_dev, float* p_dev, void* stream) {
  NvtxRange nvtx_("unocg_apply_K32_dev");
  if (!ctx || !d_dev || !p_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->have_phase || !ctx->have_props) return fail(ctx, UNOCG_ERR_STATE, "microstructure/properties missing");
  if (instance < 0 || instance >= ctx->B) return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance out of range");
  StencilArgs<float> a{};
  a.g = ctx->g; a.c = ctx->c; a.BL = 1; a.L = 1;
  a.phase = ctx->phase + (long long)instance * ctx->g.n;
  a.mat = material(ctx);
  a.mat.m64 += (long long)instance * ctx->n_phases * 2;
  a.mat.m32 += (long long)instance * ctx->n_phases * 2;
  a.d = d_dev; a.p = p_dev; a.sc = nullptr; a.standalone = 1;
  a.ku_tma = ku_tma_choice(ctx); a.err = ctx->flags + 6; a.spin_limit = ctx->spin_limit;
  cudaStream_t s = (cudaStream_t)stream;
  CK(order_after(&ctx->join_ev, ctx->stream, s));
  CK(launch_ku<float>(a, s));
  CK(order_after(&ctx->join_ev, s, ctx->stream));
  return UNOCG_OK;
}

extern "C" int unocg_set_ku_tile(unocg_ctx* ctx, int tile) {
  if (!ctx || tile < -1 || tile > kKuTiles) return fail(ctx, UNOCG_ERR_INVALID_ARG, "invalid K d tile");
  if (tile > 0 && !ku_tile_ok(ctx->g, ctx->c, tile))
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "K d tile shape not available for this grid / physics");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->ku_tile = tile;
  free_graph(ctx);  // the captured launches hold the old shape
  return UNOCG_OK;
}

extern "C" int unocg_get_ku_tile(unocg_ctx* ctx, int* tile) {
  if (!ctx || !tile) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  *tile = ku_tma_choice(ctx);
  return UNOCG_OK;
}

// Times `reps` launches of the FP32 K d over all B x L fields of the context (standalone mode,
// CUDA events on the context stream, after one warm-up launch) for the earlier kernels
// (times[0]), every TMA tile shape (times[1..8]) and every vector-march shape (times[9..16]),
// NaN where the grid does not allow it; keeps the fastest and returns its index in *best.
extern "C" int unocg_autotune_ku(unocg_ctx* ctx, int reps, double* times, int* best) {
  if (!ctx || reps < 1 || !times) return fail(ctx, UNOCG_ERR_INVALID_ARG, "invalid autotune arguments");
  if (!ctx->have_phase || !ctx->have_props || ctx->L < 1)
    return fail(ctx, UNOCG_ERR_STATE, "set microstructure, phase properties and loads first");
  int rc = ensure_workspace(ctx, UNOCG_MIXED, UNOCG_PRECOND_UNO);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const size_t fld = (size_t)ctx->B * ctx->L * ctx->c * ctx->g.n;
  // a smooth, nonzero direction (its values do not change the time)
  CK(cudaMemsetAsync(ctx->f32.d, 0x3c, fld * sizeof(float), ctx->stream));
  double bt = 1e300;
  int bk = 0;
  const int saved = ctx->ku_tile;
  for (int k = 0; k <= kKuTiles && rc == UNOCG_OK; ++k) {
    times[k] = std::nan("");
    if (!ku_tile_ok(ctx->g, ctx->c, k)) continue;
    ctx->ku_tile = k;
    StencilArgs<float> a = ku_args<float>(ctx);
    a.standalone = 1;
    float ms = 0.f;
    cudaError_t e = launch_ku<float>(a, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_ku<float>(a, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) { rc = fail(ctx, UNOCG_ERR_CUDA, std::string("K d autotune: ") + cudaGetErrorString(e)); break; }
    times[k] = ms / reps;
    if (times[k] < bt) { bt = times[k]; bk = k; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) { ctx->ku_tile = saved; return rc; }
  int flag = 0;
  CK(cudaMemcpy(&flag, ctx->flags + 6, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    ctx->ku_tile = saved;
    CK(cudaMemset(ctx->flags + 6, 0, sizeof(int)));
    return fail(ctx, UNOCG_ERR_DEVICE_TIMEOUT, "K d autotune: a wait for a tile copy expired");
  }
  ctx->ku_tile = bk;
  free_graph(ctx);
  if (best) *best = bk;
  return UNOCG_OK;
}

extern "C" int unocg_apply_uno_dev(unocg_ctx* ctx, int instance, const double* r_dev, double* s_dev, void* stream) {
  NvtxRange nvtx_("unocg_apply_uno_dev");
  if (!ctx || !r_dev || !s_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (instance < 0 || instance >= ctx->B) return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance out of range");
  if (ctx->wkind < 0) return fail(ctx, UNOCG_ERR_STATE, "set UNO weights first");
  if (ctx->q_dirty) {
    int rc = build_weights(ctx);
    if (rc) return rc;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(order_after(&ctx->join_ev, ctx->stream, s));
  double2* hat = nullptr;
  double2* shat = nullptr;
  const size_t m = (size_t)ctx->c * ctx->g.nh;
  CK(cudaMallocAsync(&hat, m * sizeof(double2), s));
  CK(cudaMallocAsync(&shat, m * sizeof(double2), s));
  PlaneFwdArgs<double> pf{};
  pf.g = ctx->g; pf.c = ctx->c; pf.BL = 1; pf.src = r_dev; pf.hat = hat; pf.ft = tables(ctx, true); pf.standalone = 1;
  cudaError_t e = fwd_transform<double>(pf, s, 0);
  if (e == cudaSuccess) {
    LineArgs<double, double> la{};
    la.g = ctx->g; la.c = ctx->c; la.BL = 1; la.L = 1; la.hat = hat; la.shat = shat;
    la.Q = ctx->Q64 + (ctx->Bq > 1 ? (long long)instance * ctx->g.nh * (ctx->c == 1 ? 1 : 6) : 0);
    la.q_inst_stride = 0; la.scale = 1.0 / (double)ctx->g.n; la.ft = tables(ctx, true); la.standalone = 1;
    e = launch_line<double, double>(la, 0, s);
  }
  if (e == cudaSuccess) {
    PlaneInvArgs<double> pi{};
    pi.g = ctx->g; pi.c = ctx->c; pi.BL = 1; pi.shat = shat; pi.dst = s_dev; pi.ft = tables(ctx, true); pi.standalone = 1;
    e = inv_transform<double>(pi, s);
  }
  cudaFreeAsync(hat, s);
  cudaFreeAsync(shat, s);
  if (e != cudaSuccess) return fail(ctx, UNOCG_ERR_CUDA, cudaGetErrorString(e));
  CK(order_after(&ctx->join_ev, s, ctx->stream));
  return UNOCG_OK;
}

// ------------------------------------------------------------------ allocation-free UNO apply
// unocg_apply_uno_dev takes its two spectra from cudaMallocAsync.  Some callers cannot allocate
// at the moment they apply the preconditioner: a framework whose caching allocator already owns
// the device memory (the stream-ordered pool then has no room), a latency-bound loop that must
// not enter the allocator, or a deployment that needs its device footprint fixed when the
// library loads.  unocg_apply_uno_dev_noalloc serves them from this file-scope scratch instead.
// Its two halves hold the forward spectrum T r and the multiplied spectrum Q T r; nothing in it
// has to start at zero (the forward pass writes every value of the first half before the axis-1
// pass reads it, and the axis-1 pass writes every value of the second half).
constexpr size_t kNoAllocSpectrum = 524288;  // complex FP64 values per half (8 MiB each)
static __device__ __align__(256) double2 g_noalloc_scratch[2 * kNoAllocSpectrum];

namespace {
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocAddr {
  unsigned long long ctx_id;
  double2* addr;
};
std::mutex g_noalloc_mu;
NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices] = {};

// Address of the scratch in the current context of the current device, looked up once per
// context (with that device current) and cached under the context's id: a context destroyed
// and created again (cudaDeviceReset) loads the module again, and the address is looked up anew.
cudaError_t noalloc_scratch(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  // the context current on this thread; none yet if this thread has made no runtime call that
  // needs one (the symbol lookup below then binds the device's primary context)
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id) == cudaSuccess;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocAddr& c = g_noalloc_addr[dev];
  if (!have_id || !c.addr || c.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!have_id) {
      e = current_context_id(&id);
      if (e != cudaSuccess) return e;
    }
    c.addr = static_cast<double2*>(p);
    c.ctx_id = id;
  }
  *out = c.addr;
  return cudaSuccess;
}
}  // namespace

extern "C" int unocg_apply_uno_dev_noalloc(unocg_ctx* ctx, int instance, const double* r_dev, double* s_dev,
                                           void* stream) {
  if (!ctx || !r_dev || !s_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (instance < 0 || instance >= ctx->B) return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance out of range");
  if (ctx->wkind < 0) return fail(ctx, UNOCG_ERR_STATE, "set UNO weights first");
  // preparing the weights allocates: they must already be on the device
  if (ctx->q_dirty)
    return fail(ctx, UNOCG_ERR_STATE,
                "UNO weights are not prepared on the device (set the phase properties, then the weights)");
  const size_t m = (size_t)ctx->c * ctx->g.nh;
  if (m > kNoAllocSpectrum)
    return fail(ctx, UNOCG_ERR_INVALID_ARG,
                "grid too large for the static scratch: c*N1*N2*(N3/2+1) = " + std::to_string(m) +
                    " complex values, the limit is " + std::to_string(kNoAllocSpectrum));
  double2* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return fail(ctx, UNOCG_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  double2* hat = scratch;
  double2* shat = scratch + kNoAllocSpectrum;
  cudaStream_t s = (cudaStream_t)stream;
  e = order_after(&ctx->join_ev, ctx->stream, s);
  if (e != cudaSuccess) return fail(ctx, UNOCG_ERR_CUDA, cudaGetErrorString(e));
  PlaneFwdArgs<double> pf{};
  pf.g = ctx->g; pf.c = ctx->c; pf.BL = 1; pf.src = r_dev; pf.hat = hat; pf.ft = tables(ctx, true); pf.standalone = 1;
  e = fwd_transform<double>(pf, s, 0);
  if (e == cudaSuccess) {
    LineArgs<double, double> la{};
    la.g = ctx->g; la.c = ctx->c; la.BL = 1; la.L = 1; la.hat = hat; la.shat = shat;
    la.Q = ctx->Q64 + (ctx->Bq > 1 ? (long long)instance * ctx->g.nh * (ctx->c == 1 ? 1 : 6) : 0);
    la.q_inst_stride = 0; la.scale = 1.0 / (double)ctx->g.n; la.ft = tables(ctx, true); la.standalone = 1;
    e = launch_line<double, double>(la, 0, s);
  }
  if (e == cudaSuccess) {
    PlaneInvArgs<double> pi{};
    pi.g = ctx->g; pi.c = ctx->c; pi.BL = 1; pi.shat = shat; pi.dst = s_dev; pi.ft = tables(ctx, true); pi.standalone = 1;
    e = inv_transform<double>(pi, s);
  }
  if (e == cudaSuccess) e = order_after(&ctx->join_ev, s, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, UNOCG_ERR_CUDA, cudaGetErrorString(e));
  return UNOCG_OK;
}

extern "C" int unocg_rhs_dev(unocg_ctx* ctx, int instance, int load, double* f_dev, void* stream) {
  if (!ctx || !f_dev) return fail(ctx, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!ctx->have_phase || !ctx->have_props || !ctx->have_loads) return fail(ctx, UNOCG_ERR_STATE, "inputs missing");
  if (instance < 0 || instance >= ctx->B || load < 0 || load >= ctx->L)
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "instance/load out of range");
  InitArgs<double> ia{};
  ia.g = ctx->g; ia.c = ctx->c; ia.L = 1;
  ia.phase = ctx->phase + (long long)instance * ctx->g.n;
  ia.mat = material(ctx);
  ia.mat.m64 += (long long)instance * ctx->n_phases * 2;
  ia.mat.m32 += (long long)instance * ctx->n_phases * 2;
  ia.loads = ctx->loads_d + (long long)load * ctx->dim;
  ia.f64 = f_dev;
  cudaStream_t s = (cudaStream_t)stream;
  CK(order_after(&ctx->join_ev, ctx->stream, s));
  CK(launch_init<double>(ia, 1, s));
  CK(order_after(&ctx->join_ev, s, ctx->stream));
  return UNOCG_OK;
}

// ------------------------------------------------------------------ standalone UNO operator
static int ufail(unocg_uno* op, int code, const std::string& m) {
  if (op) op->err = m;
  return code;
}
#define UCK(...)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (__VA_ARGS__);                                                               \
    if (e_ != cudaSuccess) return ufail(op, e_ == cudaErrorMemoryAllocation ? UNOCG_ERR_OOM : UNOCG_ERR_CUDA, \
                                        std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" int unocg_uno_create(unocg_uno** out, int c, int n1, int n2, int n3) {
  if (!out || (c != 1 && c != 3) || !grid_ok(n1, n2, n3)) return UNOCG_ERR_INVALID_ARG;
  Grid g{n1, n2, n3, n3 / 2 + 1, (long long)n1 * n2 * n3, (long long)n1 * n2 * (n3 / 2 + 1), 1.0 / n1};
  grid_scales(g);
  if (!grid_supported(g, 8) || line_smem_bytes(g, c, 8, 2) > 220 * 1024) return UNOCG_ERR_INVALID_ARG;
  unocg_uno* op = new unocg_uno();
  *out = op;
  op->c = c;
  op->g = g;
  factor_plan(n1, &op->p1);
  factor_plan(n2, &op->p2);
  factor_plan(n3 / 2, &op->p3h);
  UCK(upload_twiddles<float>(op->tw32, n1, n2, n3));
  const size_t m = (size_t)g.nh * (c == 1 ? 1 : 6);
  UCK(cudaMalloc(&op->Q32, m * sizeof(float)));
  UCK(cudaMalloc(&op->Qtmp, m * sizeof(float)));
  UCK(cudaMalloc(&op->gq, m * sizeof(float)));
  UCK(cudaMalloc(&op->gq2, m * sizeof(float)));
  UCK(cudaMalloc(&op->mscratch, modes_grad_scratch_doubles() * sizeof(double)));
  return UNOCG_OK;
}

extern "C" void unocg_uno_destroy(unocg_uno* op) {
  if (!op) return;
  cudaDeviceSynchronize();
  void* ptrs[] = {op->Q32, op->Qtmp, op->hat, op->shat, op->ghat, op->gq, op->gq2, op->mscratch,
                  op->tw32[0], op->tw32[1], op->tw32[2], op->tw32[3]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete op;
}

extern "C" const char* unocg_uno_last_error(const unocg_uno* op) { return op ? op->err.c_str() : "null operator"; }

static FftTables uno_tables(unocg_uno* op) {
  FftTables t;
  t.p1 = op->p1; t.p2 = op->p2; t.p3h = op->p3h;
  t.tw1 = op->tw32[0]; t.tw2 = op->tw32[1]; t.tw3h = op->tw32[2]; t.tw3 = op->tw32[3];
  return t;
}

extern "C" int unocg_uno_set_theta_dev(unocg_uno* op, const float* theta_dev, void* stream) {
  if (!op || !theta_dev) return UNOCG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  op->theta = theta_dev;
  op->modes_M = -1;
  UCK(launch_psi32(theta_dev, op->Qtmp, op->g.nh, op->c, s));
  UCK(launch_symmetrize32(op->Qtmp, op->Q32, op->g, op->c == 1 ? 1 : 6, 1, s));
  return UNOCG_OK;
}

extern "C" int unocg_uno_set_modes_dev(unocg_uno* op, int M, const float* w_dev, void* stream) {
  if (!op || !w_dev) return UNOCG_ERR_INVALID_ARG;
  if (!modes_fit(op->g, M)) return ufail(op, UNOCG_ERR_INVALID_ARG, "mode set [-M,M]^2 x [0,M] does not fit the grid");
  cudaStream_t s = (cudaStream_t)stream;
  op->theta = w_dev;
  op->modes_M = M;
  UCK(launch_modes_expand32(w_dev, M, op->g, op->c, op->Qtmp, s));
  UCK(launch_symmetrize32(op->Qtmp, op->Q32, op->g, op->c == 1 ? 1 : 6, 1, s));
  return UNOCG_OK;
}

static int uno_ensure(unocg_uno* op, int batch) {
  size_t need = (size_t)batch * op->c * op->g.nh;
  if (need <= op->cap) return UNOCG_OK;
  if (op->hat) { cudaFree(op->hat); cudaFree(op->shat); cudaFree(op->ghat); }
  op->hat = op->shat = op->ghat = nullptr;
  UCK(cudaMalloc(&op->hat, need * sizeof(float2)));
  UCK(cudaMalloc(&op->shat, need * sizeof(float2)));
  UCK(cudaMalloc(&op->ghat, need * sizeof(float2)));
  op->cap = need;
  return UNOCG_OK;
}

extern "C" int unocg_uno_apply_dev(unocg_uno* op, int batch, const float* r_dev, float* s_dev, void* stream) {
  NvtxRange nvtx_("unocg_uno_apply_dev");
  if (!op || batch < 1 || !r_dev || !s_dev) return UNOCG_ERR_INVALID_ARG;
  if (!op->theta) return ufail(op, UNOCG_ERR_STATE, "set theta first");
  int rc = uno_ensure(op, batch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  PlaneFwdArgs<float> pf{};
  pf.g = op->g; pf.c = op->c; pf.BL = batch; pf.src = r_dev; pf.hat = op->hat; pf.ft = uno_tables(op); pf.standalone = 1;
  UCK(fwd_transform<float>(pf, s, 0));
  LineArgs<float, float> la{};
  la.g = op->g; la.c = op->c; la.BL = batch; la.L = 1; la.hat = op->hat; la.shat = op->shat;
  la.Q = op->Q32; la.q_inst_stride = 0; la.scale = 1.0 / (double)op->g.n; la.ft = uno_tables(op); la.standalone = 1;
  UCK(launch_line<float, float>(la, 0, s));
  PlaneInvArgs<float> pi{};
  pi.g = op->g; pi.c = op->c; pi.BL = batch; pi.shat = op->shat; pi.dst = s_dev; pi.ft = uno_tables(op); pi.standalone = 1;
  UCK(inv_transform<float>(pi, s));
  return UNOCG_OK;
}

// Features of the second-order training (Sec. 5.4; Eq. (features-c-1), Eq. (features-c-2) and
// the c = 3 set of App. C): raw sums over the batch, per half-grid mode (unitary transform,
// multiplicity w_k), in the order of the unique block entries: for the pair (i, j) of the entry,
// w_k Re(conj(T f)_i (T f)_j) (+ the (j, i) term off the diagonal) -- the a features -- and the
// same with conj(T u)_i -- half the b features.  These are the per-mode accumulations of the
// weight gradient with the adjoint field replaced by T f or T u, from the same kernels.
extern "C" int unocg_uno_features_dev(unocg_uno* op, int batch, const float* f_dev, const float* u_dev, float* ab_dev,
                                      int accumulate, void* stream) {
  if (!op || batch < 1 || !f_dev || !u_dev || !ab_dev) return UNOCG_ERR_INVALID_ARG;
  int rc = uno_ensure(op, batch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nh = (size_t)op->g.nh;
  const size_t NQ = op->c == 1 ? 1 : 6;
  if (!accumulate) UCK(cudaMemsetAsync(ab_dev, 0, 2 * nh * NQ * sizeof(float), s));
  PlaneFwdArgs<float> pf{};
  pf.g = op->g; pf.c = op->c; pf.BL = batch; pf.src = f_dev; pf.hat = op->hat; pf.ft = uno_tables(op); pf.standalone = 1;
  UCK(fwd_transform<float>(pf, s, 0));
  pf.src = u_dev;
  pf.hat = op->ghat;
  UCK(fwd_transform<float>(pf, s, 0));
  LineArgs<float, float> la{};
  la.g = op->g; la.c = op->c; la.BL = batch; la.L = 1; la.hat = op->hat; la.shat = op->shat; la.ghat = op->ghat;
  la.Q = op->Q32; la.q_inst_stride = 0; la.scale = 1.0 / (double)op->g.n; la.ft = uno_tables(op);
  la.standalone = 1; la.gq = ab_dev + nh * NQ;  // sums of w Re(conj(T u)_i (T f)_j) per entry
  UCK(launch_line<float, float>(la, 1, s));
  la.ghat = op->hat;
  la.gq = ab_dev;  // sums of w Re(conj(T f)_i (T f)_j) per entry
  UCK(launch_line<float, float>(la, 1, s));
  return UNOCG_OK;
}

extern "C" int unocg_uno_backward_dev(unocg_uno* op, int batch, const float* r_dev, const float* gs_dev,
                                      float* gr_dev, float* gtheta_dev, void* stream) {
  NvtxRange nvtx_("unocg_uno_backward_dev");
  if (!op || batch < 1 || !r_dev || !gs_dev) return UNOCG_ERR_INVALID_ARG;
  if (!op->theta) return ufail(op, UNOCG_ERR_STATE, "set theta first");
  int rc = uno_ensure(op, batch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int NQ = op->c == 1 ? 1 : 6;
  PlaneFwdArgs<float> pf{};
  pf.g = op->g; pf.c = op->c; pf.BL = batch; pf.src = r_dev; pf.hat = op->hat; pf.ft = uno_tables(op); pf.standalone = 1;
  UCK(fwd_transform<float>(pf, s, 0));
  pf.src = gs_dev;
  pf.hat = op->ghat;
  UCK(fwd_transform<float>(pf, s, 0));
  UCK(cudaMemsetAsync(op->gq, 0, (size_t)op->g.nh * NQ * sizeof(float), s));
  LineArgs<float, float> la{};
  la.g = op->g; la.c = op->c; la.BL = batch; la.L = 1; la.hat = op->hat; la.shat = op->shat; la.ghat = op->ghat;
  la.Q = op->Q32; la.q_inst_stride = 0; la.scale = 1.0 / (double)op->g.n; la.ft = uno_tables(op);
  la.standalone = 1; la.gq = op->gq;
  UCK(launch_line<float, float>(la, 1, s));
  if (gr_dev) {
    PlaneInvArgs<float> pi{};
    pi.g = op->g; pi.c = op->c; pi.BL = batch; pi.shat = op->shat; pi.dst = gr_dev; pi.ft = uno_tables(op); pi.standalone = 1;
    UCK(inv_transform<float>(pi, s));
  }
  if (gtheta_dev) {
    // Q_sym = S psi(theta) with S the (self-adjoint) plane averaging: dL/dpsi = S dL/dQ_sym
    UCK(launch_symmetrize32(op->gq, op->gq2, op->g, NQ, 1, s));
    if (op->modes_M >= 0)
      UCK(launch_modes_grad(op->theta, op->modes_M, op->g, op->c, op->gq2, op->mscratch, gtheta_dev, s));
    else
      UCK(launch_psi_grad(op->theta, op->gq2, gtheta_dev, op->g.nh, op->c, s));
  }
  return UNOCG_OK;
}


// ------------------------------------------------------------------ tuning
extern "C" int unocg_set_tuning(unocg_ctx* ctx, int radix_order, int path) {
  if (!ctx || radix_order < 0 || radix_order > 2 || (path != 1 && path != 2)) return fail(ctx, UNOCG_ERR_INVALID_ARG, "invalid tuning");
  FftPlan p1{}, p2{}, p3h{};
  if (!factor_plan(ctx->g.n1, &p1, radix_order) || !factor_plan(ctx->g.n2, &p2, radix_order) ||
      !factor_plan(ctx->g.n3 / 2, &p3h, radix_order))
    return fail(ctx, UNOCG_ERR_INVALID_ARG, "radix plan");
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->p1 = p1;
  ctx->p2 = p2;
  ctx->p3h = p3h;
  ctx->radix_order = radix_order;
  ctx->tuned_path = path;
  free_graph(ctx);  // the captured launches hold the old plans
  return UNOCG_OK;
}

// Times `reps` solves (CUDA events on the context stream, after one warm-up solve that also
// builds the graph) for each radix order (0..2) and loop driver (graph, persistent); writes the
// mean milliseconds to times[order * 2 + (driver == persistent)] (NaN where the persistent
// kernel does not fit) and keeps the fastest setting.
extern "C" int unocg_autotune(unocg_ctx* ctx, const unocg_solve_opts* o, int reps, double* times) {
  if (!ctx || !o || reps < 1 || !times) return fail(ctx, UNOCG_ERR_INVALID_ARG, "invalid autotune arguments");
  double best = 1e300;
  int bo = 0, bp = 1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = UNOCG_OK;
  for (int order = 0; order < 3 && rc == UNOCG_OK; ++order)
    for (int path = 1; path <= 2 && rc == UNOCG_OK; ++path) {
      double* t = times + order * 2 + (path - 1);
      *t = std::nan("");
      unocg_solve_opts oo = *o;
      oo.use_graph = path;
      if (path == 2 && !persistent_fits(ctx, &oo)) continue;
      rc = unocg_set_tuning(ctx, order, path);
      if (rc) break;
      rc = unocg_solve(ctx, &oo, nullptr);
      if (rc) break;
      float ms = 0.f;
      if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = fail(ctx, UNOCG_ERR_CUDA, "event"); break; }
      for (int r = 0; r < reps && rc == UNOCG_OK; ++r) rc = unocg_solve_async(ctx, &oo);
      if (rc) break;
      if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = fail(ctx, UNOCG_ERR_CUDA, "event timing"); break; }
      rc = unocg_solve_wait(ctx, nullptr);
      if (rc) break;
      *t = ms / reps;
      if (*t < best) { best = *t; bo = order; bp = path; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  return unocg_set_tuning(ctx, bo, bp);
}
