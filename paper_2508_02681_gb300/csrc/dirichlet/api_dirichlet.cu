// C ABI of the Dirichlet-BC solver (include/unocg.h, unocg_dir_*): Algorithm 1 / Algorithm 2
// on the free nodes of a grid whose fluctuation vanishes on the boundary (Sec. 6.1, Sec. 6.2),
// with the sine transform as the unitary transform of the UNO preconditioner (Dirichlet row of
// Table (fnocg-mode-selection-2d)).  The loop runs in one CUDA graph with a conditional WHILE
// node; mixed precision adds a conditional IF node for the FP64 residual replacement.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../element.cuh"
#include "dargs.h"
#include "unocg.h"

using namespace unocg;

namespace {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

enum DTicket { DT_CHECK = 0, DT_QMUL = 1, DT_KU = 2, DT_CHECK2 = 3, DT_JAC = 4, DT_N = 8 };

bool dfactor_plan(int N, FftPlan* p) {
  p->N = N;
  p->nst = 0;
  int m = N;
  while (m % 8 == 0) { p->radix[p->nst++] = 8; m /= 8; }
  while (m % 4 == 0) { p->radix[p->nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p->radix[p->nst++] = 2; m /= 2; }
  while (m % 3 == 0) { p->radix[p->nst++] = 3; m /= 3; }
  while (m % 5 == 0) { p->radix[p->nst++] = 5; m /= 5; }
  return m == 1 && p->nst <= 12;
}

template <typename T>
cudaError_t dupload_twiddles(void** dst, int N) {
  std::vector<cplx<T>> w(N);
  for (int m = 0; m < N; ++m) {
    const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)N;
    w[m] = mk<T>((T)std::cos(ang), (T)std::sin(ang));
  }
  cudaError_t e = cudaMalloc(dst, N * sizeof(cplx<T>));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, w.data(), N * sizeof(cplx<T>), cudaMemcpyHostToDevice);
}

struct DFields {
  void *r = nullptr, *p = nullptr, *q = nullptr, *hat = nullptr, *invdiag = nullptr;
  void* u = nullptr;  // FP32 solution increment (mixed precision only)
};

struct DKey {
  int precond = -1, precision = -1, max_iter = 0, replace_every = 0, L = 0;
  double tol = 0.0, replace_drop = 0.0;
  bool operator==(const DKey& o) const {
    return precond == o.precond && precision == o.precision && max_iter == o.max_iter &&
           replace_every == o.replace_every && L == o.L && tol == o.tol && replace_drop == o.replace_drop;
  }
};

}  // namespace

struct unocg_dir {
  int physics = 0, c = 1, dim = 3, B = 1, L = 0, n_phases = 0;
  DGrid g{};
  cudaStream_t stream = nullptr, own_stream = nullptr;
  cudaEvent_t join_ev = nullptr;  // orders the `_dev` entry points against the context stream
  std::string err;
  FftPlan plan[3]{};
  void* tw64[3] = {nullptr, nullptr, nullptr};
  void* tw32[3] = {nullptr, nullptr, nullptr};
  uint8_t* phase = nullptr;
  double* mat64 = nullptr;
  float* mat32 = nullptr;
  std::vector<double> props;
  double* loads_d = nullptr;
  std::vector<double> loads;
  // weights: unscaled unique entries on the host, scaled copies on the device
  int wkind = -1, Bq = 1;
  std::vector<double> Qh;
  double* Q64 = nullptr;
  float* Q32 = nullptr;
  bool f32_spd_ok = false;
  // CG state
  double *f64 = nullptr, *u64 = nullptr;
  DFields f64f, f32f;
  CgScal* sc = nullptr;
  double* part = nullptr;
  size_t part_len = 0;
  unsigned int* tickets = nullptr;
  int* flags = nullptr;
  double* ceff = nullptr;
  double *stage_a = nullptr, *stage_b = nullptr, *stage_f = nullptr;  // operator-level I/O
  int lines3[2], w2[2], w1[2];  // [0] FP64, [1] FP32
  // pass engines per precision ([0] FP64, [1] FP32): axes 3 and 2 as register plane passes (0,
  // N2 = N3 a power of two, Dirichlet faces everywhere), shared-memory plane passes (1, the plane
  // fits a block) or separate axis-3 and axis-2 passes (2); set at creation, or by the autotuner
  int plane_engine[2] = {2, 2};
  int np = 0, pa = -1, pb = -1; // periodic axes (two: k_dmixq between the axis-1 passes)
  bool line_reg_p[2] = {false, false};  // register-resident axis-1 pass with Q ([0] FP64, [1] FP32)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DKey key;
  bool solved = false, phase_set = false;
  int last_precision = 0;
};

namespace {

int dfail(unocg_dir* d, int code, const std::string& msg) {
  if (d) d->err = msg;
  return code;
}

#define DCK(x)                                                                          \
  do {                                                                                  \
    cudaError_t e__ = (x);                                                              \
    if (e__ != cudaSuccess)                                                             \
      return dfail(d, e__ == cudaErrorMemoryAllocation ? UNOCG_ERR_OOM : UNOCG_ERR_CUDA, \
                   std::string(#x ": ") + cudaGetErrorString(e__));                     \
  } while (0)

bool dim_ok(int n) {
  FftPlan p;
  return n >= 2 && n <= 512 && dfactor_plan(n, &p) && dfactor_plan(2 * n, &p);
}

// even position count W <= cap with c W lines of length 2N in the shared-memory budget
int fit_w(int N, int c, int eb, int cap) {
  int w = 2;
  while (w + 2 <= cap && dst_smem_bytes(N, c * (w + 2), eb) <= 96 * 1024) w += 2;
  return w;
}

Material dmaterial(unocg_dir* d) {
  Material m;
  m.n_phases = d->n_phases;
  m.m64 = d->mat64;
  m.m32 = d->mat32;
  return m;
}

DstTables dtables(unocg_dir* d, bool fp64) {
  DstTables t;
  for (int a = 0; a < 3; ++a) {
    t.p[a] = d->plan[a];
    t.tw[a] = fp64 ? d->tw64[a] : d->tw32[a];
  }
  return t;
}

void dfree_graph(unocg_dir* d) {
  if (d->exec) cudaGraphExecDestroy(d->exec);
  if (d->graph) cudaGraphDestroy(d->graph);
  d->exec = nullptr;
  d->graph = nullptr;
  d->key = DKey{};
}

void free_fields(DFields& f) {
  cudaFree(f.r); cudaFree(f.p); cudaFree(f.q); cudaFree(f.hat); cudaFree(f.invdiag); cudaFree(f.u);
  f = DFields{};
}

// symmetric c x c block from unique entries (paper order v1=Q11 v2=Q22 v3=Q12 v4=Q33 v5=Q23 v6=Q13)
void block_of(const double* v, int c, double Q[3][3]) {
  if (c == 1) { Q[0][0] = v[0]; return; }
  Q[0][0] = v[0]; Q[1][1] = v[1]; Q[0][1] = Q[1][0] = v[2];
  Q[2][2] = v[3]; Q[1][2] = Q[2][1] = v[4]; Q[0][2] = Q[2][0] = v[5];
}
void entries_of(const double Q[3][3], int c, double* v) {
  if (c == 1) { v[0] = Q[0][0]; return; }
  v[0] = Q[0][0]; v[1] = Q[1][1]; v[2] = Q[0][1]; v[3] = Q[2][2]; v[4] = Q[1][2]; v[5] = Q[0][2];
}
// lambda_min(Q) > eps by Sylvester's criterion on Q - eps I
bool spd_block(const double Q[3][3], int c, double eps) {
  if (c == 1) return Q[0][0] > eps;
  const double a = Q[0][0] - eps, b = Q[1][1] - eps, e = Q[2][2] - eps;
  if (!(a > 0.0)) return false;
  if (!(a * b - Q[0][1] * Q[0][1] > 0.0)) return false;
  const double det = a * (b * e - Q[1][2] * Q[1][2]) - Q[0][1] * (Q[0][1] * e - Q[1][2] * Q[0][2]) +
                     Q[0][2] * (Q[0][1] * Q[1][2] - b * Q[0][2]);
  return det > 0.0;
}
// local parametrization psi (Sec. 5.2.2): theta^2 (c = 1), L L^T with L lower triangular,
// L00 = t1, L11 = t2, L10 = t3, L22 = t4, L21 = t5, L20 = t6 (c = 3)
void psi_block(const double* t, int c, double Q[3][3]) {
  if (c == 1) { Q[0][0] = t[0] * t[0]; return; }
  double L[3][3] = {{t[0], 0, 0}, {t[2], t[1], 0}, {t[5], t[4], t[3]}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += L[i][k] * L[j][k];
      Q[i][j] = s;
    }
}

// Reference weights: Q(k) = (t_k^T K_ref t_k)^-1 per mode, with K_ref the stiffness of the
// homogeneous medium mt (kappa, or lambda and mu): the interior stencil of the 8 element
// matrices, transformed with sum_j S[k,j] S[k,j+d] = 1 (d = 0), cos(pi (k+1) / N) (d = +-1),
// the eigenvalue relations of the sine basis for the shift operators.
void reference_weights(const DGrid& g, int c, const double* mt, double* out) {
  const int C = c == 1 ? 1 : 6;
  double sten[3][3][3][3][3] = {};
  for (int o = 0; o < 8; ++o)
    for (int ob = 0; ob < 8; ++ob) {
      const int d1 = cbit(ob, 0) - cbit(o, 0), d2 = cbit(ob, 1) - cbit(o, 1), d3 = cbit(ob, 2) - cbit(o, 2);
      for (int i = 0; i < c; ++i)
        for (int k = 0; k < c; ++k) {
          const double v = c == 1 ? mt[0] * Klap(o, ob) : mt[0] * Klam(o, i, ob, k) + mt[1] * Kmu(o, i, ob, k);
          sten[d1 + 1][d2 + 1][d3 + 1][i][k] += v * g.pg.h;
        }
    }
  const int m[3] = {g.m1, g.m2, g.m3};
  const int n[3] = {g.n1, g.n2, g.n3};
  // per axis and offset d in {-1, 0, 1}: sum_j conj(t_k[j]) t_k[j + d] of the basis vector of
  // mode k; sine basis (Dirichlet axis): 1 and cos(pi (k+1) / N); Fourier basis (periodic
  // axis, the paper's transform): exp(-2 pi i k d / N)
  std::vector<std::complex<double>> gd[3];
  for (int a = 0; a < 3; ++a) {
    gd[a].resize((size_t)m[a] * 3);
    for (int k = 0; k < m[a]; ++k)
      for (int d = -1; d <= 1; ++d) {
        std::complex<double> v;
        if (g.bc[a]) v = d == 0 ? 1.0 : std::cos(M_PI * (double)(k + 1) / (double)n[a]);
        else v = std::polar(1.0, -2.0 * M_PI * (double)((long long)k * d) / (double)n[a]);
        gd[a][k * 3 + d + 1] = v;
      }
  }
  for (int k1 = 0; k1 < g.m1; ++k1)
    for (int k2 = 0; k2 < g.m2; ++k2)
      for (int k3 = 0; k3 < g.m3; ++k3) {
        double Bk[3][3] = {};
        for (int s1 = 0; s1 < 3; ++s1)
          for (int s2 = 0; s2 < 3; ++s2)
            for (int s3 = 0; s3 < 3; ++s3) {
              // the imaginary parts cancel over +-d (symmetric stencil)
              const double w = (gd[0][k1 * 3 + s1] * gd[1][k2 * 3 + s2] * gd[2][k3 * 3 + s3]).real();
              for (int i = 0; i < c; ++i)
                for (int k = 0; k < c; ++k) Bk[i][k] += w * sten[s1][s2][s3][i][k];
            }
        double Q[3][3] = {};
        if (c == 1) {
          Q[0][0] = 1.0 / Bk[0][0];
        } else {
          const double det = Bk[0][0] * (Bk[1][1] * Bk[2][2] - Bk[1][2] * Bk[2][1]) -
                             Bk[0][1] * (Bk[1][0] * Bk[2][2] - Bk[1][2] * Bk[2][0]) +
                             Bk[0][2] * (Bk[1][0] * Bk[2][1] - Bk[1][1] * Bk[2][0]);
          Q[0][0] = (Bk[1][1] * Bk[2][2] - Bk[1][2] * Bk[2][1]) / det;
          Q[0][1] = (Bk[0][2] * Bk[2][1] - Bk[0][1] * Bk[2][2]) / det;
          Q[0][2] = (Bk[0][1] * Bk[1][2] - Bk[0][2] * Bk[1][1]) / det;
          Q[1][1] = (Bk[0][0] * Bk[2][2] - Bk[0][2] * Bk[2][0]) / det;
          Q[1][2] = (Bk[0][2] * Bk[1][0] - Bk[0][0] * Bk[1][2]) / det;
          Q[2][2] = (Bk[0][0] * Bk[1][1] - Bk[0][1] * Bk[1][0]) / det;
          Q[1][0] = Q[0][1]; Q[2][0] = Q[0][2]; Q[2][1] = Q[1][2];
        }
        entries_of(Q, c, out + (((long long)k1 * g.m2 + k2) * g.m3 + k3) * C);
      }
}

// check the host weights, then upload them scaled by prod_a 2 / N_a (FP64 and FP32 copies)
int finish_weights(unocg_dir* d, double spd_eps) {
  const int C = d->c == 1 ? 1 : 6;
  const size_t m = (size_t)d->g.nf * C;
  // normalization of T^T Q T: 2 / N per sine axis, 1 / N per Hartley axis
  double scale = 1.0;
  const int ns[3] = {d->g.n1, d->g.n2, d->g.n3};
  for (int a = 0; a < 3; ++a) scale *= (d->g.bc[a] ? 2.0 : 1.0) / ns[a];
  std::vector<double> s64(d->Qh.size());
  std::vector<float> s32(d->Qh.size());
  bool ok64 = true, ok32 = true;
  for (size_t i = 0; i < d->Qh.size(); i += C) {
    double Q[3][3], Qf[3][3], vf[6];
    block_of(&d->Qh[i], d->c, Q);
    if (!std::isfinite(Q[0][0]) || !spd_block(Q, d->c, spd_eps)) ok64 = false;
    for (int k = 0; k < C; ++k) {
      s64[i + k] = d->Qh[i + k] * scale;
      s32[i + k] = (float)s64[i + k];
      vf[k] = (double)s32[i + k] / scale;
    }
    block_of(vf, d->c, Qf);
    if (!spd_block(Qf, d->c, spd_eps)) ok32 = false;
  }
  if (!ok64) {
    d->wkind = -1;
    return dfail(d, UNOCG_ERR_NOT_SPD, "UNO weights fail the safety check lambda_min(Q(k)) > eps");
  }
  d->f32_spd_ok = ok32;
  cudaFree(d->Q64);
  cudaFree(d->Q32);
  d->Q64 = nullptr;
  d->Q32 = nullptr;
  DCK(cudaMalloc(&d->Q64, d->Bq * m * sizeof(double)));
  DCK(cudaMalloc(&d->Q32, d->Bq * m * sizeof(float)));
  DCK(cudaMemcpy(d->Q64, s64.data(), d->Bq * m * sizeof(double), cudaMemcpyHostToDevice));
  DCK(cudaMemcpy(d->Q32, s32.data(), d->Bq * m * sizeof(float), cudaMemcpyHostToDevice));
  return UNOCG_OK;
}

int ensure_workspace(unocg_dir* d, int precision, int precond) {
  const int BL = d->B * d->L;
  const size_t n = (size_t)BL * d->c * d->g.ne;
  const bool fp64 = precision == UNOCG_FP64;
  DFields& f = fp64 ? d->f64f : d->f32f;
  const size_t eb = fp64 ? 8 : 4;
  if (!d->f64) DCK(cudaMalloc(&d->f64, n * sizeof(double)));
  if (!d->u64) DCK(cudaMalloc(&d->u64, n * sizeof(double)));
  if (!f.r) DCK(cudaMalloc(&f.r, n * eb));
  if (!f.p) DCK(cudaMalloc(&f.p, n * eb));
  if (!f.q) DCK(cudaMalloc(&f.q, n * eb));
  if (!fp64 && !f.u) DCK(cudaMalloc(&f.u, n * eb));
  if (precond == UNOCG_PRECOND_UNO && !f.hat) DCK(cudaMalloc(&f.hat, n * eb));
  if (precond == UNOCG_PRECOND_JACOBI && !f.invdiag)
    DCK(cudaMalloc(&f.invdiag, (size_t)d->B * d->c * d->g.ne * eb));
  size_t need = (size_t)BL * std::max({(size_t)dku_blocks(d->g, d->c), (size_t)djac_blocks(d->g),
                                       (size_t)(d->np == 2 ? dmixq_blocks(d->g, d->pa, d->pb) : 0),
                                       (size_t)(d->line_reg_p[0] || d->line_reg_p[1] ? dline_reg_blocks(d->g) : 0),
                                       (size_t)dpass_blocks(d->g, d->c, DP_QMUL, std::min(d->w1[0], d->w1[1]))});
  if (d->part_len < need) {
    cudaFree(d->part);
    d->part = nullptr;
    DCK(cudaMalloc(&d->part, need * sizeof(double)));
    d->part_len = need;
  }
  if (!d->sc) DCK(cudaMalloc(&d->sc, BL * sizeof(CgScal)));
  return UNOCG_OK;
}

struct DPlan {
  unocg_solve_opts o;
  int mixed;
};

template <typename T> DFields& dfields(unocg_dir* d) { return sizeof(T) == 8 ? d->f64f : d->f32f; }
template <typename T> int pidx() { return sizeof(T) == 8 ? 0 : 1; }

template <typename T>
DPassArgs<T> pass_args(unocg_dir* d, int mode, const LoopCtl& ctl, int after_replace) {
  DFields& f = dfields<T>(d);
  DPassArgs<T> a{};
  a.g = d->g; a.c = d->c; a.BL = d->B * d->L; a.L = d->L;
  a.lines = mode == DP_MID ? d->w2[pidx<T>()]
          : (mode == DP_QMUL || mode == DP_MID1) ? d->w1[pidx<T>()] : d->lines3[pidx<T>()];
  a.hat = (T*)f.hat; a.r = (T*)f.r; a.q = (const T*)f.q; a.p = (T*)f.p;
  a.u = sizeof(T) == 8 ? (T*)d->u64 : (T*)f.u;
  a.Q = sizeof(T) == 8 ? (const void*)d->Q64 : (const void*)d->Q32;
  a.q_inst_stride = d->Bq > 1 ? d->g.nf * (d->c == 1 ? 1 : 6) : 0;
  a.sc = d->sc;
  a.red = Reduce{d->part, d->tickets + (mode == DP_QMUL ? DT_QMUL : after_replace ? DT_CHECK2 : DT_CHECK)};
  a.ctl = ctl; a.after_replace = after_replace; a.standalone = 0;
  a.t = dtables(d, sizeof(T) == 8);
  return a;
}

template <typename T>
DJacArgs<T> jac_args(unocg_dir* d, const DPlan& pl, const LoopCtl& ctl, int part, int after_replace) {
  DFields& f = dfields<T>(d);
  DJacArgs<T> a{};
  a.g = d->g; a.c = d->c; a.BL = d->B * d->L; a.L = d->L;
  a.r = (T*)f.r; a.q = (const T*)f.q; a.p = (T*)f.p;
  a.u = sizeof(T) == 8 ? (T*)d->u64 : (T*)f.u;
  a.invdiag = pl.o.precond == UNOCG_PRECOND_JACOBI ? (const T*)f.invdiag : nullptr;
  a.sc = d->sc;
  a.red = Reduce{d->part, d->tickets + (part == 1 ? DT_JAC : after_replace ? DT_CHECK2 : DT_CHECK)};
  a.ctl = ctl; a.after_replace = after_replace;
  return a;
}

template <typename T>
cudaError_t enq_check(unocg_dir* d, cudaStream_t s, const DPlan& pl, const LoopCtl& ctl, int after_replace) {
  if (pl.o.precond == UNOCG_PRECOND_UNO) {
    if (d->plane_engine[pidx<T>()] == 0) return launch_dplane_reg<T>(pass_args<T>(d, DP_FIRST, ctl, after_replace), 1, s);
    if (d->plane_engine[pidx<T>()] == 1) return launch_dplane<T>(pass_args<T>(d, DP_FIRST, ctl, after_replace), 1, s);
    return launch_dpass<T>(pass_args<T>(d, DP_FIRST, ctl, after_replace), DP_FIRST, s);
  }
  return launch_djac<T>(jac_args<T>(d, pl, ctl, 0, after_replace), 0, s);
}

template <typename T>
cudaError_t enq_pre(unocg_dir* d, cudaStream_t s, const DPlan& pl, const LoopCtl& ctl) {
  const int BL = d->B * d->L;
  DFields& f = dfields<T>(d);
  cudaError_t e = cudaMemsetAsync(d->sc, 0, BL * sizeof(CgScal), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->tickets, 0, DT_N * sizeof(unsigned int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->flags + 2, 0, 2 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  DInitArgs ia{};
  ia.g = d->g; ia.c = d->c; ia.L = d->L; ia.phase = d->phase; ia.mat = dmaterial(d); ia.loads = d->loads_d;
  ia.f64 = d->f64; ia.u64 = d->u64; ia.u32 = sizeof(T) == 8 ? nullptr : f.u;
  ia.r = f.r; ia.p = f.p; ia.q = f.q; ia.fp64 = sizeof(T) == 8;
  e = launch_dinit(ia, BL, s);
  if (e != cudaSuccess) return e;
  if (pl.o.precond == UNOCG_PRECOND_JACOBI) {
    DDiagArgs da{d->g, d->c, d->phase, dmaterial(d), f.invdiag, sizeof(T) == 8};
    e = launch_ddiag(da, d->B, s);
    if (e != cudaSuccess) return e;
  }
  return enq_check<T>(d, s, pl, ctl, 0);
}

template <typename T>
cudaError_t enq_ku(unocg_dir* d, cudaStream_t s) {
  DFields& f = dfields<T>(d);
  DKuArgs<T> ka{};
  ka.g = d->g; ka.c = d->c; ka.BL = d->B * d->L; ka.L = d->L; ka.phase = d->phase; ka.mat = dmaterial(d);
  ka.p = (const T*)f.p; ka.q = (T*)f.q; ka.sc = d->sc; ka.red = Reduce{d->part, d->tickets + DT_KU};
  ka.standalone = 0;
  return launch_dku<T>(ka, s);
}

// the transform passes between the forward plane pass (end of the previous iteration) and K p
template <typename T>
cudaError_t enq_precond(unocg_dir* d, cudaStream_t s, const LoopCtl& ctl, int standalone_lines_dummy = 0) {
  (void)standalone_lines_dummy;
  cudaError_t e = cudaSuccess;
  const bool plane = d->plane_engine[pidx<T>()] != 2;
  if (!plane) e = launch_dpass<T>(pass_args<T>(d, DP_MID, ctl, 0), DP_MID, s);
  if (e != cudaSuccess) return e;
  if (d->np == 2) {
    DPassArgs<T> m1 = pass_args<T>(d, DP_MID1, ctl, 0);
    e = launch_dpass<T>(m1, DP_MID1, s);
    if (e == cudaSuccess) e = launch_dmixq<T>(pass_args<T>(d, DP_QMUL, ctl, 0), d->pa, d->pb, s);
    if (e == cudaSuccess) e = launch_dpass<T>(m1, DP_MID1, s);
  } else if (d->line_reg_p[pidx<T>()]) {
    e = launch_dline_reg<T>(pass_args<T>(d, DP_QMUL, ctl, 0), s);
  } else {
    e = launch_dpass<T>(pass_args<T>(d, DP_QMUL, ctl, 0), DP_QMUL, s);
  }
  if (e != cudaSuccess) return e;
  if (d->plane_engine[pidx<T>()] == 0) return launch_dplane_reg<T>(pass_args<T>(d, DP_LAST, ctl, 0), 0, s);
  if (plane) return launch_dplane<T>(pass_args<T>(d, DP_LAST, ctl, 0), 0, s);
  e = launch_dpass<T>(pass_args<T>(d, DP_MID, ctl, 0), DP_MID, s);
  if (e == cudaSuccess) e = launch_dpass<T>(pass_args<T>(d, DP_LAST, ctl, 0), DP_LAST, s);
  return e;
}

template <typename T>
cudaError_t enq_body(unocg_dir* d, cudaStream_t s, const DPlan& pl, const LoopCtl& ctl) {
  cudaError_t e = cudaSuccess;
  if (pl.o.precond == UNOCG_PRECOND_UNO) {
    e = enq_precond<T>(d, s, ctl);
  } else {
    e = launch_djac<T>(jac_args<T>(d, pl, ctl, 1, 0), 1, s);
    if (e == cudaSuccess) e = launch_djac<T>(jac_args<T>(d, pl, ctl, 2, 0), 2, s);
  }
  if (e == cudaSuccess) e = enq_ku<T>(d, s);
  if (e == cudaSuccess) e = enq_check<T>(d, s, pl, ctl, 0);
  return e;
}

template <typename T>
DResArgs<T> res_args(unocg_dir* d, T* r, int only_pending) {
  DResArgs<T> ra{};
  ra.g = d->g; ra.c = d->c; ra.BL = d->B * d->L; ra.L = d->L; ra.phase = d->phase; ra.mat = dmaterial(d);
  ra.u64 = d->u64; ra.f64 = d->f64; ra.r = r; ra.sc = d->sc; ra.only_pending = only_pending;
  return ra;
}

// mixed precision: r = f - K u in FP64 for the pending pairs, then their residual check
// mixed precision keeps rref = f - K u64 in the f64 field (FP64; f at the start): a replacement
// brings it up to date with the FP32 increment in float-pair arithmetic, writes r = rref, then
// folds the increment into u64.  FP64 recomputes r = f - K u64.
template <typename T>
cudaError_t enq_replace(unocg_dir* d, cudaStream_t s, const DPlan& pl, const LoopCtl& ctl) {
  cudaError_t e = cudaSuccess;
  if (sizeof(T) == 4) {
    e = launch_dreplace(res_args<float>(d, (float*)d->f32f.r, 1), (const float*)d->f32f.u, 1, s);
    if (e == cudaSuccess) e = launch_dfold(d->g, d->c, d->B * d->L, d->u64, (float*)d->f32f.u, d->sc, 1, s);
    if (e == cudaSuccess) e = enq_check<T>(d, s, pl, ctl, 1);
    return e;
  }
  if (e == cudaSuccess) e = launch_dres<T>(res_args<T>(d, (T*)dfields<T>(d).r, 1), s);
  if (e != cudaSuccess) return e;
  return enq_check<T>(d, s, pl, ctl, 1);
}

// reported true residual (max |f - K u| of the final iterate) and the averaged flux / stress
template <typename T>
cudaError_t enq_post(unocg_dir* d, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (sizeof(T) == 4) {
    // reported true residual: rref brought up to date with the last increment, then the fold
    e = launch_dreplace(res_args<float>(d, nullptr, 0), (const float*)d->f32f.u, 0, s);
    if (e == cudaSuccess) e = launch_dfold(d->g, d->c, d->B * d->L, d->u64, (float*)d->f32f.u, d->sc, 0, s);
  } else {
    e = launch_dres<T>(res_args<T>(d, (T*)nullptr, 0), s);
  }
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d->ceff, 0, (size_t)d->B * d->dim * d->L * sizeof(double), s);
  if (e != cudaSuccess) return e;
  DAvgArgs aa{};
  aa.g = d->g; aa.c = d->c; aa.L = d->L; aa.phase = d->phase; aa.mat = dmaterial(d); aa.loads = d->loads_d;
  aa.u64 = d->u64; aa.out = d->ceff;
  return launch_davg(aa, d->B, s);
}

template <typename T>
int build_graph(unocg_dir* d, const DPlan& pl) {
  cudaStream_t cs = nullptr, bs = nullptr, rs = nullptr;
  DCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  DCK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  DCK(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus st;
  cudaGraph_t cg = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, nullptr, nullptr, nullptr);
  cudaGraphConditionalHandle hw = 0, hi = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, cg, 0, cudaGraphCondAssignDefault);
  LoopCtl ctl{};
  ctl.tol = pl.o.tol; ctl.max_iter = pl.o.max_iter; ctl.mixed = pl.mixed;
  ctl.replace_every = pl.o.replace_every; ctl.replace_drop = pl.o.replace_drop; ctl.flexible = 0;
  ctl.h_while = hw; ctl.set_while = 1; ctl.set_if = 0;
  ctl.counters = d->flags + 2;
  if (e == cudaSuccess) e = enq_pre<T>(d, cs, pl, ctl);
  cudaGraphNodeParams wp{};
  if (e == cudaSuccess) {
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphNode_t wnode;
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
    e = cudaStreamBeginCaptureToGraph(bs, wp.conditional.phGraph_out[0], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    LoopCtl bctl = ctl;
    if (e == cudaSuccess && pl.mixed) {
      e = cudaGraphConditionalHandleCreate(&hi, wp.conditional.phGraph_out[0], 0, cudaGraphCondAssignDefault);
      bctl.h_if = hi;
      bctl.set_if = 1;
    }
    if (e == cudaSuccess) e = enq_body<T>(d, bs, pl, bctl);
    if (e == cudaSuccess && pl.mixed) {
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaGraph_t bg = nullptr;
      cudaGraphNode_t inode;
      cudaGraphNodeParams ip{};
      e = cudaStreamGetCaptureInfo(bs, &st, nullptr, &bg, &deps, nullptr, &nd);
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
        if (e == cudaSuccess) e = enq_replace<T>(d, rs, pl, rctl);
        cudaGraph_t tmp;
        cudaError_t e2 = cudaStreamEndCapture(rs, &tmp);
        if (e == cudaSuccess) e = e2;
      }
    }
    cudaGraph_t tmp;
    cudaError_t e2 = cudaStreamEndCapture(bs, &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = enq_post<T>(d, cs);
  cudaError_t e3 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e3;
  cudaStreamDestroy(cs);
  cudaStreamDestroy(bs);
  cudaStreamDestroy(rs);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return dfail(d, UNOCG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return dfail(d, UNOCG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  dfree_graph(d);
  d->graph = g;
  d->exec = ex;
  return UNOCG_OK;
}

// Host-driven loop (use_graph = 0; profiling tools see every launch): one residual check per
// iteration read back by the host.
template <typename T>
int run_host_loop(unocg_dir* d, const DPlan& pl) {
  cudaStream_t s = d->stream;
  LoopCtl ctl{};
  ctl.tol = pl.o.tol; ctl.max_iter = pl.o.max_iter; ctl.mixed = pl.mixed;
  ctl.replace_every = pl.o.replace_every; ctl.replace_drop = pl.o.replace_drop; ctl.flexible = 0;
  ctl.active_flag = d->flags; ctl.replace_flag = d->flags + 1;
  ctl.counters = d->flags + 2;
  DCK(enq_pre<T>(d, s, pl, ctl));
  int hf[2] = {0, 0};
  const long long cap = 4LL * pl.o.max_iter + 16;
  for (long long it = 0; it < cap; ++it) {
    DCK(cudaMemcpyAsync(hf, d->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    DCK(cudaStreamSynchronize(s));
    if (!hf[0]) break;
    DCK(enq_body<T>(d, s, pl, ctl));
    if (pl.mixed) {
      DCK(cudaMemcpyAsync(hf, d->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      DCK(cudaStreamSynchronize(s));
      if (hf[1]) {
        LoopCtl rctl = ctl;
        rctl.active_flag = nullptr;  // keep the loop running; the next check decides
        DCK(enq_replace<T>(d, s, pl, rctl));
      }
    }
  }
  DCK(enq_post<T>(d, s));
  return UNOCG_OK;
}

bool have_inputs(unocg_dir* d) { return d->phase_set && d->mat64 && d->L > 0; }

}  // namespace

// ------------------------------------------------------------------ create / destroy
extern "C" int unocg_dir_create_bc(unocg_dir** out, int physics, int batch, int n1, int n2, int n3, double L0,
                                   const int* bc) {
  if (!out || !bc) return UNOCG_ERR_INVALID_ARG;
  *out = nullptr;
  if ((physics != UNOCG_THERMAL && physics != UNOCG_ELASTIC) || batch < 1 || !(L0 > 0.0)) return UNOCG_ERR_INVALID_ARG;
  if (!dim_ok(n1) || !dim_ok(n2) || !dim_ok(n3)) return UNOCG_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (bc[a] != 0 && bc[a] != 1) return UNOCG_ERR_INVALID_ARG;
  if (!bc[0] && !bc[1] && !bc[2]) return UNOCG_ERR_INVALID_ARG;  // all periodic: unocg_create
  unocg_dir* d = new unocg_dir();
  *out = d;
  d->physics = physics;
  d->c = physics == UNOCG_THERMAL ? 1 : 3;
  d->dim = physics == UNOCG_THERMAL ? 3 : 6;
  d->B = batch;
  DGrid& g = d->g;
  g.n1 = n1; g.n2 = n2; g.n3 = n3;
  const int ns[3] = {n1, n2, n3};
  for (int a = 0; a < 3; ++a) {
    g.bc[a] = bc[a];
    g.o[a] = bc[a];
    if (!bc[a]) {
      if (d->np == 0) d->pa = a;
      else d->pb = a;
      ++d->np;
    }
  }
  g.m1 = n1 - bc[0]; g.m2 = n2 - bc[1]; g.m3 = n3 - bc[2];
  g.ne = (long long)n1 * n2 * n3;
  g.nf = (long long)g.m1 * g.m2 * g.m3;
  g.pg.n1 = n1; g.pg.n2 = n2; g.pg.n3 = n3; g.pg.n3h = n3 / 2 + 1;
  g.pg.n = g.ne;
  g.pg.nh = (long long)n1 * n2 * (n3 / 2 + 1);
  g.pg.h = L0 / n1;
  grid_scales(g.pg);
  for (int a = 0; a < 3; ++a) {
    const int Lt = bc[a] ? 2 * ns[a] : ns[a];  // sine: odd-extended pairs; Hartley: plain pairs
    dfactor_plan(Lt, &d->plan[a]);
    DCK(dupload_twiddles<double>(&d->tw64[a], Lt));
    DCK(dupload_twiddles<float>(&d->tw32[a], Lt));
  }
  for (int p = 0; p < 2; ++p) {
    const int eb = p == 0 ? 8 : 4;
    d->lines3[p] = dst_lines_for(n3, eb, 32);
    d->w2[p] = fit_w(n2, 1, eb, 32);
    d->w1[p] = fit_w(n1, d->c, eb, d->c == 1 ? 32 : 16);
    // one plane per block pays while two blocks fit an SM (measured: FP32 64^3 7.5 vs 8.6 ms per
    // solve; FP64 64^3 with 130 KB planes 30.0 vs 26.4 ms)
    d->plane_engine[p] = dplane_smem_bytes(g, eb) <= 110 * 1024 ? 1 : 2;
  }
  const bool all_dir = bc[0] && bc[1] && bc[2];
  if (all_dir && dplane_reg_ok(g)) d->plane_engine[0] = d->plane_engine[1] = 0;
  d->line_reg_p[0] = all_dir && dline_reg_ok(g, d->c, 8);
  d->line_reg_p[1] = all_dir && dline_reg_ok(g, d->c, 4);
  DCK(cudaStreamCreateWithFlags(&d->own_stream, cudaStreamNonBlocking));
  d->stream = d->own_stream;
  DCK(cudaMalloc(&d->phase, (size_t)batch * g.ne));
  DCK(cudaMalloc(&d->tickets, DT_N * sizeof(unsigned int)));
  DCK(cudaMemset(d->tickets, 0, DT_N * sizeof(unsigned int)));
  DCK(cudaMalloc(&d->flags, 8 * sizeof(int)));
  DCK(cudaMemset(d->flags, 0, 8 * sizeof(int)));
  return UNOCG_OK;
}

extern "C" int unocg_dir_create(unocg_dir** out, int physics, int batch, int n1, int n2, int n3, double L0) {
  const int bc[3] = {1, 1, 1};
  return unocg_dir_create_bc(out, physics, batch, n1, n2, n3, L0, bc);
}

extern "C" void unocg_dir_destroy(unocg_dir* d) {
  if (!d) return;
  if (d->stream) cudaStreamSynchronize(d->stream);
  dfree_graph(d);
  free_fields(d->f64f);
  free_fields(d->f32f);
  for (int a = 0; a < 3; ++a) {
    cudaFree(d->tw64[a]);
    cudaFree(d->tw32[a]);
  }
  cudaFree(d->phase); cudaFree(d->mat64); cudaFree(d->mat32); cudaFree(d->loads_d);
  cudaFree(d->Q64); cudaFree(d->Q32); cudaFree(d->f64); cudaFree(d->u64);
  cudaFree(d->sc); cudaFree(d->part); cudaFree(d->tickets); cudaFree(d->flags); cudaFree(d->ceff);
  cudaFree(d->stage_a); cudaFree(d->stage_b); cudaFree(d->stage_f);
  if (d->own_stream) cudaStreamDestroy(d->own_stream);
  if (d->join_ev) cudaEventDestroy(d->join_ev);
  delete d;
}

extern "C" const char* unocg_dir_last_error(const unocg_dir* d) { return d ? d->err.c_str() : "null context"; }

extern "C" int unocg_dir_set_stream(unocg_dir* d, void* stream) {
  if (!d) return UNOCG_ERR_INVALID_ARG;
  d->stream = stream ? (cudaStream_t)stream : d->own_stream;
  return UNOCG_OK;
}

extern "C" int unocg_dir_set_microstructure(unocg_dir* d, const uint8_t* phase, int n_phases) {
  if (!d || !phase) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (n_phases < 1 || n_phases > 256) return dfail(d, UNOCG_ERR_INVALID_ARG, "n_phases must be 1..256");
  const size_t n = (size_t)d->B * d->g.ne;
  for (size_t i = 0; i < n; ++i)
    if (phase[i] >= n_phases) return dfail(d, UNOCG_ERR_INVALID_ARG, "phase label out of range");
  if (n_phases != d->n_phases) {
    cudaFree(d->mat64);
    cudaFree(d->mat32);
    d->mat64 = nullptr;
    d->mat32 = nullptr;
    d->props.clear();
  }
  d->n_phases = n_phases;
  DCK(cudaStreamSynchronize(d->stream));  // a solve in flight may still read the previous inputs
  DCK(cudaMemcpy(d->phase, phase, n, cudaMemcpyHostToDevice));
  d->phase_set = true;
  d->solved = false;
  return UNOCG_OK;
}

extern "C" int unocg_dir_set_phase_properties(unocg_dir* d, const double* props) {
  if (!d || !props) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (d->n_phases < 1) return dfail(d, UNOCG_ERR_STATE, "set the microstructure first");
  const int per = d->c == 1 ? 1 : 2;
  const size_t cnt = (size_t)d->B * d->n_phases;
  std::vector<double> m64(2 * cnt);
  std::vector<float> m32(2 * cnt);
  for (size_t i = 0; i < cnt; ++i) {
    if (d->c == 1) {
      const double k = props[i];
      if (!(k > 0.0) || !std::isfinite(k)) return dfail(d, UNOCG_ERR_INVALID_ARG, "conductivity must be positive");
      m64[2 * i] = k;
      m64[2 * i + 1] = 0.0;
    } else {
      const double E = props[2 * i], nu = props[2 * i + 1];
      if (!(E > 0.0) || !(nu > -1.0) || !(nu < 0.5)) return dfail(d, UNOCG_ERR_INVALID_ARG, "need E > 0, -1 < nu < 0.5");
      m64[2 * i] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
      m64[2 * i + 1] = E / (2.0 * (1.0 + nu));
    }
    m32[2 * i] = (float)m64[2 * i];
    m32[2 * i + 1] = (float)m64[2 * i + 1];
  }
  if (!d->mat64) DCK(cudaMalloc(&d->mat64, 2 * cnt * sizeof(double)));
  if (!d->mat32) DCK(cudaMalloc(&d->mat32, 2 * cnt * sizeof(float)));
  DCK(cudaStreamSynchronize(d->stream));
  DCK(cudaMemcpy(d->mat64, m64.data(), 2 * cnt * sizeof(double), cudaMemcpyHostToDevice));
  DCK(cudaMemcpy(d->mat32, m32.data(), 2 * cnt * sizeof(float), cudaMemcpyHostToDevice));
  d->props = m64;
  (void)per;
  if (d->wkind == UNOCG_W_REFERENCE_MEDIUM) d->wkind = -2;  // rebuild from the new phases on demand
  d->solved = false;
  return UNOCG_OK;
}

extern "C" int unocg_dir_set_macro_load(unocg_dir* d, int n_loads, const double* loads) {
  if (!d || !loads || n_loads < 1) return dfail(d, UNOCG_ERR_INVALID_ARG, "invalid loads");
  for (int i = 0; i < n_loads * d->dim; ++i)
    if (!std::isfinite(loads[i])) return dfail(d, UNOCG_ERR_INVALID_ARG, "non-finite load");
  if (n_loads != d->L) {
    dfree_graph(d);
    free_fields(d->f64f);
    free_fields(d->f32f);
    cudaFree(d->f64); cudaFree(d->u64); cudaFree(d->sc); cudaFree(d->loads_d); cudaFree(d->ceff);
    d->f64 = d->u64 = nullptr;
    d->sc = nullptr;
    d->loads_d = nullptr;
    d->ceff = nullptr;
    d->L = n_loads;
  }
  d->loads.assign(loads, loads + (size_t)n_loads * d->dim);
  if (!d->loads_d) DCK(cudaMalloc(&d->loads_d, d->loads.size() * sizeof(double)));
  if (!d->ceff) DCK(cudaMalloc(&d->ceff, (size_t)d->B * d->dim * d->L * sizeof(double)));
  DCK(cudaStreamSynchronize(d->stream));
  DCK(cudaMemcpy(d->loads_d, d->loads.data(), d->loads.size() * sizeof(double), cudaMemcpyHostToDevice));
  d->solved = false;
  return UNOCG_OK;
}

static int build_reference(unocg_dir* d, double spd_eps) {
  const int C = d->c == 1 ? 1 : 6;
  d->Bq = d->B;
  d->Qh.assign((size_t)d->B * d->g.nf * C, 0.0);
  for (int b = 0; b < d->B; ++b) {
    double mt[2] = {0.0, 0.0};
    for (int p = 0; p < d->n_phases; ++p) {
      mt[0] += d->props[2 * ((size_t)b * d->n_phases + p)] / d->n_phases;
      mt[1] += d->props[2 * ((size_t)b * d->n_phases + p) + 1] / d->n_phases;
    }
    reference_weights(d->g, d->c, mt, d->Qh.data() + (size_t)b * d->g.nf * C);
  }
  d->wkind = UNOCG_W_REFERENCE_MEDIUM;
  return finish_weights(d, spd_eps);
}

extern "C" int unocg_dir_set_uno_weights(unocg_dir* d, int kind, const void* w, int dtype, double spd_eps) {
  if (!d) return UNOCG_ERR_INVALID_ARG;
  const int C = d->c == 1 ? 1 : 6;
  const size_t m = (size_t)d->g.nf * C;
  if (kind == UNOCG_W_REFERENCE_MEDIUM) {
    if (d->props.empty()) return dfail(d, UNOCG_ERR_STATE, "set the phase properties first");
    return build_reference(d, spd_eps);
  }
  if (kind != UNOCG_W_BLOCKS && kind != UNOCG_W_THETA) return dfail(d, UNOCG_ERR_INVALID_ARG, "unknown weight kind");
  if (!w || (dtype != UNOCG_DTYPE_F64 && dtype != UNOCG_DTYPE_F32)) return dfail(d, UNOCG_ERR_INVALID_ARG, "invalid weights");
  d->Bq = 1;
  d->Qh.assign(m, 0.0);
  for (size_t i = 0; i < m; i += C) {
    double v[6];
    for (int k = 0; k < C; ++k) v[k] = dtype == UNOCG_DTYPE_F64 ? ((const double*)w)[i + k] : ((const float*)w)[i + k];
    if (kind == UNOCG_W_THETA) {
      double Q[3][3];
      psi_block(v, d->c, Q);
      entries_of(Q, d->c, &d->Qh[i]);
    } else {
      for (int k = 0; k < C; ++k) d->Qh[i + k] = v[k];
    }
  }
  if (d->np > 0) {
    // conjugate modes of the periodic axes: Q(k) <- (Q(k) + Q(-k)) / 2, -k negating every
    // periodic index (the condition for a real output of the paper's Fourier-domain operator,
    // under which the Hartley passes apply the same operator)
    const int m[3] = {d->g.m1, d->g.m2, d->g.m3};
    std::vector<double> sym(d->Qh.size());
    for (int k1 = 0; k1 < m[0]; ++k1)
      for (int k2 = 0; k2 < m[1]; ++k2)
        for (int k3 = 0; k3 < m[2]; ++k3) {
          const int q1 = d->g.bc[0] ? k1 : (m[0] - k1) % m[0];
          const int q2 = d->g.bc[1] ? k2 : (m[1] - k2) % m[1];
          const int q3 = d->g.bc[2] ? k3 : (m[2] - k3) % m[2];
          const size_t i = (((size_t)k1 * m[1] + k2) * m[2] + k3) * C;
          const size_t j = (((size_t)q1 * m[1] + q2) * m[2] + q3) * C;
          for (int e = 0; e < C; ++e) sym[i + e] = 0.5 * (d->Qh[i + e] + d->Qh[j + e]);
        }
    d->Qh.swap(sym);
  }
  d->wkind = kind;
  return finish_weights(d, spd_eps);
}

extern "C" int unocg_dir_set_uno_modes(unocg_dir* d, int M, const void* w, int dtype, double spd_eps) {
  if (!d || !w || (dtype != UNOCG_DTYPE_F64 && dtype != UNOCG_DTYPE_F32)) return dfail(d, UNOCG_ERR_INVALID_ARG, "invalid weights");
  if (d->np > 0) return dfail(d, UNOCG_ERR_INVALID_ARG, "the mode layout needs Dirichlet faces on every axis");
  if (M < 0 || 2 * M + 1 > d->g.m1 || 2 * M + 1 > d->g.m2 || 2 * M + 1 > d->g.m3)
    return dfail(d, UNOCG_ERR_INVALID_ARG, "mode set [0, 2M]^3 larger than the free grid");
  const int C = d->c == 1 ? 1 : 6;
  auto wv = [&](long long i) { return dtype == UNOCG_DTYPE_F64 ? ((const double*)w)[i] : (double)((const float*)w)[i]; };
  double t[6], W0[3][3] = {};
  for (int k = 0; k < C; ++k) t[k] = wv(k);
  psi_block(t, d->c, W0);
  double e0[6];
  entries_of(W0, d->c, e0);
  d->Bq = 1;
  d->Qh.assign((size_t)d->g.nf * C, 0.0);
  for (long long i = 0; i < d->g.nf; ++i)
    for (int k = 0; k < C; ++k) d->Qh[i * C + k] = e0[k];
  const int K = 2 * M + 1;
  long long idx = 1;
  for (int k1 = 0; k1 < K; ++k1)
    for (int k2 = 0; k2 < K; ++k2)
      for (int k3 = 0; k3 < K; ++k3, ++idx) {
        for (int k = 0; k < C; ++k) t[k] = wv(idx * C + k);
        double Qm[3][3] = {}, em[6];
        psi_block(t, d->c, Qm);
        entries_of(Qm, d->c, em);
        const long long mode = ((long long)k1 * d->g.m2 + k2) * d->g.m3 + k3;
        for (int k = 0; k < C; ++k) d->Qh[mode * C + k] += em[k];
      }
  d->wkind = UNOCG_W_MODES;
  return finish_weights(d, spd_eps);
}

extern "C" int unocg_dir_get_uno_weights(unocg_dir* d, int instance, double* out) {
  if (!d || !out) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (d->wkind == -2) {
    int rc = build_reference(d, 0.0);
    if (rc) return rc;
  }
  if (d->wkind < 0) return dfail(d, UNOCG_ERR_STATE, "set UNO weights first");
  if (instance < 0 || instance >= d->B) return dfail(d, UNOCG_ERR_INVALID_ARG, "instance out of range");
  const size_t m = (size_t)d->g.nf * (d->c == 1 ? 1 : 6);
  std::memcpy(out, d->Qh.data() + (d->Bq > 1 ? instance * m : 0), m * sizeof(double));
  return UNOCG_OK;
}

// ------------------------------------------------------------------ solve
extern "C" int unocg_dir_solve_async(unocg_dir* d, const unocg_solve_opts* o) {
  NvtxRange nvtx_("unocg_dir_solve_async");
  if (!d || !o) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!have_inputs(d)) return dfail(d, UNOCG_ERR_STATE, "set microstructure, phase properties and loads first");
  if (o->precond < 0 || o->precond > 2 || (o->precision != UNOCG_FP64 && o->precision != UNOCG_MIXED) ||
      !(o->tol > 0.0) || o->max_iter < 1 || o->replace_every < 0 || !(o->replace_drop >= 0.0) ||
      !(o->replace_drop < 1.0) || o->flexible)
    return dfail(d, UNOCG_ERR_INVALID_ARG, "invalid solve options (flexible CG is not available with Dirichlet BC)");
  if (o->precond == UNOCG_PRECOND_UNO) {
    if (d->wkind == -2) {
      int rc = build_reference(d, 0.0);
      if (rc) return rc;
    }
    if (d->wkind < 0) return dfail(d, UNOCG_ERR_STATE, "set UNO weights first");
    if (o->precision == UNOCG_MIXED && !d->f32_spd_ok)
      return dfail(d, UNOCG_ERR_NOT_SPD, "UNO weights fail the safety check after rounding to FP32");
  }
  DPlan pl;
  pl.o = *o;
  pl.mixed = o->precision == UNOCG_MIXED;
  if (!pl.mixed) {
    pl.o.replace_every = 0;
    pl.o.replace_drop = 0.0;
  }
  int rc = ensure_workspace(d, o->precision, o->precond);
  if (rc) return rc;
  if (o->use_graph == 0) {
    rc = pl.mixed ? run_host_loop<float>(d, pl) : run_host_loop<double>(d, pl);
    if (rc) return rc;
  } else {
    DKey k;
    k.precond = o->precond; k.precision = o->precision; k.max_iter = o->max_iter;
    k.replace_every = pl.o.replace_every; k.replace_drop = pl.o.replace_drop; k.L = d->L; k.tol = o->tol;
    if (!d->exec || !(k == d->key)) {
      rc = pl.mixed ? build_graph<float>(d, pl) : build_graph<double>(d, pl);
      if (rc) return rc;
      d->key = k;
    }
    DCK(cudaGraphLaunch(d->exec, d->stream));
  }
  d->last_precision = o->precision;
  d->solved = true;
  return UNOCG_OK;
}

extern "C" int unocg_dir_solve_wait(unocg_dir* d, unocg_solve_info* info) {
  if (!d) return UNOCG_ERR_INVALID_ARG;
  if (!d->solved) return dfail(d, UNOCG_ERR_STATE, "no solve in flight");
  DCK(cudaStreamSynchronize(d->stream));
  DCK(cudaGetLastError());
  const int BL = d->B * d->L;
  std::vector<CgScal> hs(BL);
  DCK(cudaMemcpy(hs.data(), d->sc, BL * sizeof(CgScal), cudaMemcpyDeviceToHost));
  int status = UNOCG_OK, mx = 0;
  for (int i = 0; i < BL; ++i) {
    const CgScal& s = hs[i];
    const int st = s.done ? s.status : UNOCG_ERR_NOT_CONVERGED;
    if (status == UNOCG_OK && st != UNOCG_OK) status = st;
    mx = std::max(mx, s.iters);
    if (info) {
      const double f0 = s.r0max;
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
  DCK(cudaMemcpy(ctl, d->flags, 8 * sizeof(int), cudaMemcpyDeviceToHost));
  if (info) {
    info->status = status;
    info->max_iters = mx;
    info->checks = ctl[2];
    info->replacements = ctl[3];
  }
  if (status != UNOCG_OK) d->err = status == UNOCG_ERR_NOT_CONVERGED ? "not converged within max_iter" : "CG breakdown";
  return status;
}

extern "C" int unocg_dir_solve(unocg_dir* d, const unocg_solve_opts* o, unocg_solve_info* info) {
  int rc = unocg_dir_solve_async(d, o);
  if (rc) return rc;
  return unocg_dir_solve_wait(d, info);
}

// ------------------------------------------------------------------ outputs
static int ensure_stage(unocg_dir* d) {
  const size_t ne = (size_t)d->c * d->g.ne, nf = (size_t)d->c * d->g.nf;
  if (!d->stage_a) DCK(cudaMalloc(&d->stage_a, ne * sizeof(double)));
  if (!d->stage_b) DCK(cudaMalloc(&d->stage_b, ne * sizeof(double)));
  if (!d->stage_f) DCK(cudaMalloc(&d->stage_f, nf * sizeof(double)));
  return UNOCG_OK;
}

extern "C" int unocg_dir_get_fluctuation_dev(unocg_dir* d, int instance, int load, double* out_dev, void* stream) {
  if (!d || !out_dev) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!d->solved) return dfail(d, UNOCG_ERR_STATE, "no solution");
  if (instance < 0 || instance >= d->B || load < 0 || load >= d->L)
    return dfail(d, UNOCG_ERR_INVALID_ARG, "instance/load out of range");
  const double* src = d->u64 + ((size_t)instance * d->L + load) * d->c * d->g.ne;
  cudaStream_t s = (cudaStream_t)stream;
  DCK(order_after(&d->join_ev, d->stream, s));
  DCK(launch_dgather(d->g, d->c, src, out_dev, s));
  DCK(order_after(&d->join_ev, s, d->stream));
  return UNOCG_OK;
}

extern "C" int unocg_dir_get_fluctuation(unocg_dir* d, int instance, int load, double* out) {
  if (!d || !out) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!d->solved) return dfail(d, UNOCG_ERR_STATE, "no solution");
  if (instance < 0 || instance >= d->B || load < 0 || load >= d->L)
    return dfail(d, UNOCG_ERR_INVALID_ARG, "instance/load out of range");
  int rc = ensure_stage(d);
  if (rc) return rc;
  const size_t n = (size_t)d->g.nf;
  std::vector<double> soa((size_t)d->c * n);
  const double* src = d->u64 + ((size_t)instance * d->L + load) * d->c * d->g.ne;
  DCK(launch_dgather(d->g, d->c, src, d->stage_f, d->stream));
  DCK(cudaMemcpyAsync(soa.data(), d->stage_f, soa.size() * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  DCK(cudaStreamSynchronize(d->stream));
  for (size_t i = 0; i < n; ++i)
    for (int k = 0; k < d->c; ++k) out[i * d->c + k] = soa[k * n + i];
  return UNOCG_OK;
}

extern "C" int unocg_dir_get_effective_tensor(unocg_dir* d, double* out) {
  if (!d || !out) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!d->solved) return dfail(d, UNOCG_ERR_STATE, "no solution");
  DCK(cudaStreamSynchronize(d->stream));
  DCK(cudaMemcpy(out, d->ceff, (size_t)d->B * d->dim * d->L * sizeof(double), cudaMemcpyDeviceToHost));
  return UNOCG_OK;
}

// ------------------------------------------------------------------ operator-level entry points
extern "C" int unocg_dir_apply_K_dev(unocg_dir* d, int instance, const double* p_dev, double* q_dev, void* stream) {
  NvtxRange nvtx_("unocg_dir_apply_K_dev");
  if (!d || !p_dev || !q_dev) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (!d->phase_set || !d->mat64) return dfail(d, UNOCG_ERR_STATE, "set microstructure and phase properties first");
  if (instance < 0 || instance >= d->B) return dfail(d, UNOCG_ERR_INVALID_ARG, "instance out of range");
  int rc = ensure_stage(d);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  DCK(order_after(&d->join_ev, d->stream, s));
  DCK(launch_dscatter(d->g, d->c, p_dev, d->stage_a, s));
  DKuArgs<double> ka{};
  ka.g = d->g; ka.c = d->c; ka.BL = 1; ka.L = 1;
  ka.phase = d->phase + (size_t)instance * d->g.ne;
  Material m = dmaterial(d);
  m.m64 += (size_t)instance * d->n_phases * 2;
  m.m32 += (size_t)instance * d->n_phases * 2;
  ka.mat = m;
  ka.p = d->stage_a; ka.q = d->stage_b; ka.standalone = 1;
  DCK(launch_dku<double>(ka, s));
  DCK(launch_dgather(d->g, d->c, d->stage_b, q_dev, s));
  DCK(order_after(&d->join_ev, s, d->stream));
  return UNOCG_OK;
}

extern "C" int unocg_dir_apply_uno_dev(unocg_dir* d, int instance, const double* r_dev, double* s_dev, void* stream) {
  NvtxRange nvtx_("unocg_dir_apply_uno_dev");
  if (!d || !r_dev || !s_dev) return dfail(d, UNOCG_ERR_INVALID_ARG, "null argument");
  if (d->wkind == -2) {
    int rc = build_reference(d, 0.0);
    if (rc) return rc;
  }
  if (d->wkind < 0) return dfail(d, UNOCG_ERR_STATE, "set UNO weights first");
  if (instance < 0 || instance >= d->B) return dfail(d, UNOCG_ERR_INVALID_ARG, "instance out of range");
  int rc = ensure_stage(d);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  DCK(order_after(&d->join_ev, d->stream, s));
  DCK(launch_dscatter(d->g, d->c, r_dev, d->stage_a, s));
  LoopCtl ctl{};
  DPassArgs<double> a = pass_args<double>(d, DP_FIRST, ctl, 0);
  a.BL = 1; a.L = 1; a.standalone = 1; a.src = d->stage_a; a.hat = d->stage_b; a.out = d->stage_a;
  a.Q = d->Q64 + (d->Bq > 1 ? (size_t)instance * d->g.nf * (d->c == 1 ? 1 : 6) : 0);
  a.q_inst_stride = 0;
  auto with = [&](int lines) {
    DPassArgs<double> b = a;
    b.lines = lines;
    return b;
  };
  const bool plane = d->plane_engine[0] != 2;
  if (d->plane_engine[0] == 0) DCK(launch_dplane_reg<double>(a, 1, s));
  else if (plane) DCK(launch_dplane<double>(a, 1, s));
  else {
    DCK(launch_dpass<double>(with(d->lines3[0]), DP_FIRST, s));
    DCK(launch_dpass<double>(with(d->w2[0]), DP_MID, s));
  }
  if (d->np == 2) {
    DCK(launch_dpass<double>(with(d->w1[0]), DP_MID1, s));
    DCK(launch_dmixq<double>(a, d->pa, d->pb, s));
    DCK(launch_dpass<double>(with(d->w1[0]), DP_MID1, s));
  } else if (d->line_reg_p[0]) {
    DCK(launch_dline_reg<double>(a, s));
  } else {
    DCK(launch_dpass<double>(with(d->w1[0]), DP_QMUL, s));
  }
  if (d->plane_engine[0] == 0) DCK(launch_dplane_reg<double>(a, 0, s));
  else if (plane) DCK(launch_dplane<double>(a, 0, s));
  else {
    DCK(launch_dpass<double>(with(d->w2[0]), DP_MID, s));
    DCK(launch_dpass<double>(with(d->lines3[0]), DP_LAST, s));
  }
  DCK(launch_dgather(d->g, d->c, d->stage_a, s_dev, s));
  DCK(order_after(&d->join_ev, s, d->stream));
  return UNOCG_OK;
}


// ------------------------------------------------------------------ tuning
extern "C" int unocg_dir_set_tuning(unocg_dir* d, int precision, int plane_engine, int line_engine) {
  if (!d || (precision != UNOCG_FP64 && precision != UNOCG_MIXED) || plane_engine < 0 || plane_engine > 2 ||
      line_engine < 0 || line_engine > 1)
    return dfail(d, UNOCG_ERR_INVALID_ARG, "invalid tuning");
  const int p = precision == UNOCG_FP64 ? 0 : 1;
  const int eb = p == 0 ? 8 : 4;
  const bool all_dir = d->g.bc[0] && d->g.bc[1] && d->g.bc[2];
  int dev = 0, smem_max = 0;
  DCK(cudaGetDevice(&dev));
  DCK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (plane_engine == 0 && !(all_dir && dplane_reg_ok(d->g)))
    return dfail(d, UNOCG_ERR_INVALID_ARG, "register plane passes need Dirichlet faces and N2 = N3 a power of two <= 128");
  if (plane_engine == 1 && dplane_smem_bytes(d->g, eb) > (size_t)smem_max)
    return dfail(d, UNOCG_ERR_INVALID_ARG, "the plane does not fit a block's shared memory");
  if (line_engine == 0 && !(all_dir && dline_reg_ok(d->g, d->c, eb)))
    return dfail(d, UNOCG_ERR_INVALID_ARG, "register axis-1 pass needs Dirichlet faces, c = 1 and N1 a power of two <= 128");
  DCK(cudaStreamSynchronize(d->stream));
  d->plane_engine[p] = plane_engine;
  d->line_reg_p[p] = line_engine == 0;
  size_t need = (size_t)d->B * d->L * (size_t)(d->line_reg_p[p] ? dline_reg_blocks(d->g) : 0);
  if (need > d->part_len) {
    cudaFree(d->part);
    d->part = nullptr;
    DCK(cudaMalloc(&d->part, need * sizeof(double)));
    d->part_len = need;
  }
  dfree_graph(d);
  return UNOCG_OK;
}

// Times `reps` solves of `opts` (events on the context stream, after a warm-up solve that builds
// the graph) for every applicable pair (plane engine 0..2, axis-1 engine 0..1) of the solve's
// precision; times[plane * 2 + line] = mean milliseconds (NaN where not applicable); keeps the
// fastest.
extern "C" int unocg_dir_autotune(unocg_dir* d, const unocg_solve_opts* o, int reps, double* times) {
  if (!d || !o || reps < 1 || !times) return dfail(d, UNOCG_ERR_INVALID_ARG, "invalid autotune arguments");
  double best = 1e300;
  int bpl = -1, bli = -1;
  cudaEvent_t e0, e1;
  DCK(cudaEventCreate(&e0));
  DCK(cudaEventCreate(&e1));
  int rc = UNOCG_OK;
  for (int pe = 0; pe < 3 && rc == UNOCG_OK; ++pe)
    for (int le = 0; le < 2 && rc == UNOCG_OK; ++le) {
      double* t = times + pe * 2 + le;
      *t = std::nan("");
      if (d->np == 2 && le == 0) continue;  // two periodic axes: the axis-1 passes are fixed
      if (unocg_dir_set_tuning(d, o->precision, pe, le) != UNOCG_OK) continue;
      rc = unocg_dir_solve(d, o, nullptr);
      if (rc) break;
      float ms = 0.f;
      if (cudaEventRecord(e0, d->stream) != cudaSuccess) { rc = dfail(d, UNOCG_ERR_CUDA, "event"); break; }
      for (int r = 0; r < reps && rc == UNOCG_OK; ++r) rc = unocg_dir_solve_async(d, o);
      if (rc) break;
      if (cudaEventRecord(e1, d->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = dfail(d, UNOCG_ERR_CUDA, "event timing"); break; }
      rc = unocg_dir_solve_wait(d, nullptr);
      if (rc) break;
      *t = ms / reps;
      if (*t < best) { best = *t; bpl = pe; bli = le; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (bpl < 0) return dfail(d, UNOCG_ERR_STATE, "no applicable pass engine");
  return unocg_dir_set_tuning(d, o->precision, bpl, bli);
}
