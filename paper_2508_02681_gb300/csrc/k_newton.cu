// Second-order UNO training (Algorithm 4, Sec. 5.4; c = 3: App. C) on the device: Newton-Raphson
// on the paper's bypass-plus-modes weights w = [w_0; w_1 .. w_n] from the precomputed features.
//
// Per mode k of the learned set the loss is quadratic in the unique block entries v (paper
// order): L_k(v) = sum_m a_{k,m} (Q(v)^2)_m - b_k . v = (1/2) v^T H_k v - b_k . v with
// H_k[e][f] = sum_m a_{k,m} (E_e E_f + E_f E_e)_m (E_e the symmetric unit matrix of entry e);
// for c = 1 this is a v^2 - b v, for c = 2 the loss of Eq. (features-c-2).  Every mode outside
// the learned set sees only the bypass, so those modes enter through the sums a_rest, b_rest.
// With v = psi(w_0) + psi(w_k) on the learned modes and psi(w_0) elsewhere (psi = L L^T, L lower
// triangular holding the parameters), gradient and Hessian follow by the chain rule; the Hessian
// is an arrow of P x P blocks (P = C = c(c+1)/2): the bypass couples to every mode, the modes do
// not couple to each other.  One step is an O(n) block Schur-complement solve:
//   D_k = H_kk + lambda I,   S = H_00 + lambda I - sum_k H_0k D_k^-1 H_k0,
//   S x_0 = g_0 - sum_k H_0k D_k^-1 g_k,   x_k = D_k^-1 (g_k - H_k0 x_0),   w <- w - x,
// with Levenberg-Marquardt damping lambda: a step is taken only if it lowers the loss, else
// lambda grows and the step is recomputed.
//
// Kernels: k_newton_modes (one thread per mode: H_k, the chain rule, D_k^-1 by Cholesky, the
// per-block partial sums of the Schur complement and of the loss), k_newton_bypass (one block:
// the fixed-order sum of the partials, S and its Cholesky solve for x_0), k_newton_update (one
// thread per mode: x_k, the trial weights and the partials of the trial loss), k_newton_loss
// (one block: the trial loss).  The host drives the damping.
#include <algorithm>
#include <cmath>
#include <utility>
#include <string>
#include <vector>
#include "common.cuh"
#include "../../include/unocg.h"

namespace unocg {
namespace {

constexpr int NMAX = 6;          // entries / parameters per mode (c = 3)
constexpr int kNewtonThreads = 128;

struct NewtonTables {
  int c, C;                       // components, entries (= parameters) per mode
  int ei[NMAX], ej[NMAX];         // entry e is Q[ei][ej]
  int lr[NMAX], lq[NMAX];         // parameter p sits at L[lr][lq]
  double T[NMAX][NMAX][NMAX];     // (E_e E_f + E_f E_e)_m
  double D2[NMAX][NMAX][NMAX];    // d^2 v_e / dw_p dw_q (constant)
};

// Partials of one block: Schur sum [P*P], its right-hand-side sum [P], sum of H_k [C*C], sum of
// the entry gradients [C], loss, max |H_kk|, failure count.
constexpr int kPartVals = NMAX * NMAX + NMAX + NMAX * NMAX + NMAX + 3;

struct NewtonArgs {
  int n;                          // learned modes
  const double* ak;               // [n][C]
  const double* bk;               // [n][C]
  const double* a_rest;           // [C]
  const double* b_rest;           // [C]
  const double* w;                // [1 + n][C] current weights
  double* wt;                     // [1 + n][C] trial weights
  double* dg;                     // [n][C]    D_k^-1 g_k
  double* dh;                     // [n][C][C] D_k^-1 H_k0
  double* part;                   // [blocks][kPartVals]
  double* part2;                  // [blocks] trial-loss partials
  double* out;                    // [0] loss(w), [1] loss(trial), [2] max|H_kk|, [3] failures
  int blocks;
  double lambda;
};

__device__ void psi_jac(const NewtonTables& t, const double* w, double* v, double (*J)[NMAX]) {
  double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int p = 0; p < t.C; ++p) L[t.lr[p]][t.lq[p]] = w[p];
  for (int e = 0; e < t.C; ++e) {
    double s = 0.0;
    for (int k = 0; k < t.c; ++k) s += L[t.ei[e]][k] * L[t.ej[e]][k];
    v[e] = s;
    if (J)
      for (int p = 0; p < t.C; ++p)
        J[e][p] = (t.ei[e] == t.lr[p] ? L[t.ej[e]][t.lq[p]] : 0.0) + (t.ej[e] == t.lr[p] ? L[t.ei[e]][t.lq[p]] : 0.0);
  }
}

__device__ void hess_entries(const NewtonTables& t, const double* a, double (*H)[NMAX]) {
  for (int e = 0; e < t.C; ++e)
    for (int f = 0; f < t.C; ++f) {
      double s = 0.0;
      for (int m = 0; m < t.C; ++m) s += a[m] * t.T[e][f][m];
      H[e][f] = s;
    }
}

// Cholesky factor of the symmetric n x n matrix A in place (lower); false if not positive definite
__device__ bool cholesky(double (*A)[NMAX], int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    A[j][j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
      A[i][j] = s / d;
    }
  }
  return true;
}
__device__ void chol_solve(const double (*Lf)[NMAX], int n, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= Lf[i][k] * x[k];
    x[i] = s / Lf[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= Lf[k][i] * x[k];
    x[i] = s / Lf[i][i];
  }
}

__device__ double quad_loss(const NewtonTables& t, const double (*H)[NMAX], const double* b, const double* v) {
  double s = 0.0;
  for (int e = 0; e < t.C; ++e) {
    double hv = 0.0;
    for (int f = 0; f < t.C; ++f) hv += H[e][f] * v[f];
    s += 0.5 * v[e] * hv - b[e] * v[e];
  }
  return s;
}

// block sum of `cnt` values per thread into part[blockIdx.x * stride + ...] (fixed order)
__device__ void block_partials(double* vals, int cnt, double* sh, double* dst) {
  for (int j = 0; j < cnt; ++j) {
    double s = block_sum(vals[j], sh);
    if (threadIdx.x == 0) dst[j] = s;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kNewtonThreads) k_newton_modes(const __grid_constant__ NewtonTables t, NewtonArgs a) {
  __shared__ double sh[32];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = t.C, C = t.C;
  double vals[kPartVals];
  for (int j = 0; j < kPartVals; ++j) vals[j] = 0.0;
  double hmax = 0.0;
  if (k < a.n) {
    double v0[NMAX], J0[NMAX][NMAX], u[NMAX], Ji[NMAX][NMAX], vi[NMAX], H[NMAX][NMAX], G[NMAX];
    psi_jac(t, a.w, v0, J0);
    psi_jac(t, a.w + (1 + k) * C, u, Ji);
    for (int e = 0; e < C; ++e) vi[e] = v0[e] + u[e];
    hess_entries(t, a.ak + k * C, H);
    const double* b = a.bk + k * C;
    for (int e = 0; e < C; ++e) {
      double s = -b[e];
      for (int f = 0; f < C; ++f) s += H[e][f] * vi[f];
      G[e] = s;
    }
    double gi[NMAX], H0i[NMAX][NMAX], D[NMAX][NMAX];
    for (int p = 0; p < P; ++p) {
      double s = 0.0;
      for (int e = 0; e < C; ++e) s += Ji[e][p] * G[e];
      gi[p] = s;
    }
    for (int p = 0; p < P; ++p)
      for (int q = 0; q < P; ++q) {
        double s0 = 0.0, si = 0.0;
        for (int e = 0; e < C; ++e) {
          double hj = 0.0;
          for (int f = 0; f < C; ++f) hj += H[e][f] * Ji[f][q];
          s0 += J0[e][p] * hj;
          si += Ji[e][p] * hj;
        }
        for (int e = 0; e < C; ++e) si += G[e] * t.D2[e][p][q];
        H0i[p][q] = s0;
        D[p][q] = si;
        hmax = fmax(hmax, fabs(si));
      }
    for (int p = 0; p < P; ++p) D[p][p] += a.lambda;
    double* dg = a.dg + k * C;
    double* dh = a.dh + (long long)k * C * C;
    if (cholesky(D, P)) {
      double x[NMAX];
      for (int p = 0; p < P; ++p) x[p] = gi[p];
      chol_solve(D, P, x);
      for (int p = 0; p < P; ++p) dg[p] = x[p];
      // columns of D^-1 H_k0 (H_k0 = H_0k^T)
      double Y[NMAX][NMAX];
      for (int q = 0; q < P; ++q) {
        for (int p = 0; p < P; ++p) x[p] = H0i[q][p];
        chol_solve(D, P, x);
        for (int p = 0; p < P; ++p) Y[p][q] = x[p];
      }
      for (int p = 0; p < P; ++p)
        for (int q = 0; q < P; ++q) dh[p * C + q] = Y[p][q];
      // Schur partials: H_0k D^-1 H_k0 and H_0k D^-1 g_k
      for (int p = 0; p < P; ++p) {
        for (int q = 0; q < P; ++q) {
          double s = 0.0;
          for (int r = 0; r < P; ++r) s += H0i[p][r] * Y[r][q];
          vals[p * NMAX + q] = s;
        }
        double s = 0.0;
        for (int r = 0; r < P; ++r) s += H0i[p][r] * dg[r];
        vals[NMAX * NMAX + p] = s;
      }
    } else {
      vals[kPartVals - 1] = 1.0;  // D_k not positive definite
    }
    for (int e = 0; e < C; ++e) {
      for (int f = 0; f < C; ++f) vals[NMAX * NMAX + NMAX + e * NMAX + f] = H[e][f];
      vals[2 * NMAX * NMAX + NMAX + e] = G[e];
    }
    vals[2 * NMAX * NMAX + 2 * NMAX] = quad_loss(t, H, b, vi);
  }
  block_partials(vals, kPartVals - 2, sh, a.part + (long long)blockIdx.x * kPartVals);
  // max |H_kk| and the failure count
  const double hblock = block_max(hmax, sh);
  const double fails = block_sum(vals[kPartVals - 1], sh);
  if (threadIdx.x == 0) {
    a.part[(long long)blockIdx.x * kPartVals + kPartVals - 2] = hblock;
    a.part[(long long)blockIdx.x * kPartVals + kPartVals - 1] = fails;
  }
}

// One thread: sums the partials in block order, forms S and solves for x_0 (written to wt[0]
// as the trial bypass), records loss(w), max |H_kk| and the failure count.
__global__ void k_newton_bypass(const __grid_constant__ NewtonTables t, NewtonArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int P = t.C, C = t.C;
  double acc[kPartVals];
  for (int j = 0; j < kPartVals; ++j) acc[j] = 0.0;
  double hmax = 0.0;
  for (int bidx = 0; bidx < a.blocks; ++bidx) {
    const double* p = a.part + (long long)bidx * kPartVals;
    for (int j = 0; j < kPartVals - 2; ++j) acc[j] += p[j];
    hmax = fmax(hmax, p[kPartVals - 2]);
    acc[kPartVals - 1] += p[kPartVals - 1];
  }
  double v0[NMAX], J0[NMAX][NMAX], Hr[NMAX][NMAX], Gall[NMAX];
  psi_jac(t, a.w, v0, J0);
  hess_entries(t, a.a_rest, Hr);
  for (int e = 0; e < C; ++e) {
    double s = -a.b_rest[e] + acc[2 * NMAX * NMAX + NMAX + e];
    for (int f = 0; f < C; ++f) s += Hr[e][f] * v0[f];
    Gall[e] = s;
  }
  const double loss = quad_loss(t, Hr, a.b_rest, v0) + acc[2 * NMAX * NMAX + 2 * NMAX];
  double S[NMAX][NMAX], rhs[NMAX];
  for (int p = 0; p < P; ++p) {
    double g0 = 0.0;
    for (int e = 0; e < C; ++e) g0 += J0[e][p] * Gall[e];
    rhs[p] = g0 - acc[NMAX * NMAX + p];
    for (int q = 0; q < P; ++q) {
      double s = 0.0;
      for (int e = 0; e < C; ++e) {
        double hj = 0.0;
        for (int f = 0; f < C; ++f) hj += (Hr[e][f] + acc[NMAX * NMAX + NMAX + e * NMAX + f]) * J0[f][q];
        s += J0[e][p] * hj;
      }
      for (int e = 0; e < C; ++e) s += Gall[e] * t.D2[e][p][q];
      S[p][q] = s - acc[p * NMAX + q] + (p == q ? a.lambda : 0.0);
    }
  }
  double fails = acc[kPartVals - 1];
  if (fails == 0.0 && cholesky(S, P)) {
    chol_solve(S, P, rhs);
    for (int p = 0; p < P; ++p) a.wt[p] = a.w[p] - rhs[p];
  } else {
    fails += 1.0;
    for (int p = 0; p < P; ++p) a.wt[p] = a.w[p];
  }
  a.out[0] = loss;
  a.out[2] = hmax;
  a.out[3] = fails;
}

// One thread per mode: x_k = D_k^-1 g_k - D_k^-1 H_k0 x_0, trial weights and trial-loss partials.
__global__ void __launch_bounds__(kNewtonThreads) k_newton_update(const __grid_constant__ NewtonTables t, NewtonArgs a) {
  __shared__ double sh[32];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int P = t.C, C = t.C;
  double lt = 0.0;
  if (k < a.n) {
    double x0[NMAX];
    for (int p = 0; p < P; ++p) x0[p] = a.w[p] - a.wt[p];
    const double* dg = a.dg + k * C;
    const double* dh = a.dh + (long long)k * C * C;
    double wk[NMAX];
    for (int p = 0; p < P; ++p) {
      double s = dg[p];
      for (int q = 0; q < P; ++q) s -= dh[p * C + q] * x0[q];
      wk[p] = a.w[(1 + k) * C + p] - s;
      a.wt[(1 + k) * C + p] = wk[p];
    }
    double v0[NMAX], u[NMAX], vi[NMAX], H[NMAX][NMAX];
    psi_jac(t, a.wt, v0, nullptr);
    psi_jac(t, wk, u, nullptr);
    for (int e = 0; e < C; ++e) vi[e] = v0[e] + u[e];
    hess_entries(t, a.ak + k * C, H);
    lt = quad_loss(t, H, a.bk + k * C, vi);
  }
  const double s = block_sum(lt, sh);
  if (threadIdx.x == 0) a.part2[blockIdx.x] = s;
}

__global__ void k_newton_loss(const __grid_constant__ NewtonTables t, NewtonArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int bidx = 0; bidx < a.blocks; ++bidx) s += a.part2[bidx];
  double v0[NMAX], Hr[NMAX][NMAX];
  psi_jac(t, a.wt, v0, nullptr);
  hess_entries(t, a.a_rest, Hr);
  a.out[1] = s + quad_loss(t, Hr, a.b_rest, v0);
}

NewtonTables make_tables(int c) {
  NewtonTables t{};
  t.c = c;
  t.C = c * (c + 1) / 2;
  // entry order (paper): c = 1 (Q11); c = 2 (Q11, Q22, Q12); c = 3 (Q11, Q22, Q12, Q33, Q23, Q13)
  static const int E3[6][2] = {{0, 0}, {1, 1}, {0, 1}, {2, 2}, {1, 2}, {0, 2}};
  // parameter positions in L: c = 2 (w1 -> L11, w2 -> L22, w3 -> L21);
  // c = 3 (L11, L22, L21, L33, L32, L31)
  static const int L3[6][2] = {{0, 0}, {1, 1}, {1, 0}, {2, 2}, {2, 1}, {2, 0}};
  for (int e = 0; e < t.C; ++e) {
    t.ei[e] = E3[e][0];
    t.ej[e] = E3[e][1];
    t.lr[e] = L3[e][0];
    t.lq[e] = L3[e][1];
  }
  double E[NMAX][3][3] = {};
  for (int e = 0; e < t.C; ++e) E[e][t.ei[e]][t.ej[e]] = E[e][t.ej[e]][t.ei[e]] = 1.0;
  for (int e = 0; e < t.C; ++e)
    for (int f = 0; f < t.C; ++f) {
      double M[3][3] = {};
      for (int i = 0; i < c; ++i)
        for (int j = 0; j < c; ++j)
          for (int k = 0; k < c; ++k) M[i][j] += E[e][i][k] * E[f][k][j] + E[f][i][k] * E[e][k][j];
      for (int m = 0; m < t.C; ++m) t.T[e][f][m] = M[t.ei[m]][t.ej[m]];
    }
  // d^2 (L L^T)_{ij} / dL_{r q} dL_{r' q'} = [i = r][j = r'][q = q'] + [j = r][i = r'][q = q']
  for (int e = 0; e < t.C; ++e)
    for (int p = 0; p < t.C; ++p)
      for (int q = 0; q < t.C; ++q)
        t.D2[e][p][q] = ((t.ei[e] == t.lr[p] && t.ej[e] == t.lr[q] && t.lq[p] == t.lq[q]) ? 1.0 : 0.0) +
                        ((t.ej[e] == t.lr[p] && t.ei[e] == t.lr[q] && t.lq[p] == t.lq[q]) ? 1.0 : 0.0);
  return t;
}

}  // namespace
}  // namespace unocg

using namespace unocg;

struct unocg_newton {
  int c = 1, C = 1, n = 0, blocks = 1;
  NewtonTables t{};
  double *ak = nullptr, *bk = nullptr, *rest = nullptr, *w = nullptr, *wt = nullptr, *dg = nullptr,
         *dh = nullptr, *part = nullptr, *part2 = nullptr, *out = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

static int nfail(unocg_newton* o, int code, const std::string& m) {
  if (o) o->err = m;
  return code;
}
#define NCK(...)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                  \
    if (e_ != cudaSuccess)                                                           \
      return nfail(o, e_ == cudaErrorMemoryAllocation ? UNOCG_ERR_OOM : UNOCG_ERR_CUDA, \
                   std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));       \
  } while (0)

extern "C" int unocg_newton_create(unocg_newton** out, int c, int n_modes) {
  if (!out || (c != 1 && c != 2 && c != 3) || n_modes < 0) return UNOCG_ERR_INVALID_ARG;
  unocg_newton* o = new unocg_newton();
  *out = o;
  o->c = c;
  o->C = c * (c + 1) / 2;
  o->n = n_modes;
  o->blocks = std::max(1, (n_modes + kNewtonThreads - 1) / kNewtonThreads);
  o->t = make_tables(c);
  const size_t C = o->C, n = n_modes;
  NCK(cudaStreamCreateWithFlags(&o->stream, cudaStreamNonBlocking));
  NCK(cudaMalloc(&o->ak, std::max<size_t>(1, n * C) * sizeof(double)));
  NCK(cudaMalloc(&o->bk, std::max<size_t>(1, n * C) * sizeof(double)));
  NCK(cudaMalloc(&o->rest, 2 * C * sizeof(double)));
  NCK(cudaMalloc(&o->w, (1 + n) * C * sizeof(double)));
  NCK(cudaMalloc(&o->wt, (1 + n) * C * sizeof(double)));
  NCK(cudaMalloc(&o->dg, std::max<size_t>(1, n * C) * sizeof(double)));
  NCK(cudaMalloc(&o->dh, std::max<size_t>(1, n * C * C) * sizeof(double)));
  NCK(cudaMalloc(&o->part, (size_t)o->blocks * kPartVals * sizeof(double)));
  NCK(cudaMalloc(&o->part2, (size_t)o->blocks * sizeof(double)));
  NCK(cudaMalloc(&o->out, 4 * sizeof(double)));
  return UNOCG_OK;
}

extern "C" void unocg_newton_destroy(unocg_newton* o) {
  if (!o) return;
  if (o->stream) cudaStreamSynchronize(o->stream);
  for (double* p : {o->ak, o->bk, o->rest, o->w, o->wt, o->dg, o->dh, o->part, o->part2, o->out})
    if (p) cudaFree(p);
  if (o->stream) cudaStreamDestroy(o->stream);
  delete o;
}

extern "C" const char* unocg_newton_last_error(const unocg_newton* o) { return o ? o->err.c_str() : "null object"; }

extern "C" int unocg_newton_set_features(unocg_newton* o, const double* ak, const double* bk, const double* a_rest,
                                         const double* b_rest) {
  if (!o || (!ak && o->n) || (!bk && o->n) || !a_rest || !b_rest) return nfail(o, UNOCG_ERR_INVALID_ARG, "null argument");
  const size_t C = o->C, n = o->n;
  for (size_t i = 0; i < n * C; ++i)
    if (!std::isfinite(ak[i]) || !std::isfinite(bk[i])) return nfail(o, UNOCG_ERR_INVALID_ARG, "non-finite feature");
  if (n) {
    NCK(cudaMemcpy(o->ak, ak, n * C * sizeof(double), cudaMemcpyHostToDevice));
    NCK(cudaMemcpy(o->bk, bk, n * C * sizeof(double), cudaMemcpyHostToDevice));
  }
  NCK(cudaMemcpy(o->rest, a_rest, C * sizeof(double), cudaMemcpyHostToDevice));
  NCK(cudaMemcpy(o->rest + C, b_rest, C * sizeof(double), cudaMemcpyHostToDevice));
  return UNOCG_OK;
}

extern "C" int unocg_newton_run(unocg_newton* o, const double* w0, int max_steps, double tol, double* w_out,
                                double* hist, int* n_hist) {
  if (!o || !w0 || !w_out || max_steps < 0 || !(tol >= 0.0)) return nfail(o, UNOCG_ERR_INVALID_ARG, "invalid argument");
  const size_t C = o->C, n = o->n;
  NCK(cudaMemcpy(o->w, w0, (1 + n) * C * sizeof(double), cudaMemcpyHostToDevice));
  NewtonArgs a{};
  a.n = o->n; a.ak = o->ak; a.bk = o->bk; a.a_rest = o->rest; a.b_rest = o->rest + C;
  a.dg = o->dg; a.dh = o->dh; a.part = o->part; a.part2 = o->part2; a.out = o->out; a.blocks = o->blocks;
  double* cur = o->w;
  double* trial = o->wt;
  std::vector<double> h;
  double lam = 0.0;
  auto trial_step = [&](double* res) -> int {
    a.w = cur;
    a.wt = trial;
    a.lambda = lam;
    k_newton_modes<<<o->blocks, kNewtonThreads, 0, o->stream>>>(o->t, a);
    k_newton_bypass<<<1, 32, 0, o->stream>>>(o->t, a);
    k_newton_update<<<o->blocks, kNewtonThreads, 0, o->stream>>>(o->t, a);
    k_newton_loss<<<1, 32, 0, o->stream>>>(o->t, a);
    NCK(cudaGetLastError());
    NCK(cudaMemcpyAsync(res, o->out, 4 * sizeof(double), cudaMemcpyDeviceToHost, o->stream));
    NCK(cudaStreamSynchronize(o->stream));
    return UNOCG_OK;
  };
  double res[4];
  int rc = trial_step(res);
  if (rc) return rc;
  h.push_back(res[0]);
  for (int step = 0; step < max_steps; ++step) {
    bool taken = false;
    while (true) {
      if (res[3] == 0.0 && res[1] <= h.back()) {
        taken = true;
        break;
      }
      lam = std::max(2.0 * lam, 1e-12 * std::max(1.0, res[2]));
      if (lam > 1e30) break;
      rc = trial_step(res);
      if (rc) return rc;
    }
    if (!taken) break;
    std::swap(cur, trial);
    h.push_back(res[1]);
    lam *= 0.1;
    const double last = h[h.size() - 1], prev = h[h.size() - 2];
    if (std::fabs(prev - last) <= tol * std::max(1.0, std::fabs(last))) break;
    rc = trial_step(res);
    if (rc) return rc;
  }
  NCK(cudaMemcpy(w_out, cur, (1 + n) * C * sizeof(double), cudaMemcpyDeviceToHost));
  if (n_hist) {
    const int cap = *n_hist;
    const int cnt = (int)h.size();
    if (hist)
      for (int i = 0; i < cnt && i < cap; ++i) hist[i] = h[i];
    *n_hist = cnt;
  }
  return UNOCG_OK;
}
