// Set-up kernels for the UNO weights (run once per weight/property change, not per iteration).
//
//  * Reference-medium weights (FANS, Sec. 4.3.4): Q(k) = S_ref(k)^{-1} for k != 0 and
//    Q(0) = 0.  The Fourier symbol of the homogeneous trilinear stencil is a tensor product of
//    the 1D FE stiffness and mass symbols K1(t) = 2 - 2 cos t, M1(t) = (2 + cos t)/3 and
//    G(t) = sin t, with t_a = 2 pi k_a / N_a (times h):
//      thermal  S = kappa sum_a K1(t_a) M1(t_b) M1(t_c)
//      elastic  S_aa = (lambda + 2 mu) K1(t_a) M1 M1 + mu sum_{b != a} K1(t_b) M1(t_a) M1(t_c)
//               S_ab = (lambda + mu) G(t_a) G(t_b) M1(t_c)
//  * Local parametrization psi (Sec. 5.2.2 / App. B.1): Q = L L^T from C = c(c+1)/2 values.
//  * Symmetrization of the self-conjugate half-grid planes (Q(-k) = Q(k) keeps P real).
//  * Safety check of the Remark after Algorithm 2 via Sylvester's criterion on Q(k) - eps I.
//  * Rounding to BF16 / FP32 for the mixed-precision path.
// Entries are stored in the paper's order v1=Q11 v2=Q22 v3=Q12 v4=Q33 v5=Q23 v6=Q13 (App. B.2).
#include "kargs.h"
#include "setup.h"

namespace unocg {

__device__ __forceinline__ void mode_angles(const Grid& g, long long m, double* t) {
  const long long M = (long long)g.n2 * g.n3h;
  int k1 = (int)(m / M);
  int rem = (int)(m % M);
  int k2 = rem / g.n3h, k3 = rem % g.n3h;
  t[0] = 2.0 * k1 / g.n1;  // in units of pi
  t[1] = 2.0 * k2 / g.n2;
  t[2] = 2.0 * k3 / g.n3;
}

__global__ void k_ref_q(RefQArgs a) {
  const long long nh = a.g.nh;
  const int b = blockIdx.y;
  const double* ref = a.ref + 2 * b;  // (kappa or lambda, mu)
  const int NQ = a.c == 1 ? 1 : 6;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < nh; m += (long long)gridDim.x * blockDim.x) {
    double t[3], cs[3], sn[3], K1[3], M1[3];
    mode_angles(a.g, m, t);
    for (int x = 0; x < 3; ++x) {
      sincospi(t[x], &sn[x], &cs[x]);
      K1[x] = 2.0 - 2.0 * cs[x];
      M1[x] = (2.0 + cs[x]) / 3.0;
    }
    double* q = a.Q + ((long long)b * nh + m) * NQ;
    if (m == 0) {
      for (int i = 0; i < NQ; ++i) q[i] = 0.0;
      continue;
    }
    const double h = a.g.h;
    if (a.c == 1) {
      double S = ref[0] * h * (K1[0] * M1[1] * M1[2] + M1[0] * K1[1] * M1[2] + M1[0] * M1[1] * K1[2]);
      q[0] = 1.0 / S;
    } else {
      const double la = ref[0], mu = ref[1];
      double S[3][3];
      for (int x = 0; x < 3; ++x) {
        int y = (x + 1) % 3, z = (x + 2) % 3;
        S[x][x] = h * ((la + 2.0 * mu) * K1[x] * M1[y] * M1[z] +
                       mu * (K1[y] * M1[x] * M1[z] + K1[z] * M1[x] * M1[y]));
        S[x][y] = S[y][x] = h * (la + mu) * sn[x] * sn[y] * M1[z];
      }
      // inverse of the symmetric 3x3 block by its adjugate
      double c00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
      double c01 = S[1][2] * S[2][0] - S[1][0] * S[2][2];
      double c02 = S[1][0] * S[2][1] - S[1][1] * S[2][0];
      double det = S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02;
      double id = 1.0 / det;
      double i00 = c00 * id, i01 = c01 * id, i02 = c02 * id;
      double i11 = (S[0][0] * S[2][2] - S[0][2] * S[2][0]) * id;
      double i12 = (S[0][2] * S[1][0] - S[0][0] * S[1][2]) * id;
      double i22 = (S[0][0] * S[1][1] - S[0][1] * S[1][0]) * id;
      q[0] = i00; q[1] = i11; q[2] = i01; q[3] = i22; q[4] = i12; q[5] = i02;
    }
  }
}

// psi: theta (FP64 or FP32) -> entries
template <typename TI, typename TO>
__global__ void k_psi(const TI* theta, TO* Q, long long nh, int c) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < nh; m += (long long)gridDim.x * blockDim.x) {
    if (c == 1) {
      double t = (double)theta[m];
      Q[m] = (TO)(t * t);
    } else {
      const TI* th = theta + m * 6;
      double t1 = th[0], t2 = th[1], t3 = th[2], t4 = th[3], t5 = th[4], t6 = th[5];
      // L = [[t1, 0, 0], [t3, t2, 0], [t6, t5, t4]],  Q = L L^T (Eq. (local-param-3))
      TO* q = Q + m * 6;
      q[0] = (TO)(t1 * t1);
      q[1] = (TO)(t3 * t3 + t2 * t2);
      q[2] = (TO)(t1 * t3);
      q[3] = (TO)(t6 * t6 + t5 * t5 + t4 * t4);
      q[4] = (TO)(t3 * t6 + t2 * t5);
      q[5] = (TO)(t1 * t6);
    }
  }
}

// chain rule through psi: gtheta = (d entries / d theta)^T gq
__global__ void k_psi_grad(const float* theta, const float* gq, float* gtheta, long long nh, int c) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < nh; m += (long long)gridDim.x * blockDim.x) {
    if (c == 1) {
      gtheta[m] = 2.0f * theta[m] * gq[m];
    } else {
      const float* th = theta + m * 6;
      const float* g = gq + m * 6;
      float t1 = th[0], t2 = th[1], t3 = th[2], t4 = th[3], t5 = th[4], t6 = th[5];
      float* o = gtheta + m * 6;
      o[0] = 2.f * t1 * g[0] + t3 * g[2] + t6 * g[5];
      o[1] = 2.f * t2 * g[1] + t5 * g[4];
      o[2] = 2.f * t3 * g[1] + t1 * g[2] + t6 * g[4];
      o[3] = 2.f * t4 * g[3];
      o[4] = 2.f * t5 * g[3] + t2 * g[4];
      o[5] = 2.f * t6 * g[3] + t3 * g[4] + t1 * g[5];
    }
  }
}

// ---------------------------------------------------------------- bypass + limited mode set
// Eq. (fnocg-parametrization) with the periodic mode set K_M = [-M, M]^2 x [0, M] minus {0}:
// weights w[0] (bypass W = psi(w[0]), every mode) and w[1 + i] (mode i, order: k1 slowest from
// -M, then k2 from -M, then k3 from 0).  Mode index of a half-grid position, or -1.
__device__ __forceinline__ int mode_index(int k1, int k2, int k3, const Grid& g, int M) {
  const int s1 = 2 * k1 <= g.n1 ? k1 : k1 - g.n1;
  const int s2 = 2 * k2 <= g.n2 ? k2 : k2 - g.n2;
  if (s1 < -M || s1 > M || s2 < -M || s2 > M || k3 > M) return -1;
  if (s1 == 0 && s2 == 0 && k3 == 0) return -1;
  const int lin = ((s1 + M) * (2 * M + 1) + (s2 + M)) * (M + 1) + k3;
  const int zero = (M * (2 * M + 1) + M) * (M + 1);
  return lin > zero ? lin - 1 : lin;
}

// unique entries of psi(th) (paper order) added to q
template <typename TI>
__device__ __forceinline__ void psi_add(const TI* th, int c, double* q) {
  if (c == 1) {
    const double t = (double)th[0];
    q[0] += t * t;
    return;
  }
  const double t1 = th[0], t2 = th[1], t3 = th[2], t4 = th[3], t5 = th[4], t6 = th[5];
  q[0] += t1 * t1;
  q[1] += t3 * t3 + t2 * t2;
  q[2] += t1 * t3;
  q[3] += t6 * t6 + t5 * t5 + t4 * t4;
  q[4] += t3 * t6 + t2 * t5;
  q[5] += t1 * t6;
}

// raw entries W + K(k) on the half grid (made even on the self-conjugate planes afterwards)
template <typename TI, typename TO>
__global__ void k_modes_expand(const TI* w, int M, Grid g, int c, TO* Q) {
  const int NQ = c == 1 ? 1 : 6;
  const long long MM = (long long)g.n2 * g.n3h;
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < g.nh; m += (long long)gridDim.x * blockDim.x) {
    const int k1 = (int)(m / MM), rem = (int)(m % MM);
    const int k2 = rem / g.n3h, k3 = rem % g.n3h;
    double q[6] = {0, 0, 0, 0, 0, 0};
    psi_add(w, c, q);
    const int i = mode_index(k1, k2, k3, g, M);
    if (i >= 0) psi_add(w + (long long)(1 + i) * NQ, c, q);
    for (int e = 0; e < NQ; ++e) Q[m * NQ + e] = (TO)q[e];
  }
}

// (d entries / d theta)^T g for one weight vector
__device__ __forceinline__ void psi_grad_one(const float* th, const float* gv, int c, float* o) {
  if (c == 1) {
    o[0] = 2.0f * th[0] * gv[0];
    return;
  }
  const float t1 = th[0], t2 = th[1], t3 = th[2], t4 = th[3], t5 = th[4], t6 = th[5];
  o[0] = 2.f * t1 * gv[0] + t3 * gv[2] + t6 * gv[5];
  o[1] = 2.f * t2 * gv[1] + t5 * gv[4];
  o[2] = 2.f * t3 * gv[1] + t1 * gv[2] + t6 * gv[4];
  o[3] = 2.f * t4 * gv[3];
  o[4] = 2.f * t5 * gv[3] + t2 * gv[4];
  o[5] = 2.f * t6 * gv[3] + t3 * gv[4] + t1 * gv[5];
}

// per-block sums of the entry gradients over all half-grid modes (the bypass acts on each)
constexpr int kModesGradParts = 128;
__global__ void __launch_bounds__(256) k_modes_grad_sum(const float* gq, long long nh, int NQ, double* part) {
  __shared__ double red[6][8];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < nh; m += (long long)gridDim.x * blockDim.x)
    for (int e = 0; e < NQ; ++e) acc[e] += (double)gq[m * NQ + e];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = 0; e < NQ; ++e) {
    double v = acc[e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[e][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[threadIdx.x][k];
    part[blockIdx.x * 6 + threadIdx.x] = v;
  }
}

// gw[0] from the summed gradient, gw[1 + i] from the gradient at mode i
__global__ void k_modes_grad(const float* w, int M, Grid g, int c, const float* gq, const double* part, int nparts,
                             float* gw) {
  const int NQ = c == 1 ? 1 : 6;
  const int n_modes = (2 * M + 1) * (2 * M + 1) * (M + 1) - 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_modes; i += gridDim.x * blockDim.x) {
    int lin = i;
    if (lin >= (M * (2 * M + 1) + M) * (M + 1)) ++lin;  // skip k = 0
    const int k3 = lin % (M + 1), t = lin / (M + 1);
    const int s2 = t % (2 * M + 1) - M, s1 = t / (2 * M + 1) - M;
    const int k1 = s1 < 0 ? s1 + g.n1 : s1, k2 = s2 < 0 ? s2 + g.n2 : s2;
    const long long m = ((long long)k1 * g.n2 + k2) * g.n3h + k3;
    psi_grad_one(w + (long long)(1 + i) * NQ, gq + m * NQ, c, gw + (long long)(1 + i) * NQ);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float sum[6];
    for (int e = 0; e < NQ; ++e) {
      double v = 0.0;
      for (int k = 0; k < nparts; ++k) v += part[k * 6 + e];
      sum[e] = (float)v;
    }
    psi_grad_one(w, sum, c, gw);
  }
}

// Average the entries of (k1, k2) and (-k1, -k2) on the planes k3 = 0 and k3 = N3/2.
template <typename TQ>
__global__ void k_symmetrize(const TQ* in, TQ* out, Grid g, int NQ, int nb) {
  const long long nh = g.nh;
  const long long M = (long long)g.n2 * g.n3h;
  const long long tot = nh * nb;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    long long b = x / nh, m = x % nh;
    int k1 = (int)(m / M);
    int rem = (int)(m % M);
    int k2 = rem / g.n3h, k3 = rem % g.n3h;
    const TQ* src = in + b * nh * NQ;
    bool self_conj = (k3 == 0) || (2 * k3 == g.n3);
    long long mm = ((long long)((g.n1 - k1) % g.n1) * g.n2 + (g.n2 - k2) % g.n2) * g.n3h + k3;
    for (int i = 0; i < NQ; ++i) {
      double v = (double)src[m * NQ + i];
      if (self_conj) v = 0.5 * (v + (double)src[mm * NQ + i]);
      out[(b * nh + m) * NQ + i] = (TQ)v;
    }
  }
}

// Sylvester's criterion on Q(k) - eps I for every k != 0 (entries read as TQ): counts failures
// and records the smallest leading minor ratio seen.
template <typename TQ>
__global__ void k_spd_check(const TQ* Q, long long nh, int nb, int c, double eps, unsigned long long* fails) {
  const int NQ = c == 1 ? 1 : 6;
  const long long tot = nh * nb;
  unsigned long long cnt = 0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    long long m = x % nh;
    if (m == 0) continue;  // the k = 0 mode may share the null space of K (Remark after Alg. 2)
    const TQ* q = Q + x * NQ;
    bool ok;
    if (c == 1) {
      double v = (double)q[0];
      ok = (v - eps > 0.0) && !isnan(v);
    } else {
      double a = (double)q[0] - eps, d = (double)q[1] - eps, f = (double)q[3] - eps;
      double b = (double)q[2], e = (double)q[4], cc = (double)q[5];
      double m1 = a;
      double m2 = a * d - b * b;
      double m3 = a * (d * f - e * e) - b * (b * f - e * cc) + cc * (b * e - d * cc);
      ok = m1 > 0.0 && m2 > 0.0 && m3 > 0.0;
    }
    if (!ok) cnt++;
  }
  if (cnt) atomicAdd(fails, cnt);
}

template <typename TO>
__global__ void k_convert(const double* in, TO* out, long long m);
template <>
__global__ void k_convert<float>(const double* in, float* out, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
template <>
__global__ void k_convert<__nv_bfloat16>(const double* in, __nv_bfloat16* out, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn((float)in[i]);
}

// phase table: (kappa) or (E, nu) -> per-phase (kappa, 0) or (lambda, mu), FP64 and FP32
__global__ void k_material(const double* props, double* m64, float* m32, int count, int physics) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double a, b;
  if (physics == 1) {
    a = props[i];
    b = 0.0;
  } else {
    double E = props[2 * i], nu = props[2 * i + 1];
    a = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    b = E / (2.0 * (1.0 + nu));
  }
  m64[2 * i] = a;
  m64[2 * i + 1] = b;
  m32[2 * i] = (float)a;
  m32[2 * i + 1] = (float)b;
}

// reference medium per instance: arithmetic mean over the phases of kappa or (lambda, mu)
__global__ void k_ref_props(const double* m64, double* ref, int B, int n_phases) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s0 = 0.0, s1 = 0.0;
  for (int p = 0; p < n_phases; ++p) {
    s0 += m64[(b * n_phases + p) * 2];
    s1 += m64[(b * n_phases + p) * 2 + 1];
  }
  ref[2 * b] = s0 / n_phases;
  ref[2 * b + 1] = s1 / n_phases;
}

static int blocks_for(long long m) {
  long long b = (m + 255) / 256;
  if (b > 2048) b = 2048;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_ref_q(const RefQArgs& a, int B, cudaStream_t s) {
  k_ref_q<<<dim3(blocks_for(a.g.nh), B), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_psi64(const double* theta, double* Q, long long nh, int c, cudaStream_t s) {
  k_psi<double, double><<<blocks_for(nh), 256, 0, s>>>(theta, Q, nh, c);
  return cudaGetLastError();
}
cudaError_t launch_psi32(const float* theta, float* Q, long long nh, int c, cudaStream_t s) {
  k_psi<float, float><<<blocks_for(nh), 256, 0, s>>>(theta, Q, nh, c);
  return cudaGetLastError();
}
cudaError_t launch_modes_expand64(const double* w, int M, const Grid& g, int c, double* Q, cudaStream_t s) {
  k_modes_expand<double, double><<<blocks_for(g.nh), 256, 0, s>>>(w, M, g, c, Q);
  return cudaGetLastError();
}
cudaError_t launch_modes_expand32(const float* w, int M, const Grid& g, int c, float* Q, cudaStream_t s) {
  k_modes_expand<float, float><<<blocks_for(g.nh), 256, 0, s>>>(w, M, g, c, Q);
  return cudaGetLastError();
}
size_t modes_grad_scratch_doubles() { return (size_t)kModesGradParts * 6; }
cudaError_t launch_modes_grad(const float* w, int M, const Grid& g, int c, const float* gq, double* scratch, float* gw,
                              cudaStream_t s) {
  k_modes_grad_sum<<<kModesGradParts, 256, 0, s>>>(gq, g.nh, c == 1 ? 1 : 6, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_modes = (2 * M + 1) * (2 * M + 1) * (M + 1) - 1;
  k_modes_grad<<<(n_modes + 255) / 256 + 1, 256, 0, s>>>(w, M, g, c, gq, scratch, kModesGradParts, gw);
  return cudaGetLastError();
}
cudaError_t launch_psi_grad(const float* theta, const float* gq, float* gtheta, long long nh, int c, cudaStream_t s) {
  k_psi_grad<<<blocks_for(nh), 256, 0, s>>>(theta, gq, gtheta, nh, c);
  return cudaGetLastError();
}
cudaError_t launch_symmetrize64(const double* in, double* out, const Grid& g, int NQ, int nb, cudaStream_t s) {
  k_symmetrize<double><<<blocks_for(g.nh * nb), 256, 0, s>>>(in, out, g, NQ, nb);
  return cudaGetLastError();
}
cudaError_t launch_symmetrize32(const float* in, float* out, const Grid& g, int NQ, int nb, cudaStream_t s) {
  k_symmetrize<float><<<blocks_for(g.nh * nb), 256, 0, s>>>(in, out, g, NQ, nb);
  return cudaGetLastError();
}
cudaError_t launch_spd_check64(const double* Q, long long nh, int nb, int c, double eps, unsigned long long* fails, cudaStream_t s) {
  k_spd_check<double><<<blocks_for(nh * nb), 256, 0, s>>>(Q, nh, nb, c, eps, fails);
  return cudaGetLastError();
}
cudaError_t launch_spd_check16(const __nv_bfloat16* Q, long long nh, int nb, int c, double eps, unsigned long long* fails, cudaStream_t s) {
  k_spd_check<__nv_bfloat16><<<blocks_for(nh * nb), 256, 0, s>>>(Q, nh, nb, c, eps, fails);
  return cudaGetLastError();
}
cudaError_t launch_convert32(const double* in, float* out, long long m, cudaStream_t s) {
  k_convert<float><<<blocks_for(m), 256, 0, s>>>(in, out, m);
  return cudaGetLastError();
}
cudaError_t launch_convert16(const double* in, __nv_bfloat16* out, long long m, cudaStream_t s) {
  k_convert<__nv_bfloat16><<<blocks_for(m), 256, 0, s>>>(in, out, m);
  return cudaGetLastError();
}
cudaError_t launch_material(const double* props, double* m64, float* m32, int count, int physics, cudaStream_t s) {
  k_material<<<(count + 127) / 128, 128, 0, s>>>(props, m64, m32, count, physics);
  return cudaGetLastError();
}
cudaError_t launch_ref_props(const double* m64, double* ref, int B, int n_phases, cudaStream_t s) {
  k_ref_props<<<(B + 127) / 128, 128, 0, s>>>(m64, ref, B, n_phases);
  return cudaGetLastError();
}

}  // namespace unocg
