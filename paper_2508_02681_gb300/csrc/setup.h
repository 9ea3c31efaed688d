// Host launchers of the weight / material set-up kernels (k_setup.cu).
#pragma once
#include "common.cuh"

namespace unocg {

struct RefQArgs {
  Grid g;
  int c;
  const double* ref;  // [B][2]: kappa_ref or (lambda_ref, mu_ref)
  double* Q;          // [B][nh][C]
};

cudaError_t launch_ref_q(const RefQArgs& a, int B, cudaStream_t s);
cudaError_t launch_psi64(const double* theta, double* Q, long long nh, int c, cudaStream_t s);
cudaError_t launch_psi32(const float* theta, float* Q, long long nh, int c, cudaStream_t s);
cudaError_t launch_psi_grad(const float* theta, const float* gq, float* gtheta, long long nh, int c, cudaStream_t s);
// bypass + limited mode set (Eq. (fnocg-parametrization)): raw half-grid entries W + K(k) from
// weights [1 + n_modes][C]; gradient of the weights from the entry gradient (even part)
cudaError_t launch_modes_expand64(const double* w, int M, const Grid& g, int c, double* Q, cudaStream_t s);
cudaError_t launch_modes_expand32(const float* w, int M, const Grid& g, int c, float* Q, cudaStream_t s);
size_t modes_grad_scratch_doubles();
cudaError_t launch_modes_grad(const float* w, int M, const Grid& g, int c, const float* gq, double* scratch, float* gw,
                              cudaStream_t s);
cudaError_t launch_symmetrize64(const double* in, double* out, const Grid& g, int NQ, int nb, cudaStream_t s);
cudaError_t launch_symmetrize32(const float* in, float* out, const Grid& g, int NQ, int nb, cudaStream_t s);
cudaError_t launch_spd_check64(const double* Q, long long nh, int nb, int c, double eps, unsigned long long* fails, cudaStream_t s);
cudaError_t launch_spd_check16(const __nv_bfloat16* Q, long long nh, int nb, int c, double eps, unsigned long long* fails, cudaStream_t s);
cudaError_t launch_convert32(const double* in, float* out, long long m, cudaStream_t s);
cudaError_t launch_convert16(const double* in, __nv_bfloat16* out, long long m, cudaStream_t s);
cudaError_t launch_material(const double* props, double* m64, float* m32, int count, int physics, cudaStream_t s);
cudaError_t launch_ref_props(const double* m64, double* ref, int B, int n_phases, cudaStream_t s);

}  // namespace unocg
