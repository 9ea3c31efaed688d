// Device-side bookkeeping of the CG loop (Algorithm 1 / Algorithm 2): the stopping test and
// iteration count after each residual update, the scalar updates of the search direction and
// step width, and the conditional-graph control of the device-resident loop.
#pragma once
#include "common.cuh"
#include "../../include/unocg.h"

namespace unocg {

struct LoopCtl {
  double tol;                       // relative: stop when ||r||_inf <= tol ||r_0||_inf
  int max_iter;
  int mixed;                        // mixed precision: verify convergence by a true residual
  int replace_every;                // mixed: replacement after this many iterations since the last
  double replace_drop;              // mixed: replacement once ||r|| < replace_drop * ||r|| at the last
  int flexible;                     // Polak-Ribiere coefficient
  cudaGraphConditionalHandle h_while;
  cudaGraphConditionalHandle h_if;
  int set_while, set_if;            // which handles this launch sets
  int* active_flag;                 // optional: 1 while any (instance, load) is still iterating
  int* replace_flag;                // optional: 1 when a residual replacement is due
  int* counters;                    // optional: [0] residual checks after CG steps, [1] after replacements
};

// Residual check after r <- r - alpha p (or after a replacement, `after_replace`).  Runs in the
// last block of the residual-update kernel over all (instance, load) pairs.
__device__ inline void residual_decision(CgScal* sc, int BL, const LoopCtl& ctl, int after_replace) {
  for (int bl = threadIdx.x; bl < BL; bl += blockDim.x) {
    CgScal& s = sc[bl];
    if (s.done) continue;
    // a check after a replacement concerns only the replaced pairs
    if (after_replace && !s.need_replace) continue;
    s.just_replaced = after_replace;
    double rmax = bits_to_double(s.rmax_bits);
    s.rmax_bits = 0ull;
    s.rmax = rmax;
    if (!s.started) {
      s.r0max = rmax;
      s.rrep = rmax;
      s.rep_iter = 0;
      s.started = 1;
    }
    if (after_replace) {
      s.need_replace = 0;
      s.true_res = (s.r0max > 0.0) ? rmax / s.r0max : 0.0;
      s.rrep = rmax;
      s.rep_iter = s.iters;
    }
    if (isnan(rmax) || isinf(rmax)) {
      s.done = 1;
      s.status = UNOCG_ERR_BREAKDOWN;
      continue;
    }
    bool conv = rmax <= ctl.tol * s.r0max;
    // mixed precision: a true residual confirms convergence, replaces r periodically, and
    // replaces it whenever it has fallen by replace_drop since the last replacement
    if (ctl.mixed && !after_replace && s.iters > 0 &&
        (conv || (ctl.replace_every > 0 && s.iters - s.rep_iter >= ctl.replace_every) ||
         rmax <= ctl.replace_drop * s.rrep)) {
      s.need_replace = 1;
      continue;
    }
    if (conv) {
      s.done = 1;
      s.status = UNOCG_OK;
    } else if (s.iters >= ctl.max_iter) {
      s.done = 1;
      s.status = UNOCG_ERR_NOT_CONVERGED;
    } else {
      s.iters += 1;
    }
  }
  __syncthreads();
  int any_active = 0, any_replace = 0;
  for (int bl = threadIdx.x; bl < BL; bl += blockDim.x) {
    any_active |= !sc[bl].done;
    any_replace |= sc[bl].need_replace;
  }
  any_active = __syncthreads_or(any_active);
  any_replace = __syncthreads_or(any_replace);
  if (threadIdx.x == 0) {
    if (ctl.counters) atomicAdd(ctl.counters + (after_replace ? 1 : 0), 1);
    if (ctl.set_while) cudaGraphSetConditional(ctl.h_while, any_active ? 1u : 0u);
    if (ctl.set_if) cudaGraphSetConditional(ctl.h_if, any_replace ? 1u : 0u);
    if (ctl.active_flag) *ctl.active_flag = any_active;
    if (ctl.replace_flag) *ctl.replace_flag = any_replace;
  }
}

// gamma_new = r . s is final: new search-direction coefficient (Algorithm 1, line "d <- s +
// (gamma1/gamma0) d"), or the Polak-Ribiere value in the flexible variant.
__device__ inline void direction_update(CgScal& s, double gamma, double rs_old, int flexible) {
  if (isnan(gamma) || !(gamma > 0.0)) {
    s.done = 1;
    s.status = UNOCG_ERR_BREAKDOWN;
    s.beta = 0.0;
    return;
  }
  double g0 = (s.iters <= 1) ? 1.0 : s.gamma;
  s.gamma_prev = g0;
  s.gamma = gamma;
  if (s.iters <= 1) s.beta = 0.0;
  else s.beta = flexible ? (gamma - rs_old) / g0 : gamma / g0;
}

// d . p is final: step width alpha = gamma / (d . p).
__device__ inline void step_update(CgScal& s, double dp) {
  if (isnan(dp) || !(dp > 0.0)) {
    s.done = 1;
    s.status = UNOCG_ERR_BREAKDOWN;
    s.alpha = 0.0;
    return;
  }
  s.alpha = s.gamma / dp;
}

}  // namespace unocg
