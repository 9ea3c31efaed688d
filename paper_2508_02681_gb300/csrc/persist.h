// Arguments and launcher of the persistent UNO-CG kernel (k_persist.cu).
#pragma once
#include "kargs.h"

namespace unocg {

template <typename T, typename QT> struct PersistArgs {
  PlaneFwdArgs<T> pf;   // r, p, hat (= r_hat), transforms
  LineArgs<T, QT> la;   // r_hat, s_hat, Q, tile width
  PlaneInvArgs<T> pi;   // s_hat, d, u
  StencilArgs<T> ka;    // d, p, phase labels, materials
  FoldArgs<T> fo;       // u64, u32, d (mixed precision replacement)
  const double* loads;  // [L][3 or 6]
  CgScal* sc;           // final per-pair state (written by block 0)
  double* part;         // per-task partial sums
  long long off_max, off_line, off_ku;
  unsigned int* bar;    // grid barrier: [0] arrivals, [1] generation
  int* err;             // barrier timeout flag
  int* counters;        // [0] residual checks after CG steps, [1] after replacements
  LoopCtl ctl;
  int B, L, BL;
  int n_line_tasks, n_ku_tasks, n_tr_tasks, n_fold_chunks;
  long long spin_limit; // SM clock cycles a barrier may wait
};

// values of the thermal K d tile (node halo of d + element conductivities), see ku_task.cuh
#ifndef UNOCG_KU_TZ
#define UNOCG_KU_TZ 4
#endif
constexpr size_t kPersistKuTileValues = (UNOCG_KU_TZ + 2) * 10 * 34 + (UNOCG_KU_TZ + 1) * 9 * 33;

// dynamic shared memory of the persistent kernel
inline size_t persist_smem_bytes(const Grid& g, int c, int tb, int cplx_bytes, int BL, int B, int n_phases,
                                 int t_bytes) {
  const int P = (g.n3h % 2 == 0) ? g.n3h + 1 : g.n3h;
  size_t nA = 2 * (size_t)g.n2 * P;
  size_t nL = 2 * (size_t)g.n1 * c * tb;
  if (nL > nA) nA = nL;
  const size_t nK = kPersistKuTileValues / 2 + 1;  // K d halo tile, in complex units
  if (nK > nA) nA = nK;
  size_t bytes = (nA + g.n3 / 2 + g.n2 + g.n3 + g.n1) * cplx_bytes;
  bytes += (size_t)BL * sizeof(CgScal);
  bytes += (size_t)B * 2 * n_phases * (sizeof(double) + t_bytes);
  return bytes;
}

template <typename T, typename QT>
cudaError_t launch_persist(PersistArgs<T, QT>& a, cudaStream_t s, int sm_count);

}  // namespace unocg
