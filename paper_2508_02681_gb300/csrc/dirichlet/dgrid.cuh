// Dirichlet boundary conditions on the voxel grid (Sec. 4.1, Sec. 6): N1 x N2 x N3 voxels,
// (N1+1)(N2+1)(N3+1) nodes, the fluctuation fixed to zero on every boundary node, so only the
// M_a = N_a - 1 interior nodes per axis carry unknowns.
//
// Device fields live on the N1 x N2 x N3 node grid of the periodic discretization: node i_a = 0
// stands for both boundary faces of axis a (node N_a wraps to it) and holds zero in every
// solution, direction and residual field, interior node j_a (0 <= j_a < M_a) is node j_a + 1.
// With zeros there, the periodic stencil at an interior node is exactly the Dirichlet one (its
// eight voxels j + 1 - o never wrap, and its neighbours on the faces read zero), so the K d,
// right-hand-side, diagonal and voxel-average functions of the periodic path serve unchanged;
// only the rows of the boundary nodes are ignored.  The sine transform reads and writes the
// interior nodes only.
#pragma once
#include "../common.cuh"

namespace unocg {

// Boundary conditions per axis (mixed BC, Sec. 6.2): an axis with bc[a] = 1 has Dirichlet faces
// (node 0 held at zero, N_a - 1 free nodes, offset o_a = 1); bc[a] = 0 is periodic (all N_a
// nodes free, o_a = 0).  The same embedding serves every combination.
struct DGrid {
  int n1, n2, n3;   // voxels per axis (= nodes per axis of the embedding grid)
  int m1, m2, m3;   // free nodes per axis (N - 1 Dirichlet, N periodic)
  int bc[3];        // 1: Dirichlet faces along the axis, 0: periodic
  int o[3];         // free index j is node j + o (o = bc)
  long long ne;     // voxels = nodes of the embedding grid (field stride per component)
  long long nf;     // free nodes
  Grid pg;          // the embedding grid as a periodic grid (stencil functions)
};

// embedding-grid node of free node index f (j3 fastest)
__device__ __forceinline__ long long dnode_of_free(const DGrid& g, long long f, int& i1, int& i2, int& i3) {
  const int j3 = (int)(f % g.m3);
  const long long r = f / g.m3;
  i2 = (int)(r % g.m2) + g.o[1];
  i1 = (int)(r / g.m2) + g.o[0];
  i3 = j3 + g.o[2];
  return ((long long)i1 * g.n2 + i2) * g.n3 + i3;
}

__device__ __forceinline__ bool dfree_node(const DGrid& g, int i1, int i2, int i3) {
  return !(g.bc[0] && i1 == 0) && !(g.bc[1] && i2 == 0) && !(g.bc[2] && i3 == 0);
}

__device__ __forceinline__ bool dinterior(const DGrid& g, long long node) {
  const int i3 = (int)(node % g.n3);
  const long long r = node / g.n3;
  const int i2 = (int)(r % g.n2), i1 = (int)(r / g.n2);
  return dfree_node(g, i1, i2, i3);
}

}  // namespace unocg
