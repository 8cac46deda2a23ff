// Common device/host definitions of the GB300 generalized Stokes library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

// Geometry of one mesh level as the kernels see it.
struct Geom {
  int dim;
  int n[3];        // cells per axis
  int nv[3];       // velocity nodes per axis = 2n+1
  int npn[3];      // pressure nodes per axis = n+1
  long long Nv, Np, Nc;
  unsigned faces;  // Dirichlet faces (bit 2a: lower face of axis a, bit 2a+1: upper face)
  const uint8_t* vmask;  // per velocity node, 1 = constrained; NULL -> faces only
  const uint8_t* pmask;  // per pressure node, 1 = constrained; NULL -> none
  const uint8_t* cvoid;  // per cell, 1 = obstacle; NULL -> none
  const uint16_t* ccmask;  // 2D meshes with obstacles: per cell, bit la + 3 lb = local node constrained,
                           // bit 15 = obstacle cell; NULL -> derive from the faces
  double h[3];
};

// Level-constant coefficients of the cell operators (all in the arithmetic type T).
// Integer 1D matrices (see gs_cell.cuh) carry the exact rational entries; these scalars carry
// the mesh widths and the common denominators.
template <typename T>
struct OpCoef {
  // viscous + mass block (eta-scaled terms are multiplied by eta_K per cell)
  T mm;            // 2D: alpha hx hy / 900      3D: alpha hx hy hz / 27000
  T km[3];         // 2D: [0] hy/(90 hx) [1] hx/(90 hy)   3D: [a] = prod_{b!=a} h_b / (2700 h_a)
  T ex[3];         // 2D: 1/36 (all)      3D: h_a / 1080
  T eta_scale;     // multiplies eta_K (1 normally, 0 for a pure mass operator)
  // divergence block
  T bd[3];         // 2D: [0] hy/36 [1] hx/36      3D: [a] = prod_{b!=a} h_b / 216
  // pressure mass (Schur): prod h / 6^d, multiplied by 1/eta_K per cell
  T pm;
};

__host__ __device__ inline bool face_constrained(const Geom& g, int I, int J, int K) {
  unsigned f = g.faces;
  if ((f & 1u) && I == 0) return true;
  if ((f & 2u) && I == g.nv[0] - 1) return true;
  if ((f & 4u) && J == 0) return true;
  if ((f & 8u) && J == g.nv[1] - 1) return true;
  if (g.dim == 3) {
    if ((f & 16u) && K == 0) return true;
    if ((f & 32u) && K == g.nv[2] - 1) return true;
  }
  return false;
}

__device__ __forceinline__ bool vnode_constrained(const Geom& g, long long node, int I, int J, int K) {
  if (g.vmask) return g.vmask[node] != 0;
  return face_constrained(g, I, J, K);
}

__device__ __forceinline__ bool pnode_constrained(const Geom& g, long long q) {
  return g.pmask ? (g.pmask[q] != 0) : false;
}

__device__ __forceinline__ bool cell_void(const Geom& g, long long c) {
  return g.cvoid ? (g.cvoid[c] != 0) : false;
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

}  // namespace gs
