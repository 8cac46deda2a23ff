// Rigid-body deflation of stiff inclusions (finest velocity level): projections Z^T r, the small
// dense solve y = E^-1 c, and the update x += Z y.  Not part of the paper's method: stiff
// inclusions below the coarse-cell size have near-rigid motions that no coarse level of the
// V-cycle represents (Sec. 4 resolves the interface on the coarsest mesh instead).
//
// Z holds, per inclusion k, its rigid motions on the velocity nodes of its cells (constrained
// nodes excluded from the node list): the d translations e_a, then the rotations about the
// inclusion's node centroid c_k, 2D (-(y - c_y), x - c_x), 3D e_ax x (x - c_k) for ax = x, y, z.
// Vectors over the modes have nt = 3 (2D) or 6 (3D) entries per inclusion.  Inclusions share no
// node (they are node-connected components), so the update is free of write conflicts.
#include "gs_kernels.h"

namespace gs {

namespace {
constexpr int DTPB = 256;

// mode values of node (dx, dy, dz) relative to the centroid, for a vector v (component a)
__device__ __forceinline__ void rigid_dots(int dim, double dx, double dy, double dz, const double* v, double* s) {
  if (dim == 2) {
    s[0] += v[0];
    s[1] += v[1];
    s[2] += -dy * v[0] + dx * v[1];
  } else {
    s[0] += v[0];
    s[1] += v[1];
    s[2] += v[2];
    s[3] += -dz * v[1] + dy * v[2];  // e_x x d = (0, -dz, dy)
    s[4] += dz * v[0] - dx * v[2];   // e_y x d = (dz, 0, -dx)
    s[5] += -dy * v[0] + dx * v[1];  // e_z x d = (-dy, dx, 0)
  }
}

__device__ __forceinline__ void node_offset(const DeflArgs& a, int n, double& dx, double& dy, double& dz,
                                            const double* cen) {
  const int I = n % a.g.nv[0];
  const int J = (n / a.g.nv[0]) % a.g.nv[1];
  const int K = a.g.dim == 3 ? n / (a.g.nv[0] * a.g.nv[1]) : 0;
  dx = I * (0.5 * a.g.h[0]) - cen[0];
  dy = J * (0.5 * a.g.h[1]) - cen[1];
  dz = a.g.dim == 3 ? K * (0.5 * a.g.h[2]) - cen[2] : 0.0;
}
}  // namespace

// c[k * nt + t] = (Z^T r) for mode t of inclusion k (one block per inclusion, fixed reduction order)
template <typename T>
struct DeflDotsK {
  struct Args { DeflArgs d; const T* r; double* c; };
  static constexpr int THREADS = DTPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& A, int blk, int) {
    __shared__ double sh[6][DTPB / 32];
    const DeflArgs& a = A.d;
    const int k = blk;
    const int nt = a.g.dim == 2 ? 3 : 6;
    const double* cen = a.cen + 3 * k;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int i = a.off[k] + threadIdx.x; i < a.off[k + 1]; i += DTPB) {
      const int n = a.nodes[i];
      double dx, dy, dz;
      node_offset(a, n, dx, dy, dz, cen);
      double v[3] = {0, 0, 0};
      for (int c = 0; c < a.g.dim; ++c) v[c] = (double)A.r[c * a.g.Nv + n];
      rigid_dots(a.g.dim, dx, dy, dz, v, s);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      double x = s[t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) sh[t][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < nt) {
      double x = 0.0;
      for (int q = 0; q < DTPB / 32; ++q) x += sh[threadIdx.x][q];
      A.c[k * nt + threadIdx.x] = x;
    }
  }
};

// y = Einv c (dense M x M, one warp per row)
struct DeflGemvK {
  struct Args { const double* Einv; int M; const double* c; double* y; };
  static constexpr int THREADS = DTPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    const int row = (blk * DTPB + (int)threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= a.M) return;
    double s = 0.0;
    for (int j = lane; j < a.M; j += 32) s += a.Einv[(long long)row * a.M + j] * a.c[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) a.y[row] = s;
  }
};

// x += Z y on the inclusions' nodes (one block per inclusion)
template <typename T>
struct DeflAddK {
  struct Args { DeflArgs d; const double* y; T* x; };
  static constexpr int THREADS = DTPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& A, int blk, int) {
    const DeflArgs& a = A.d;
    const int k = blk;
    const int nt = a.g.dim == 2 ? 3 : 6;
    const double* cen = a.cen + 3 * k;
    const double* y = A.y + k * nt;
    for (int i = a.off[k] + threadIdx.x; i < a.off[k + 1]; i += DTPB) {
      const int n = a.nodes[i];
      double dx, dy, dz;
      node_offset(a, n, dx, dy, dz, cen);
      double u[3];
      if (a.g.dim == 2) {
        u[0] = y[0] - dy * y[2];
        u[1] = y[1] + dx * y[2];
        u[2] = 0.0;
      } else {
        // translations + sum_ax y_ax (e_ax x d)
        u[0] = y[0] + dz * y[4] - dy * y[5];
        u[1] = y[1] - dz * y[3] + dx * y[5];
        u[2] = y[2] + dy * y[3] - dx * y[4];
      }
      for (int c = 0; c < a.g.dim; ++c) A.x[c * a.g.Nv + n] += (T)u[c];
    }
  }
};

template <typename T>
cudaError_t launch_defl_dots(const DeflArgs& d, const T* r, double* c, cudaStream_t st) {
  return submit<DeflDotsK<T>>({d, r, c}, d.ninc, 0, st);
}
cudaError_t launch_defl_gemv(const double* Einv, int M, const double* c, double* y, cudaStream_t st) {
  return submit<DeflGemvK>({Einv, M, c, y}, ((long long)M * 32 + DTPB - 1) / DTPB, 0, st);
}
template <typename T>
cudaError_t launch_defl_add(const DeflArgs& d, const double* y, T* x, cudaStream_t st) {
  return submit<DeflAddK<T>>({d, y, x}, d.ninc, 0, st);
}

template cudaError_t launch_defl_dots<float>(const DeflArgs&, const float*, double*, cudaStream_t);
template cudaError_t launch_defl_dots<double>(const DeflArgs&, const double*, double*, cudaStream_t);
template cudaError_t launch_defl_add<float>(const DeflArgs&, const double*, float*, cudaStream_t);
template cudaError_t launch_defl_add<double>(const DeflArgs&, const double*, double*, cudaStream_t);

}  // namespace gs
