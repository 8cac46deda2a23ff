// Tiled Q1 node operators on the pressure grid: the pressure Laplacian K_p of the
// Cahouet-Chabard Schur term and the 1/eta-weighted pressure mass M_p(1/eta) (Schur
// approximation of the block preconditioner, Sec. 4 variant).
//
// A CTA owns a box of pressure nodes (32 x 8 in 2D, 8 x 8 x 4 in 3D, one thread per node).  It
// stages, with cp.async, the box plus a one-node halo of the input vector (constrained entries
// and nodes outside the mesh zero-filled) and one scalar per touching cell (0 for obstacle
// cells and cells outside the mesh, the cell weight for K_p (1, or abar / alpha_K with alpha
// per cell), pm / eta for the mass).  Each thread then sums
// its <= 2^d cells x 2^d nodes from shared memory and applies the epilogue (apply, residual,
// or fused Chebyshev step).  The cell matrices are
//   K_p:  w_K sum_a kc[a] (K1 in direction a, Pi elsewhere),   K1 = [1 -1; -1 1], Pi = [2 1; 1 2],
//   mass: pm / eta_K  prod_a Pi,                            pm = prod h / 6^d.
#include "gs_kernels.h"

namespace gs {

namespace {
template <int DIM>
struct Q1Box;
template <>
struct Q1Box<2> { static constexpr int B0 = 32, B1 = 8, B2 = 1; };
template <>
struct Q1Box<3> { static constexpr int B0 = 8, B1 = 8, B2 = 4; };

template <typename T>
__device__ __forceinline__ void cp_async_q1(T* smem, const T* gmem, bool load) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(load ? 4 : 0));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(load ? 8 : 0));
}
}  // namespace

template <typename T, int DIM, int OP, int MODE>
__device__ __forceinline__ void q1tile_body(const Q1Args<T>& A, int bid) {
  using Bx = Q1Box<DIM>;
  constexpr int B0 = Bx::B0, B1 = Bx::B1, B2 = Bx::B2;
  constexpr int X0 = B0 + 2, X1 = B1 + 2, X2 = DIM == 3 ? B2 + 2 : 1;  // staged nodes
  constexpr int C0 = B0 + 1, C1 = B1 + 1, C2 = DIM == 3 ? B2 + 1 : 1;  // staged cells
  __shared__ T sx[X0 * X1 * X2];
  __shared__ T sc[C0 * C1 * C2];
  const Geom& g = A.g;
  const int nb0 = (g.npn[0] + B0 - 1) / B0, nb1 = (g.npn[1] + B1 - 1) / B1;
  int blk = bid;
  const int b0 = blk % nb0;
  blk /= nb0;
  const int b1 = blk % nb1;
  const int b2 = blk / nb1;
  const int o0 = b0 * B0, o1 = b1 * B1, o2 = DIM == 3 ? b2 * B2 : 0;
  const int tid = threadIdx.x;

  // stage x (box + halo); constrained entries -> 0
  for (int i = tid; i < X0 * X1 * X2; i += 256) {
    const int i0 = i % X0, i1 = (i / X0) % X1, i2 = i / (X0 * X1);
    const int P = o0 - 1 + i0, Q = o1 - 1 + i1, R = DIM == 3 ? o2 - 1 + i2 : 0;
    bool inr = P >= 0 && P < g.npn[0] && Q >= 0 && Q < g.npn[1];
    if (DIM == 3) inr = inr && R >= 0 && R < g.npn[2];
    const long long q = inr ? P + (long long)g.npn[0] * (Q + (long long)g.npn[1] * R) : 0;
    const bool con = inr && A.cmask && A.cmask[q];
    cp_async_q1(sx + i, A.x + q, inr && !con);
  }
  // one scalar per touching cell
  for (int i = tid; i < C0 * C1 * C2; i += 256) {
    const int i0 = i % C0, i1 = (i / C0) % C1, i2 = i / (C0 * C1);
    const int c0 = o0 - 1 + i0, c1 = o1 - 1 + i1, c2 = DIM == 3 ? o2 - 1 + i2 : 0;
    bool inr = c0 >= 0 && c0 < g.n[0] && c1 >= 0 && c1 < g.n[1];
    if (DIM == 3) inr = inr && c2 >= 0 && c2 < g.n[2];
    T v = T(0);
    if (inr) {
      const long long cell = c0 + (long long)g.n[0] * (c1 + (long long)g.n[1] * c2);
      if (!cell_void(g, cell)) v = OP == Q1_PLAP ? (A.eta ? A.eta[cell] : T(1)) : A.pm / A.eta[cell];
    }
    sc[i] = v;
  }
  // this thread's node and its epilogue operands (issued before the wait)
  const int t0 = tid % B0, t1 = (tid / B0) % B1, t2 = DIM == 3 ? tid / (B0 * B1) : 0;
  const int P = o0 + t0, Q = o1 + t1, R = o2 + t2;
  bool mine = P < g.npn[0] && Q < g.npn[1];
  if (DIM == 3) mine = mine && R < g.npn[2];
  const long long q = mine ? P + (long long)g.npn[0] * (Q + (long long)g.npn[1] * R) : 0;
  T bq = T(0), dq = T(0), diq = T(0);
  bool con = false;
  if (mine) {
    con = A.cmask && A.cmask[q];
    if (MODE != TILE_APPLY) bq = A.b[q];
    if (MODE == TILE_CHEB) {
      diq = A.dinv[q];
      if (A.use_d) dq = A.d[q];
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (!mine) return;

  // sum over the touching cells (cx: 0 = cell below, node is its local 1; 1 = cell above, local 0)
  T acc = T(0);
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const int lc = (t0 + cx) + C0 * ((t1 + cy) + C1 * (DIM == 3 ? t2 + cz : 0));
        const T s = sc[lc];
        const int qa = 1 - cx, qb = 1 - cy, qc = 1 - cz;
        T cellsum = T(0);
#pragma unroll
        for (int rc = 0; rc < (DIM == 3 ? 2 : 1); ++rc)
#pragma unroll
          for (int rb = 0; rb < 2; ++rb)
#pragma unroll
            for (int ra = 0; ra < 2; ++ra) {
              const int si = (t0 + cx + ra) + X0 * ((t1 + cy + rb) + X1 * (DIM == 3 ? t2 + cz + rc : 0));
              const T pa = qa == ra ? T(2) : T(1), pb = qb == rb ? T(2) : T(1);
              T w;
              if (OP == Q1_PLAP) {
                const T ka = qa == ra ? T(1) : T(-1), kb = qb == rb ? T(1) : T(-1);
                if (DIM == 2) {
                  w = A.kc[0] * ka * pb + A.kc[1] * pa * kb;
                } else {
                  const T pc = qc == rc ? T(2) : T(1), kk = qc == rc ? T(1) : T(-1);
                  w = A.kc[0] * ka * pb * pc + A.kc[1] * pa * kb * pc + A.kc[2] * pa * pb * kk;
                }
              } else {
                w = pa * pb;
                if (DIM == 3) w *= (qc == rc ? T(2) : T(1));
              }
              cellsum += w * sx[si];
            }
        acc += s * cellsum;
      }
  const T xq = con ? A.x[q] : sx[(t0 + 1) + X0 * ((t1 + 1) + X1 * (DIM == 3 ? t2 + 1 : 0))];
  const T kq = con ? xq : acc;
  if (MODE == TILE_APPLY) {
    A.y[q] = kq;
  } else if (MODE == TILE_RESID) {
    A.y[q] = bq - kq;
  } else {
    const T r = bq - kq;
    T dn = A.c2 * diq * r;
    if (A.use_d) dn += A.c1 * dq;
    A.d[q] = dn;
    A.xout[q] = xq + dn;
  }
}

template <typename T, int DIM, int OP, int MODE>
struct Q1TileK {
  using Args = Q1Args<T>;
  static constexpr int THREADS = 256, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) { q1tile_body<T, DIM, OP, MODE>(a, blk); }
};

template <typename T, int DIM, int OP>
static cudaError_t q1_dispatch_mode(int mode, const Q1Args<T>& a, cudaStream_t st) {
  using Bx = Q1Box<DIM>;
  const long long nblk = (long long)((a.g.npn[0] + Bx::B0 - 1) / Bx::B0) * ((a.g.npn[1] + Bx::B1 - 1) / Bx::B1) *
                         (DIM == 3 ? (a.g.npn[2] + Bx::B2 - 1) / Bx::B2 : 1);
  if (mode == TILE_APPLY) return submit<Q1TileK<T, DIM, OP, TILE_APPLY>>(a, nblk, 0, st);
  if (mode == TILE_RESID) return submit<Q1TileK<T, DIM, OP, TILE_RESID>>(a, nblk, 0, st);
  return submit<Q1TileK<T, DIM, OP, TILE_CHEB>>(a, nblk, 0, st);
}

template <typename T>
cudaError_t launch_q1tile(int op, int mode, const Q1Args<T>& a, cudaStream_t st) {
  if (a.g.dim == 2)
    return op == Q1_PLAP ? q1_dispatch_mode<T, 2, Q1_PLAP>(mode, a, st) : q1_dispatch_mode<T, 2, Q1_PMASS>(mode, a, st);
  return op == Q1_PLAP ? q1_dispatch_mode<T, 3, Q1_PLAP>(mode, a, st) : q1_dispatch_mode<T, 3, Q1_PMASS>(mode, a, st);
}

template cudaError_t launch_q1tile<float>(int, int, const Q1Args<float>&, cudaStream_t);
template cudaError_t launch_q1tile<double>(int, int, const Q1Args<double>&, cudaStream_t);

}  // namespace gs
