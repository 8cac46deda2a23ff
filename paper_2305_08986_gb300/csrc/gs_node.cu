// Node-gather kernels: diagonal of A, multigrid transfers, and the 1/eta-weighted pressure
// mass (Schur approximation).  One thread per output node; every output is written once.
#include "gs_cell.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {
constexpr int TPB = 256;

__device__ __forceinline__ void unflat(long long idx, const int* ext, int dim, int& I, int& J, int& K) {
  if (idx < (1LL << 31)) {  // 32-bit division (a 64-bit one takes several times the instructions)
    const unsigned u = (unsigned)idx, e0 = (unsigned)ext[0], e1 = (unsigned)ext[1];
    const unsigned q = u / e0;
    I = (int)(u - q * e0);
    J = (int)(q % e1);
    K = dim == 3 ? (int)(q / e1) : 0;
    return;
  }
  I = (int)(idx % ext[0]);
  idx /= ext[0];
  J = (int)(idx % ext[1]);
  K = dim == 3 ? (int)(idx / ext[1]) : 0;
}

inline unsigned nblk(long long n) { return (unsigned)((n + TPB - 1) / TPB); }
}  // namespace

// ---- diag(A) (Sec. 4: the Jacobi preconditioner of Cheb(A, diag(A), k_A)) ----------------------
template <typename T, int DIM>
__global__ void k_diagA(const Geom g, const OpCoef<T> c, const T* __restrict__ eta, const T* __restrict__ alpha,
                        T* __restrict__ out, int invert) {
  const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= g.Nv) return;
  int I, J, K;
  unflat(node, g.nv, DIM, I, J, K);
  const bool con = vnode_constrained(g, node, I, J, K);
  T acc[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) acc[a] = T(0);
  if (!con) {
    // cells touching the node along each axis and the node's local index in them
    int cl[3][2], ll[3][2], cnt[3];
    const int idx[3] = {I, J, K};
    for (int ax = 0; ax < DIM; ++ax) {
      const int v = idx[ax];
      cnt[ax] = 0;
      if (v & 1) {
        cl[ax][0] = v >> 1; ll[ax][0] = 1; cnt[ax] = 1;
      } else {
        if ((v >> 1) - 1 >= 0) { cl[ax][cnt[ax]] = (v >> 1) - 1; ll[ax][cnt[ax]] = 2; cnt[ax]++; }
        if ((v >> 1) < g.n[ax]) { cl[ax][cnt[ax]] = v >> 1; ll[ax][cnt[ax]] = 0; cnt[ax]++; }
      }
    }
    const int c2n = DIM == 3 ? cnt[2] : 1;
    for (int k = 0; k < c2n; ++k)
      for (int j = 0; j < cnt[1]; ++j)
        for (int i = 0; i < cnt[0]; ++i) {
          const long long cell = cl[0][i] + (long long)g.n[0] * (cl[1][j] + (long long)g.n[1] * (DIM == 3 ? cl[2][k] : 0));
          if (cell_void(g, cell)) continue;
          const T e = eta[cell] * c.eta_scale;
          OpCoef<T> cK = c;  // the cell's mass coefficient (alpha per cell)
          if (alpha) cK.mm = c.mm * alpha[cell];
#pragma unroll
          for (int a = 0; a < DIM; ++a)
            acc[a] += cell_diagA<T>(DIM, a, ll[0][i], ll[1][j], DIM == 3 ? ll[2][k] : 0, e, cK);
        }
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    T v = con ? T(1) : acc[a];
    out[a * g.Nv + node] = invert ? T(1) / v : v;
  }
}

template <typename T>
cudaError_t launch_diagA(const Geom& g, const OpCoef<T>& c, const T* eta, const T* alpha, T* out, int invert,
                         cudaStream_t st) {
  if (g.dim == 2)
    k_diagA<T, 2><<<nblk(g.Nv), TPB, 0, st>>>(g, c, eta, alpha, out, invert);
  else
    k_diagA<T, 3><<<nblk(g.Nv), TPB, 0, st>>>(g, c, eta, alpha, out, invert);
  return launched(cudaGetLastError());
}

// ---- transfers: P = Q2 interpolation of the coarse field at the fine nodes (Sec. 4, nested
// meshes); R = P^T.  1D weights: fine 2C <- coarse C (1); fine 4c+1 <- (3/8, 3/4, -1/8) on
// coarse (2c, 2c+1, 2c+2); fine 4c+3 <- (-1/8, 3/4, 3/8).  Constrained fine rows and
// constrained coarse columns are removed. -----------------------------------------------------

// weights of coarse node C seen from fine nodes, in five slots at offsets f - 2C = -3, -1, 0, 1, 3:
// even C: (-1/8, 3/8, 1, 3/8, -1/8); odd C: (-, 3/4, 1, 3/4, -); ok marks the slots that exist
// (inside the fine mesh, and the inner three for odd C).  Fixed slots, so the arrays stay in
// registers when the loops over them are unrolled.  The weights and their pairwise products are
// dyadic and exact in FP32, so they are kept in float (FP64 arithmetic is far slower on this GPU);
// the results are the same bits.
__device__ __forceinline__ void restrict_stencil(int C, int nvf, int (&fi)[5], float (&w)[5], bool (&ok)[5]) {
  const bool odd = C & 1;
  const int off[5] = {-3, -1, 0, 1, 3};
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    fi[t] = 2 * C + off[t];
    ok[t] = fi[t] >= 0 && fi[t] < nvf && (!odd || (t >= 1 && t <= 3));
  }
  w[0] = w[4] = -0.125f;
  w[1] = w[3] = odd ? 0.75f : 0.375f;
  w[2] = 1.0f;
}

// Optional start of the coarse level's Chebyshev smoother from zero, fused into the restriction
// that produces its right-hand side: d = x = dinv * rc * inv_theta (the same expression as the
// separate start kernel, so the same bits).  d == NULL: restriction only.
template <typename T>
struct ChebStart {
  const T* dinv;
  T inv_theta;
  T* d;
  T* x;
};

template <typename T>
struct XferArgs {
  Geom gf, gc;
  const T* in;
  T* out;
  ChebStart<T> cs;
};

template <typename T, int DIM>
__device__ __forceinline__ void restrict_body(const Geom& gf, const Geom& gc, const T* __restrict__ rf,
                                              T* __restrict__ rc, const ChebStart<T>& cs, int blk) {
  const long long node = blk * (long long)blockDim.x + threadIdx.x;
  if (node >= gc.Nv) return;
  int I, J, K;
  unflat(node, gc.nv, DIM, I, J, K);
  const bool con = vnode_constrained(gc, node, I, J, K);
  T acc[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) acc[a] = T(0);
  if (!con) {
    int fx[5], fy[5], fz[5];
    float wx[5], wy[5], wz[5];
    bool okx[5], oky[5], okz[5];
    restrict_stencil(I, gf.nv[0], fx, wx, okx);
    restrict_stencil(J, gf.nv[1], fy, wy, oky);
    if (DIM == 3) {
      restrict_stencil(K, gf.nv[2], fz, wz, okz);
    } else {
      fz[0] = 0; wz[0] = 1.0f; okz[0] = true;
    }
    // the existing fine nodes in slot order (z, then y, then x innermost)
#pragma unroll
    for (int k = 0; k < (DIM == 3 ? 5 : 1); ++k) {
      if (!okz[k]) continue;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        if (!oky[j]) continue;
        const T wjk = T(wy[j] * wz[k]);  // exact in float
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          if (!okx[i]) continue;
          const long long fn = fx[i] + (long long)gf.nv[0] * (fy[j] + (long long)gf.nv[1] * fz[k]);
          if (vnode_constrained(gf, fn, fx[i], fy[j], fz[k])) continue;
          const T w = T(wx[i]) * wjk;
#pragma unroll
          for (int a = 0; a < DIM; ++a) acc[a] += w * rf[a * gf.Nv + fn];
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) rc[a * gc.Nv + node] = acc[a];
  if (cs.d) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const long long i = a * gc.Nv + node;
      const T v = cs.dinv[i] * acc[a] * cs.inv_theta;
      cs.d[i] = v;
      cs.x[i] = v;
    }
  }
}

__device__ __forceinline__ int prolong_stencil(int I, int* ci, float* w) {
  if (!(I & 1)) { ci[0] = I >> 1; w[0] = 1.0f; return 1; }
  const int c = I >> 2;  // coarse cell
  if ((I & 3) == 1) {
    ci[0] = 2 * c; ci[1] = 2 * c + 1; ci[2] = 2 * c + 2;
    w[0] = 0.375f; w[1] = 0.75f; w[2] = -0.125f;
  } else {
    ci[0] = 2 * c; ci[1] = 2 * c + 1; ci[2] = 2 * c + 2;
    w[0] = -0.125f; w[1] = 0.75f; w[2] = 0.375f;
  }
  return 3;
}

template <typename T, int DIM>
__device__ __forceinline__ void prolong_add_body(const Geom& gf, const Geom& gc, const T* __restrict__ xc,
                                                 T* __restrict__ xf, int blk) {
  const long long node = blk * (long long)blockDim.x + threadIdx.x;
  if (node >= gf.Nv) return;
  int I, J, K;
  unflat(node, gf.nv, DIM, I, J, K);
  if (vnode_constrained(gf, node, I, J, K)) return;
  int cx[3], cy[3], cz[3];
  float wx[3], wy[3], wz[3];
  const int mx = prolong_stencil(I, cx, wx);
  const int my = prolong_stencil(J, cy, wy);
  int mz = 1;
  cz[0] = 0; wz[0] = 1.0f;
  if (DIM == 3) mz = prolong_stencil(K, cz, wz);
  T acc[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) acc[a] = T(0);
  for (int k = 0; k < mz; ++k)
    for (int j = 0; j < my; ++j) {
      const T wjk = T(wy[j] * wz[k]);  // exact in float
      for (int i = 0; i < mx; ++i) {
        const long long cn = cx[i] + (long long)gc.nv[0] * (cy[j] + (long long)gc.nv[1] * cz[k]);
        if (vnode_constrained(gc, cn, cx[i], cy[j], cz[k])) continue;
        const T w = T(wx[i]) * wjk;
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[a] += w * xc[a * gc.Nv + cn];
      }
    }
#pragma unroll
  for (int a = 0; a < DIM; ++a) xf[a * gf.Nv + node] += acc[a];
}

template <typename T, int DIM>
struct RestrictK {
  using Args = XferArgs<T>;
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    restrict_body<T, DIM>(a.gf, a.gc, a.in, a.out, a.cs, blk);
  }
};
template <typename T, int DIM>
struct ProlongAddK {
  using Args = XferArgs<T>;
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    prolong_add_body<T, DIM>(a.gf, a.gc, a.in, a.out, blk);
  }
};

template <typename T>
cudaError_t launch_restrict(const Geom& gf, const Geom& gc, const T* rf, T* rc, cudaStream_t st, const T* dinv,
                            T inv_theta, T* d, T* x) {
  const XferArgs<T> a{gf, gc, rf, rc, ChebStart<T>{dinv, inv_theta, d, x}};
  if (gf.dim == 2) return submit<RestrictK<T, 2>>(a, nblk(gc.Nv), 0, st);
  return submit<RestrictK<T, 3>>(a, nblk(gc.Nv), 0, st);
}

template <typename T>
cudaError_t launch_prolong_add(const Geom& gf, const Geom& gc, const T* xc, T* xf, cudaStream_t st) {
  const XferArgs<T> a{gf, gc, xc, xf};
  if (gf.dim == 2) return submit<ProlongAddK<T, 2>>(a, nblk(gf.Nv), 0, st);
  return submit<ProlongAddK<T, 3>>(a, nblk(gf.Nv), 0, st);
}

// ---- pressure mass M_p(1/eta): cell matrix (prod h / 6^d) eta_K^{-1} Pi x Pi (x Pi) ---------------
template <typename T, int DIM, int MODE>
__global__ void k_pmass(const PMassArgs<T> A) {
  const Geom& g = A.g;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.Np) return;
  int I, J, K;
  unflat(q, g.npn, DIM, I, J, K);
  const bool con = !A.raw && pnode_constrained(g, q);
  T mx = T(0);
  if (!con) {
    const int idx[3] = {I, J, K};
    int cl[3][2], cnt[3];
    for (int ax = 0; ax < DIM; ++ax) {
      cnt[ax] = 0;
      if (idx[ax] - 1 >= 0) cl[ax][cnt[ax]++] = idx[ax] - 1;
      if (idx[ax] < g.n[ax]) cl[ax][cnt[ax]++] = idx[ax];
    }
    const int c2n = DIM == 3 ? cnt[2] : 1;
    for (int k = 0; k < c2n; ++k)
      for (int j = 0; j < cnt[1]; ++j)
        for (int i = 0; i < cnt[0]; ++i) {
          const int c0 = cl[0][i], c1 = cl[1][j], c2 = DIM == 3 ? cl[2][k] : 0;
          const long long cell = c0 + (long long)g.n[0] * (c1 + (long long)g.n[1] * c2);
          if (cell_void(g, cell)) continue;
          const int la = I - c0, lb = J - c1, lc = DIM == 3 ? K - c2 : 0;  // local node of q
          T s = T(0);
          for (int rc = 0; rc < (DIM == 3 ? 2 : 1); ++rc)
            for (int rb = 0; rb < 2; ++rb)
              for (int ra = 0; ra < 2; ++ra) {
                const long long r = (c0 + ra) + (long long)g.npn[0] * ((c1 + rb) + (long long)g.npn[1] * (c2 + rc));
                if (!A.raw && pnode_constrained(g, r)) continue;
                int w = (la == ra ? 2 : 1) * (lb == rb ? 2 : 1);
                if (DIM == 3) w *= (lc == rc ? 2 : 1);
                s += T(w) * A.x[r];
              }
          mx += A.unit ? s : s / A.eta[cell];
        }
    mx *= A.c.pm;
  }
  const T mq = con ? A.x[q] : mx;
  if (MODE == TILE_APPLY) {
    A.y[q] = mq;
  } else {
    const T r = A.b[q] - mq;
    T dn = A.c2 * A.dinv[q] * r;
    if (A.use_d) dn += A.c1 * A.d[q];
    A.d[q] = dn;
    A.xout[q] = A.x[q] + dn;
  }
}

template <typename T, int DIM>
__global__ void k_pdiag(const Geom g, const OpCoef<T> c, const T* __restrict__ eta, T* __restrict__ dinv) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.Np) return;
  int I, J, K;
  unflat(q, g.npn, DIM, I, J, K);
  if (pnode_constrained(g, q)) { dinv[q] = T(1); return; }
  const int idx[3] = {I, J, K};
  int cl[3][2], cnt[3];
  for (int ax = 0; ax < DIM; ++ax) {
    cnt[ax] = 0;
    if (idx[ax] - 1 >= 0) cl[ax][cnt[ax]++] = idx[ax] - 1;
    if (idx[ax] < g.n[ax]) cl[ax][cnt[ax]++] = idx[ax];
  }
  T s = T(0);
  const int c2n = DIM == 3 ? cnt[2] : 1;
  for (int k = 0; k < c2n; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i) {
        const long long cell = cl[0][i] + (long long)g.n[0] * (cl[1][j] + (long long)g.n[1] * (DIM == 3 ? cl[2][k] : 0));
        if (cell_void(g, cell)) continue;
        s += T(1) / eta[cell];
      }
  dinv[q] = T(1) / (s * c.pm * T(DIM == 3 ? 8 : 4));
}

template <typename T>
cudaError_t launch_pmass(int mode, PMassArgs<T> a, cudaStream_t st) {
  if (!a.raw && !a.unit) {
    Q1Args<T> q{};
    q.g = a.g;
    q.pm = a.c.pm;
    q.eta = a.eta;
    q.cmask = a.g.pmask;
    q.x = a.x; q.y = a.y; q.b = a.b; q.d = a.d; q.dinv = a.dinv; q.xout = a.xout;
    q.c1 = a.c1; q.c2 = a.c2; q.use_d = a.use_d;
    return launch_q1tile<T>(Q1_PMASS, mode, q, st);
  }
  const unsigned nb = nblk(a.g.Np);
  if (a.g.dim == 2) {
    if (mode == TILE_APPLY) k_pmass<T, 2, TILE_APPLY><<<nb, TPB, 0, st>>>(a);
    else k_pmass<T, 2, TILE_CHEB><<<nb, TPB, 0, st>>>(a);
  } else {
    if (mode == TILE_APPLY) k_pmass<T, 3, TILE_APPLY><<<nb, TPB, 0, st>>>(a);
    else k_pmass<T, 3, TILE_CHEB><<<nb, TPB, 0, st>>>(a);
  }
  return launched(cudaGetLastError());
}

template <typename T>
cudaError_t launch_pdiag(const Geom& g, const OpCoef<T>& c, const T* eta, T* dinv, cudaStream_t st) {
  if (g.dim == 2)
    k_pdiag<T, 2><<<nblk(g.Np), TPB, 0, st>>>(g, c, eta, dinv);
  else
    k_pdiag<T, 3><<<nblk(g.Np), TPB, 0, st>>>(g, c, eta, dinv);
  return launched(cudaGetLastError());
}

#define INST(T)                                                                                    \
  template cudaError_t launch_diagA<T>(const Geom&, const OpCoef<T>&, const T*, const T*, T*, int, cudaStream_t); \
  template cudaError_t launch_restrict<T>(const Geom&, const Geom&, const T*, T*, cudaStream_t, const T*, T, T*, T*); \
  template cudaError_t launch_prolong_add<T>(const Geom&, const Geom&, const T*, T*, cudaStream_t); \
  template cudaError_t launch_pmass<T>(int, PMassArgs<T>, cudaStream_t);                           \
  template cudaError_t launch_pdiag<T>(const Geom&, const OpCoef<T>&, const T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace gs

// ---- pressure Laplacian K_p (Cahouet-Chabard term of the Schur approximation) ----------------------
namespace gs {

template <typename T, int DIM>
__global__ void k_plap_diag(const Geom g, const T k0, const T k1, const T k2, const T* __restrict__ w,
                            const uint8_t* __restrict__ cmask, T* __restrict__ dinv) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.Np) return;
  if (cmask[q]) { dinv[q] = T(1); return; }
  int I, J, K;
  unflat(q, g.npn, DIM, I, J, K);
  const int idx[3] = {I, J, K};
  int cl[3][2], cnt[3];
  for (int ax = 0; ax < DIM; ++ax) {
    cnt[ax] = 0;
    if (idx[ax] - 1 >= 0) cl[ax][cnt[ax]++] = idx[ax] - 1;
    if (idx[ax] < g.n[ax]) cl[ax][cnt[ax]++] = idx[ax];
  }
  T wsum = T(0);  // sum of the active touching cells' weights
  const int c2n = DIM == 3 ? cnt[2] : 1;
  for (int k = 0; k < c2n; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i) {
        const long long cell = cl[0][i] + (long long)g.n[0] * (cl[1][j] + (long long)g.n[1] * (DIM == 3 ? cl[2][k] : 0));
        if (!cell_void(g, cell)) wsum += w ? w[cell] : T(1);
      }
  const T per_cell = DIM == 2 ? T(2) * (k0 + k1) : T(4) * (k0 + k1 + k2);
  dinv[q] = T(1) / (wsum * per_cell);
}

template <typename T>
struct PXferArgs {
  Geom gf, gc;
  const uint8_t* mf;
  const uint8_t* mc;
  const T* in;
  T* out;
  ChebStart<T> cs;
};

template <typename T, int DIM>
__device__ __forceinline__ void p_restrict_body(const Geom& gf, const Geom& gc, const uint8_t* __restrict__ mf,
                                                const uint8_t* __restrict__ mc, const T* __restrict__ rf,
                                                T* __restrict__ rc, const ChebStart<T>& cs, int blk) {
  const long long q = blk * (long long)blockDim.x + threadIdx.x;
  if (q >= gc.Np) return;
  if (mc[q]) {
    rc[q] = T(0);
    if (cs.d) cs.d[q] = cs.x[q] = cs.dinv[q] * T(0) * cs.inv_theta;
    return;
  }
  int I, J, K;
  unflat(q, gc.npn, DIM, I, J, K);
  const int idx[3] = {I, J, K};
  // fine nodes 2C - 1, 2C, 2C + 1 per axis with weights 1/2, 1, 1/2; ok marks those inside the
  // fine mesh (fixed slots: the arrays stay in registers)
  int f[3][3];
  T w[3][3];
  bool ok[3][3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax >= DIM) {
      f[ax][0] = 0; w[ax][0] = T(1); ok[ax][0] = true; ok[ax][1] = ok[ax][2] = false;
      continue;
    }
    const int C = idx[ax];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      f[ax][t] = 2 * C - 1 + t;
      ok[ax][t] = f[ax][t] >= 0 && f[ax][t] < gf.npn[ax];
    }
    w[ax][0] = w[ax][2] = T(0.5);
    w[ax][1] = T(1);
  }
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!ok[2][k]) continue;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (!ok[1][j]) continue;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (!ok[0][i]) continue;
        const long long fq = f[0][i] + (long long)gf.npn[0] * (f[1][j] + (long long)gf.npn[1] * f[2][k]);
        if (mf[fq]) continue;
        acc += w[0][i] * w[1][j] * w[2][k] * rf[fq];
      }
    }
  }
  rc[q] = acc;
  if (cs.d) {  // start of the coarse level's Chebyshev smoother (ChebStart)
    const T v = cs.dinv[q] * acc * cs.inv_theta;
    cs.d[q] = v;
    cs.x[q] = v;
  }
}

template <typename T, int DIM>
__device__ __forceinline__ void p_prolong_add_body(const Geom& gf, const Geom& gc, const uint8_t* __restrict__ mf,
                                                   const uint8_t* __restrict__ mc, const T* __restrict__ xc,
                                                   T* __restrict__ xf, int blk) {
  const long long q = blk * (long long)blockDim.x + threadIdx.x;
  if (q >= gf.Np) return;
  if (mf[q]) return;
  int I, J, K;
  unflat(q, gf.npn, DIM, I, J, K);
  const int idx[3] = {I, J, K};
  // even fine coordinate v: coarse v / 2 with weight 1; odd: coarse (v - 1) / 2 and (v + 1) / 2 with
  // weights 1/2 (fixed slots: the arrays stay in registers)
  int cidx[3][2];
  T w[3][2];
  bool ok[3][2];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax >= DIM) {
      cidx[ax][0] = 0; w[ax][0] = T(1); ok[ax][0] = true; ok[ax][1] = false;
      continue;
    }
    const int v = idx[ax];
    const bool odd = v & 1;
    cidx[ax][0] = v >> 1;
    cidx[ax][1] = (v >> 1) + 1;
    w[ax][0] = odd ? T(0.5) : T(1);
    w[ax][1] = T(0.5);
    ok[ax][0] = true;
    ok[ax][1] = odd;
  }
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (!ok[2][k]) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (!ok[1][j]) continue;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (!ok[0][i]) continue;
        const long long cq = cidx[0][i] + (long long)gc.npn[0] * (cidx[1][j] + (long long)gc.npn[1] * cidx[2][k]);
        if (mc[cq]) continue;
        acc += w[0][i] * w[1][j] * w[2][k] * xc[cq];
      }
    }
  }
  xf[q] += acc;
}

template <typename T, int DIM>
struct PRestrictK {
  using Args = PXferArgs<T>;
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    p_restrict_body<T, DIM>(a.gf, a.gc, a.mf, a.mc, a.in, a.out, a.cs, blk);
  }
};
template <typename T, int DIM>
struct PProlongAddK {
  using Args = PXferArgs<T>;
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    p_prolong_add_body<T, DIM>(a.gf, a.gc, a.mf, a.mc, a.in, a.out, blk);
  }
};

template <typename T>
struct MaskCopyK {  // may run in place
  struct Args { const T* in; const uint8_t* mask; T* out; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)nblk * blockDim.x)
      a.out[i] = a.mask[i] ? T(0) : a.in[i];
  }
};
template <typename T>
struct CcCombineK {
  struct Args { const T* m; const T* v; const uint8_t* mask; T alpha; T* z; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < a.n; i += (long long)nblk * blockDim.x)
      a.z[i] = -(a.m[i] + a.alpha * (a.mask[i] ? T(0) : a.v[i]));
  }
};

template <typename T>
cudaError_t launch_plap(int mode, PLapArgs<T> a, cudaStream_t st) {
  Q1Args<T> q{};
  q.g = a.g;
  for (int i = 0; i < 3; ++i) q.kc[i] = a.kc[i];
  q.cmask = a.cmask;
  q.eta = a.w;  // Q1_PLAP: the per-cell weight
  q.x = a.x; q.y = a.y; q.b = a.b; q.d = a.d; q.dinv = a.dinv; q.xout = a.xout;
  q.c1 = a.c1; q.c2 = a.c2; q.use_d = a.use_d;
  return launch_q1tile<T>(Q1_PLAP, mode, q, st);
}

template <typename T>
cudaError_t launch_plap_diag(const Geom& g, const T* kc, const T* w, const uint8_t* cmask, T* dinv, cudaStream_t st) {
  if (g.dim == 2)
    k_plap_diag<T, 2><<<nblk(g.Np), TPB, 0, st>>>(g, kc[0], kc[1], kc[2], w, cmask, dinv);
  else
    k_plap_diag<T, 3><<<nblk(g.Np), TPB, 0, st>>>(g, kc[0], kc[1], kc[2], w, cmask, dinv);
  return launched(cudaGetLastError());
}
template <typename T>
cudaError_t launch_p_restrict(const Geom& gf, const Geom& gc, const uint8_t* mf, const uint8_t* mc, const T* rf, T* rc,
                              cudaStream_t st, const T* dinv, T inv_theta, T* d, T* x) {
  const PXferArgs<T> a{gf, gc, mf, mc, rf, rc, ChebStart<T>{dinv, inv_theta, d, x}};
  if (gf.dim == 2) return submit<PRestrictK<T, 2>>(a, nblk(gc.Np), 0, st);
  return submit<PRestrictK<T, 3>>(a, nblk(gc.Np), 0, st);
}
template <typename T>
cudaError_t launch_p_prolong_add(const Geom& gf, const Geom& gc, const uint8_t* mf, const uint8_t* mc, const T* xc,
                                 T* xf, cudaStream_t st) {
  const PXferArgs<T> a{gf, gc, mf, mc, xc, xf, ChebStart<T>{nullptr, T(0), nullptr, nullptr}};
  if (gf.dim == 2) return submit<PProlongAddK<T, 2>>(a, nblk(gf.Np), 0, st);
  return submit<PProlongAddK<T, 3>>(a, nblk(gf.Np), 0, st);
}
template <typename T>
cudaError_t launch_mask_copy(const T* in, const uint8_t* mask, T* out, long long n, cudaStream_t st) {
  return submit<MaskCopyK<T>>({in, mask, out, n}, nblk(n), 0, st);
}
template <typename T>
cudaError_t launch_cc_combine(const T* m, const T* v, const uint8_t* mask, T alpha, T* z, long long n, cudaStream_t st) {
  return submit<CcCombineK<T>>({m, v, mask, alpha, z, n}, nblk(n), 0, st);
}

#define INSTP(T)                                                                                          \
  template cudaError_t launch_plap<T>(int, PLapArgs<T>, cudaStream_t);                                    \
  template cudaError_t launch_plap_diag<T>(const Geom&, const T*, const T*, const uint8_t*, T*, cudaStream_t); \
  template cudaError_t launch_p_restrict<T>(const Geom&, const Geom&, const uint8_t*, const uint8_t*,      \
                                            const T*, T*, cudaStream_t, const T*, T, T*, T*);             \
  template cudaError_t launch_p_prolong_add<T>(const Geom&, const Geom&, const uint8_t*, const uint8_t*,   \
                                               const T*, T*, cudaStream_t);                               \
  template cudaError_t launch_mask_copy<T>(const T*, const uint8_t*, T*, long long, cudaStream_t);        \
  template cudaError_t launch_cc_combine<T>(const T*, const T*, const uint8_t*, T, T*, long long, cudaStream_t);
INSTP(float)
INSTP(double)
#undef INSTP

// ---- corrector stage: diagonal of rho (C + S) (setup, FP64) ----------------------------------
// diag_i += rho sum_q W_q phi_i(q) (v° . grad phi_i)(q) + rho r_K sum_q W_q (v° . grad phi_i)(q)^2
// summed over the active cells around free velocity node i (the same value for both components).
__global__ void k_diag_conv(Geom g, const double* __restrict__ vc, const double* __restrict__ rk, double rho,
                            double* __restrict__ diag) {
  const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= g.Nv) return;
  const int I = (int)(node % g.nv[0]), J = (int)(node / g.nv[0]);
  if (g.vmask ? g.vmask[node] != 0 : face_constrained(g, I, J, 0)) return;
  const double hx = g.h[0], hy = g.h[1];
  double acc = 0.0;
  for (int cb = 0; cb < 2; ++cb)
    for (int ca = 0; ca < 2; ++ca) {
      // cells containing the node: column (I - 1) / 2 or I / 2 (both for an even, interior I)
      const int c0 = (I % 2 == 0) ? (ca == 0 ? I / 2 : I / 2 - 1) : (ca == 0 ? I / 2 : -1);
      const int c1 = (J % 2 == 0) ? (cb == 0 ? J / 2 : J / 2 - 1) : (cb == 0 ? J / 2 : -1);
      if (c0 < 0 || c0 >= g.n[0] || c1 < 0 || c1 >= g.n[1]) continue;
      const long long cell = c0 + (long long)g.n[0] * c1;
      if (cell_void(g, cell)) continue;
      const int la = I - 2 * c0, lb = J - 2 * c1;
      double vx[9], vy[9];
      for (int q = 0; q < 9; ++q) vx[q] = vy[q] = 0.0;
      for (int jb = 0; jb < 3; ++jb)
        for (int ja = 0; ja < 3; ++ja) {
          const long long nd = (2 * c0 + ja) + (long long)g.nv[0] * (2 * c1 + jb);
          const double v0 = vc[nd], v1 = vc[g.Nv + nd];
          for (int qb = 0; qb < 3; ++qb)
            for (int qa = 0; qa < 3; ++qa) {
              const double ph = GaussQ2::phi(qa, ja) * GaussQ2::phi(qb, jb);
              vx[qa + 3 * qb] += ph * v0;
              vy[qa + 3 * qb] += ph * v1;
            }
        }
      const double r = rk[cell];
      for (int qb = 0; qb < 3; ++qb)
        for (int qa = 0; qa < 3; ++qa) {
          const int q = qa + 3 * qb;
          const double W = GaussQ2::w(qa) * GaussQ2::w(qb) * hx * hy;
          const double phi = GaussQ2::phi(qa, la) * GaussQ2::phi(qb, lb);
          const double adv = vx[q] * GaussQ2::dq(qa, la) * GaussQ2::phi(qb, lb) / hx +
                             vy[q] * GaussQ2::phi(qa, la) * GaussQ2::dq(qb, lb) / hy;
          acc += W * (phi * adv + r * adv * adv);
        }
    }
  diag[node] += rho * acc;
  diag[g.Nv + node] += rho * acc;
}
// 3D: the same sum over the (up to 8) active cells around the node, v° interpolated to the 27 Gauss
// points of each cell by sum factorisation (one axis at a time).
__global__ void k_diag_conv3(Geom g, const double* __restrict__ vc, const double* __restrict__ rk, double rho,
                             double* __restrict__ diag) {
  const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= g.Nv) return;
  const int I = (int)(node % g.nv[0]);
  const int J = (int)((node / g.nv[0]) % g.nv[1]);
  const int K = (int)(node / ((long long)g.nv[0] * g.nv[1]));
  if (g.vmask ? g.vmask[node] != 0 : face_constrained(g, I, J, K)) return;
  const int X[3] = {I, J, K};
  const double jac = g.h[0] * g.h[1] * g.h[2];
  double acc = 0.0;
  for (int cs = 0; cs < 8; ++cs) {
    int cl[3], ll[3];
    bool ok = true;
    for (int ax = 0; ax < 3; ++ax) {
      const int side = (cs >> ax) & 1;  // 0: the cell at or above the node, 1: the cell below an even node
      const int c = (X[ax] % 2 == 0) ? (side == 0 ? X[ax] / 2 : X[ax] / 2 - 1) : (side == 0 ? X[ax] / 2 : -1);
      if (c < 0 || c >= g.n[ax]) ok = false;
      cl[ax] = c;
      ll[ax] = X[ax] - 2 * c;
    }
    if (!ok) continue;
    const long long cell = cl[0] + (long long)g.n[0] * (cl[1] + (long long)g.n[1] * cl[2]);
    if (cell_void(g, cell)) continue;
    double v[3][27];
    for (int b = 0; b < 3; ++b) {
      double a0[27], a1[27];
      for (int jc = 0; jc < 3; ++jc)  // nodal values of component b
        for (int jb = 0; jb < 3; ++jb)
          for (int ja = 0; ja < 3; ++ja)
            a0[ja + 3 * jb + 9 * jc] =
                vc[b * g.Nv + (2 * cl[0] + ja) + (long long)g.nv[0] * ((2 * cl[1] + jb) + (long long)g.nv[1] * (2 * cl[2] + jc))];
      for (int jc = 0; jc < 3; ++jc)  // along x
        for (int jb = 0; jb < 3; ++jb)
          for (int qa = 0; qa < 3; ++qa) {
            double t = 0.0;
            for (int ja = 0; ja < 3; ++ja) t += GaussQ2::phi(qa, ja) * a0[ja + 3 * jb + 9 * jc];
            a1[qa + 3 * jb + 9 * jc] = t;
          }
      for (int jc = 0; jc < 3; ++jc)  // along y
        for (int qb = 0; qb < 3; ++qb)
          for (int qa = 0; qa < 3; ++qa) {
            double t = 0.0;
            for (int jb = 0; jb < 3; ++jb) t += GaussQ2::phi(qb, jb) * a1[qa + 3 * jb + 9 * jc];
            a0[qa + 3 * qb + 9 * jc] = t;
          }
      for (int qc = 0; qc < 3; ++qc)  // along z
        for (int qb = 0; qb < 3; ++qb)
          for (int qa = 0; qa < 3; ++qa) {
            double t = 0.0;
            for (int jc = 0; jc < 3; ++jc) t += GaussQ2::phi(qc, jc) * a0[qa + 3 * qb + 9 * jc];
            v[b][qa + 3 * qb + 9 * qc] = t;
          }
    }
    const double r = rk[cell];
    for (int qc = 0; qc < 3; ++qc)
      for (int qb = 0; qb < 3; ++qb)
        for (int qa = 0; qa < 3; ++qa) {
          const int q = qa + 3 * qb + 9 * qc;
          const double W = GaussQ2::w(qa) * GaussQ2::w(qb) * GaussQ2::w(qc) * jac;
          const double pa = GaussQ2::phi(qa, ll[0]), pb = GaussQ2::phi(qb, ll[1]), pc = GaussQ2::phi(qc, ll[2]);
          const double phi = pa * pb * pc;
          const double adv = v[0][q] * GaussQ2::dq(qa, ll[0]) * pb * pc / g.h[0] +
                             v[1][q] * pa * GaussQ2::dq(qb, ll[1]) * pc / g.h[1] +
                             v[2][q] * pa * pb * GaussQ2::dq(qc, ll[2]) / g.h[2];
          acc += W * (phi * adv + r * adv * adv);
        }
  }
  for (int a = 0; a < 3; ++a) diag[a * g.Nv + node] += rho * acc;
}
cudaError_t launch_diag_conv(const Geom& g, const double* vc, const double* rk, double rho, double* diag,
                             cudaStream_t st) {
  if (g.dim == 3) {
    k_diag_conv3<<<nblk(g.Nv), TPB, 0, st>>>(g, vc, rk, rho, diag);
    return launched(cudaGetLastError(), 1);
  }
  k_diag_conv<<<nblk(g.Nv), TPB, 0, st>>>(g, vc, rk, rho, diag);
  return launched(cudaGetLastError(), 1);
}

template <typename T>
__global__ void k_reciprocal(const double* __restrict__ in, T* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)(1.0 / in[i]);
}
template <typename T>
cudaError_t launch_reciprocal(const double* in, T* out, long long n, cudaStream_t st) {
  k_reciprocal<T><<<nblk(n), TPB, 0, st>>>(in, out, n);
  return launched(cudaGetLastError(), 1);
}
template cudaError_t launch_reciprocal<float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_reciprocal<double>(const double*, double*, long long, cudaStream_t);

}  // namespace gs
