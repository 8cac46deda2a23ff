// Kernels of the saddle-point multigrid with the block smoother K_j (Sec. 4, Eq. "smoother"):
// the Schur diagonal diag(B diag(A)^{-1} B^T) that preconditions ChebMINRES, the two inner
// products of one MINRES step and the smoother's update of the level iterate.
//
// One MINRES step from zero for S w = v with preconditioner P = D_S^{-1} (one Chebyshev step of
// Cheb(S, D_S, 1); its 1/theta scaling cancels in MINRES) is w = a z with z = P v and
// a = (z . S z) / ((S z) . P (S z)): the minimiser of the P-norm of the residual over span{z}.
#include "gs_kernels.h"

namespace gs {

namespace {
constexpr int TPB = 256;
inline unsigned nblk(long long n) {
  long long b = (n + TPB - 1) / TPB;
  return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// fixed-tree block sum, valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// 1D Q1 x Q2 integrals on the reference interval, times 6: N[a][b] = 6 int psi_a phi_b,
// G[a][b] = 6 int psi_a phi_b' (psi: Q1 basis on {0, 1}; phi: Q2 basis on {0, 1/2, 1})
__device__ __forceinline__ int n1d(int a, int b) { return a == 0 ? (b == 0 ? 1 : (b == 1 ? 2 : 0)) : (b == 0 ? 0 : (b == 1 ? 2 : 1)); }
__device__ __forceinline__ int g1d(int a, int b) { return a == 0 ? (b == 0 ? -5 : (b == 1 ? 4 : 1)) : (b == 0 ? -1 : (b == 1 ? -4 : 5)); }
}  // namespace

#define GS_FOR(i, n) \
  for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)nblk * blockDim.x)

// D_S[q] = sum over free velocity entries (j, a) of B[q, (j, a)]^2 / A[(j, a), (j, a)], with the
// assembled entry B[q, (j, a)] = sum over the active cells K holding q and j of
// -bd[a] G(q_a, j_a) prod_{b != a} N(q_b, j_b) (local 1D indices of q and j in K).  One thread per
// pressure node; out = 1 / D_S (invert, 0 where D_S = 0, e.g. constrained nodes) or D_S.
template <typename T>
struct SchurDiagK {
  struct Args { Geom g; OpCoef<double> c; const T* dinv; T* out; int invert; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& A, int blk, int nblk) {
    const Geom& g = A.g;
    const int dim = g.dim;
    GS_FOR(q, g.Np) {
      const int Q[3] = {(int)(q % g.npn[0]), (int)((q / g.npn[0]) % g.npn[1]),
                        dim == 3 ? (int)(q / ((long long)g.npn[0] * g.npn[1])) : 0};
      double ds = 0.0;
      if (!pnode_constrained(g, q)) {
        int lo[3], hi[3];
        for (int b = 0; b < 3; ++b) {
          if (b >= dim) { lo[b] = hi[b] = 0; continue; }
          lo[b] = max(2 * Q[b] - 2, 0);
          hi[b] = min(2 * Q[b] + 2, g.nv[b] - 1);
        }
        for (int K = lo[2]; K <= hi[2]; ++K)
          for (int J = lo[1]; J <= hi[1]; ++J)
            for (int I = lo[0]; I <= hi[0]; ++I) {
              const int V[3] = {I, J, K};
              const long long node = I + (long long)g.nv[0] * (J + (long long)g.nv[1] * K);
              if (vnode_constrained(g, node, I, J, K)) continue;
              for (int a = 0; a < dim; ++a) {
                double bij = 0.0;
                // cells c with c_b in {Q_b - 1, Q_b} holding node V (local index V_b - 2 c_b in 0..2)
                for (int dc = 0; dc < (dim == 3 ? 2 : 1); ++dc)
                  for (int db = 0; db < 2; ++db)
                    for (int da = 0; da < 2; ++da) {
                      const int cc[3] = {Q[0] - 1 + da, Q[1] - 1 + db, dim == 3 ? Q[2] - 1 + dc : 0};
                      bool ok = true;
                      double prod = 1.0;
                      for (int b = 0; b < dim && ok; ++b) {
                        const int lv = V[b] - 2 * cc[b];
                        if (cc[b] < 0 || cc[b] >= g.n[b] || lv < 0 || lv > 2) { ok = false; break; }
                        const int lq = Q[b] - cc[b];
                        prod *= (b == a) ? (double)g1d(lq, lv) : (double)n1d(lq, lv);
                      }
                      if (!ok) continue;
                      const long long cell = cc[0] + (long long)g.n[0] * (cc[1] + (long long)g.n[1] * cc[2]);
                      if (cell_void(g, cell)) continue;
                      bij += prod;
                    }
                bij *= -A.c.bd[a];
                ds += bij * bij * (double)A.dinv[a * g.Nv + node];
              }
            }
      }
      A.out[q] = A.invert ? (T)(ds > 0.0 ? 1.0 / ds : 0.0) : (T)ds;
    }
  }
};

// part[0 * G + blk] = partial sum of z . q, part[1 * G + blk] = of q . (dsinv q)  (G = nblk blocks)
template <typename T>
struct SchurDotsK {
  struct Args { const T* z; const T* q; const T* dsinv; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sh[TPB / 32];
    double s0 = 0.0, s1 = 0.0;
    GS_FOR(i, a.n) {
      const double qi = (double)a.q[i];
      s0 += (double)a.z[i] * qi;
      s1 += qi * (double)a.dsinv[i] * qi;
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
      a.part[blk] = s0;
      a.part[nblk + blk] = s1;
    }
  }
};

// Smoother update with a = s[0] / s[1] (0 when s[1] = 0):
//   x_u = x_u + wt + a y   (velocity, n_u entries),   x_p = x_p - a z   (pressure, n_p entries);
// zero: the iterate starts from zero (x is not read).
template <typename T>
struct MonoUpdateK {
  struct Args { T* xu; T* xp; const T* wt; const T* y; const T* z; const double* s; long long nu, np; int zero; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sal;  // the step length once per block (FP64 division)
    if (threadIdx.x == 0) {
      const double s1 = a.s[1];
      sal = s1 > 0.0 ? a.s[0] / s1 : 0.0;
    }
    __syncthreads();
    const T al = (T)sal;
    GS_FOR(i, a.nu + a.np) {
      if (i < a.nu) {
        const T v = a.wt[i] + al * a.y[i];
        a.xu[i] = a.zero ? v : a.xu[i] + v;
      } else {
        const long long k = i - a.nu;
        const T v = -al * a.z[k];
        a.xp[k] = a.zero ? v : a.xp[k] + v;
      }
    }
  }
};

// out = a * b (elementwise)
template <typename T>
struct MulK {
  struct Args { const T* a; const T* b; T* out; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    GS_FOR(i, a.n) a.out[i] = a.a[i] * a.b[i];
  }
};

// y += x
template <typename T>
struct AddK {
  struct Args { const T* x; T* y; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    GS_FOR(i, a.n) a.y[i] += a.x[i];
  }
};

template <typename T>
cudaError_t launch_schur_diag(const Geom& g, const OpCoef<double>& c, const T* dinv, T* out, int invert,
                              cudaStream_t st) {
  return submit<SchurDiagK<T>>({g, c, dinv, out, invert}, nblk(g.Np), 0, st);
}
template <typename T>
cudaError_t launch_schur_dots(const T* z, const T* q, const T* dsinv, long long n, double* part, int G, double* out,
                              cudaStream_t st) {
  cudaError_t e = submit<SchurDotsK<T>>({z, q, dsinv, n, part}, G, 0, st);
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(part, 2, G, out, st);
}
template <typename T>
cudaError_t launch_mono_update(T* xu, T* xp, const T* wt, const T* y, const T* z, const double* s, long long nu,
                               long long np, int zero, cudaStream_t st) {
  return submit<MonoUpdateK<T>>({xu, xp, wt, y, z, s, nu, np, zero}, nblk(nu + np), 0, st);
}
template <typename T>
cudaError_t launch_mul(const T* a, const T* b, T* out, long long n, cudaStream_t st) {
  return submit<MulK<T>>({a, b, out, n}, nblk(n), 0, st);
}

template <typename T>
cudaError_t launch_add(const T* x, T* y, long long n, cudaStream_t st) {
  return submit<AddK<T>>({x, y, n}, nblk(n), 0, st);
}

// ---- ChebBiCGStab(1, 1): one preconditioned BiCGStab step for S w = q from zero (van der Vorst;
// shadow residual = q, preconditioner P = D_S^{-1}), the Schur solve of the saddle-point smoother
// when the velocity block is not symmetric (corrector stage):
//   z1 = P q, v = S z1, alpha = (q . q) / (q . v), s = q - alpha v, z2 = P s, t = S z2,
//   omega = (t . s) / (t . t), w = alpha z1 + omega z2;
// alpha = 0 and omega = 0 when q . v = 0 (the iteration stops at w = 0), omega = 0 when t = 0.

// part[blk] = sum a . b, part[nblk + blk] = sum c . d over the block's entries (FP64 sums)
template <typename T>
struct Dot2K {
  struct Args { const T* a; const T* b; const T* c; const T* d; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sh[TPB / 32];
    double s0 = 0.0, s1 = 0.0;
    GS_FOR(i, a.n) {
      s0 += (double)a.a[i] * (double)a.b[i];
      s1 += (double)a.c[i] * (double)a.d[i];
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
      a.part[blk] = s0;
      a.part[nblk + blk] = s1;
    }
  }
};

// s = q - alpha v (in place of v), z2 = P s, with alpha = s1[0] / s1[1] (0 when s1[1] = 0)
template <typename T>
struct BicgSK {
  struct Args { const T* q; T* v; const T* dsinv; T* z2; const double* s1; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sal;
    if (threadIdx.x == 0) sal = a.s1[1] != 0.0 ? a.s1[0] / a.s1[1] : 0.0;
    __syncthreads();
    const T al = (T)sal;
    GS_FOR(i, a.n) {
      const T sv = a.q[i] - al * a.v[i];
      a.v[i] = sv;
      a.z2[i] = a.dsinv[i] * sv;
    }
  }
};

// x_u (+)= wt + alpha y1 + omega y2,  x_p (+)= -(alpha z1 + omega z2)   (the step works on the
// negated right-hand side q = r_p - B wt; zero: the iterate starts from zero)
template <typename T>
struct MonoUpdate2K {
  struct Args {
    T* xu; T* xp; const T* wt; const T* y1; const T* y2; const T* z1; const T* z2; const double* s1;
    const double* s2; long long nu, np; int zero;
  };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sal, som;
    if (threadIdx.x == 0) {
      const bool ok = a.s1[1] != 0.0;
      sal = ok ? a.s1[0] / a.s1[1] : 0.0;
      som = (ok && a.s2[1] > 0.0) ? a.s2[0] / a.s2[1] : 0.0;
    }
    __syncthreads();
    const T al = (T)sal, om = (T)som;
    GS_FOR(i, a.nu + a.np) {
      if (i < a.nu) {
        const T v = a.wt[i] + al * a.y1[i] + om * a.y2[i];
        a.xu[i] = a.zero ? v : a.xu[i] + v;
      } else {
        const long long k = i - a.nu;
        const T v = -(al * a.z1[k] + om * a.z2[k]);
        a.xp[k] = a.zero ? v : a.xp[k] + v;
      }
    }
  }
};

template <typename T>
cudaError_t launch_dot2(const T* a, const T* b, const T* c, const T* d, long long n, double* part, int G,
                        double* out, cudaStream_t st) {
  cudaError_t e = submit<Dot2K<T>>({a, b, c, d, n, part}, G, 0, st);
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(part, 2, G, out, st);
}
template <typename T>
cudaError_t launch_bicg_s(const T* q, T* v, const T* dsinv, T* z2, const double* s1, long long n, cudaStream_t st) {
  return submit<BicgSK<T>>({q, v, dsinv, z2, s1, n}, nblk(n), 0, st);
}
template <typename T>
cudaError_t launch_mono_update2(T* xu, T* xp, const T* wt, const T* y1, const T* y2, const T* z1, const T* z2,
                                const double* s1, const double* s2, long long nu, long long np, int zero,
                                cudaStream_t st) {
  return submit<MonoUpdate2K<T>>({xu, xp, wt, y1, y2, z1, z2, s1, s2, nu, np, zero}, nblk(nu + np), 0, st);
}
#define INSTB(T)                                                                                                   \
  template cudaError_t launch_dot2<T>(const T*, const T*, const T*, const T*, long long, double*, int, double*,    \
                                      cudaStream_t);                                                               \
  template cudaError_t launch_bicg_s<T>(const T*, T*, const T*, T*, const double*, long long, cudaStream_t);       \
  template cudaError_t launch_mono_update2<T>(T*, T*, const T*, const T*, const T*, const T*, const T*,            \
                                              const double*, const double*, long long, long long, int, cudaStream_t);
INSTB(float)
INSTB(double)
#undef INSTB

#define INSTM(T)                                                                                                  \
  template cudaError_t launch_schur_diag<T>(const Geom&, const OpCoef<double>&, const T*, T*, int, cudaStream_t); \
  template cudaError_t launch_schur_dots<T>(const T*, const T*, const T*, long long, double*, int, double*,       \
                                            cudaStream_t);                                                        \
  template cudaError_t launch_mono_update<T>(T*, T*, const T*, const T*, const T*, const double*, long long,       \
                                             long long, int, cudaStream_t);                                       \
  template cudaError_t launch_mul<T>(const T*, const T*, T*, long long, cudaStream_t);                           \
  template cudaError_t launch_add<T>(const T*, T*, long long, cudaStream_t);
INSTM(float)
INSTM(double)
#undef INSTM

}  // namespace gs
