// Vector kernels of the Krylov / multigrid path: casts, Chebyshev start, Lanczos helpers,
// deterministic multi-dot reductions (FGMRES Gram-Schmidt, Sec. 5), multi-axpy updates,
// pressure-mean projection, lifting, and the dense FP64 coarse solve.
#include <atomic>

#include "gs_kernels.h"

namespace gs {

static std::atomic<long long> g_launches{0};
Recorder*& current_recorder() {
  static thread_local Recorder* r = nullptr;
  return r;
}
cudaError_t launched(cudaError_t e, int kernels) {
  if (e == cudaSuccess) g_launches.fetch_add(kernels, std::memory_order_relaxed);
  return e;
}
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

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

// deterministic block sum (fixed tree); result valid in thread 0
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
}  // namespace

// grid-stride loop of one instance: element indices of block blk out of nblk
#define GS_FOR(i, n) \
  for (long long i = blk * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)nblk * blockDim.x)

template <typename T>
struct ChebInit0K {
  struct Args { const T* b; const T* dinv; T inv_theta; T* d; T* x; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    GS_FOR(i, a.n) {
      const T v = a.dinv[i] * a.b[i] * a.inv_theta;
      a.d[i] = v;
      a.x[i] = v;
    }
  }
};
template <typename T>
cudaError_t launch_cheb_init0(const T* b, const T* dinv, T inv_theta, T* d, T* x, long long n, cudaStream_t st) {
  return submit<ChebInit0K<T>>({b, dinv, inv_theta, d, x, n}, nblk(n), 0, st);
}

template <typename TI, typename TO>
struct CastK {  // may run in place
  struct Args { const TI* in; TO* out; long long n; TO scale; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    GS_FOR(i, a.n) a.out[i] = a.scale * (TO)a.in[i];
  }
};
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* in, TO* out, long long n, TO scale, cudaStream_t st) {
  return submit<CastK<TI, TO>>({in, out, n, scale}, nblk(n), 0, st);
}

template <typename T>
__global__ void k_zero_constrained_u(const Geom g, T* v) {
  const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node >= g.Nv) return;
  const int I = (int)(node % g.nv[0]);
  const int J = (int)((node / g.nv[0]) % g.nv[1]);
  const int K = g.dim == 3 ? (int)(node / ((long long)g.nv[0] * g.nv[1])) : 0;
  if (vnode_constrained(g, node, I, J, K))
    for (int a = 0; a < g.dim; ++a) v[a * g.Nv + node] = T(0);
}
template <typename T>
cudaError_t launch_zero_constrained_u(const Geom& g, T* v, cudaStream_t st) {
  k_zero_constrained_u<T><<<nblk(g.Nv), TPB, 0, st>>>(g, v);
  return launched(cudaGetLastError());
}

// Lanczos on S = D^{-1/2} A D^{-1/2}:  t = sqrt(dinv) v ;  w = sqrt(dinv) (A t) - beta v_prev
template <typename T>
__global__ void k_lanczos_pre(const T* __restrict__ dinv, const T* __restrict__ v, T* __restrict__ t, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    t[i] = sqrt(dinv[i]) * v[i];
}
template <typename T>
__global__ void k_lanczos_post(const T* __restrict__ dinv, const T* y, const T* __restrict__ vprev,
                               T beta_prev, T* w, long long n) {  // y and w may alias
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w[i] = sqrt(dinv[i]) * y[i] - beta_prev * vprev[i];
}
template <typename T>
cudaError_t launch_lanczos_pre(const T* dinv, const T* v, T* t, long long n, cudaStream_t st) {
  k_lanczos_pre<T><<<nblk(n), TPB, 0, st>>>(dinv, v, t, n);
  return launched(cudaGetLastError());
}
template <typename T>
cudaError_t launch_lanczos_post(const T* dinv, const T* y, const T* vprev, T beta_prev, T* w, long long n,
                                cudaStream_t st) {
  k_lanczos_post<T><<<nblk(n), TPB, 0, st>>>(dinv, y, vprev, beta_prev, w, n);
  return launched(cudaGetLastError());
}

// ---- multi-dot: part[i*G + blk] = sum over the block's elements of V[i][e] w[e] ------------------
// Tall-skinny V^T w: every thread keeps KB accumulators, so w is read once per KB basis vectors
// and the block reduces KB sums at once (one barrier pair per KB vectors).  Deterministic: the
// element-to-thread assignment and the reduction tree are fixed by the launch shape.
template <typename T, int KB>
struct DotsK {
  struct Args { const T* V; long long ldv; int k; const T* w; long long n; double* part; int self_dot; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sh[KB + 1][32];
    const T* __restrict__ V = a.V;
    const T* __restrict__ w = a.w;
    const long long ldv = a.ldv, n = a.n;
    const int k = a.k;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i0 = 0; i0 < k || (i0 == 0 && a.self_dot); i0 += KB) {
      const int kb = max(0, min(KB, k - i0));
      const bool self = a.self_dot && i0 == 0;  // w . w rides along with the first block of vectors
      double acc[KB], accw = 0.0;
#pragma unroll
      for (int i = 0; i < KB; ++i) acc[i] = 0.0;
      GS_FOR(e, n) {
        const double we = (double)w[e];
        if (self) accw += we * we;
#pragma unroll
        for (int i = 0; i < KB; ++i)
          if (i < kb) acc[i] += (double)V[(i0 + i) * ldv + e] * we;
      }
#pragma unroll
      for (int i = 0; i <= KB; ++i) {
        double v = i < KB ? acc[i] : accw;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i][wid] = v;
      }
      __syncthreads();
      if (threadIdx.x < kb) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += sh[threadIdx.x][q];
        a.part[(long long)(i0 + threadIdx.x) * nblk + blk] = t;
      }
      if (self && threadIdx.x == 32) {  // the row after the k dot products
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += sh[KB][q];
        a.part[(long long)k * nblk + blk] = t;
      }
      __syncthreads();
    }
  }
};
template <typename T>
cudaError_t launch_dots_partial(const T* V, long long ldv, int k, const T* w, long long n, double* part, int G,
                                cudaStream_t st) {
  if (k <= 1) return submit<DotsK<T, 1>>({V, ldv, k, w, n, part, 0}, G, 0, st);
  return submit<DotsK<T, 8>>({V, ldv, k, w, n, part, 0}, G, 0, st);
}
cudaError_t launch_dots_norm_partial(const double* V, long long ldv, int k, const double* w, long long n, double* part,
                                     int G, cudaStream_t st) {
  return submit<DotsK<double, 8>>({V, ldv, k, w, n, part, 1}, G, 0, st);
}

// w <- w + sign * sum_i coef[i] V[i], and per-block partial sums of the new |w|^2
struct MultiAxpyNormK {
  struct Args { const double* V; long long ldv; int k; const double* coef; double sign; double* w; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    extern __shared__ double cs[];
    __shared__ double sh[32];
    const double* __restrict__ V = a.V;
    double* __restrict__ w = a.w;
    const int k = a.k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = a.sign * a.coef[i];
    __syncthreads();
    double s = 0.0;
    GS_FOR(e, a.n) {
      double acc = w[e];
      for (int i = 0; i < k; ++i) acc += cs[i] * V[i * a.ldv + e];
      w[e] = acc;
      s += acc * acc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
      a.part[blk] = t;
    }
  }
};
cudaError_t launch_multi_axpy_norm(const double* V, long long ldv, int k, const double* coef, double sign, double* w,
                                   long long n, double* part, int G, cudaStream_t st) {
  return submit<MultiAxpyNormK>({V, ldv, k, coef, sign, w, n, part}, G, sizeof(double) * (k > 0 ? k : 1), st);
}

// ---- Krylov basis in double-float form (GB300: FP64 is 1/74 of the FP32 rate) ----------------------
// A basis vector is stored as float2 (hi, lo) with value hi + lo (48 significant bits, same 8 bytes
// as a double).  Products hi/lo x hi/lo are formed exactly with an FMA for hi*hi plus the two
// cross terms, and sums are carried as unevaluated float pairs (TwoSum + renormalisation), so the
// Gram-Schmidt dot products and updates run on the FP32 pipes at ~48-bit accuracy.
__device__ __forceinline__ float2 df_split(double a) {
  const float h = (float)a;
  return make_float2(h, (float)(a - (double)h));
}
__device__ __forceinline__ double df_join(float2 v) { return (double)v.x + (double)v.y; }
// acc += a * b
__device__ __forceinline__ void df_fma(float2& acc, float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = acc.x + p;
  const float bb = s - acc.x;
  const float err = (acc.x - (s - bb)) + (p - bb);
  const float lo = acc.y + err + e;
  const float hi = s + lo;
  acc.y = lo - (hi - s);
  acc.x = hi;
}

template <int KB>
struct DotsDfK {
  struct Args { const float2* V; long long ldv; int k; const double* w; long long n; double* part; int self_dot; };
  static constexpr int THREADS = TPB, MINB = 3;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sh[KB + 1][32];
    const float2* __restrict__ V = a.V;
    const double* __restrict__ w = a.w;
    const long long ldv = a.ldv, n = a.n;
    const int k = a.k;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long stride = (long long)nblk * blockDim.x;
    for (int i0 = 0; i0 < k; i0 += KB) {
      const int kb = min(KB, k - i0);
      const bool self = a.self_dot && i0 == 0;
      float2 acc[KB];
      double accw = 0.0;
#pragma unroll
      for (int i = 0; i < KB; ++i) acc[i] = make_float2(0.f, 0.f);
      const float2* Vb = V + i0 * ldv;
      long long e = blk * (long long)blockDim.x + threadIdx.x;
      // two elements per iteration, every load issued before the double-float arithmetic
      for (; e + stride < n; e += 2 * stride) {
        const double wd0 = w[e], wd1 = w[e + stride];
        float2 v0[KB], v1[KB];
#pragma unroll
        for (int i = 0; i < KB; ++i) {
          v0[i] = i < kb ? Vb[i * ldv + e] : make_float2(0.f, 0.f);
          v1[i] = i < kb ? Vb[i * ldv + e + stride] : make_float2(0.f, 0.f);
        }
        if (self) accw += wd0 * wd0 + wd1 * wd1;
        const float2 we0 = df_split(wd0), we1 = df_split(wd1);
#pragma unroll
        for (int i = 0; i < KB; ++i) {
          df_fma(acc[i], v0[i], we0);
          df_fma(acc[i], v1[i], we1);
        }
      }
      if (e < n) {
        const double wd = w[e];
        if (self) accw += wd * wd;
        const float2 we = df_split(wd);
#pragma unroll
        for (int i = 0; i < KB; ++i)
          if (i < kb) df_fma(acc[i], Vb[i * ldv + e], we);
      }
#pragma unroll
      for (int i = 0; i <= KB; ++i) {
        double v = i < KB ? df_join(acc[i]) : accw;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i][wid] = v;
      }
      __syncthreads();
      if (threadIdx.x < kb) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += sh[threadIdx.x][q];
        a.part[(long long)(i0 + threadIdx.x) * nblk + blk] = t;
      }
      if (self && threadIdx.x == 32) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += sh[KB][q];
        a.part[(long long)k * nblk + blk] = t;
      }
      __syncthreads();
    }
  }
};
cudaError_t launch_dots_partial_df(const float2* V, long long ldv, int k, const double* w, long long n, double* part,
                                   int G, int self_dot, cudaStream_t st) {
  return submit<DotsDfK<8>>({V, ldv, k, w, n, part, self_dot}, G, 0, st);
}

// Arithmetic of a Krylov basis element: double-float pairs (float2, products on the FP32 pipes)
// or IEEE doubles (FP64 fused multiply-add).  The fused CGS2 kernels below are written once for both.
template <typename B>
struct BasisOps;
template <>
struct BasisOps<float2> {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 split(double a) { return df_split(a); }
  static __device__ __forceinline__ double join(float2 v) { return df_join(v); }
  static __device__ __forceinline__ void fma(float2& acc, float2 a, float2 b) { df_fma(acc, a, b); }
};
template <>
struct BasisOps<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double split(double a) { return a; }
  static __device__ __forceinline__ double join(double v) { return v; }
  static __device__ __forceinline__ void fma(double& acc, double a, double b) { acc = ::fma(a, b, acc); }
};

// part[i * nblk + blk] = partial sums of V[i] . w (i < k <= 64): a block stages a 256-element strip
// of w in shared memory (in the basis arithmetic), and warp q dots basis rows q, q + 8, q + 16, ...
// against it (coalesced rows, eight loads in flight per thread); every row and w are read once.
// The dot-only counterpart of MultiAxpyDotsK's second phase.
template <typename B>
struct DotsStripK {
  using O = BasisOps<B>;
  static constexpr int KW = 8;  // basis vectors per warp
  struct Args { const B* V; long long ldv; int k; const double* w; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 4;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ B wt[TPB];
    const B* __restrict__ V = a.V;
    const long long ldv = a.ldv, n = a.n;
    const int k = a.k;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    B acc[KW];
#pragma unroll
    for (int q = 0; q < KW; ++q) acc[q] = O::zero();
    for (long long base = (long long)blk * TPB; base < n; base += (long long)nblk * TPB) {
      const long long e = base + tid;
      wt[tid] = e < n ? O::split(a.w[e]) : O::zero();
      __syncthreads();
#pragma unroll
      for (int q = 0; q < KW; ++q) {
        const int i = wid + 8 * q;
        if (i < k) {
          const B* Vi = V + i * ldv + base;
          B v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int el = lane + 32 * t;
            v[t] = base + el < n ? Vi[el] : O::zero();
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) O::fma(acc[q], v[t], wt[lane + 32 * t]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      const int i = wid + 8 * q;
      if (i < k) {
        double v = O::join(acc[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) a.part[(long long)i * nblk + blk] = v;
      }
    }
  }
};
// Both dot blocks of classical Gram-Schmidt evaluated through the Gram matrix (option orth = 2) for
// rows r0 .. r0 + k - 1 of the basis (a chunk of at most 64): part[(r0 + i) * nblk + blk] = partials
// of V[r0 + i] . w and part[(kt + r0 + i) * nblk + blk] = partials of V[r0 + i] . u, with u the newest
// basis vector (one new column of G = V^T V) and kt the basis size.  Like DotsStripK, with a second
// staged strip; every basis row is read once for both dots.
template <typename B>
struct DotsStrip2K {
  using O = BasisOps<B>;
  static constexpr int KW = 8;
  struct Args { const B* V; long long ldv; int r0; int k; int kt; const B* U; const double* w; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 3;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ B wt[TPB];
    __shared__ B ut[TPB];
    const B* __restrict__ V = a.V + (long long)a.r0 * a.ldv;
    const long long ldv = a.ldv, n = a.n;
    const int k = a.k;
    const B* __restrict__ U = a.U;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    B accw[KW], accu[KW];
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      accw[q] = O::zero();
      accu[q] = O::zero();
    }
    for (long long base = (long long)blk * TPB; base < n; base += (long long)nblk * TPB) {
      const long long e = base + tid;
      wt[tid] = e < n ? O::split(a.w[e]) : O::zero();
      ut[tid] = e < n ? U[e] : O::zero();
      __syncthreads();
#pragma unroll
      for (int q = 0; q < KW; ++q) {
        const int i = wid + 8 * q;
        if (i < k) {
          const B* Vi = V + i * ldv + base;
          B v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int el = lane + 32 * t;
            v[t] = base + el < n ? Vi[el] : O::zero();
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            O::fma(accw[q], v[t], wt[lane + 32 * t]);
            O::fma(accu[q], v[t], ut[lane + 32 * t]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      const int i = wid + 8 * q;
      if (i < k) {
        double v = O::join(accw[q]), u = O::join(accu[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          v += __shfl_down_sync(0xffffffffu, v, o);
          u += __shfl_down_sync(0xffffffffu, u, o);
        }
        if (lane == 0) {
          a.part[(long long)(a.r0 + i) * nblk + blk] = v;
          a.part[(long long)(a.kt + a.r0 + i) * nblk + blk] = u;
        }
      }
    }
  }
};
// all kt rows, in launches of at most 64 rows; u = V[kt - 1]
template <typename B>
cudaError_t launch_dots_strip2(const B* V, long long ldv, int kt, const double* w, long long n, double* part, int G,
                               cudaStream_t st) {
  constexpr int KMAX = 8 * DotsStrip2K<B>::KW;
  if (kt < 1) return cudaErrorInvalidValue;
  const B* U = V + (long long)(kt - 1) * ldv;
  for (int r0 = 0; r0 < kt; r0 += KMAX) {
    const int k = kt - r0 < KMAX ? kt - r0 : KMAX;
    cudaError_t e = submit<DotsStrip2K<B>>({V, ldv, r0, k, kt, U, w, n, part}, G, 0, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t launch_dots_strip2_df(const float2* V, long long ldv, int k, const double* w, long long n, double* part,
                                  int G, cudaStream_t st) {
  return launch_dots_strip2<float2>(V, ldv, k, w, n, part, G, st);
}
cudaError_t launch_dots_strip2_fp64(const double* V, long long ldv, int k, const double* w, long long n, double* part,
                                    int G, cudaStream_t st) {
  return launch_dots_strip2<double>(V, ldv, k, w, n, part, G, st);
}

// Gram-matrix form of the second Gram-Schmidt pass: with d = [V^T w ; V^T v_{k-1}] (2k values),
// store column k - 1 of G = V^T V (and its mirror row), then c = h1 + (h1 - G h1), h1 = V^T w.  In
// exact arithmetic c is the CGS2 coefficient vector h1 + V^T (w - V h1); the update w - V c follows.
// One block of 256 threads; any k <= ldg.
struct GramCorrK {
  struct Args { const double* d; double* G; int ldg; int k; double* c; double* zero; };
  static constexpr int THREADS = 256, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int, int) {
    const int k = a.k;
    for (int i = threadIdx.x; i < k; i += THREADS) {
      const double g = a.d[k + i];
      a.G[(long long)i * a.ldg + (k - 1)] = g;
      a.G[(long long)(k - 1) * a.ldg + i] = g;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += THREADS) {
      double s = 0.0;
      for (int l = 0; l < k; ++l) s = fma(a.G[(long long)i * a.ldg + l], a.d[l], s);
      const double h = a.d[i];
      a.c[i] = h + (h - s);
      if (a.zero) a.zero[i] = 0.0;  // a second coefficient slot that callers add to c
    }
  }
};
cudaError_t launch_gram_correct(const double* d, double* G, int ldg, int k, double* c, double* zero,
                                cudaStream_t st) {
  if (k < 1 || k > ldg) return cudaErrorInvalidValue;
  return submit<GramCorrK>({d, G, ldg, k, c, zero}, 1, 0, st);
}

template <typename B>
cudaError_t launch_dots_strip(const B* V, long long ldv, int k, const double* w, long long n, double* part, int G,
                              cudaStream_t st) {
  if (k > 8 * DotsStripK<B>::KW) return cudaErrorInvalidValue;
  return submit<DotsStripK<B>>({V, ldv, k, w, n, part}, G, 0, st);
}
cudaError_t launch_dots_strip_df(const float2* V, long long ldv, int k, const double* w, long long n, double* part,
                                 int G, cudaStream_t st) {
  return launch_dots_strip<float2>(V, ldv, k, w, n, part, G, st);
}
cudaError_t launch_dots_strip_fp64(const double* V, long long ldv, int k, const double* w, long long n, double* part,
                                   int G, cudaStream_t st) {
  return launch_dots_strip<double>(V, ldv, k, w, n, part, G, st);
}

// w <- w + sign * sum_i coef[i] V[i] (sum carried in the basis arithmetic), partial sums of |w|^2
template <typename B>
struct MultiAxpyNormBK {
  using O = BasisOps<B>;
  struct Args { const B* V; long long ldv; int k; const double* coef; double sign; double* w; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    extern __shared__ __align__(16) unsigned char cs_raw[];
    B* cs2 = reinterpret_cast<B*>(cs_raw);
    __shared__ double sh[32];
    const B* __restrict__ V = a.V;
    double* __restrict__ w = a.w;
    const long long ldv = a.ldv;
    const int k = a.k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs2[i] = O::split(a.sign * a.coef[i]);
    __syncthreads();
    double s = 0.0;
    GS_FOR(e, a.n) {
      const double we = w[e];
      B acc = O::zero();
      int i = 0;
      for (; i + 8 <= k; i += 8) {  // eight basis loads in flight per thread
        B v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = V[(i + u) * ldv + e];
#pragma unroll
        for (int u = 0; u < 8; ++u) O::fma(acc, cs2[i + u], v[u]);
      }
      for (; i < k; ++i) O::fma(acc, cs2[i], V[i * ldv + e]);
      const double r = we + O::join(acc);
      w[e] = r;
      s += r * r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
      a.part[blk] = t;
    }
  }
};
cudaError_t launch_multi_axpy_norm_df(const float2* V, long long ldv, int k, const double* coef, double sign, double* w,
                                      long long n, double* part, int G, cudaStream_t st) {
  return submit<MultiAxpyNormBK<float2>>({V, ldv, k, coef, sign, w, n, part}, G, sizeof(float2) * (k > 0 ? k : 1), st);
}
cudaError_t launch_multi_axpy_norm_fp64(const double* V, long long ldv, int k, const double* coef, double sign,
                                        double* w, long long n, double* part, int G, cudaStream_t st) {
  return submit<MultiAxpyNormBK<double>>({V, ldv, k, coef, sign, w, n, part}, G, sizeof(double) * (k > 0 ? k : 1), st);
}

// First CGS2 update fused with the second pass's dot products:
//   w <- w + sign * sum_i coef[i] V[i]            (sum in the basis arithmetic, FP64 result)
//   part[i * nblk + blk] = sum over the block's elements of V[i] . w_new
// The block walks its elements in rounds of 256: every thread updates one element and keeps the
// new value in shared memory, then warp q accumulates the dot products of basis vectors q, q + 8,
// q + 16, ... over the round's 256 elements (coalesced rows; the rows were just read by the update,
// so they come from L1/L2).  One pass over V from HBM instead of two.
template <typename B>
struct MultiAxpyDotsK {
  using O = BasisOps<B>;
  static constexpr int KW = 8;  // basis vectors per warp (k <= 64)
  struct Args { const B* V; long long ldv; int k; const double* coef; double sign; double* w; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 4;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    extern __shared__ __align__(16) unsigned char cs_raw[];
    B* cs2 = reinterpret_cast<B*>(cs_raw);
    __shared__ B wt[TPB];
    const B* __restrict__ V = a.V;
    double* __restrict__ w = a.w;
    const long long ldv = a.ldv, n = a.n;
    const int k = a.k;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < k; i += blockDim.x) cs2[i] = O::split(a.sign * a.coef[i]);
    B acc[KW];
#pragma unroll
    for (int q = 0; q < KW; ++q) acc[q] = O::zero();
    __syncthreads();
    for (long long base = (long long)blk * TPB; base < n; base += (long long)nblk * TPB) {
      const long long e = base + tid;
      B wdf = O::zero();
      if (e < n) {
        B s = O::zero();
        int i = 0;
        for (; i + 8 <= k; i += 8) {
          B v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = V[(i + u) * ldv + e];
#pragma unroll
          for (int u = 0; u < 8; ++u) O::fma(s, cs2[i + u], v[u]);
        }
        for (; i < k; ++i) O::fma(s, cs2[i], V[i * ldv + e]);
        const double r = w[e] + O::join(s);
        w[e] = r;
        wdf = O::split(r);
      }
      wt[tid] = wdf;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < KW; ++q) {
        const int i = wid + 8 * q;
        if (i < k) {
          const B* Vi = V + i * ldv + base;
          B v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int el = lane + 32 * t;
            v[t] = base + el < n ? Vi[el] : O::zero();
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) O::fma(acc[q], v[t], wt[lane + 32 * t]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      const int i = wid + 8 * q;
      if (i < k) {
        double v = O::join(acc[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) a.part[(long long)i * nblk + blk] = v;
      }
    }
  }
};
cudaError_t launch_multi_axpy_dots_df(const float2* V, long long ldv, int k, const double* coef, double sign, double* w,
                                      long long n, double* part, int G, cudaStream_t st) {
  if (k > 8 * MultiAxpyDotsK<float2>::KW) return cudaErrorInvalidValue;
  return submit<MultiAxpyDotsK<float2>>({V, ldv, k, coef, sign, w, n, part}, G, sizeof(float2) * (k > 0 ? k : 1), st);
}
cudaError_t launch_multi_axpy_dots_fp64(const double* V, long long ldv, int k, const double* coef, double sign,
                                        double* w, long long n, double* part, int G, cudaStream_t st) {
  if (k > 8 * MultiAxpyDotsK<double>::KW) return cudaErrorInvalidValue;
  return submit<MultiAxpyDotsK<double>>({V, ldv, k, coef, sign, w, n, part}, G, sizeof(double) * (k > 0 ? k : 1), st);
}

// v_df <- w / sqrt(nrm2) in double-float form, and the same vector as double in vd
struct ScaleDfK {
  struct Args { const double* w; const double* nrm2; float2* v; double* vd; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    // the scale once per block: FP64 division and square root are slow on the FP64 pipe
    __shared__ double ssc;
    if (threadIdx.x == 0) ssc = 1.0 / sqrt(a.nrm2[0]);
    __syncthreads();
    const double sc = ssc;
    GS_FOR(i, a.n) {
      const double x = a.w[i] * sc;
      a.v[i] = df_split(x);
      a.vd[i] = x;
    }
  }
};
cudaError_t launch_scale_by_rnorm_df(const double* w, const double* nrm2, float2* v, double* vd, long long n,
                                     cudaStream_t st) {
  unsigned g = nblk(n);
  if (g > 152u * 16u) g = 152u * 16u;
  return submit<ScaleDfK>({w, nrm2, v, vd, n}, g, 0, st);
}

struct ReduceK {
  struct Args { const double* part; int G; double* out; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    __shared__ double sh[32];
    const int i = blk;
    double s = 0.0;
    for (int b = threadIdx.x; b < a.G; b += blockDim.x) s += a.part[(long long)i * a.G + b];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) a.out[i] = s;
  }
};
cudaError_t launch_reduce_partials(const double* part, int k, int G, double* out, cudaStream_t st) {
  return submit<ReduceK>({part, G, out}, k, 0, st);
}

struct MultiAxpyK {
  struct Args { const double* V; long long ldv; int k; const double* coef; double sign; double* w; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    extern __shared__ double cs[];
    const double* __restrict__ V = a.V;
    double* __restrict__ w = a.w;
    const int k = a.k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = a.sign * a.coef[i];
    __syncthreads();
    GS_FOR(e, a.n) {
      double acc = w[e];
      for (int i = 0; i < k; ++i) acc += cs[i] * V[i * a.ldv + e];
      w[e] = acc;
    }
  }
};
cudaError_t launch_multi_axpy(const double* V, long long ldv, int k, const double* coef, double sign, double* w,
                              long long n, cudaStream_t st) {
  unsigned g = nblk(n);
  if (g > 152u * 16u) g = 152u * 16u;
  return submit<MultiAxpyK>({V, ldv, k, coef, sign, w, n}, g, sizeof(double) * (k > 0 ? k : 1), st);
}

struct ScaleK {
  struct Args { const double* w; const double* nrm2; double* v; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double ssc;  // the scale once per block (FP64 division and square root)
    if (threadIdx.x == 0) ssc = 1.0 / sqrt(a.nrm2[0]);
    __syncthreads();
    const double s = ssc;
    GS_FOR(i, a.n) a.v[i] = a.w[i] * s;
  }
};
cudaError_t launch_scale_by_rnorm(const double* w, const double* nrm2, double* v, long long n, cudaStream_t st) {
  unsigned g = nblk(n);
  if (g > 152u * 16u) g = 152u * 16u;
  return submit<ScaleK>({w, nrm2, v, n}, g, 0, st);
}

__global__ void k_add_vec(double* a, const double* b, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) a[i] += b[i];
}
cudaError_t launch_add_vec(double* a, const double* b, int k, cudaStream_t st) {
  k_add_vec<<<(k + 63) / 64, 64, 0, st>>>(a, b, k);
  return launched(cudaGetLastError());
}

struct MaskedSumK {
  struct Args { const double* x; const uint8_t* mask; long long n; double* part; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    __shared__ double sh[32];
    double s = 0.0;
    GS_FOR(e, a.n)
      if (!a.mask || !a.mask[e]) s += a.x[e];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) a.part[blk] = s;
  }
};
cudaError_t launch_masked_sum_partial(const double* x, const uint8_t* mask, long long n, double* part, int G,
                                      cudaStream_t st) {
  return submit<MaskedSumK>({x, mask, n, part}, G, 0, st);
}
struct SubScalarK {
  struct Args { double* x; const uint8_t* mask; long long n; const double* sum; double inv_count; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    const double m = a.sum[0] * a.inv_count;
    GS_FOR(e, a.n)
      if (!a.mask || !a.mask[e]) a.x[e] -= m;
  }
};
cudaError_t launch_sub_scalar_masked(double* x, const uint8_t* mask, long long n, const double* sum,
                                     double inv_count, cudaStream_t st) {
  return submit<SubScalarK>({x, mask, n, sum, inv_count}, nblk(n), 0, st);
}

// ---- dense coarse solve (explicit inverse of A_0 on its free unknowns) ------------------------------
template <typename T>
struct CoarseGatherK {
  struct Args { const T* b; const int* freeidx; int nf; double* tmp; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    const int i = blk * blockDim.x + threadIdx.x;
    if (i < a.nf) a.tmp[i] = (double)a.b[a.freeidx[i]];
  }
};
template <typename T>
struct CoarseGemvK {
  struct Args { const double* Ainv; const int* freeidx; int nf; const double* tmp; T* y; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    const int warp = (blk * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.nf) return;
    const double* row = a.Ainv + (long long)warp * a.nf;
    double s = 0.0;
    for (int j = lane; j < a.nf; j += 32) s += row[j] * a.tmp[j];
    s = warp_sum(s);
    if (lane == 0) a.y[a.freeidx[warp]] = (T)s;
  }
};
template <typename T>
struct ZeroK {
  struct Args { T* y; long long n; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    GS_FOR(i, a.n) a.y[i] = T(0);
  }
};
template <typename T>
cudaError_t launch_coarse_solve(const double* Ainv, const int* freeidx, int nf, const T* b, T* y, long long n,
                                double* tmp, cudaStream_t st) {
  cudaError_t e = submit<CoarseGatherK<T>>({b, freeidx, nf, tmp}, (nf + TPB - 1) / TPB, 0, st);
  if (e != cudaSuccess) return e;
  e = submit<ZeroK<T>>({y, n}, nblk(n), 0, st);
  if (e != cudaSuccess) return e;
  return submit<CoarseGemvK<T>>({Ainv, freeidx, nf, tmp, y}, ((long long)nf * 32 + TPB - 1) / TPB, 0, st);
}

// y[0..n) = 0 (no read of y: safe on uninitialised memory)
template <typename T>
cudaError_t launch_fill_zero(T* y, long long n, cudaStream_t st) {
  return submit<ZeroK<T>>({y, n}, nblk(n), 0, st);
}
template cudaError_t launch_fill_zero<double>(double*, long long, cudaStream_t);

// dst = [s0[0..n0) | s1[0..n1) | s2[0..n2)]: the host-bound scalars of one instance in one place
struct Gather3K {
  struct Args { const double* s[3]; int n[3]; double* dst; };
  static constexpr int THREADS = 64, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int, int) {
    int off = 0;
    for (int q = 0; q < 3; ++q) {
      for (int i = threadIdx.x; i < a.n[q]; i += blockDim.x) a.dst[off + i] = a.s[q][i];
      off += a.n[q];
    }
  }
};
cudaError_t launch_gather3(const double* s0, int n0, const double* s1, int n1, const double* s2, int n2, double* dst,
                           cudaStream_t st) {
  Gather3K::Args a{{s0, s1, s2}, {n0, n1, n2}, dst};
  return submit<Gather3K>(a, 1, 0, st);
}

// Gauss-Jordan inversion of an SPD matrix (no pivoting), one pivot per pair of launches.
__global__ void k_gj_save(const double* __restrict__ A, int n, int k, double* __restrict__ row, double* __restrict__ col) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    row[i] = A[(long long)k * n + i];
    col[i] = A[(long long)i * n + k];
  }
}
__global__ void k_gj_update(double* __restrict__ A, int n, int k, const double* __restrict__ row,
                            const double* __restrict__ col) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  const double p = row[k];
  double v;
  if (i == k && j == k) v = 1.0 / p;
  else if (i == k) v = row[j] / p;
  else if (j == k) v = -col[i] / p;
  else v = A[idx] - col[i] * row[j] / p;
  A[idx] = v;
}
cudaError_t launch_gj_save(const double* A, int n, int k, double* row, double* col, cudaStream_t st) {
  k_gj_save<<<(n + TPB - 1) / TPB, TPB, 0, st>>>(A, n, k, row, col);
  return launched(cudaGetLastError());
}
cudaError_t launch_gj_update(double* A, int n, int k, const double* row, const double* col, cudaStream_t st) {
  k_gj_update<<<nblk((long long)n * n), TPB, 0, st>>>(A, n, k, row, col);
  return launched(cudaGetLastError());
}

template <typename T>
__global__ void k_axpby(const T* __restrict__ x, T* __restrict__ y, T a, T b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
template <typename T>
cudaError_t launch_axpby(const T* x, T* y, T a, T b, long long n, cudaStream_t st) {
  k_axpby<T><<<nblk(n), TPB, 0, st>>>(x, y, a, b, n);
  return launched(cudaGetLastError());
}

__device__ __forceinline__ bool full_constrained(const Geom& geo, long long i) {
  const long long n_u = geo.dim * geo.Nv;
  if (i < n_u) {
    const long long node = i % geo.Nv;
    const int I = (int)(node % geo.nv[0]);
    const int J = (int)((node / geo.nv[0]) % geo.nv[1]);
    const int K = geo.dim == 3 ? (int)(node / ((long long)geo.nv[0] * geo.nv[1])) : 0;
    return geo.vmask ? geo.vmask[node] != 0 : face_constrained(geo, I, J, K);
  }
  return geo.pmask ? geo.pmask[i - n_u] != 0 : false;
}

struct CopyConstrainedK {
  struct Args { const double* v; double* z; Geom geo; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    const long long N = a.geo.dim * a.geo.Nv + a.geo.Np;
    GS_FOR(i, N)
      if (full_constrained(a.geo, i)) a.z[i] = a.v[i];
  }
};
cudaError_t launch_copy_constrained(const double* v, double* z, const Geom& geo, cudaStream_t st) {
  const long long N = geo.dim * geo.Nv + geo.Np;
  return submit<CopyConstrainedK>({v, z, geo}, nblk(N), 0, st);
}

// The preconditioner's result back in FGMRES precision, z = [(double) zu | (double) zp], with the
// constrained entries copied from v instead (the saddle matrix is the identity there): the two
// casts and the constrained copy above in one pass.  One thread per velocity node, all of its
// components (its mesh position, and so its constraint, is found once), then one per pressure
// node.  Each entry of z depends only on the same entry of v, zu or zp, so z may alias v.
template <typename T>
struct PrecondOutK {
  struct Args { const T* zu; const T* zp; const double* v; double* z; Geom geo; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    const Geom& g = a.geo;
    const long long Nv = g.Nv, n_u = g.dim * Nv;
    const bool idx32 = Nv < (1LL << 31);
    GS_FOR(i, Nv + g.Np) {
      if (i < Nv) {
        bool con;
        if (g.vmask) {
          con = g.vmask[i] != 0;
        } else if (idx32) {
          const unsigned node = (unsigned)i, n0 = (unsigned)g.nv[0], n1 = (unsigned)g.nv[1];
          const unsigned q = node / n0;
          con = face_constrained(g, (int)(node - q * n0), (int)(q % n1), g.dim == 3 ? (int)(q / n1) : 0);
        } else {
          const long long q = i / g.nv[0];
          con = face_constrained(g, (int)(i - q * g.nv[0]), (int)(q % g.nv[1]), g.dim == 3 ? (int)(q / g.nv[1]) : 0);
        }
        for (int c = 0; c < g.dim; ++c) {
          const long long e = c * Nv + i;
          a.z[e] = con ? a.v[e] : (double)a.zu[e];
        }
      } else {
        const long long p = i - Nv;
        const bool con = g.pmask != nullptr && g.pmask[p] != 0;
        a.z[n_u + p] = con ? a.v[n_u + p] : (double)a.zp[p];
      }
    }
  }
};
template <typename T>
cudaError_t launch_precond_out(const T* zu, const T* zp, const double* v, double* z, const Geom& geo,
                               cudaStream_t st) {
  return submit<PrecondOutK<T>>({zu, zp, v, z, geo}, nblk(geo.Nv + geo.Np), 0, st);
}

// the preconditioner's input in its own precision: u = (T) v[0, n_u), p = (T) v[n_u, n_u + n_p)
template <typename T>
struct PrecondInK {
  struct Args { const double* v; T* u; T* p; long long n_u, n_p; };
  static constexpr int THREADS = TPB, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int nblk) {
    GS_FOR(i, a.n_u + a.n_p) {
      const T x = (T)a.v[i];
      if (i < a.n_u) a.u[i] = x;
      else a.p[i - a.n_u] = x;
    }
  }
};
template <typename T>
cudaError_t launch_precond_in(const double* v, T* u, T* p, long long n_u, long long n_p, cudaStream_t st) {
  return submit<PrecondInK<T>>({v, u, p, n_u, n_p}, nblk(n_u + n_p), 0, st);
}

// rhs = Mf - Kg on free entries, g on constrained entries (velocity then pressure)
__global__ void k_combine_lift(const double* __restrict__ Mf, const double* __restrict__ Kg,
                               const double* __restrict__ g, const Geom geo, double* __restrict__ rhs) {
  const long long N = geo.dim * geo.Nv + geo.Np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    rhs[i] = full_constrained(geo, i) ? g[i] : Mf[i] - Kg[i];
  }
}
cudaError_t launch_combine_lift(const double* Mf, const double* Kg, const double* g, const uint8_t*, const uint8_t*,
                                const Geom& geo, double* rhs, cudaStream_t st) {
  const long long N = geo.dim * geo.Nv + geo.Np;
  k_combine_lift<<<nblk(N), TPB, 0, st>>>(Mf, Kg, g, geo, rhs);
  return launched(cudaGetLastError());
}

#define INST(T)                                                                                       \
  template cudaError_t launch_cheb_init0<T>(const T*, const T*, T, T*, T*, long long, cudaStream_t); \
  template cudaError_t launch_zero_constrained_u<T>(const Geom&, T*, cudaStream_t);                   \
  template cudaError_t launch_lanczos_pre<T>(const T*, const T*, T*, long long, cudaStream_t);        \
  template cudaError_t launch_lanczos_post<T>(const T*, const T*, const T*, T, T*, long long, cudaStream_t); \
  template cudaError_t launch_dots_partial<T>(const T*, long long, int, const T*, long long, double*, int, cudaStream_t); \
  template cudaError_t launch_axpby<T>(const T*, T*, T, T, long long, cudaStream_t);                 \
  template cudaError_t launch_coarse_solve<T>(const double*, const int*, int, const T*, T*, long long, double*, cudaStream_t); \
  template cudaError_t launch_precond_out<T>(const T*, const T*, const double*, double*, const Geom&, cudaStream_t); \
  template cudaError_t launch_precond_in<T>(const double*, T*, T*, long long, long long, cudaStream_t);
INST(float)
INST(double)
#undef INST
template cudaError_t launch_cast<double, float>(const double*, float*, long long, float, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, long long, double, cudaStream_t);
template cudaError_t launch_cast<double, double>(const double*, double*, long long, double, cudaStream_t);
template cudaError_t launch_cast<float, float>(const float*, float*, long long, float, cudaStream_t);

}  // namespace gs
