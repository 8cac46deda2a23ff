// Host-side launch wrappers of the device kernels (internal to libgs.so).
#pragma once
#include <cuda_runtime.h>

#include "gs_batch.cuh"
#include "gs_common.cuh"

namespace gs {

// Process-wide count of kernels this library has launched (returned by every launch wrapper).
cudaError_t launched(cudaError_t e, int kernels = 1);
long long launches_total();

enum TileMode { TILE_APPLY = 0, TILE_RESID = 1, TILE_CHEB = 2 };

// Arguments of the cell-tile operator kernel.  Velocity vectors have length dim*Nv
// (component-blocked), pressure vectors Np.
template <typename T>
struct TileArgs {
  Geom g;
  OpCoef<T> c;
  const T* eta;   // per cell
  const T* alpha; // per cell factor of the mass term (alpha_K; NULL: 1, alpha then lives in c.mm)
  const T* xu;    // velocity input (A and B), CHEB: current iterate
  const T* xp;    // pressure input (B^T)
  T* yu;          // velocity output (APPLY / RESID)
  T* yp;          // pressure output (B)
  const T* bu;    // velocity right-hand side (RESID / CHEB)
  const T* bp;    // pressure right-hand side (RESID)
  T* d;           // CHEB: search direction (in/out)
  const T* dinv;  // CHEB: inverse diagonal
  T* xout;        // CHEB: next iterate (must not alias xu)
  T c1, c2;       // CHEB: d <- c1 d + c2 dinv r   (c1 ignored when use_d == 0)
  int use_d;
  int raw;        // 1: no constraint elimination (operator of the unconstrained forms)
  int* err;       // device word set nonzero when a bounded wait of the kernel gave up (may be NULL)
  // corrector stage: conv = 1 adds rho (C + S) to A, conv = 2 the symmetric part of that term
  int conv;
  const T* vc;    // the convective field v° on this level (d N_v entries, component-blocked)
  const T* rk;    // streamline parameter r_K per cell
  T rho, ihx, ihy, wq;  // density, 1 / h_x, 1 / h_y, h_x h_y (3D: h_x h_y h_z)
  T ihz;                // 1 / h_z (3D)
  int tiles[3];
  T* part;        // 3D FP32: per-tile partial sums of the nodes on shared tile faces (gs_tile.cu,
                  // tile3nh_body; NULL: the halo tiles are used)
  int shape;      // 2D velocity-block variant (0 / 1 / 2: tiles of 16 / 17 / 8 rows of evaluated cells,
                  // 3: the strip kernel of gs_strip2d.cuh; other operator blocks: 3 -> tiles of 8);
                  // 3D: 0 / 1 -> tiles of 8 x 8 x 8 / 8 x 8 x 4 evaluated cells
};
constexpr int kTileShapes2D = 4;   // velocity-block variants the autotuner times
constexpr int kTileHeights2D = 3;  // tile variants of the full saddle operator
// 3D cell tiles (TileArgs::shape): 0 -> 8 x 8 x 8, 1 -> 8 x 8 x 4 evaluated cells; every variant
// sums a node's cell contributions in the same order, so the choice does not change any result
constexpr int kTileShapes3D = 2;
// FP32 3D velocity block without halo cells (gs_tile.cu, tile3nh_body): tiles of 8 x 8 x 4 cells, a
// 17 x 17 x 9 node box each; the partial-sum buffer holds 3 boxes (one per component) per tile
constexpr int kNH3Cells0 = 8, kNH3Cells1 = 8, kNH3Cells2 = 4;
constexpr int kNH3Box = (2 * kNH3Cells0 + 1) * (2 * kNH3Cells1 + 1) * (2 * kNH3Cells2 + 1);
inline long long nh3_part_elems(const int n[3]) {
  const long long t = (long long)((n[0] + kNH3Cells0 - 1) / kNH3Cells0) * ((n[1] + kNH3Cells1 - 1) / kNH3Cells1) *
                      ((n[2] + kNH3Cells2 - 1) / kNH3Cells2);
  return t * 3 * kNH3Box;
}
constexpr int tile3d_depth(int shape) { return shape == 1 ? 4 : 8; }

// Which blocks of the saddle operator a launch computes.
enum TileOps { OPS_A = 1, OPS_BT = 2, OPS_B = 4 };

template <typename T>
cudaError_t launch_tile(int dim, int mode, int ops, TileArgs<T> a, cudaStream_t st);
template <typename T>
cudaError_t launch_tile2d(int mode, int ops, TileArgs<T> a, cudaStream_t st);
template <typename T>
cudaError_t launch_strip2d(int mode, TileArgs<T> a, cudaStream_t st);
// one CTA whose bounded mbarrier wait runs out (about a second) and sets *err
cudaError_t launch_wait_probe(int* err, cudaStream_t st);
// the same operators with the corrector-stage terms (TileArgs::conv != 0), 32 x 8 tiles
template <typename T>
cudaError_t launch_tile2d_conv(int mode, int ops, const TileArgs<T>& a, cudaStream_t st);
// diag += diag(rho (C + S)) on every free velocity node (both components); FP64
cudaError_t launch_diag_conv(const Geom& g, const double* vc, const double* rk, double rho, double* diag,
                             cudaStream_t st);
// out[i] = 1 / in[i]
template <typename T>
cudaError_t launch_reciprocal(const double* in, T* out, long long n, cudaStream_t st);

template <typename T>
cudaError_t launch_diagA(const Geom& g, const OpCoef<T>& c, const T* eta, const T* alpha, T* out, int invert,
                         cudaStream_t st);
// rc = R rf; with d != NULL also the start of the coarse level's Chebyshev smoother from zero,
// d = x = dinv * rc * inv_theta (the expression of launch_cheb_init0)
template <typename T>
cudaError_t launch_restrict(const Geom& gf, const Geom& gc, const T* rf, T* rc, cudaStream_t st,
                            const T* dinv = nullptr, T inv_theta = T(0), T* d = nullptr, T* x = nullptr);
template <typename T>
cudaError_t launch_prolong_add(const Geom& gf, const Geom& gc, const T* xc, T* xf, cudaStream_t st);

// Pressure mass M_p(1/eta): APPLY y = M x;  CHEB: r = b - M x_in, d = c1 d + c2 dinv r,
// x_out = x_in + d.
template <typename T>
struct PMassArgs {
  Geom g;
  OpCoef<T> c;
  const T* eta;
  const T* x;
  T* y;
  const T* b;
  T* d;
  const T* dinv;
  T* xout;
  T c1, c2;
  int use_d;
  int raw;   // 1: no constraint elimination
  int unit;  // 1: unit cell weight (plain Q1 mass) instead of 1/eta
};
template <typename T>
cudaError_t launch_pmass(int mode, PMassArgs<T> a, cudaStream_t st);
template <typename T>
cudaError_t launch_pdiag(const Geom& g, const OpCoef<T>& c, const T* eta, T* dinv, cudaStream_t st);

// Pressure Laplacian K_p (Q1 stiffness over active cells; nodes with cmask != 0 are identity
// rows / zero columns).  Cell matrix: sum_a kc[a] (K1 in direction a, Pi elsewhere), with
// K1 = [1 -1; -1 1], Pi = [2 1; 1 2], kc[a] = prod_{b != a} h_b / (6^(d-1) h_a).
// Modes as for the tile kernel: APPLY y = K x; RESID y = b - K x; CHEB fused Chebyshev step.
template <typename T>
struct PLapArgs {
  Geom g;
  T kc[3];
  const T* w;  // per-cell weight (abar / alpha_K with alpha per cell); NULL: 1
  const uint8_t* cmask;
  const T* x;
  T* y;
  const T* b;
  T* d;
  const T* dinv;
  T* xout;
  T c1, c2;
  int use_d;
};
template <typename T>
cudaError_t launch_plap(int mode, PLapArgs<T> a, cudaStream_t st);
template <typename T>
cudaError_t launch_plap_diag(const Geom& g, const T* kc, const T* w, const uint8_t* cmask, T* dinv, cudaStream_t st);
// Q1 transfers between pressure levels (bilinear interpolation and its transpose)
template <typename T>
cudaError_t launch_p_restrict(const Geom& gf, const Geom& gc, const uint8_t* mf, const uint8_t* mc, const T* rf,
                              T* rc, cudaStream_t st, const T* dinv = nullptr, T inv_theta = T(0), T* d = nullptr,
                              T* x = nullptr);
template <typename T>
cudaError_t launch_p_prolong_add(const Geom& gf, const Geom& gc, const uint8_t* mf, const uint8_t* mc, const T* xc,
                                 T* xf, cudaStream_t st);
// Tiled Q1 operators (gs_q1tile.cu): OP = Q1_PLAP (K_p, cell scalar eta[cell], or 1 when eta is
// NULL: the per-cell weight) or Q1_PMASS (M_p(1/eta), cell scalar pm / eta); cmask (may be NULL)
// marks identity rows / zero columns.
enum Q1Op { Q1_PLAP = 0, Q1_PMASS = 1 };
template <typename T>
struct Q1Args {
  Geom g;
  T kc[3];
  T pm;
  const T* eta;
  const uint8_t* cmask;
  const T* x;
  T* y;
  const T* b;
  T* d;
  const T* dinv;
  T* xout;
  T c1, c2;
  int use_d;
};
template <typename T>
cudaError_t launch_q1tile(int op, int mode, const Q1Args<T>& a, cudaStream_t st);
// out[i] = mask[i] ? 0 : in[i]   (may run in place)
template <typename T>
cudaError_t launch_mask_copy(const T* in, const uint8_t* mask, T* out, long long n, cudaStream_t st);
// z[i] = -(m[i] + alpha * (mask[i] ? 0 : v[i]))   (Cahouet-Chabard combination)
template <typename T>
cudaError_t launch_cc_combine(const T* m, const T* v, const uint8_t* mask, T alpha, T* z, long long n,
                              cudaStream_t st);

// ---- vector kernels ----
template <typename T>
cudaError_t launch_cheb_init0(const T* b, const T* dinv, T inv_theta, T* d, T* x, long long n,
                              cudaStream_t st);
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* in, TO* out, long long n, TO scale, cudaStream_t st);
template <typename T>
cudaError_t launch_zero_constrained_u(const Geom& g, T* v, cudaStream_t st);
template <typename T>
cudaError_t launch_lanczos_pre(const T* dinv, const T* v, T* t, long long n, cudaStream_t st);
template <typename T>
cudaError_t launch_lanczos_post(const T* dinv, const T* y, const T* vprev, T beta_prev, T* w,
                                long long n, cudaStream_t st);

// partial sums: part[i * G + block] = sum over block's chunk of V[i][e] * w[e], i < k
template <typename T>
cudaError_t launch_dots_partial(const T* V, long long ldv, int k, const T* w, long long n,
                                double* part, int G, cudaStream_t st);
cudaError_t launch_reduce_partials(const double* part, int k, int G, double* out, cudaStream_t st);
// Gram-Schmidt through the Gram matrix (orth = 2): dots of the basis with w and with its newest row,
// then the correction of the coefficients (gs_blas.cu)
cudaError_t launch_dots_strip2_df(const float2* V, long long ldv, int k, const double* w, long long n, double* part,
                                  int G, cudaStream_t st);
cudaError_t launch_dots_strip2_fp64(const double* V, long long ldv, int k, const double* w, long long n, double* part,
                                    int G, cudaStream_t st);
cudaError_t launch_gram_correct(const double* d, double* G, int ldg, int k, double* c, double* zero,
                                cudaStream_t st);
// k dot products V[i] . w plus w . w in row k of part (rows 0..k)
cudaError_t launch_dots_norm_partial(const double* V, long long ldv, int k, const double* w, long long n,
                                     double* part, int G, cudaStream_t st);
// w <- w + sign * sum_i coef[i] V[i]; part[block] = partial sums of the new |w|^2 (G blocks)
cudaError_t launch_multi_axpy_norm(const double* V, long long ldv, int k, const double* coef, double sign,
                                   double* w, long long n, double* part, int G, cudaStream_t st);
// Krylov basis stored in double-float form (float2 hi + lo): the same operations on FP32 pipes
cudaError_t launch_dots_partial_df(const float2* V, long long ldv, int k, const double* w, long long n,
                                   double* part, int G, int self_dot, cudaStream_t st);
cudaError_t launch_multi_axpy_norm_df(const float2* V, long long ldv, int k, const double* coef, double sign,
                                      double* w, long long n, double* part, int G, cudaStream_t st);
// part[i * G + block] = partial sums of V[i] . w (k <= 64; strips of w staged in shared memory,
// every row read once)
cudaError_t launch_dots_strip_df(const float2* V, long long ldv, int k, const double* w, long long n, double* part,
                                 int G, cudaStream_t st);
// w <- w + sign * sum_i coef[i] V[i], then part[i * G + block] = partial sums of V[i] . w_new
// (first CGS2 update fused with the second pass's dots; k <= 64)
cudaError_t launch_multi_axpy_dots_df(const float2* V, long long ldv, int k, const double* coef, double sign,
                                      double* w, long long n, double* part, int G, cudaStream_t st);
cudaError_t launch_scale_by_rnorm_df(const double* w, const double* nrm2, float2* v, double* vd, long long n,
                                     cudaStream_t st);
// the same three fused CGS2 passes on an IEEE FP64 basis (FP64 products and sums)
cudaError_t launch_dots_strip_fp64(const double* V, long long ldv, int k, const double* w, long long n, double* part,
                                   int G, cudaStream_t st);
cudaError_t launch_multi_axpy_dots_fp64(const double* V, long long ldv, int k, const double* coef, double sign,
                                        double* w, long long n, double* part, int G, cudaStream_t st);
cudaError_t launch_multi_axpy_norm_fp64(const double* V, long long ldv, int k, const double* coef, double sign,
                                        double* w, long long n, double* part, int G, cudaStream_t st);
// w <- w + sign * sum_i coef[i] V[i]   (coef on device)
cudaError_t launch_multi_axpy(const double* V, long long ldv, int k, const double* coef, double sign,
                              double* w, long long n, cudaStream_t st);
// v <- w * (1 / sqrt(nrm2[0]))   (nrm2 on device)
cudaError_t launch_scale_by_rnorm(const double* w, const double* nrm2, double* v, long long n,
                                  cudaStream_t st);
cudaError_t launch_add_vec(double* a, const double* b, int k, cudaStream_t st);  // a += b (small)
// x[i] -= mean over pressure entries that are free; pmask may be NULL; sum on device
cudaError_t launch_masked_sum_partial(const double* x, const uint8_t* mask, long long n,
                                      double* part, int G, cudaStream_t st);
cudaError_t launch_sub_scalar_masked(double* x, const uint8_t* mask, long long n, const double* sum,
                                     double inv_count, cudaStream_t st);
// coarse dense solve: y[free[i]] = sum_j Ainv[i][j] b[free[j]], y[constrained] = 0
template <typename T>
cudaError_t launch_coarse_solve(const double* Ainv, const int* freeidx, int nf, const T* b, T* y,
                                long long n, double* tmp, cudaStream_t st);
cudaError_t launch_gj_save(const double* A, int n, int k, double* row, double* col, cudaStream_t st);
cudaError_t launch_gj_update(double* A, int n, int k, const double* row, const double* col,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_fill_zero(T* y, long long n, cudaStream_t st);
// dst = [s0[0..n0) | s1[0..n1) | s2[0..n2)]  (one block)
cudaError_t launch_gather3(const double* s0, int n0, const double* s1, int n1, const double* s2, int n2, double* dst,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_axpby(const T* x, T* y, T a, T b, long long n, cudaStream_t st);  // y = a x + b y
// z[i] = v[i] on every constrained entry of a full vector [u | p] (finest level)
cudaError_t launch_copy_constrained(const double* v, double* z, const Geom& geo, cudaStream_t st);
// z = [(double) zu | (double) zp] with z[i] = v[i] on every constrained entry (finest level)
template <typename T>
cudaError_t launch_precond_out(const T* zu, const T* zp, const double* v, double* z, const Geom& geo,
                               cudaStream_t st);
// u = (T) v[0, n_u), p = (T) v[n_u, n_u + n_p)
template <typename T>
cudaError_t launch_precond_in(const double* v, T* u, T* p, long long n_u, long long n_p, cudaStream_t st);
cudaError_t launch_combine_lift(const double* Mf, const double* Kg, const double* g,
                                const uint8_t* vmask, const uint8_t* pmask, const Geom& geo,
                                double* rhs, cudaStream_t st);

// ---- rigid-body deflation of stiff inclusions (gs_defl.cu) ----
struct DeflArgs {
  Geom g;             // finest level
  const int* nodes;   // unconstrained velocity nodes of every inclusion's cells, concatenated
  const int* off;     // ninc + 1 offsets into nodes
  const double* cen;  // per inclusion: centroid of all its cells' nodes (3 doubles)
  int ninc;
};
// c[k * nt + t] = projection of r on mode t of inclusion k (nt = 3 in 2D, 6 in 3D)
template <typename T>
cudaError_t launch_defl_dots(const DeflArgs& d, const T* r, double* c, cudaStream_t st);
// y = Einv c (M x M dense)
cudaError_t launch_defl_gemv(const double* Einv, int M, const double* c, double* y, cudaStream_t st);
// x += Z y
template <typename T>
cudaError_t launch_defl_add(const DeflArgs& d, const double* y, T* x, cudaStream_t st);


// ---- saddle-point multigrid with the block smoother K_j (gs_mono.cu) ----
// out[q] = diag(B diag(A)^{-1} B^T)[q] from the inverse velocity diagonal dinv (invert = 0), or its
// inverse with 0 where it vanishes (invert = 1); constrained pressure nodes give 0
template <typename T>
cudaError_t launch_schur_diag(const Geom& g, const OpCoef<double>& c, const T* dinv, T* out, int invert,
                              cudaStream_t st);
// out[0] = z . q, out[1] = q . (dsinv q) (G blocks of partial sums in part, fixed reduction order)
template <typename T>
cudaError_t launch_schur_dots(const T* z, const T* q, const T* dsinv, long long n, double* part, int G, double* out,
                              cudaStream_t st);
// a = s[0] / s[1] (0 if s[1] = 0); x_u (+)= wt + a y, x_p (+)= -a z  (zero: overwrite)
template <typename T>
cudaError_t launch_mono_update(T* xu, T* xp, const T* wt, const T* y, const T* z, const double* s, long long nu,
                               long long np, int zero, cudaStream_t st);
// ChebBiCGStab(1, 1) pieces (corrector stage): out[0] = a . b, out[1] = c . d; s = q - alpha v (in
// v) and z2 = dsinv s with alpha = s1[0] / s1[1]; the smoother update with alpha and omega = s2[0] / s2[1]
template <typename T>
cudaError_t launch_dot2(const T* a, const T* b, const T* c, const T* d, long long n, double* part, int G,
                        double* out, cudaStream_t st);
template <typename T>
cudaError_t launch_bicg_s(const T* q, T* v, const T* dsinv, T* z2, const double* s1, long long n, cudaStream_t st);
template <typename T>
cudaError_t launch_mono_update2(T* xu, T* xp, const T* wt, const T* y1, const T* y2, const T* z1, const T* z2,
                                const double* s1, const double* s2, long long nu, long long np, int zero,
                                cudaStream_t st);
template <typename T>
cudaError_t launch_mul(const T* a, const T* b, T* out, long long n, cudaStream_t st);  // out = a * b
template <typename T>
cudaError_t launch_add(const T* x, T* y, long long n, cudaStream_t st);  // y += x

}  // namespace gs
