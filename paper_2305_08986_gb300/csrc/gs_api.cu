// Host side of libgs.so: level hierarchy, setup (diagonals, Lanczos bounds, dense coarse
// inverse), the velocity V-cycle, the block-triangular preconditioner, FGMRES with CGS2, and
// the extern "C" entry points declared in include/gs.h.
//
// Every device buffer is carved out of the caller's workspace (no device allocation here);
// every launch goes to the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gs.h"
#include "gs_kernels.h"
#include "gs_slot.h"

using namespace gs;

namespace {

thread_local std::string g_err;

gs_status fail(gs_status s, const std::string& why) {
  g_err = why;
  return s;
}

#define CK(...)                                                                        \
  do {                                                                                 \
    cudaError_t e__ = (__VA_ARGS__);                                                   \
    if (e__ != cudaSuccess)                                                            \
      return fail(GS_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__)); \
  } while (0)

#define CKS(...)                               \
  do {                                         \
    gs_status s__ = (__VA_ARGS__);             \
    if (s__ != GS_OK) return s__;              \
  } while (0)

// kernel classes reported by gs_profile_read
enum KClass { K_SADDLE64 = 0, K_CHEB, K_RESID, K_BT, K_TRANSFER, K_COARSE, K_SCHUR, K_DOTS, K_AXPY, K_VEC, K_MONO,
              K_NCLASS };
const char* const kclass_name[K_NCLASS] = {"saddle_fp64", "cheb_step", "residual_A", "gradient_BT", "transfer",
                                           "coarse_solve", "schur_step", "gram_schmidt_dots", "krylov_axpy",
                                           "vector_misc", "saddle_smoother"};

struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(long long count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += (size_t)(count > 0 ? count : 1) * sizeof(T);
    return p;
  }
};

struct Level {
  int n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  long long Nv = 0, Np = 0, Nc = 0, nu = 0;
  bool has_void = false;
  std::vector<uint8_t> hvoid, hvmask, hpmask;
  std::vector<double> heta;
  std::vector<double> halpha;  // alpha per cell (when given per cell; coarse: mean of active children)
  Geom g{};
  OpCoef<double> c64{};
  OpCoef<float> c32{};
  double* eta64 = nullptr;
  float* eta32 = nullptr;
  double* alpha64 = nullptr;  // alpha per cell, or NULL (alpha then lives in the coefficients)
  float* alpha32 = nullptr;
  void* pw = nullptr;         // weights abar / alpha_K of the pressure Laplacian (MG precision), or NULL
  uint8_t *vmask = nullptr, *pmask = nullptr, *cvoid = nullptr;
  std::vector<uint16_t> hccmask;  // 2D with obstacles: per cell, constrained local nodes + obstacle bit
  uint16_t* ccmask = nullptr;
  void *xA = nullptr, *xB = nullptr, *b = nullptr, *d = nullptr, *dinv = nullptr;
  double lam_hi = 0.0;
  int* errw = nullptr;  // the context's device error word (bounded waits that gave up)
  // corrector stage (option corrector): v° on this level (injected), r_K per cell
  std::vector<double> hvc, hrk;
  double* vc64 = nullptr;
  float* vc32 = nullptr;
  double* rk64 = nullptr;
  float* rk32 = nullptr;
  float* part3 = nullptr;  // 3D: partial sums of the FP32 halo-free tiles (shared by all levels)
  int conv = 0;         // 1 while the context is in the corrector stage
  double rho = 0.0;
  // pressure Laplacian level (Cahouet-Chabard term): constraint mask, MG vectors, bound
  std::vector<uint8_t> hpc;
  uint8_t* pcmask = nullptr;
  void *pxA = nullptr, *pxB = nullptr, *pb = nullptr, *pd = nullptr, *pdinv = nullptr;
  double plam_hi = 0.0;
  double pkc[3] = {0, 0, 0};
  int shape = 0;  // 2D tile height variant of this level's multigrid kernels (TileArgs::shape)
  // saddle-point multigrid (precond_kind 1): level vectors [u | p] (iterate ms, right-hand side
  // mr, residual mres), the first Ahat solve mwt, Schur work vectors mz / mq, the inverse Schur
  // diagonal dsinv and the pressure constraint mask mpm (all zero without obstacle cells)
  void *ms = nullptr, *mr = nullptr, *mres = nullptr, *mwt = nullptr, *mz = nullptr, *mq = nullptr;
  void *my1 = nullptr, *mz2 = nullptr;  // corrector stage: the second BiCGStab direction (y1, z2)
  void* dsinv = nullptr;
  uint8_t* mpm = nullptr;
};

// State of the resumable FGMRES that the batching engine drives (see gs_slot.h).
struct KState {
  enum Phase { NONE = 0, INIT, RESID, ITER, FINAL, DONE };
  enum Pend { P_NONE = 0, P_SCALE, P_XUPDATE, P_ZERO_X };
  int phase = NONE, pend = P_NONE;
  const double* b = nullptr;
  double* x = nullptr;
  double tol = 0.0;
  bool from_conv = false, from_max = false, project_final = true;
  int it = 0, extra = 0, j = 0, kx = 0;
  double bnorm = 0.0, rel = 0.0;
  std::vector<double> H, cs, sn, g, y;
  const double* ydev = nullptr;
  gs_status result = GS_OK;
  std::string err;
  bool body_ok = false;
  Recorder body;
  const void* zu = nullptr;
  const void* zp = nullptr;
};

}  // namespace

struct gs_ctx {
  int dim = 2, L = 1;
  gs_options opt{};
  double alpha = 0.0;        // alpha, or abar = max alpha_K when alpha is given per cell
  bool alpha_cells = false;
  cudaStream_t st = nullptr;
  bool fp32 = true;
  std::vector<Level> lv;
  long long N = 0, nu = 0, np = 0;
  bool nullspace = false;
  long long n_pfree = 0;
  // Schur step vectors (finest level, MG precision)
  void *p_b = nullptr, *p_xA = nullptr, *p_xB = nullptr, *p_d = nullptr, *p_dinv = nullptr;
  // Cahouet-Chabard Schur term: allocated unless schur_kind == 1, active when cc is set
  bool cc_alloc = false, cc = false, psingular = false;
  int nfp = 0;
  std::vector<int> hpfree;
  double* PAinv = nullptr;
  int* pcfree = nullptr;
  double* pctmp = nullptr;
  // dense coarse inverse
  int nf = 0;
  std::vector<int> hfree;
  double* Ainv = nullptr;
  int* cfree = nullptr;
  double *ctmp = nullptr, *gjrow = nullptr, *gjcol = nullptr;
  int* errw = nullptr;  // device word: nonzero after a kernel's bounded wait gave up
  // saddle-point multigrid (precond_kind 1): dense coarse saddle inverse on its free unknowns
  // (velocity free entries, then free pressure entries offset by d N_v of level 0), MINRES sums,
  // finest-level right-hand side and cycle sum (mono_cycles > 1)
  bool mono = false;
  int nmf = 0;
  std::vector<int> hmfree;
  double* MAinv = nullptr;
  int* mcfree = nullptr;
  double *mctmp = nullptr, *msc = nullptr, *msc2 = nullptr;
  void *mb = nullptr, *mx = nullptr;
  // Krylov (FP64)
  double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *t1 = nullptr, *t2 = nullptr;
  double* vcur = nullptr;  // current basis vector as double (input of the preconditioner)
  int saddle_shape = 0;    // 2D tile height variant of the FP64 saddle operator
  // rigid-body deflation of stiff inclusions on the finest level (option deflate = 1)
  int defl_ninc = 0, defl_M = 0, defl_m = 0;  // inclusions, modes (ninc x nt), modes kept
  std::vector<int> hd_nodes, hd_off;
  std::vector<double> hd_cen;
  std::vector<uint8_t> hd_keep;
  int *d_nodes = nullptr, *d_off = nullptr;
  double *d_cen = nullptr, *d_Einv = nullptr, *d_c = nullptr, *d_y = nullptr;
  DeflArgs defl{};
  double* part = nullptr;
  int G = 1;   // blocks of the multi-dot partial sums
  int GA = 1;  // blocks of the fused axpy + norm (G * (m + 2) >= GA partial sums)
  int GF = 1;  // blocks of the fused CGS2 update + dots (one wave, 4 CTAs per SM)
  double* dsc = nullptr;
  double* gram = nullptr;  // orth = 2: G = V^T V of the current restart cycle, (m + 1) x (m + 1)
  double* gsc = nullptr;   // orth = 2: [V^T w ; V^T v_j], 2 (m + 2) values
  double* hpin = nullptr;
  int last_it = 0;
  double last_rel = 0.0;
  size_t footprint = 0;
  // CUDA graph of the preconditioner body (captured on cap_st at the second application)
  cudaStream_t cap_st = nullptr;
  cudaGraphExec_t pgraph = nullptr;
  const void* g_zu = nullptr;
  const void* g_zp = nullptr;
  long long pcalls = 0;
  int pgraph_kernels = 0;
  // optional per-kernel-class timing (CUDA event pairs on the context stream)
  bool prof = false;
  std::vector<cudaEvent_t> evs;
  size_t ev_used = 0;
  struct ProfRec {
    int cls;
    int level;  // multigrid level of the launch (-1: not tied to a level)
    size_t ev;
  };
  std::vector<ProfRec> recs;
  int prof_lv = -1;  // level tag of the launches being enqueued
  // batching engine state
  KState ks;
};

namespace {

long prof_begin(gs_ctx* c, int cls) {
  if (!c->prof) return -1;
  if (c->ev_used + 2 > c->evs.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { c->prof = false; return -1; }
      c->evs.push_back(e);
    }
  }
  const size_t i = c->ev_used;
  c->ev_used += 2;
  cudaEventRecord(c->evs[i], c->st);
  c->recs.push_back({cls, c->prof_lv, i});
  return (long)i;
}
void prof_end(gs_ctx* c, long i) {
  if (i >= 0) cudaEventRecord(c->evs[(size_t)i + 1], c->st);
}

// Tags the launches enqueued while it lives with multigrid level l (profiling only).
struct LevelTag {
  gs_ctx* c;
  int old;
  LevelTag(gs_ctx* cc, int l) : c(cc), old(cc->prof_lv) { c->prof_lv = l; }
  ~LevelTag() { c->prof_lv = old; }
};

#define KL(cls, ...)                      \
  do {                                    \
    const long p__ = prof_begin(c, cls);  \
    CK(__VA_ARGS__);                      \
    prof_end(c, p__);                     \
  } while (0)

int opt_or(int v, int d) { return v > 0 ? v : d; }

const double kReorthKappa = 0.70710678118654752440;  // 1/sqrt(2)

gs_options normalize_opts(const gs_options* o) {
  gs_options r{};
  if (o) r = *o;
  r.cheb_degree = opt_or(r.cheb_degree, 4);
  r.smooth_steps = opt_or(r.smooth_steps, 1);
  r.restart = opt_or(r.restart, 50);
  r.max_iter = opt_or(r.max_iter, 1000);
  r.mg_precision = (r.mg_precision == 64) ? 64 : 32;
  r.schur_degree = opt_or(r.schur_degree, 4);
  r.lanczos_steps = opt_or(r.lanczos_steps, 12);
  r.coarse_mode = r.coarse_mode == 1 ? 1 : 0;
  r.schur_kind = (r.schur_kind == 1 || r.schur_kind == 2) ? r.schur_kind : 0;
  // public 0 / 2 -> Gram-matrix CGS2 (internal 2), 1 -> selective (1), 3 -> explicit CGS2 (internal 0)
  r.orth = r.orth == 1 ? 1 : (r.orth == 3 ? 0 : 2);
  r.graphs = r.graphs == 1 ? 1 : 0;
  r.plap_degree = opt_or(r.plap_degree, 2);
  // 0 (default) and 1: IEEE FP64 basis; 2: double-float basis (stored internally as 0 / 1 = double-float / FP64)
  r.krylov_fp64 = r.krylov_fp64 == 2 ? 0 : 1;
  r.tile_autotune = (r.tile_autotune >= 1 && r.tile_autotune <= 5) ? r.tile_autotune : 0;
  r.corrector = r.corrector == 1 ? 1 : 0;
  r.deflate = r.deflate == 1 ? 1 : 0;
  r.precond_kind = r.precond_kind == 1 ? 1 : 0;
  r.mono_smooth = opt_or(r.mono_smooth, 2);
  r.mono_cycles = opt_or(r.mono_cycles, 1);
  return r;
}

template <typename T>
OpCoef<T> make_coef(int dim, const double* h, double alpha) {
  OpCoef<T> c{};
  if (dim == 2) {
    const double hx = h[0], hy = h[1];
    c.mm = (T)(alpha * hx * hy / 900.0);
    c.km[0] = (T)(hy / (90.0 * hx));
    c.km[1] = (T)(hx / (90.0 * hy));
    c.km[2] = 0;
    c.ex[0] = c.ex[1] = c.ex[2] = (T)(1.0 / 36.0);
    c.bd[0] = (T)(hy / 36.0);
    c.bd[1] = (T)(hx / 36.0);
    c.bd[2] = 0;
    c.pm = (T)(hx * hy / 36.0);
  } else {
    const double hx = h[0], hy = h[1], hz = h[2];
    c.mm = (T)(alpha * hx * hy * hz / 27000.0);
    c.km[0] = (T)(hy * hz / (2700.0 * hx));
    c.km[1] = (T)(hx * hz / (2700.0 * hy));
    c.km[2] = (T)(hx * hy / (2700.0 * hz));
    c.ex[0] = (T)(hx / 1080.0);
    c.ex[1] = (T)(hy / 1080.0);
    c.ex[2] = (T)(hz / 1080.0);
    c.bd[0] = (T)(hy * hz / 216.0);
    c.bd[1] = (T)(hx * hz / 216.0);
    c.bd[2] = (T)(hx * hy / 216.0);
    c.pm = (T)(hx * hy * hz / 216.0);
  }
  c.eta_scale = (T)1;
  return c;
}

// inclusions whose rigid motions the deflation space can hold (workspace capacity)
const int kDeflMaxInclusions = 256;
gs_status plan_deflation(gs_ctx* c, const gs_mesh* m);

// ---- host planning: level sizes, obstacle flags, constraint masks, coarse eta -----------------
gs_status plan(const gs_mesh* m, int L, const double* eta, gs_ctx* c, const double* alpha_cells = nullptr) {
  if (!m) return fail(GS_EINVAL, "mesh is NULL");
  if (m->dim != 2 && m->dim != 3) return fail(GS_EINVAL, "dim must be 2 or 3");
  if (L < 1 || L > 16) return fail(GS_EINVAL, "levels must be in [1, 16]");
  const int dim = m->dim;
  for (int a = 0; a < dim; ++a) {
    if (m->n[a] < 1) return fail(GS_EINVAL, "cells per axis must be >= 1");
    if (!(m->len[a] > 0.0)) return fail(GS_EINVAL, "domain extent must be > 0");
    if (m->n[a] % (1 << (L - 1)) != 0)
      return fail(GS_EINVAL, "cells per axis must be divisible by 2^(levels-1)");
    if (m->n[a] > (1 << 24)) return fail(GS_EINVAL, "mesh too large");
  }
  c->dim = dim;
  c->L = L;
  c->lv.assign(L, Level());
  for (int l = L - 1; l >= 0; --l) {
    Level& lv = c->lv[l];
    for (int a = 0; a < 3; ++a) {
      lv.n[a] = a < dim ? (m->n[a] >> (L - 1 - l)) : 1;
      lv.h[a] = a < dim ? m->len[a] / lv.n[a] : 1.0;
    }
    lv.Nc = (long long)lv.n[0] * lv.n[1] * lv.n[2];
    lv.Nv = (long long)(2 * lv.n[0] + 1) * (2 * lv.n[1] + 1) * (dim == 3 ? 2 * lv.n[2] + 1 : 1);
    lv.Np = (long long)(lv.n[0] + 1) * (lv.n[1] + 1) * (dim == 3 ? lv.n[2] + 1 : 1);
    lv.nu = dim * lv.Nv;
  }
  // obstacle flags and eta per level (finest from input; coarse: all children void / mean of active)
  Level& F = c->lv[L - 1];
  F.hvoid.assign(F.Nc, 0);
  bool any_void = false;
  if (m->cell_void) {
    for (long long i = 0; i < F.Nc; ++i) {
      F.hvoid[i] = m->cell_void[i] ? 1 : 0;
      any_void |= F.hvoid[i] != 0;
    }
  }
  if (eta) {
    F.heta.assign(eta, eta + F.Nc);
    if (alpha_cells) {
      F.halpha.assign(alpha_cells, alpha_cells + F.Nc);
      double amax = 0.0;
      for (long long i = 0; i < F.Nc; ++i) {
        if (F.hvoid[i]) continue;
        if (!(std::isfinite(alpha_cells[i]) && alpha_cells[i] >= 0.0))
          return fail(GS_EINVAL, "alpha must be finite and >= 0 on active cells");
        amax = std::max(amax, alpha_cells[i]);
      }
      c->alpha = amax;
    }
    for (long long i = 0; i < F.Nc; ++i)
      if (!(std::isfinite(eta[i]) && eta[i] > 0.0) && !F.hvoid[i])
        return fail(GS_EINVAL, "eta must be positive and finite on active cells");
  }
  for (int l = L - 2; l >= 0; --l) {
    Level& C = c->lv[l];
    const Level& Fi = c->lv[l + 1];
    C.hvoid.assign(C.Nc, 0);
    if (eta) C.heta.assign(C.Nc, 1.0);
    const bool pa = !Fi.halpha.empty();
    if (pa) C.halpha.assign(C.Nc, 0.0);
    for (int k = 0; k < C.n[2]; ++k)
      for (int j = 0; j < C.n[1]; ++j)
        for (int i = 0; i < C.n[0]; ++i) {
          const long long cc = i + (long long)C.n[0] * (j + (long long)C.n[1] * k);
          int nact = 0, nch = 0;
          double s = 0.0, sa = 0.0;
          for (int dk = 0; dk < (dim == 3 ? 2 : 1); ++dk)
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di) {
                const long long fc = (2 * i + di) + (long long)Fi.n[0] * ((2 * j + dj) + (long long)Fi.n[1] * (dim == 3 ? 2 * k + dk : 0));
                nch++;
                if (!Fi.hvoid[fc]) {
                  nact++;
                  if (eta) s += Fi.heta[fc];
                  if (pa) sa += Fi.halpha[fc];
                }
              }
          C.hvoid[cc] = (nact == 0) ? 1 : 0;
          if (eta && nact > 0) C.heta[cc] = s / nact;
          if (pa && nact > 0) C.halpha[cc] = sa / nact;
          (void)nch;
        }
  }
  for (int l = 0; l < L; ++l) {
    Level& lv = c->lv[l];
    lv.has_void = any_void;
    if (!any_void) continue;
    const int nv0 = 2 * lv.n[0] + 1, nv1 = 2 * lv.n[1] + 1, nv2 = dim == 3 ? 2 * lv.n[2] + 1 : 1;
    lv.hvmask.assign(lv.Nv, 0);
    Geom gtmp{};
    gtmp.dim = dim;
    gtmp.faces = m->dirichlet_faces;
    gtmp.nv[0] = nv0; gtmp.nv[1] = nv1; gtmp.nv[2] = nv2;
    for (int K = 0; K < nv2; ++K)
      for (int J = 0; J < nv1; ++J)
        for (int I = 0; I < nv0; ++I)
          if (face_constrained(gtmp, I, J, K)) lv.hvmask[I + (long long)nv0 * (J + (long long)nv1 * K)] = 1;
    for (int k = 0; k < lv.n[2]; ++k)
      for (int j = 0; j < lv.n[1]; ++j)
        for (int i = 0; i < lv.n[0]; ++i) {
          const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
          if (!lv.hvoid[cc]) continue;
          for (int lc = 0; lc < (dim == 3 ? 3 : 1); ++lc)
            for (int lb = 0; lb < 3; ++lb)
              for (int la = 0; la < 3; ++la)
                lv.hvmask[(2 * i + la) + (long long)nv0 * ((2 * j + lb) + (long long)nv1 * (dim == 3 ? 2 * k + lc : 0))] = 1;
        }
    {
      const int np0 = lv.n[0] + 1, np1 = lv.n[1] + 1;
      lv.hpmask.assign(lv.Np, 1);
      for (int k = 0; k < lv.n[2]; ++k)
        for (int j = 0; j < lv.n[1]; ++j)
          for (int i = 0; i < lv.n[0]; ++i) {
            const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
            if (lv.hvoid[cc]) continue;
            for (int lc = 0; lc < (dim == 3 ? 2 : 1); ++lc)
              for (int lb = 0; lb < 2; ++lb)
                for (int la = 0; la < 2; ++la)
                  lv.hpmask[(i + la) + (long long)np0 * ((j + lb) + (long long)np1 * (dim == 3 ? k + lc : 0))] = 0;
          }
    }
  }
  // free unknowns of the coarse level
  Level& C0 = c->lv[0];
  c->hfree.clear();
  if (c->opt.coarse_mode != 1) {
    Geom gtmp{};
    gtmp.dim = dim;
    gtmp.faces = m->dirichlet_faces;
    gtmp.nv[0] = 2 * C0.n[0] + 1; gtmp.nv[1] = 2 * C0.n[1] + 1; gtmp.nv[2] = dim == 3 ? 2 * C0.n[2] + 1 : 1;
    for (int a = 0; a < dim; ++a)
      for (long long node = 0; node < C0.Nv; ++node) {
        const int I = (int)(node % gtmp.nv[0]);
        const int J = (int)((node / gtmp.nv[0]) % gtmp.nv[1]);
        const int K = (int)(node / ((long long)gtmp.nv[0] * gtmp.nv[1]));
        const bool con = C0.has_void ? C0.hvmask[node] != 0 : face_constrained(gtmp, I, J, K);
        if (!con) c->hfree.push_back((int)(a * C0.Nv + node));
      }
  }
  c->nf = (int)c->hfree.size();
  if ((long long)c->nf * c->nf > (1LL << 31)) return fail(GS_EINVAL, "coarsest level too large for the dense solve; use more levels");
  const Level& Fl = c->lv[L - 1];
  c->nu = Fl.nu;
  c->np = Fl.Np;
  c->N = Fl.nu + Fl.Np;
  c->nullspace = m->dirichlet_faces == ((1u << (2 * dim)) - 1u);
  c->n_pfree = Fl.Np;
  if (Fl.has_void) {
    c->n_pfree = 0;
    for (auto v : Fl.hpmask) c->n_pfree += v ? 0 : 1;
  }
  // saddle-point multigrid: free unknowns of the dense coarse saddle solve
  c->mono = c->opt.precond_kind == 1;
  c->hmfree.clear();
  if (c->mono && c->opt.deflate == 1) return fail(GS_EINVAL, "deflation applies to the block-triangular preconditioner");
  if (c->opt.corrector && c->opt.deflate == 1)
    return fail(GS_EINVAL, "the corrector stage is built without deflation");
  if (c->mono && c->opt.coarse_mode != 1) {
    c->hmfree = c->hfree;
    for (long long q = 0; q < C0.Np; ++q)
      if (!(C0.has_void && C0.hpmask[q])) c->hmfree.push_back((int)(C0.nu + q));
  }
  c->nmf = (int)c->hmfree.size();
  if ((long long)c->nmf * c->nmf > (1LL << 31)) return fail(GS_EINVAL, "coarsest level too large for the dense saddle solve");
  // pressure Laplacian of the Cahouet-Chabard term: p = 0 on pressure nodes touched by no active
  // cell and on faces without a velocity Dirichlet condition; pure Neumann if every face is
  // Dirichlet (then singular with the constant in its kernel)
  c->cc_alloc = c->opt.schur_kind != 1;
  c->hpfree.clear();
  c->nfp = 0;
  c->psingular = c->nullspace;
  if (c->cc_alloc) {
    for (int l = 0; l < L; ++l) {
      Level& lv = c->lv[l];
      const int np0 = lv.n[0] + 1, np1 = lv.n[1] + 1, np2 = dim == 3 ? lv.n[2] + 1 : 1;
      lv.hpc.assign(lv.Np, 1);
      for (int k = 0; k < lv.n[2]; ++k)
        for (int j = 0; j < lv.n[1]; ++j)
          for (int i = 0; i < lv.n[0]; ++i) {
            const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
            if (lv.hvoid[cc]) continue;
            for (int lc = 0; lc < (dim == 3 ? 2 : 1); ++lc)
              for (int lb = 0; lb < 2; ++lb)
                for (int la = 0; la < 2; ++la)
                  lv.hpc[(i + la) + (long long)np0 * ((j + lb) + (long long)np1 * (dim == 3 ? k + lc : 0))] = 0;
          }
      const int npa[3] = {np0, np1, np2};
      for (long long q = 0; q < lv.Np; ++q) {
        const int idx[3] = {(int)(q % np0), (int)((q / np0) % np1), (int)(q / ((long long)np0 * np1))};
        for (int a = 0; a < dim; ++a) {
          if (!(m->dirichlet_faces & (1u << (2 * a))) && idx[a] == 0) lv.hpc[q] = 1;
          if (!(m->dirichlet_faces & (1u << (2 * a + 1))) && idx[a] == npa[a] - 1) lv.hpc[q] = 1;
        }
      }
    }
    if (c->opt.coarse_mode != 1)
      for (long long q = 0; q < c->lv[0].Np; ++q)
        if (!c->lv[0].hpc[q]) c->hpfree.push_back((int)q);
    c->nfp = (int)c->hpfree.size();
    if ((long long)c->nfp * c->nfp > (1LL << 31)) return fail(GS_EINVAL, "coarsest pressure level too large");
  }
  CKS(plan_deflation(c, m));
  return GS_OK;
}

// ---- rigid-body deflation of stiff inclusions (finest level; kernels in gs_defl.cu) --------------
// Stiff cells: active cells with eta >= sqrt(eta_min eta_max), only when eta_max >= 1e3 eta_min;
// inclusions: connected components of stiff cells sharing a velocity node, numbered in the order
// of their first cell; per inclusion the sorted unconstrained nodes of its cells, the centroid of
// all its cells' nodes, and which of its rigid modes do not vanish on the unconstrained nodes.
gs_status plan_deflation(gs_ctx* c, const gs_mesh* m) {
  c->hd_nodes.clear();
  c->hd_off.assign(1, 0);
  c->hd_cen.clear();
  c->hd_keep.clear();
  c->defl_ninc = c->defl_M = c->defl_m = 0;
  if (c->opt.deflate != 1) return GS_OK;
  const Level& F = c->lv[c->L - 1];
  const int dim = c->dim, nt = dim == 2 ? 3 : 6;
  if (F.Nv >= (1LL << 31)) return fail(GS_EINVAL, "deflation: mesh too large for 32-bit node lists");
  if (F.heta.empty()) return GS_OK;
  double lo = INFINITY, hi = 0.0;
  for (long long i = 0; i < F.Nc; ++i)
    if (!F.hvoid[i]) { lo = std::fmin(lo, F.heta[i]); hi = std::fmax(hi, F.heta[i]); }
  if (!(hi >= 1e3 * lo)) return GS_OK;
  const double thr = std::sqrt(lo * hi);
  auto stiff = [&](long long i) { return !F.hvoid[i] && F.heta[i] >= thr; };
  const int n0 = F.n[0], n1 = F.n[1], n2 = F.n[2];
  std::vector<int> lab(F.Nc, 0);
  std::vector<std::vector<long long>> cells;
  std::vector<long long> stack;
  for (long long c0 = 0; c0 < F.Nc; ++c0) {
    if (!stiff(c0) || lab[c0]) continue;
    cells.emplace_back();
    const int id = (int)cells.size();
    lab[c0] = id;
    stack.assign(1, c0);
    while (!stack.empty()) {
      const long long cc = stack.back();
      stack.pop_back();
      cells.back().push_back(cc);
      const int i = (int)(cc % n0), j = (int)((cc / n0) % n1), k = (int)(cc / ((long long)n0 * n1));
      for (int dk = (dim == 3 ? -1 : 0); dk <= (dim == 3 ? 1 : 0); ++dk)
        for (int dj = -1; dj <= 1; ++dj)
          for (int di = -1; di <= 1; ++di) {
            const int a = i + di, b = j + dj, e = k + dk;
            if (a < 0 || a >= n0 || b < 0 || b >= n1 || e < 0 || e >= n2) continue;
            const long long cn = a + (long long)n0 * (b + (long long)n1 * e);
            if (stiff(cn) && !lab[cn]) { lab[cn] = id; stack.push_back(cn); }
          }
    }
  }
  const int nv0 = 2 * n0 + 1, nv1 = 2 * n1 + 1;
  Geom gt{};
  gt.dim = dim;
  gt.faces = m->dirichlet_faces;
  gt.nv[0] = nv0; gt.nv[1] = nv1; gt.nv[2] = dim == 3 ? 2 * n2 + 1 : 1;
  std::vector<int> stamp(F.Nv, 0);
  for (size_t q = 0; q < cells.size(); ++q) {
    std::vector<int> nodes;
    for (long long cc : cells[q]) {
      const int i = (int)(cc % n0), j = (int)((cc / n0) % n1), k = (int)(cc / ((long long)n0 * n1));
      for (int lc = 0; lc < (dim == 3 ? 3 : 1); ++lc)
        for (int lb = 0; lb < 3; ++lb)
          for (int la = 0; la < 3; ++la) {
            const long long nd = (2 * i + la) + (long long)nv0 * ((2 * j + lb) + (long long)nv1 * (dim == 3 ? 2 * k + lc : 0));
            if (stamp[nd] != (int)q + 1) { stamp[nd] = (int)q + 1; nodes.push_back((int)nd); }
          }
    }
    std::sort(nodes.begin(), nodes.end());
    double cen[3] = {0, 0, 0};
    for (int nd : nodes) {
      cen[0] += (nd % nv0) * (0.5 * F.h[0]);
      cen[1] += ((nd / nv0) % nv1) * (0.5 * F.h[1]);
      if (dim == 3) cen[2] += (nd / ((long long)nv0 * nv1)) * (0.5 * F.h[2]);
    }
    for (int a = 0; a < 3; ++a) cen[a] /= (double)nodes.size();
    double norm2[6] = {0, 0, 0, 0, 0, 0};
    for (int nd : nodes) {
      const int I = nd % nv0, J = (nd / nv0) % nv1, K = dim == 3 ? (int)(nd / ((long long)nv0 * nv1)) : 0;
      const bool con = F.has_void ? F.hvmask[nd] != 0 : face_constrained(gt, I, J, K);
      if (con) continue;
      c->hd_nodes.push_back(nd);
      const double dx = I * (0.5 * F.h[0]) - cen[0], dy = J * (0.5 * F.h[1]) - cen[1];
      const double dz = dim == 3 ? K * (0.5 * F.h[2]) - cen[2] : 0.0;
      for (int a = 0; a < dim; ++a) norm2[a] += 1.0;
      if (dim == 2) {
        norm2[2] += dx * dx + dy * dy;
      } else {
        norm2[3] += dy * dy + dz * dz;
        norm2[4] += dx * dx + dz * dz;
        norm2[5] += dx * dx + dy * dy;
      }
    }
    c->hd_off.push_back((int)c->hd_nodes.size());
    for (int a = 0; a < 3; ++a) c->hd_cen.push_back(cen[a]);
    for (int t = 0; t < nt; ++t) {
      c->hd_keep.push_back(norm2[t] > 0.0 ? 1 : 0);
      c->defl_m += norm2[t] > 0.0 ? 1 : 0;
    }
  }
  c->defl_ninc = (int)cells.size();
  c->defl_M = c->defl_ninc * nt;
  if (c->defl_ninc > kDeflMaxInclusions)
    return fail(GS_EINVAL, "deflation: more than " + std::to_string(kDeflMaxInclusions) + " stiff inclusions");
  return GS_OK;
}

// ---- device layout (dry run when ar.base == nullptr) -------------------------------------------
void layout(gs_ctx* c, Arena& ar) {
  const size_t S = c->fp32 ? 4 : 8;
  auto takeT = [&](long long n) -> void* { return S == 4 ? (void*)ar.take<float>(n) : (void*)ar.take<double>(n); };
  for (int l = 0; l < c->L; ++l) {
    Level& lv = c->lv[l];
    lv.eta64 = ar.take<double>(lv.Nc);
    lv.eta32 = ar.take<float>(lv.Nc);
    // alpha per cell (used only when gs_create_ex gets one; reserved always so that the
    // footprint does not depend on it: 12 bytes per cell)
    double* a64 = ar.take<double>(lv.Nc);
    float* a32 = ar.take<float>(lv.Nc);
    lv.alpha64 = c->alpha_cells ? a64 : nullptr;
    lv.alpha32 = c->alpha_cells ? a32 : nullptr;
    if (lv.has_void) {
      lv.cvoid = ar.take<uint8_t>(lv.Nc);
      lv.vmask = ar.take<uint8_t>(lv.Nv);
      lv.pmask = ar.take<uint8_t>(lv.Np);
      if (c->dim == 2) lv.ccmask = ar.take<uint16_t>(lv.Nc);
    }
    if (c->opt.corrector) {  // both precisions: FP32 applies are allowed on an FP64-multigrid context
      lv.vc64 = ar.take<double>(lv.nu);
      lv.rk64 = ar.take<double>(lv.Nc);
      lv.vc32 = ar.take<float>(lv.nu);
      lv.rk32 = ar.take<float>(lv.Nc);
    }
    lv.xA = takeT(lv.nu);
    lv.xB = takeT(lv.nu);
    lv.b = takeT(lv.nu);
    lv.d = takeT(lv.nu);
    lv.dinv = takeT(lv.nu);
  }
  const Level& F = c->lv[c->L - 1];
  c->p_b = takeT(F.Np);
  c->p_xA = takeT(F.Np);
  c->p_xB = takeT(F.Np);
  c->p_d = takeT(F.Np);
  c->p_dinv = takeT(F.Np);
  c->Ainv = ar.take<double>((long long)c->nf * c->nf);
  c->cfree = ar.take<int>(c->nf);
  c->ctmp = ar.take<double>(c->nf);
  c->errw = ar.take<int>(4);
  for (int l = 0; l < c->L; ++l) c->lv[l].errw = c->errw;
  if (c->dim == 3) {  // partial sums of the FP32 halo-free tiles: the finest level needs the most
    long long mx = 0;
    for (int l = 0; l < c->L; ++l) mx = std::max(mx, nh3_part_elems(c->lv[l].n));
    float* p3 = ar.take<float>(mx);
    for (int l = 0; l < c->L; ++l) c->lv[l].part3 = p3;
  }
  const int gjn = std::max(c->nf, std::max(c->nfp, c->nmf));
  c->gjrow = ar.take<double>(gjn);
  c->gjcol = ar.take<double>(gjn);
  if (c->cc_alloc) {
    for (int l = 0; l < c->L; ++l) {
      Level& lv = c->lv[l];
      lv.pcmask = ar.take<uint8_t>(lv.Np);
      void* pw = takeT(lv.Nc);
      lv.pw = c->alpha_cells ? pw : nullptr;
      lv.pxA = takeT(lv.Np);
      lv.pxB = takeT(lv.Np);
      lv.pb = takeT(lv.Np);
      lv.pd = takeT(lv.Np);
      lv.pdinv = takeT(lv.Np);
    }
    c->PAinv = ar.take<double>((long long)c->nfp * c->nfp);
    c->pcfree = ar.take<int>(c->nfp);
    c->pctmp = ar.take<double>(c->nfp);
  }
  if (c->mono) {
    for (int l = 0; l < c->L; ++l) {
      Level& lv = c->lv[l];
      lv.ms = takeT(lv.nu + lv.Np);
      lv.mr = takeT(lv.nu + lv.Np);
      lv.mres = takeT(lv.nu + lv.Np);
      lv.mwt = takeT(lv.nu);
      lv.mz = takeT(lv.Np);
      lv.mq = takeT(lv.Np);
      lv.dsinv = takeT(lv.Np);
      lv.mpm = ar.take<uint8_t>(lv.Np);
      if (c->opt.corrector) {
        lv.my1 = takeT(lv.nu);
        lv.mz2 = takeT(lv.Np);
      }
    }
    c->MAinv = ar.take<double>((long long)c->nmf * c->nmf);
    c->mcfree = ar.take<int>(c->nmf);
    c->mctmp = ar.take<double>(c->nmf);
    c->msc = ar.take<double>(2);
    c->msc2 = ar.take<double>(2);
    if (c->opt.mono_cycles > 1) {
      c->mb = takeT(F.nu + F.Np);
      c->mx = takeT(F.nu + F.Np);
    }
  }
  if (c->opt.deflate == 1) {  // capacity: every node, kDeflMaxInclusions inclusions
    const int Mmax = kDeflMaxInclusions * (c->dim == 2 ? 3 : 6);
    c->d_nodes = ar.take<int>(c->lv[c->L - 1].Nv);
    c->d_off = ar.take<int>(kDeflMaxInclusions + 1);
    c->d_cen = ar.take<double>(3LL * kDeflMaxInclusions);
    c->d_Einv = ar.take<double>((long long)Mmax * Mmax);
    c->d_c = ar.take<double>(Mmax);
    c->d_y = ar.take<double>(Mmax);
  }
  const int m = c->opt.restart;
  c->V = ar.take<double>((long long)(m + 1) * c->N);
  c->Z = ar.take<double>((long long)m * c->N);
  c->w = ar.take<double>(c->N);
  c->r = ar.take<double>(c->N);
  c->t1 = ar.take<double>(c->N);
  c->t2 = ar.take<double>(c->N);
  c->vcur = ar.take<double>(c->N);
  long long G = (c->N + 4095) / 4096;
  if (G > 152 * 3) G = 152 * 3;  // three resident CTAs per SM for the multi-dot
  if (G < 1) G = 1;
  c->G = (int)G;
  long long GA = (c->N + 1023) / 1024;
  if (GA > 152 * 16) GA = 152 * 16;
  if (GA > (long long)c->G * (m + 2)) GA = (long long)c->G * (m + 2);
  if (GA < 1) GA = 1;
  c->GA = (int)GA;
  long long GF = (c->N + 2047) / 2048;  // strips of 256 elements, at least 8 per block
  if (GF > 4 * 152) GF = 4 * 152;
  if (GF < 1) GF = 1;
  c->GF = (int)GF;
  // partial-sum rows: m + 2 dots, or both dot blocks of orth = 2 (2 k rows, k <= m + 1)
  const int prow = std::max(m + 2, 2 * (m + 1) + 2);
  c->part = ar.take<double>((long long)std::max(c->G, c->GF) * prow);
  c->dsc = ar.take<double>(4 * (m + 4));
  c->gram = ar.take<double>((long long)(m + 1) * (m + 1));
  c->gsc = ar.take<double>(2 * (m + 2));
  c->footprint = ar.off + 256;
}

void set_geom(gs_ctx* c, const gs_mesh* m) {
  for (int l = 0; l < c->L; ++l) {
    Level& lv = c->lv[l];
    Geom& g = lv.g;
    g.dim = c->dim;
    for (int a = 0; a < 3; ++a) {
      g.n[a] = lv.n[a];
      g.nv[a] = a < c->dim ? 2 * lv.n[a] + 1 : 1;
      g.npn[a] = a < c->dim ? lv.n[a] + 1 : 1;
      g.h[a] = lv.h[a];
    }
    g.Nv = lv.Nv;
    g.Np = lv.Np;
    g.Nc = lv.Nc;
    g.faces = m->dirichlet_faces;
    g.vmask = lv.vmask;
    g.pmask = lv.pmask;
    g.cvoid = lv.cvoid;
    g.ccmask = lv.ccmask;
    // alpha per cell: the coefficients carry alpha = 1 and the kernels multiply by alpha_K
    lv.c64 = make_coef<double>(c->dim, lv.h, c->alpha_cells ? 1.0 : c->alpha);
    lv.c32 = make_coef<float>(c->dim, lv.h, c->alpha_cells ? 1.0 : c->alpha);
    // Q1 stiffness coefficients kc[a] = prod_{b != a} h_b / (6^(d-1) h_a)
    for (int a = 0; a < 3; ++a) {
      if (a >= c->dim) { lv.pkc[a] = 0.0; continue; }
      double v = 1.0 / lv.h[a];
      for (int b = 0; b < c->dim; ++b)
        if (b != a) v *= lv.h[b] / 6.0;
      lv.pkc[a] = v;
    }
  }
}

// ---- small helpers ----------------------------------------------------------------------------
template <typename T>
OpCoef<T> coef(const Level& lv);
template <>
OpCoef<double> coef<double>(const Level& lv) { return lv.c64; }
template <>
OpCoef<float> coef<float>(const Level& lv) { return lv.c32; }
template <typename T>
const T* etap(const Level& lv);
template <>
const double* etap<double>(const Level& lv) { return lv.eta64; }
template <>
const float* etap<float>(const Level& lv) { return lv.eta32; }

template <typename T>
const T* alphap(const Level& lv);
template <>
const double* alphap<double>(const Level& lv) { return lv.alpha64; }
template <>
const float* alphap<float>(const Level& lv) { return lv.alpha32; }

template <typename T>
TileArgs<T> tile_args(const Level& lv) {
  TileArgs<T> a{};
  a.g = lv.g;
  a.c = coef<T>(lv);
  a.eta = etap<T>(lv);
  a.alpha = alphap<T>(lv);
  a.shape = lv.shape;
  a.err = lv.errw;
  if (sizeof(T) == 4 && lv.g.dim == 3) a.part = (T*)lv.part3;
  if (lv.conv) {
    a.conv = 1;
    a.vc = sizeof(T) == 8 ? (const T*)lv.vc64 : (const T*)lv.vc32;
    a.rk = sizeof(T) == 8 ? (const T*)lv.rk64 : (const T*)lv.rk32;
    a.rho = (T)lv.rho;
    a.ihx = (T)(1.0 / lv.h[0]);
    a.ihy = (T)(1.0 / lv.h[1]);
    a.ihz = (T)(1.0 / lv.h[2]);
    a.wq = (T)(lv.g.dim == 3 ? lv.h[0] * lv.h[1] * lv.h[2] : lv.h[0] * lv.h[1]);
  }
  return a;
}

// Report (and clear) a bounded wait that gave up in any kernel since the last check.
gs_status check_device_error(gs_ctx* c) {
  if (!c->errw) return GS_OK;
  int* h = reinterpret_cast<int*>(c->hpin);
  CK(cudaMemcpyAsync(h, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (*h != 0) {
    CK(cudaMemsetAsync(c->errw, 0, sizeof(int), c->st));
    return fail(GS_ETIMEOUT, "a kernel's wait for its staged data gave up after about a second");
  }
  return GS_OK;
}

// dot products of T vectors accumulated in FP64, result copied to host
template <typename T>
gs_status dot_host(gs_ctx* c, const T* V, long long ldv, int k, const T* w, long long n, double* out) {
  KL(K_DOTS, launch_dots_partial<T>(V, ldv, k, w, n, c->part, c->G, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, k, c->G, c->dsc, c->st));
  CK(cudaMemcpyAsync(c->hpin, c->dsc, sizeof(double) * k, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i < k; ++i) out[i] = c->hpin[i];
  return GS_OK;
}

// largest eigenvalue of the symmetric tridiagonal matrix (a, b) by Sturm-sequence bisection
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int k = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0) cnt++;
    for (int i = 1; i < k; ++i) {
      if (q == 0.0) q = 1e-300;
      q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
      if (q < 0) cnt++;
    }
    return cnt;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) >= k) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Lanczos estimate of lambda_max(D^{-1} M) for a level operator M (Sec. 4 Chebyshev bounds):
// `steps` Lanczos steps on D^{-1/2} M D^{-1/2} from a SplitMix64 start vector whose 64-bit
// counter is (seed << 32) ^ (level_code << 56) ^ i; constrained entries are zeroed.
template <typename T, typename ZeroFn, typename ApplyFn>
gs_status lanczos_core(gs_ctx* c, long long n, int level_code, T* v, T* vprev, T* t, T* w, const T* dinv,
                       ZeroFn zero, ApplyFn apply, double* lam) {
  std::vector<T> h0(n);
  const uint64_t base = ((uint64_t)((uint32_t)c->opt.seed) << 32) ^ ((uint64_t)(level_code & 0xFF) << 56);
  for (long long i = 0; i < n; ++i) {
    const uint64_t r = splitmix64(base ^ (uint64_t)i);
    h0[i] = (T)(2.0 * ((double)(r >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
  }
  CK(cudaMemcpyAsync(v, h0.data(), sizeof(T) * n, cudaMemcpyHostToDevice, c->st));
  CK(zero(v));
  double nrm2;
  CKS(dot_host<T>(c, v, n, 1, v, n, &nrm2));
  CK(launch_cast<T, T>(v, v, n, (T)(1.0 / std::sqrt(nrm2)), c->st));
  CK(cudaMemsetAsync(vprev, 0, sizeof(T) * n, c->st));
  std::vector<double> al, be;
  double beta_prev = 0.0;
  for (int j = 0; j < c->opt.lanczos_steps; ++j) {
    CK(launch_lanczos_pre<T>(dinv, v, t, n, c->st));
    CK(apply((const T*)t, w));
    CK(launch_lanczos_post<T>(dinv, w, vprev, (T)beta_prev, w, n, c->st));
    double alpha;
    CKS(dot_host<T>(c, w, n, 1, v, n, &alpha));
    CK(launch_axpby<T>(v, w, (T)(-alpha), (T)1, n, c->st));
    double bb;
    CKS(dot_host<T>(c, w, n, 1, w, n, &bb));
    const double beta = std::sqrt(bb);
    al.push_back(alpha);
    if (j == c->opt.lanczos_steps - 1 || beta == 0.0) break;
    be.push_back(beta);
    // vprev <- v ; v <- w / beta
    CK(launch_cast<T, T>(w, vprev, n, (T)(1.0 / beta), c->st));
    std::swap(v, vprev);
    beta_prev = beta;
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  *lam = 1.2 * tridiag_max_eig(al, be);
  if (!std::isfinite(*lam) || *lam <= 0.0) return fail(GS_EBREAKDOWN, "eigenvalue estimate failed");
  return GS_OK;
}

template <typename T>
gs_status lanczos(gs_ctx* c, int l) {
  Level& lv = c->lv[l];
  return lanczos_core<T>(
      c, lv.nu, l, (T*)lv.xA, (T*)lv.xB, (T*)lv.d, (T*)lv.b, (const T*)lv.dinv,
      [&](T* v) { return launch_zero_constrained_u<T>(lv.g, v, c->st); },
      [&](const T* x, T* y) {
        TileArgs<T> a = tile_args<T>(lv);
        a.xu = x;
        a.yu = y;
        if (a.conv) a.conv = 2;  // corrector stage: bounds of the symmetric part of the block
        return launch_tile<T>(c->dim, TILE_APPLY, OPS_A, a, c->st);
      },
      &lv.lam_hi);
}

template <typename T>
PLapArgs<T> plap_args(const Level& lv) {
  PLapArgs<T> a{};
  a.g = lv.g;
  for (int i = 0; i < 3; ++i) a.kc[i] = (T)lv.pkc[i];
  a.w = (const T*)lv.pw;
  a.cmask = lv.pcmask;
  return a;
}

// pressure level: the level-code field carries 0x80 | l to separate it from velocity level l
template <typename T>
gs_status plap_lanczos(gs_ctx* c, int l) {
  Level& lv = c->lv[l];
  return lanczos_core<T>(
      c, lv.Np, 0x80 | l, (T*)lv.pxA, (T*)lv.pxB, (T*)lv.pd, (T*)lv.pb, (const T*)lv.pdinv,
      [&](T* v) { return launch_mask_copy<T>(v, lv.pcmask, v, lv.Np, c->st); },
      [&](const T* x, T* y) {
        PLapArgs<T> a = plap_args<T>(lv);
        a.x = x;
        a.y = y;
        return launch_plap<T>(TILE_APPLY, a, c->st);
      },
      &lv.plam_hi);
}

// host assembly of the dense coarse matrix on its free unknowns (same closed-form 1D matrices)
// Corrector stage: the cell's rho (C + S) block (component-diagonal, 3^d x 3^d per component) added
// to the dense coarse matrix, by the 3-point Gauss rule per axis of the kernels (host copy of the
// 1D matrices): entry (p, q) = rho sum_g W_g (phi_p(g) adv_q(g) + r_K adv_p(g) adv_q(g)),
// adv_q = v° . grad phi_q.
void add_conv_cell(const Level& lv, int dim, int i, int j, int k, const std::vector<int>& map, int nf,
                   std::vector<double>& A) {
  const double s = 0.38729833462074168852;
  const double Phi[3][3] = {{0.3 + s, 0.4, 0.3 - s}, {0.0, 1.0, 0.0}, {0.3 - s, 0.4, 0.3 + s}};
  const double Dq[3][3] = {{-1.0 - 4.0 * s, 8.0 * s, 1.0 - 4.0 * s}, {-1.0, 0.0, 1.0}, {-1.0 + 4.0 * s, -8.0 * s, 1.0 + 4.0 * s}};
  const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  const int nb = dim == 2 ? 9 : 27;  // nodes of the cell = Gauss points of the cell
  const long long nv0 = 2 * lv.n[0] + 1, nv1 = 2 * lv.n[1] + 1;
  const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
  double jac = 1.0;
  for (int ax = 0; ax < dim; ++ax) jac *= lv.h[ax];
  auto idx = [](int q, int ax) { return ax == 0 ? q % 3 : (ax == 1 ? (q / 3) % 3 : q / 9); };
  long long gn[27];
  for (int q = 0; q < nb; ++q)
    gn[q] = (2 * i + idx(q, 0)) + nv0 * ((2 * j + idx(q, 1)) + nv1 * (dim == 3 ? 2 * k + idx(q, 2) : 0));
  double vq[3][27] = {};
  for (int g = 0; g < nb; ++g)
    for (int jn = 0; jn < nb; ++jn) {
      double ph = 1.0;
      for (int ax = 0; ax < dim; ++ax) ph *= Phi[idx(g, ax)][idx(jn, ax)];
      for (int b = 0; b < dim; ++b) vq[b][g] += ph * lv.hvc[b * lv.Nv + gn[jn]];
    }
  double phi[27][27], adv[27][27], W[27];
  for (int g = 0; g < nb; ++g) {
    W[g] = jac;
    for (int ax = 0; ax < dim; ++ax) W[g] *= w[idx(g, ax)];
    for (int p = 0; p < nb; ++p) {
      double ph = 1.0, ad = 0.0;
      for (int ax = 0; ax < dim; ++ax) ph *= Phi[idx(g, ax)][idx(p, ax)];
      for (int ax = 0; ax < dim; ++ax) {
        double t = vq[ax][g] * Dq[idx(g, ax)][idx(p, ax)] / lv.h[ax];
        for (int o = 0; o < dim; ++o)
          if (o != ax) t *= Phi[idx(g, o)][idx(p, o)];
        ad += t;
      }
      phi[p][g] = ph;
      adv[p][g] = ad;
    }
  }
  const double r = lv.hrk[cc];
  for (int p = 0; p < nb; ++p)
    for (int qn = 0; qn < nb; ++qn) {
      double v = 0.0;
      for (int g = 0; g < nb; ++g) v += W[g] * (phi[p][g] * adv[qn][g] + r * adv[p][g] * adv[qn][g]);
      v *= lv.rho;
      for (int a = 0; a < dim; ++a) {
        const int row = map[a * lv.Nv + gn[p]], col = map[a * lv.Nv + gn[qn]];
        if (row >= 0 && col >= 0) A[(size_t)row * nf + col] += v;
      }
    }
}

void assemble_coarse(gs_ctx* c, std::vector<double>& A) {
  const Level& lv = c->lv[0];
  const int dim = c->dim;
  const int nf = c->nf;
  A.assign((size_t)nf * nf, 0.0);
  std::vector<int> map(lv.nu, -1);
  for (int i = 0; i < nf; ++i) map[c->hfree[i]] = i;
  static const int Mi[3][3] = {{4, 2, -1}, {2, 16, 2}, {-1, 2, 4}};
  static const int Ki[3][3] = {{7, -8, 1}, {-8, 16, -8}, {1, -8, 7}};
  static const int Ei[3][3] = {{-3, -4, 1}, {4, 0, -4}, {-1, 4, 3}};
  const OpCoef<double>& cf = lv.c64;
  const int nb = dim == 2 ? 9 : 27;
  const int nv0 = 2 * lv.n[0] + 1, nv1 = 2 * lv.n[1] + 1;
  std::vector<long long> gn(nb);
  for (int k = 0; k < lv.n[2]; ++k)
    for (int j = 0; j < lv.n[1]; ++j)
      for (int i = 0; i < lv.n[0]; ++i) {
        const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
        if (lv.has_void && lv.hvoid[cc]) continue;
        const double eta = lv.heta[cc];
        const double mm = c->alpha_cells ? cf.mm * lv.halpha[cc] : cf.mm;
        for (int q = 0; q < nb; ++q) {
          const int la = q % 3, lb = (q / 3) % 3, lc = q / 9;
          gn[q] = (2 * i + la) + (long long)nv0 * ((2 * j + lb) + (long long)nv1 * (dim == 3 ? 2 * k + lc : 0));
        }
        for (int al = 0; al < dim; ++al)
          for (int be = 0; be < dim; ++be)
            for (int p = 0; p < nb; ++p) {
              const int row = map[al * lv.Nv + gn[p]];
              if (row < 0) continue;
              const int pi[3] = {p % 3, (p / 3) % 3, p / 9};
              for (int q = 0; q < nb; ++q) {
                const int col = map[be * lv.Nv + gn[q]];
                if (col < 0) continue;
                const int qi[3] = {q % 3, (q / 3) % 3, q / 9};
                double v = 0.0;
                if (al == be) {
                  const double cz = (al == 2 ? 2.0 : 1.0) * eta * cf.km[2];
                  const double cy = (al == 1 ? 2.0 : 1.0) * eta * cf.km[1];
                  const double cx = (al == 0 ? 2.0 : 1.0) * eta * cf.km[0];
                  const double Mx = Mi[pi[0]][qi[0]], My = Mi[pi[1]][qi[1]];
                  const double Kx = Ki[pi[0]][qi[0]], Ky = Ki[pi[1]][qi[1]];
                  if (dim == 2) {
                    v = Mx * (mm * My + cy * Ky) + Kx * (cx * My);
                  } else {
                    const double Mz = Mi[pi[2]][qi[2]], Kz = Ki[pi[2]][qi[2]];
                    v = Mx * (My * (mm * Mz + cz * Kz) + cy * Ky * Mz) + Kx * (cx * My * Mz);
                  }
                } else {
                  // eta (E in direction be) (E^T in direction al) (M in the third direction)
                  double prod = 1.0;
                  int third = 3 - al - be;
                  for (int ax = 0; ax < dim; ++ax) {
                    if (ax == be) prod *= Ei[pi[ax]][qi[ax]];
                    else if (ax == al) prod *= Ei[qi[ax]][pi[ax]];
                    else prod *= Mi[pi[ax]][qi[ax]];
                  }
                  const double ce = dim == 2 ? cf.ex[0] : cf.ex[third];
                  v = eta * ce * prod;
                }
                A[(size_t)row * nf + col] += v;
              }
            }
        if (lv.conv) add_conv_cell(lv, dim, i, j, k, map, nf, A);
      }
}

template <typename T>
gs_status setup_T(gs_ctx* c) {
  for (int l = 0; l < c->L; ++l) {
    Level& lv = c->lv[l];
    CK(launch_diagA<T>(lv.g, coef<T>(lv), etap<T>(lv), alphap<T>(lv), (T*)lv.dinv, 1, c->st));
  }
  for (int l = (c->opt.coarse_mode == 1 ? 0 : 1); l < c->L; ++l) CKS(lanczos<T>(c, l));
  const Level& F = c->lv[c->L - 1];
  CK(launch_pdiag<T>(F.g, coef<T>(F), etap<T>(F), (T*)c->p_dinv, c->st));
  if (c->mono)
    for (int l = (c->opt.coarse_mode == 1 ? 0 : 1); l < c->L; ++l) {
      Level& lv = c->lv[l];
      CK(launch_schur_diag<T>(lv.g, lv.c64, (const T*)lv.dinv, (T*)lv.dsinv, 1, c->st));
    }
  if (c->cc) {
    for (int l = 0; l < c->L; ++l) {
      Level& lv = c->lv[l];
      T kc[3] = {(T)lv.pkc[0], (T)lv.pkc[1], (T)lv.pkc[2]};
      CK(launch_plap_diag<T>(lv.g, kc, (const T*)lv.pw, lv.pcmask, (T*)lv.pdinv, c->st));
    }
    for (int l = (c->opt.coarse_mode == 1 ? 0 : 1); l < c->L; ++l) CKS(plap_lanczos<T>(c, l));
  }
  return GS_OK;
}

// host assembly of the dense coarse pressure Laplacian on its free nodes; with a pure Neumann
// problem the rank-one term 1 1^T / n_free makes it invertible without changing its action on
// mean-free vectors
void assemble_coarse_plap(gs_ctx* c, std::vector<double>& A) {
  const Level& lv = c->lv[0];
  const int dim = c->dim, nf = c->nfp;
  A.assign((size_t)nf * nf, 0.0);
  std::vector<int> map(lv.Np, -1);
  for (int i = 0; i < nf; ++i) map[c->hpfree[i]] = i;
  const int np0 = lv.n[0] + 1, np1 = lv.n[1] + 1;
  const int nb = dim == 2 ? 4 : 8;
  for (int k = 0; k < lv.n[2]; ++k)
    for (int j = 0; j < lv.n[1]; ++j)
      for (int i = 0; i < lv.n[0]; ++i) {
        const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
        if (lv.hvoid[cc]) continue;
        const double wK = (c->alpha_cells && lv.halpha[cc] > 0.0) ? c->alpha / lv.halpha[cc] : 1.0;  // abar / alpha_K
        for (int p = 0; p < nb; ++p) {
          const int pa = p & 1, pb = (p >> 1) & 1, pc = p >> 2;
          const int row = map[(i + pa) + (long long)np0 * ((j + pb) + (long long)np1 * (dim == 3 ? k + pc : 0))];
          if (row < 0) continue;
          for (int q = 0; q < nb; ++q) {
            const int qa = q & 1, qb = (q >> 1) & 1, qc = q >> 2;
            const int col = map[(i + qa) + (long long)np0 * ((j + qb) + (long long)np1 * (dim == 3 ? k + qc : 0))];
            if (col < 0) continue;
            const double k1a = pa == qa ? 1 : -1, ia = pa == qa ? 2 : 1;
            const double k1b = pb == qb ? 1 : -1, ib = pb == qb ? 2 : 1;
            double v;
            if (dim == 2) {
              v = lv.pkc[0] * k1a * ib + lv.pkc[1] * ia * k1b;
            } else {
              const double k1c = pc == qc ? 1 : -1, ic = pc == qc ? 2 : 1;
              v = lv.pkc[0] * k1a * ib * ic + lv.pkc[1] * ia * k1b * ic + lv.pkc[2] * ia * ib * k1c;
            }
            A[(size_t)row * nf + col] += wK * v;
          }
        }
      }
  if (c->psingular)
    for (size_t q = 0; q < A.size(); ++q) A[q] += 1.0 / nf;
}

// host assembly of the dense coarse saddle matrix M_0 = [A_0 B_0^T; B_0 0] on its free unknowns
// (the velocity block of assemble_coarse, then the free pressure nodes); B's cell entries are
// -bd[a] (Gi in direction a) (Ni elsewhere) with Ni, Gi the 1D Q1 x Q2 integrals times 6.  With
// every face Dirichlet the pressure block gets -1 1^T / n_p,free (the constant pressure is in
// the kernel of M_0; mean-free solutions of consistent systems do not change).
void assemble_coarse_saddle(gs_ctx* c, std::vector<double>& M) {
  const Level& lv = c->lv[0];
  const int dim = c->dim, nf = c->nf, n = c->nmf;
  std::vector<double> A;
  assemble_coarse(c, A);
  M.assign((size_t)n * n, 0.0);
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nf; ++j) M[(size_t)i * n + j] = A[(size_t)i * nf + j];
  std::vector<int> umap(lv.nu, -1), pmap(lv.Np, -1);
  for (int i = 0; i < nf; ++i) umap[c->hfree[i]] = i;
  for (int i = nf; i < n; ++i) pmap[c->hmfree[i] - lv.nu] = i;
  static const int Ni[2][3] = {{1, 2, 0}, {0, 2, 1}};
  static const int Gi[2][3] = {{-5, 4, 1}, {-1, -4, 5}};
  const int nv0 = 2 * lv.n[0] + 1, nv1 = 2 * lv.n[1] + 1;
  const int np0 = lv.n[0] + 1, np1 = lv.n[1] + 1;
  const int nbp = dim == 2 ? 4 : 8, nbv = dim == 2 ? 9 : 27;
  for (int k = 0; k < lv.n[2]; ++k)
    for (int j = 0; j < lv.n[1]; ++j)
      for (int i = 0; i < lv.n[0]; ++i) {
        const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
        if (lv.has_void && lv.hvoid[cc]) continue;
        for (int pq = 0; pq < nbp; ++pq) {
          const int qi[3] = {pq & 1, (pq >> 1) & 1, pq >> 2};
          const int row = pmap[(i + qi[0]) + (long long)np0 * ((j + qi[1]) + (long long)np1 * (dim == 3 ? k + qi[2] : 0))];
          if (row < 0) continue;
          for (int pv = 0; pv < nbv; ++pv) {
            const int vi[3] = {pv % 3, (pv / 3) % 3, pv / 9};
            const long long node =
                (2 * i + vi[0]) + (long long)nv0 * ((2 * j + vi[1]) + (long long)nv1 * (dim == 3 ? 2 * k + vi[2] : 0));
            for (int a = 0; a < dim; ++a) {
              const int col = umap[a * lv.Nv + node];
              if (col < 0) continue;
              double prod = 1.0;
              for (int b = 0; b < dim; ++b) prod *= (b == a) ? Gi[qi[b]][vi[b]] : Ni[qi[b]][vi[b]];
              const double v = -lv.c64.bd[a] * prod;
              M[(size_t)row * n + col] += v;
              M[(size_t)col * n + row] += v;
            }
          }
        }
      }
  if (c->nullspace && n > nf)
    for (int r = nf; r < n; ++r)
      for (int q = nf; q < n; ++q) M[(size_t)r * n + q] -= 1.0 / (n - nf);
}

// FP64 saddle operator on the finest level: y = K x (APPLY) or y = b - K x (RESID)
gs_status saddle(gs_ctx* c, int mode, const double* x, double* y, const double* b, int raw = 0);

// ---- tile-height autotuner (2D): a launch-shape choice, the results do not depend on it -------------
// Time `reps` launches of one kernel configuration (after one warm-up launch); microseconds each.
template <typename F>
gs_status time_launches(gs_ctx* c, F&& launch, int reps, double* us) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(e);
  *us = 1e3 * ms / reps;
  return GS_OK;
}

// Per level, time the fused Chebyshev step with each compiled kernel variant (2D: tile heights
// and the strip kernel; 3D: tile depths) on the level's own (scratch) vectors and keep the
// fastest; then the same for the FP64 saddle operator on the finest level.  A variant must beat
// the current choice by 2 % to replace it.
template <typename T>
gs_status autotune(gs_ctx* c) {
  const int nshape = c->dim == 2 ? kTileShapes2D : kTileShapes3D;
  const int nsaddle = c->dim == 2 ? kTileHeights2D : kTileShapes3D;
  for (int l = 0; l < c->L; ++l) {
    Level& lv = c->lv[l];
    CK(cudaMemsetAsync(lv.xA, 0, sizeof(T) * lv.nu, c->st));
    CK(cudaMemsetAsync(lv.b, 0, sizeof(T) * lv.nu, c->st));
    CK(cudaMemsetAsync(lv.d, 0, sizeof(T) * lv.nu, c->st));
    double best_us = 0.0;
    int best = 0;
    for (int s = 0; s < nshape; ++s) {
      TileArgs<T> a = tile_args<T>(lv);
      a.shape = s;
      a.xu = (const T*)lv.xA; a.bu = (const T*)lv.b; a.d = (T*)lv.d; a.dinv = (const T*)lv.dinv;
      a.xout = (T*)lv.xB; a.c1 = (T)0.5; a.c2 = (T)1; a.use_d = 1;
      double us;
      CKS(time_launches(c, [&]() { return launch_tile<T>(c->dim, TILE_CHEB, OPS_A, a, c->st); }, 4, &us));
      if (s == 0 || us < 0.98 * best_us) { best_us = us; best = s; }
    }
    lv.shape = best;
  }
  CK(cudaMemsetAsync(c->r, 0, sizeof(double) * c->N, c->st));
  double best_us = 0.0;
  int best = 0;
  for (int s = 0; s < nsaddle; ++s) {
    c->saddle_shape = s;
    double us;
    CKS(time_launches(c, [&]() -> cudaError_t {
      return saddle(c, TILE_APPLY, c->r, c->w, nullptr) == GS_OK ? cudaSuccess : cudaErrorUnknown; }, 3, &us));
    if (s == 0 || us < 0.98 * best_us) { best_us = us; best = s; }
  }
  c->saddle_shape = best;
  return GS_OK;
}

gs_status setup(gs_ctx* c) {
  CK(cudaMemsetAsync(c->errw, 0, sizeof(int) * 4, c->st));
  // upload per-level data
  for (int l = 0; l < c->L; ++l) {
    Level& lv = c->lv[l];
    std::vector<float> e32(lv.Nc);
    for (long long i = 0; i < lv.Nc; ++i) e32[i] = (float)lv.heta[i];
    CK(cudaMemcpyAsync(lv.eta64, lv.heta.data(), sizeof(double) * lv.Nc, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(lv.eta32, e32.data(), sizeof(float) * lv.Nc, cudaMemcpyHostToDevice, c->st));
    std::vector<float> a32;
    std::vector<double> w64;
    std::vector<float> w32;
    if (c->alpha_cells) {
      a32.resize(lv.Nc);
      for (long long i = 0; i < lv.Nc; ++i) a32[i] = (float)lv.halpha[i];
      CK(cudaMemcpyAsync(lv.alpha64, lv.halpha.data(), sizeof(double) * lv.Nc, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lv.alpha32, a32.data(), sizeof(float) * lv.Nc, cudaMemcpyHostToDevice, c->st));
      if (lv.pw) {  // weights abar / alpha_K of the pressure Laplacian (1 on cells without alpha)
        w64.resize(lv.Nc);
        for (long long i = 0; i < lv.Nc; ++i) w64[i] = lv.halpha[i] > 0.0 ? c->alpha / lv.halpha[i] : 1.0;
        if (c->fp32) {
          w32.assign(w64.begin(), w64.end());
          CK(cudaMemcpyAsync(lv.pw, w32.data(), sizeof(float) * lv.Nc, cudaMemcpyHostToDevice, c->st));
        } else {
          CK(cudaMemcpyAsync(lv.pw, w64.data(), sizeof(double) * lv.Nc, cudaMemcpyHostToDevice, c->st));
        }
      }
    }
    if (lv.has_void) {
      CK(cudaMemcpyAsync(lv.cvoid, lv.hvoid.data(), lv.Nc, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lv.vmask, lv.hvmask.data(), lv.Nv, cudaMemcpyHostToDevice, c->st));
      if (lv.ccmask) {
        // per cell: bit la + 3 lb for a constrained local node, bit 15 for an obstacle cell
        const long long nv0 = 2 * lv.n[0] + 1;
        lv.hccmask.assign(lv.Nc, 0);
        for (int j = 0; j < lv.n[1]; ++j)
          for (int i = 0; i < lv.n[0]; ++i) {
            const long long cc = i + (long long)lv.n[0] * j;
            unsigned m = lv.hvoid[cc] ? 0x8000u : 0u;
            for (int lb = 0; lb < 3; ++lb)
              for (int la = 0; la < 3; ++la)
                if (lv.hvmask[(2 * i + la) + nv0 * (2 * j + lb)]) m |= 1u << (la + 3 * lb);
            lv.hccmask[cc] = (uint16_t)m;
          }
        CK(cudaMemcpyAsync(lv.ccmask, lv.hccmask.data(), sizeof(uint16_t) * lv.Nc, cudaMemcpyHostToDevice, c->st));
      }
      if (lv.pmask) CK(cudaMemcpyAsync(lv.pmask, lv.hpmask.data(), lv.Np, cudaMemcpyHostToDevice, c->st));
    }
    CK(cudaStreamSynchronize(c->st));  // host staging vectors go out of scope
  }
  // coarse inverse: host assembly, device Gauss-Jordan
  if (c->nf > 0) {
    std::vector<double> A;
    assemble_coarse(c, A);
    CK(cudaMemcpyAsync(c->Ainv, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->cfree, c->hfree.data(), sizeof(int) * c->nf, cudaMemcpyHostToDevice, c->st));
    for (int k = 0; k < c->nf; ++k) {
      CK(launch_gj_save(c->Ainv, c->nf, k, c->gjrow, c->gjcol, c->st));
      CK(launch_gj_update(c->Ainv, c->nf, k, c->gjrow, c->gjcol, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
  }
  if (c->cc) {
    for (int l = 0; l < c->L; ++l) {
      Level& lv = c->lv[l];
      CK(cudaMemcpyAsync(lv.pcmask, lv.hpc.data(), lv.Np, cudaMemcpyHostToDevice, c->st));
    }
  }
  if (c->mono) {
    for (int l = 0; l < c->L; ++l) {
      Level& lv = c->lv[l];
      if (lv.has_void)
        CK(cudaMemcpyAsync(lv.mpm, lv.hpmask.data(), lv.Np, cudaMemcpyHostToDevice, c->st));
      else
        CK(cudaMemsetAsync(lv.mpm, 0, lv.Np, c->st));
    }
    if (c->nmf > 0) {
      std::vector<double> M;
      assemble_coarse_saddle(c, M);
      CK(cudaMemcpyAsync(c->MAinv, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(c->mcfree, c->hmfree.data(), sizeof(int) * c->nmf, cudaMemcpyHostToDevice, c->st));
      // Gauss-Jordan without pivoting: the velocity pivots are those of the SPD A_0, the pressure
      // pivots those of the negative definite -(B_0 A_0^{-1} B_0^T (+ 1 1^T / n))
      for (int k = 0; k < c->nmf; ++k) {
        CK(launch_gj_save(c->MAinv, c->nmf, k, c->gjrow, c->gjcol, c->st));
        CK(launch_gj_update(c->MAinv, c->nmf, k, c->gjrow, c->gjcol, c->st));
      }
      CK(cudaStreamSynchronize(c->st));
    }
  }
  if (c->cc && c->nfp > 0) {
    std::vector<double> A;
    assemble_coarse_plap(c, A);
    CK(cudaMemcpyAsync(c->PAinv, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->pcfree, c->hpfree.data(), sizeof(int) * c->nfp, cudaMemcpyHostToDevice, c->st));
    for (int k = 0; k < c->nfp; ++k) {
      CK(launch_gj_save(c->PAinv, c->nfp, k, c->gjrow, c->gjcol, c->st));
      CK(launch_gj_update(c->PAinv, c->nfp, k, c->gjrow, c->gjcol, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
  }
  if (c->fp32) CKS(setup_T<float>(c)); else CKS(setup_T<double>(c));
  CK(cudaStreamSynchronize(c->st));
  if (c->opt.tile_autotune == 0) {
    CKS(c->fp32 ? autotune<float>(c) : autotune<double>(c));
  } else if (c->dim == 3) {
    for (int l = 0; l < c->L; ++l) c->lv[l].shape = c->opt.tile_autotune == 2 ? 1 : 0;
    c->saddle_shape = c->opt.tile_autotune == 2 ? 1 : 0;
  } else if (c->dim == 2 && c->opt.tile_autotune == 5) {
    // size rule: the strip kernel where a level has enough cells to fill the GPU, 32 x 8 tiles below
    for (int l = 0; l < c->L; ++l) c->lv[l].shape = c->lv[l].Nc >= 32768 ? 3 : 2;
    c->saddle_shape = 2;
  } else if (c->dim == 2) {
    for (int l = 0; l < c->L; ++l) c->lv[l].shape = c->opt.tile_autotune - 1;
    c->saddle_shape = std::min(c->opt.tile_autotune - 1, kTileHeights2D - 1);
  }
  return GS_OK;
}

// ---- Chebyshev smoother on level l: result in lv.xA (Sec. 4, Cheb(A, diag(A), k)) -------------
// 1 / theta of a Chebyshev interval [hi / 15, hi] (the first step from zero is x = dinv b / theta)
double cheb_inv_theta(double hi) { return 1.0 / (0.5 * (hi + hi / 15.0)); }

// started: the first step from zero (d = x = dinv b / theta) was already done by the restriction
// that produced b (launch_restrict with a Chebyshev start)
template <typename T>
gs_status cheb(gs_ctx* c, int l, const T* b, bool zero_init, bool started = false) {
  const LevelTag tag__(c, l);
  Level& lv = c->lv[l];
  const double hi = lv.lam_hi, lo = hi / 15.0;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  const int k = c->opt.cheb_degree;
  T* dinv = (T*)lv.dinv;
  T* d = (T*)lv.d;
  if (zero_init) {
    if (!started) KL(K_VEC, launch_cheb_init0<T>(b, dinv, (T)(1.0 / theta), d, (T*)lv.xA, lv.nu, c->st));
  } else {
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = (const T*)lv.xA; a.bu = b; a.d = d; a.dinv = dinv; a.xout = (T*)lv.xB;
    a.c1 = 0; a.c2 = (T)(1.0 / theta); a.use_d = 0;
    KL(K_CHEB, launch_tile<T>(c->dim, TILE_CHEB, OPS_A, a, c->st));
    std::swap(lv.xA, lv.xB);
  }
  double rho = 1.0 / sigma;
  for (int t = 1; t < k; ++t) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = (const T*)lv.xA; a.bu = b; a.d = d; a.dinv = dinv; a.xout = (T*)lv.xB;
    a.c1 = (T)(rn * rho); a.c2 = (T)(2.0 * rn / delta); a.use_d = 1;
    KL(K_CHEB, launch_tile<T>(c->dim, TILE_CHEB, OPS_A, a, c->st));
    std::swap(lv.xA, lv.xB);
    rho = rn;
  }
  return GS_OK;
}

// V-cycle on level l: input lv.b, output lv.xA (started: see cheb)
template <typename T>
gs_status vcycle(gs_ctx* c, int l, bool started = false) {
  const LevelTag tag__(c, l);
  Level& lv = c->lv[l];
  if (l == 0) {
    if (c->opt.coarse_mode == 1) return cheb<T>(c, 0, (const T*)lv.b, true, started);
    KL(K_COARSE, launch_coarse_solve<T>(c->Ainv, c->cfree, c->nf, (const T*)lv.b, (T*)lv.xA, lv.nu, c->ctmp, c->st));
    return GS_OK;
  }
  for (int s = 0; s < c->opt.smooth_steps; ++s) CKS(cheb<T>(c, l, (const T*)lv.b, s == 0, s == 0 && started));
  {
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = (const T*)lv.xA; a.bu = (const T*)lv.b; a.yu = (T*)lv.d;
    KL(K_RESID, launch_tile<T>(c->dim, TILE_RESID, OPS_A, a, c->st));
  }
  // rigid-body deflation on the finest level: y = E^-1 Z^T r, added after the coarse correction
  const bool defl = l == c->L - 1 && c->defl_ninc > 0;
  if (defl) {
    KL(K_VEC, launch_defl_dots<T>(c->defl, (const T*)lv.d, c->d_c, c->st));
    KL(K_VEC, launch_defl_gemv(c->d_Einv, c->defl_M, c->d_c, c->d_y, c->st));
  }
  Level& cl = c->lv[l - 1];
  // the coarse level's first smoothing step from zero is started inside the restriction
  const bool start = c->opt.smooth_steps >= 1 && (l - 1 >= 1 || c->opt.coarse_mode == 1);
  if (start)
    KL(K_TRANSFER, launch_restrict<T>(lv.g, cl.g, (const T*)lv.d, (T*)cl.b, c->st, (const T*)cl.dinv,
                                      (T)cheb_inv_theta(cl.lam_hi), (T*)cl.d, (T*)cl.xA));
  else
    KL(K_TRANSFER, launch_restrict<T>(lv.g, cl.g, (const T*)lv.d, (T*)cl.b, c->st));
  CKS(vcycle<T>(c, l - 1, start));
  KL(K_TRANSFER, launch_prolong_add<T>(lv.g, cl.g, (const T*)cl.xA, (T*)lv.xA, c->st));
  if (defl) KL(K_VEC, launch_defl_add<T>(c->defl, c->d_y, (T*)lv.xA, c->st));
  for (int s = 0; s < c->opt.smooth_steps; ++s) CKS(cheb<T>(c, l, (const T*)lv.b, false));
  return GS_OK;
}

// S^{-1} b ~ Chebyshev-Jacobi on M_p(1/eta) from zero, Wathen interval: result in c->p_xA
template <typename T>
gs_status schur_inv(gs_ctx* c, const T* b) {
  const Level& F = c->lv[c->L - 1];
  const double lo = std::pow(0.5, c->dim), hi = std::pow(1.5, c->dim);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  KL(K_VEC, launch_cheb_init0<T>(b, (const T*)c->p_dinv, (T)(1.0 / theta), (T*)c->p_d, (T*)c->p_xA, F.Np, c->st));
  double rho = 1.0 / sigma;
  for (int t = 1; t < c->opt.schur_degree; ++t) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    PMassArgs<T> a{};
    a.g = F.g; a.c = coef<T>(F); a.eta = etap<T>(F);
    a.x = (const T*)c->p_xA; a.b = b; a.d = (T*)c->p_d; a.dinv = (const T*)c->p_dinv; a.xout = (T*)c->p_xB;
    a.c1 = (T)(rn * rho); a.c2 = (T)(2.0 * rn / delta); a.use_d = 1;
    KL(K_SCHUR, launch_pmass<T>(TILE_CHEB, a, c->st));
    std::swap(c->p_xA, c->p_xB);
    rho = rn;
  }
  return GS_OK;
}

// Chebyshev smoother of the pressure Laplacian on level l (result in lv.pxA)
template <typename T>
gs_status pcheb(gs_ctx* c, int l, const T* b, bool zero_init, bool started = false) {
  const LevelTag tag__(c, l);
  Level& lv = c->lv[l];
  const double hi = lv.plam_hi, lo = hi / 15.0;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  const int k = c->opt.plap_degree;
  T* dinv = (T*)lv.pdinv;
  T* d = (T*)lv.pd;
  if (zero_init) {
    if (!started) KL(K_SCHUR, launch_cheb_init0<T>(b, dinv, (T)(1.0 / theta), d, (T*)lv.pxA, lv.Np, c->st));
  } else {
    PLapArgs<T> a = plap_args<T>(lv);
    a.x = (const T*)lv.pxA; a.b = b; a.d = d; a.dinv = dinv; a.xout = (T*)lv.pxB;
    a.c1 = 0; a.c2 = (T)(1.0 / theta); a.use_d = 0;
    KL(K_SCHUR, launch_plap<T>(TILE_CHEB, a, c->st));
    std::swap(lv.pxA, lv.pxB);
  }
  double rho = 1.0 / sigma;
  for (int t = 1; t < k; ++t) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    PLapArgs<T> a = plap_args<T>(lv);
    a.x = (const T*)lv.pxA; a.b = b; a.d = d; a.dinv = dinv; a.xout = (T*)lv.pxB;
    a.c1 = (T)(rn * rho); a.c2 = (T)(2.0 * rn / delta); a.use_d = 1;
    KL(K_SCHUR, launch_plap<T>(TILE_CHEB, a, c->st));
    std::swap(lv.pxA, lv.pxB);
    rho = rn;
  }
  return GS_OK;
}

// V-cycle for the pressure Laplacian: input lv.pb, output lv.pxA
template <typename T>
gs_status pvcycle(gs_ctx* c, int l, bool started = false) {
  const LevelTag tag__(c, l);
  Level& lv = c->lv[l];
  if (l == 0) {
    if (c->opt.coarse_mode == 1) return pcheb<T>(c, 0, (const T*)lv.pb, true, started);
    KL(K_SCHUR, launch_coarse_solve<T>(c->PAinv, c->pcfree, c->nfp, (const T*)lv.pb, (T*)lv.pxA, lv.Np, c->pctmp, c->st));
    return GS_OK;
  }
  for (int s = 0; s < c->opt.smooth_steps; ++s) CKS(pcheb<T>(c, l, (const T*)lv.pb, s == 0, s == 0 && started));
  {
    PLapArgs<T> a = plap_args<T>(lv);
    a.x = (const T*)lv.pxA; a.b = (const T*)lv.pb; a.y = (T*)lv.pd;
    KL(K_SCHUR, launch_plap<T>(TILE_RESID, a, c->st));
  }
  Level& cl = c->lv[l - 1];
  const bool start = c->opt.smooth_steps >= 1 && (l - 1 >= 1 || c->opt.coarse_mode == 1);
  if (start)
    KL(K_SCHUR, launch_p_restrict<T>(lv.g, cl.g, lv.pcmask, cl.pcmask, (const T*)lv.pd, (T*)cl.pb, c->st,
                                     (const T*)cl.pdinv, (T)cheb_inv_theta(cl.plam_hi), (T*)cl.pd, (T*)cl.pxA));
  else
    KL(K_SCHUR, launch_p_restrict<T>(lv.g, cl.g, lv.pcmask, cl.pcmask, (const T*)lv.pd, (T*)cl.pb, c->st));
  CKS(pvcycle<T>(c, l - 1, start));
  KL(K_SCHUR, launch_p_prolong_add<T>(lv.g, cl.g, lv.pcmask, cl.pcmask, (const T*)cl.pxA, (T*)lv.pxA, c->st));
  for (int s = 0; s < c->opt.smooth_steps; ++s) CKS(pcheb<T>(c, l, (const T*)lv.pb, false));
  return GS_OK;
}

// Cahouet-Chabard term K_p^{-1} r ~ one pressure V-cycle, constrained entries zero; result in
// the finest level's pxA
template <typename T>
gs_status plap_inverse(gs_ctx* c, const T* r) {
  Level& F = c->lv[c->L - 1];
  KL(K_VEC, launch_mask_copy<T>(r, F.pcmask, (T*)F.pb, F.Np, c->st));
  CKS(pvcycle<T>(c, c->L - 1));
  return GS_OK;
}

// ---- saddle-point multigrid with the block smoother K_j (Sec. 4, Eq. "smoother") ---------------
// Level l: iterate [u | p] in lv.ms, right-hand side in lv.mr (MG precision).  One smoothing step
// x <- x + K_j (b - M_j x) applies K_j by its block factorisation
//   w~ = Ahat^{-1} r_u,   w_p = Shat^{-1} (B w~ - r_p),   w_u = w~ - Ahat^{-1} B^T w_p,
// Ahat^{-1} = Cheb(A, diag A, k_A) from zero, Shat^{-1} = one MINRES step on S = B Ahat^{-1} B^T
// with preconditioner P = D_S^{-1} = diag(B diag(A)^{-1} B^T)^{-1}: w_p = a z, z = P (B w~ - r_p),
// a = (z . S z) / ((S z) . P (S z)).  S z = B y with y = Ahat^{-1} B^T z, and Ahat^{-1} is linear,
// so Ahat^{-1} B^T w_p = a y: the second Ahat solve of the smoother is the one inside S z.  The
// kernels run on -z, -y and -S z (from r_p - B w~), which leaves a and the update unchanged.
template <typename T>
gs_status mono_smooth_step(gs_ctx* c, int l, bool zero) {
  const LevelTag tag__(c, l);
  Level& lv = c->lv[l];
  T* x = (T*)lv.ms;
  const T* b = (const T*)lv.mr;
  const T* ru = b;
  const T* rp = b + lv.nu;
  if (!zero) {  // r = b - M_j x
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = x; a.xp = x + lv.nu; a.bu = b; a.bp = b + lv.nu;
    a.yu = (T*)lv.mres; a.yp = (T*)lv.mres + lv.nu;
    KL(K_MONO, launch_tile<T>(c->dim, TILE_RESID, OPS_A | OPS_BT | OPS_B, a, c->st));
    ru = (const T*)lv.mres;
    rp = ru + lv.nu;
  }
  CKS(cheb<T>(c, l, ru, true));  // w~ = Ahat^{-1} r_u in lv.xA
  std::swap(lv.xA, lv.mwt);
  const T* wt = (const T*)lv.mwt;
  T* q = (T*)lv.mq;
  T* z = (T*)lv.mz;
  {  // q = r_p - B w~
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = wt; a.bp = rp; a.yp = q;
    KL(K_MONO, launch_tile<T>(c->dim, TILE_RESID, OPS_B, a, c->st));
  }
  KL(K_MONO, launch_mul<T>((const T*)lv.dsinv, q, z, lv.Np, c->st));  // z = P q
  {  // lv.b = B^T z
    TileArgs<T> a = tile_args<T>(lv);
    a.xp = z; a.yu = (T*)lv.b;
    KL(K_MONO, launch_tile<T>(c->dim, TILE_APPLY, OPS_BT, a, c->st));
  }
  CKS(cheb<T>(c, l, (const T*)lv.b, true));  // y = Ahat^{-1} B^T z in lv.xA
  if (lv.conv) {  // corrector stage: ChebBiCGStab(1, 1) on the negated right-hand side q
    T* y1 = (T*)lv.my1;
    T* v = (T*)lv.mres + lv.nu;  // v, then s (the residual is consumed)
    T* z2 = (T*)lv.mz2;
    KL(K_MONO, launch_cast<T, T>((const T*)lv.xA, y1, lv.nu, (T)1, c->st));  // y1 = Ahat^{-1} B^T z1
    {  // v = S z1 = B y1
      TileArgs<T> a = tile_args<T>(lv);
      a.xu = y1; a.yp = v;
      KL(K_MONO, launch_tile<T>(c->dim, TILE_APPLY, OPS_B, a, c->st));
    }
    KL(K_MONO, launch_dot2<T>(q, q, q, v, lv.Np, c->part, c->G, c->msc, c->st));  // q . q, q . v
    KL(K_MONO, launch_bicg_s<T>(q, v, (const T*)lv.dsinv, z2, c->msc, lv.Np, c->st));  // s, z2 = P s
    {  // lv.b = B^T z2
      TileArgs<T> a = tile_args<T>(lv);
      a.xp = z2; a.yu = (T*)lv.b;
      KL(K_MONO, launch_tile<T>(c->dim, TILE_APPLY, OPS_BT, a, c->st));
    }
    CKS(cheb<T>(c, l, (const T*)lv.b, true));  // y2 = Ahat^{-1} B^T z2 in lv.xA
    {  // t = S z2 = B y2 (into q)
      TileArgs<T> a = tile_args<T>(lv);
      a.xu = (const T*)lv.xA; a.yp = q;
      KL(K_MONO, launch_tile<T>(c->dim, TILE_APPLY, OPS_B, a, c->st));
    }
    KL(K_MONO, launch_dot2<T>(q, (const T*)v, q, q, lv.Np, c->part, c->G, c->msc2, c->st));  // t . s, t . t
    KL(K_MONO, launch_mono_update2<T>(x, x + lv.nu, wt, y1, (const T*)lv.xA, z, z2, c->msc, c->msc2, lv.nu, lv.Np,
                                      zero ? 1 : 0, c->st));
    return GS_OK;
  }
  {  // q = B y = S z
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = (const T*)lv.xA; a.yp = q;
    KL(K_MONO, launch_tile<T>(c->dim, TILE_APPLY, OPS_B, a, c->st));
  }
  KL(K_MONO, launch_schur_dots<T>(z, q, (const T*)lv.dsinv, lv.Np, c->part, c->G, c->msc, c->st));
  KL(K_MONO, launch_mono_update<T>(x, x + lv.nu, wt, (const T*)lv.xA, z, c->msc, lv.nu, lv.Np, zero ? 1 : 0, c->st));
  return GS_OK;
}

// one saddle-point V-cycle on level l: right-hand side lv.mr -> iterate lv.ms.  m smoothing steps
// (the first from zero), residual, Q2 / Q1 restriction, recursion, interpolation, m steps; level
// 0: dense saddle solve (coarse_mode 0) or m smoothing steps from zero.
template <typename T>
gs_status mono_vcycle(gs_ctx* c, int l) {
  const LevelTag tag__(c, l);
  Level& lv = c->lv[l];
  if (l == 0 && c->opt.coarse_mode != 1) {
    KL(K_COARSE, launch_coarse_solve<T>(c->MAinv, c->mcfree, c->nmf, (const T*)lv.mr, (T*)lv.ms, lv.nu + lv.Np,
                                        c->mctmp, c->st));
    return GS_OK;
  }
  const int m = c->opt.mono_smooth;
  for (int s = 0; s < m; ++s) CKS(mono_smooth_step<T>(c, l, s == 0));
  if (l == 0) return GS_OK;
  T* res = (T*)lv.mres;
  {
    TileArgs<T> a = tile_args<T>(lv);
    a.xu = (const T*)lv.ms; a.xp = (const T*)lv.ms + lv.nu; a.bu = (const T*)lv.mr; a.bp = (const T*)lv.mr + lv.nu;
    a.yu = res; a.yp = res + lv.nu;
    KL(K_MONO, launch_tile<T>(c->dim, TILE_RESID, OPS_A | OPS_BT | OPS_B, a, c->st));
  }
  Level& cl = c->lv[l - 1];
  KL(K_TRANSFER, launch_restrict<T>(lv.g, cl.g, res, (T*)cl.mr, c->st));
  KL(K_TRANSFER, launch_p_restrict<T>(lv.g, cl.g, lv.mpm, cl.mpm, res + lv.nu, (T*)cl.mr + cl.nu, c->st));
  CKS(mono_vcycle<T>(c, l - 1));
  KL(K_TRANSFER, launch_prolong_add<T>(lv.g, cl.g, (const T*)cl.ms, (T*)lv.ms, c->st));
  KL(K_TRANSFER, launch_p_prolong_add<T>(lv.g, cl.g, lv.mpm, cl.mpm, (const T*)cl.ms + cl.nu, (T*)lv.ms + lv.nu,
                                         c->st));
  for (int s = 0; s < m; ++s) CKS(mono_smooth_step<T>(c, l, false));
  return GS_OK;
}

// n cycles on the finest level from zero, x <- x + V(b - M x): input F.mr, output mono_out()
template <typename T>
gs_status mono_body(gs_ctx* c) {
  Level& F = c->lv[c->L - 1];
  const long long n = F.nu + F.Np;
  const int cycles = c->opt.mono_cycles;
  if (cycles > 1) KL(K_VEC, launch_cast<T, T>((const T*)F.mr, (T*)c->mb, n, (T)1, c->st));
  CKS(mono_vcycle<T>(c, c->L - 1));
  if (cycles > 1) {
    KL(K_VEC, launch_cast<T, T>((const T*)F.ms, (T*)c->mx, n, (T)1, c->st));
    for (int i = 1; i < cycles; ++i) {
      TileArgs<T> a = tile_args<T>(F);
      a.xu = (const T*)c->mx; a.xp = (const T*)c->mx + F.nu; a.bu = (const T*)c->mb; a.bp = (const T*)c->mb + F.nu;
      a.yu = (T*)F.mr; a.yp = (T*)F.mr + F.nu;
      KL(K_MONO, launch_tile<T>(c->dim, TILE_RESID, OPS_A | OPS_BT | OPS_B, a, c->st));
      CKS(mono_vcycle<T>(c, c->L - 1));
      KL(K_VEC, launch_add<T>((const T*)F.ms, (T*)c->mx, n, c->st));
    }
  }
  return GS_OK;
}

// staging of the preconditioner body: where its input is cast to and its result is left
void* body_in_u(gs_ctx* c) { return c->mono ? c->lv[c->L - 1].mr : c->lv[c->L - 1].d; }
void* body_in_p(gs_ctx* c) {
  const size_t S = c->fp32 ? 4 : 8;
  return c->mono ? (void*)((char*)c->lv[c->L - 1].mr + S * c->nu) : c->p_b;
}
const void* body_out_u(gs_ctx* c) {
  if (!c->mono) return c->lv[c->L - 1].xA;
  return c->opt.mono_cycles > 1 ? c->mx : c->lv[c->L - 1].ms;
}
const void* body_out_p(gs_ctx* c) {
  if (!c->mono) return c->p_xB;
  const size_t S = c->fp32 ? 4 : 8;
  return (const char*)body_out_u(c) + S * c->nu;
}

gs_status project_pressure(gs_ctx* c, double* x) {
  if (!c->nullspace) return GS_OK;
  const Level& F = c->lv[c->L - 1];
  double* p = x + c->nu;
  KL(K_VEC, launch_masked_sum_partial(p, F.pmask, F.Np, c->part, c->G, c->st));
  KL(K_VEC, launch_reduce_partials(c->part, 1, c->G, c->dsc + 3 * (c->opt.restart + 4) , c->st));
  KL(K_VEC, launch_sub_scalar_masked(p, F.pmask, F.Np, c->dsc + 3 * (c->opt.restart + 4), 1.0 / (double)c->n_pfree, c->st));
  return GS_OK;
}

// block upper-triangular preconditioner: z_p = -S^{-1} v_p, z_u = V(v_u - B^T z_p); constrained
// entries of z copied from v (K is the identity there); pressure mean removed
// Body of the preconditioner between the staging buffers: r_p in c->p_b, r_u in F.d (both in the
// MG precision) -> z_p in c->p_xB, z_u in F.xA.  Fixed work, no host synchronisation: captured
// once into a CUDA graph and replayed.
template <typename T>
gs_status precond_body(gs_ctx* c) {
  if (c->mono) return mono_body<T>(c);
  Level& F = c->lv[c->L - 1];
  CKS(schur_inv<T>(c, (const T*)c->p_b));
  if (c->cc) {
    // z_p = -(M_p(1/eta)^{-1} r_p + alpha K_p^{-1} r_p)  (Cahouet-Chabard)
    CKS(plap_inverse<T>(c, (const T*)c->p_b));
    KL(K_VEC, launch_cc_combine<T>((const T*)c->p_xA, (const T*)F.pxA, F.pcmask, (T)c->alpha, (T*)c->p_xB, F.Np,
                                   c->st));
  } else {
    KL(K_VEC, launch_cast<T, T>((const T*)c->p_xA, (T*)c->p_xB, F.Np, (T)(-1), c->st));  // z_p in p_xB
  }
  {
    TileArgs<T> a = tile_args<T>(F);
    a.xp = (const T*)c->p_xB; a.bu = (const T*)F.d; a.yu = (T*)F.b;
    KL(K_BT, launch_tile<T>(c->dim, TILE_RESID, OPS_BT, a, c->st));
  }
  CKS(vcycle<T>(c, c->L - 1));
  return GS_OK;
}

// capture the preconditioner body into a CUDA graph (on the private capture stream)
template <typename T>
gs_status capture_precond(gs_ctx* c) {
  cudaStream_t user = c->st;
  CK(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal));
  c->st = c->cap_st;
  gs_status s = precond_body<T>(c);
  c->st = user;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_st, &graph);
  if (s != GS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(GS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->pgraph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->pgraph = nullptr;
    return fail(GS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  // the graph leaves its results where the captured launches put them
  c->g_zu = body_out_u(c);
  c->g_zp = body_out_p(c);
  return GS_OK;
}

// block upper-triangular preconditioner: z_p = -S^{-1} v_p, z_u = V(v_u - B^T z_p); constrained
// entries of z copied from v (K is the identity there); pressure mean removed
template <typename T>
gs_status precond_T(gs_ctx* c, const double* v, double* z) {
  Level& F = c->lv[c->L - 1];
  KL(K_VEC, launch_precond_in<T>(v, (T*)body_in_u(c), (T*)body_in_p(c), F.nu, F.Np, c->st));
  const void* zu;
  const void* zp;
  const bool use_graph = c->opt.graphs == 0 && !c->prof && c->cap_st != nullptr;
  if (use_graph && !c->pgraph && c->pcalls > 0) CKS(capture_precond<T>(c));
  if (use_graph && c->pgraph) {
    CK(cudaGraphLaunch(c->pgraph, c->st));
    launched(cudaSuccess, c->pgraph_kernels);
    zu = c->g_zu;
    zp = c->g_zp;
  } else {
    const long long before = launches_total();
    CKS(precond_body<T>(c));
    c->pgraph_kernels = (int)(launches_total() - before);
    zu = body_out_u(c);
    zp = body_out_p(c);
  }
  c->pcalls++;
  KL(K_VEC, launch_precond_out<T>((const T*)zu, (const T*)zp, v, z, F.g, c->st));
  CKS(project_pressure(c, z));
  return GS_OK;
}

gs_status precond(gs_ctx* c, const double* v, double* z) {
  return c->fp32 ? precond_T<float>(c, v, z) : precond_T<double>(c, v, z);
}

// FP64 saddle operator on the finest level: y = K x (APPLY) or y = b - K x (RESID)
gs_status saddle(gs_ctx* c, int mode, const double* x, double* y, const double* b, int raw) {
  const Level& F = c->lv[c->L - 1];
  TileArgs<double> a = tile_args<double>(F);
  a.shape = c->saddle_shape;
  a.xu = x; a.xp = x + c->nu; a.yu = y; a.yp = y + c->nu;
  a.bu = b; a.bp = b ? b + c->nu : nullptr; a.raw = raw;
  KL(K_SADDLE64, launch_tile<double>(c->dim, mode, OPS_A | OPS_BT | OPS_B, a, c->st));
  return GS_OK;
}

gs_status norm2_host(gs_ctx* c, const double* x, double* out) {
  return dot_host<double>(c, x, c->N, 1, x, c->N, out);
}

// CGS2 with the double-float basis (explicit second pass): h1 = V^T w; w -= V h1 fused with h2 = V^T w (one
// pass over V); w -= V h2 with the new |w|^2.  h1, h2: j + 1 entries each, nrm: |w|^2 (device).
const int kFusedGsMax = 64;
cudaError_t dots_strip(const float2* V, long long ldv, int k, const double* w, long long n, double* part, int G,
                       cudaStream_t st) {
  return launch_dots_strip_df(V, ldv, k, w, n, part, G, st);
}
cudaError_t dots_strip(const double* V, long long ldv, int k, const double* w, long long n, double* part, int G,
                       cudaStream_t st) {
  return launch_dots_strip_fp64(V, ldv, k, w, n, part, G, st);
}
cudaError_t dots_strip2(const float2* V, long long ldv, int k, const double* w, long long n, double* part, int G,
                        cudaStream_t st) {
  return launch_dots_strip2_df(V, ldv, k, w, n, part, G, st);
}
cudaError_t dots_strip2(const double* V, long long ldv, int k, const double* w, long long n, double* part, int G,
                        cudaStream_t st) {
  return launch_dots_strip2_fp64(V, ldv, k, w, n, part, G, st);
}
cudaError_t multi_axpy_dots(const float2* V, long long ldv, int k, const double* coef, double sign, double* w,
                            long long n, double* part, int G, cudaStream_t st) {
  return launch_multi_axpy_dots_df(V, ldv, k, coef, sign, w, n, part, G, st);
}
cudaError_t multi_axpy_dots(const double* V, long long ldv, int k, const double* coef, double sign, double* w,
                            long long n, double* part, int G, cudaStream_t st) {
  return launch_multi_axpy_dots_fp64(V, ldv, k, coef, sign, w, n, part, G, st);
}
cudaError_t multi_axpy_norm_b(const float2* V, long long ldv, int k, const double* coef, double sign, double* w,
                              long long n, double* part, int G, cudaStream_t st) {
  return launch_multi_axpy_norm_df(V, ldv, k, coef, sign, w, n, part, G, st);
}
cudaError_t multi_axpy_norm_b(const double* V, long long ldv, int k, const double* coef, double sign, double* w,
                              long long n, double* part, int G, cudaStream_t st) {
  return launch_multi_axpy_norm_fp64(V, ldv, k, coef, sign, w, n, part, G, st);
}
// CGS2 with an explicit second pass in three passes over V, for a double-float (float2) or IEEE FP64 (double) basis.
template <typename B>
gs_status cgs2_fused(gs_ctx* c, const B* V, int j, double* h1, double* h2, double* nrm) {
  const long long N = c->N;
  KL(K_DOTS, dots_strip(V, N, j + 1, c->w, N, c->part, c->GF, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, j + 1, c->GF, h1, c->st));
  KL(K_AXPY, multi_axpy_dots(V, N, j + 1, h1, -1.0, c->w, N, c->part, c->GF, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, j + 1, c->GF, h2, c->st));
  KL(K_AXPY, multi_axpy_norm_b(V, N, j + 1, h2, -1.0, c->w, N, c->part, c->GA, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, 1, c->GA, nrm, c->st));
  return GS_OK;
}

// Classical Gram-Schmidt through the Gram matrix (orth = 2): one pass over V for d = [V^T w ;
// V^T v_j] (the newest basis vector, one new column of G = V^T V), c = h1 + (h1 - G h1) on the
// device, then one pass w -= V c with the new |w|^2.  In exact arithmetic c equals the CGS2
// coefficients h1 + V^T (w - V h1): the second pass's dots are replaced by G h1, so V is read twice
// instead of three times and the FP64 work is 3 instead of 4 FMAs per basis entry.
template <typename B>
gs_status cgs_gram(gs_ctx* c, const B* V, int j, double* coef, double* nrm, double* zero = nullptr) {
  const long long N = c->N;
  const int m = c->opt.restart;
  const int g2 = std::min(c->GF, 3 * 152);  // one wave of the two-vector dots (3 CTAs per SM)
  KL(K_DOTS, dots_strip2(V, N, j + 1, c->w, N, c->part, g2, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, 2 * (j + 1), g2, c->gsc, c->st));
  KL(K_DOTS, launch_gram_correct(c->gsc, c->gram, m + 1, j + 1, coef, zero, c->st));
  KL(K_AXPY, multi_axpy_norm_b(V, N, j + 1, coef, -1.0, c->w, N, c->part, c->GA, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, 1, c->GA, nrm, c->st));
  return GS_OK;
}

gs_status fgmres(gs_ctx* c, const double* b, double* x, double tol, int* its, double* relres) {
  const long long N = c->N;
  const int m = c->opt.restart;
  double bn2;
  CKS(norm2_host(c, b, &bn2));
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) return fail(GS_EBREAKDOWN, "right-hand side is not finite");
  c->last_it = 0;
  c->last_rel = 0.0;
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * N, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (its) *its = 0;
    if (relres) *relres = 0.0;
    return GS_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hc = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int it = 0, extra = 0;
  double* h1 = c->dsc;
  double* h2 = c->dsc + (m + 4);
  double* nrm = c->dsc + 2 * (m + 4);
  gs_status result = GS_OK;
  double rel = 0.0;
  for (;;) {
    CKS(saddle(c, TILE_RESID, x, c->r, b));
    double beta2;
    CKS(norm2_host(c, c->r, &beta2));
    const double beta = std::sqrt(beta2);
    if (!std::isfinite(beta)) return fail(GS_EBREAKDOWN, "residual is not finite");
    rel = beta / bnorm;
    if (rel <= tol) break;
    if (it >= c->opt.max_iter) { result = GS_ENOCONV; break; }
    CK(cudaMemcpyAsync(nrm, &beta2, sizeof(double), cudaMemcpyHostToDevice, c->st));
    const bool dfk = c->opt.krylov_fp64 == 0;  // basis in double-float form
    float2* Vdf = reinterpret_cast<float2*>(c->V);
    if (dfk)
      KL(K_AXPY, launch_scale_by_rnorm_df(c->r, nrm, Vdf, c->vcur, N, c->st));
    else
      KL(K_AXPY, launch_scale_by_rnorm(c->r, nrm, c->V, N, c->st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    bool converged = false;
    for (int j = 0; j < m; ++j) {
      const double* Vj = dfk ? c->vcur : c->V + (long long)j * N;
      double* Zj = c->Z + (long long)j * N;
      CKS(precond(c, Vj, Zj));
      CKS(saddle(c, TILE_APPLY, Zj, c->w, nullptr));
      // classical Gram-Schmidt: h = V^T w (with |w|^2 in the same pass), w -= V h (with the new
      // |w|^2 in the same pass); a second pass when |w| fell below 1/sqrt(2) of its value
      // (Daniel-Gragg-Kaufman-Stewart, orth = 1), or always (CGS2, explicit or through the Gram matrix)
      double hn;
      if (c->opt.orth == 2) {
        if (dfk)
          CKS(cgs_gram(c, (const float2*)Vdf, j, h2, nrm));
        else
          CKS(cgs_gram(c, (const double*)c->V, j, h2, nrm));
        CK(cudaMemcpyAsync(c->hpin, h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(c->hpin + (j + 1), nrm, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int i = 0; i <= j; ++i) Hc(i, j) = c->hpin[i];
        hn = std::sqrt(c->hpin[j + 1]);
      } else if (c->opt.orth != 1 && j + 1 <= kFusedGsMax) {
        // CGS2 with the first update fused into the second pass's dots: three passes over V
        if (dfk)
          CKS(cgs2_fused(c, (const float2*)Vdf, j, h1, h2, nrm));
        else
          CKS(cgs2_fused(c, (const double*)c->V, j, h1, h2, nrm));
        CK(cudaMemcpyAsync(c->hpin, h1, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(c->hpin + (j + 1), h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(c->hpin + 2 * (j + 1), nrm, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int i = 0; i <= j; ++i) Hc(i, j) = c->hpin[i];
        for (int i = 0; i <= j; ++i) Hc(i, j) += c->hpin[j + 1 + i];
        hn = std::sqrt(c->hpin[2 * (j + 1)]);
      } else {
        if (dfk)
          KL(K_DOTS, launch_dots_partial_df(Vdf, N, j + 1, c->w, N, c->part, c->G, 1, c->st));
        else
          KL(K_DOTS, launch_dots_norm_partial(c->V, N, j + 1, c->w, N, c->part, c->G, c->st));
        KL(K_DOTS, launch_reduce_partials(c->part, j + 2, c->G, h1, c->st));
        if (dfk)
          KL(K_AXPY, launch_multi_axpy_norm_df(Vdf, N, j + 1, h1, -1.0, c->w, N, c->part, c->GA, c->st));
        else
          KL(K_AXPY, launch_multi_axpy_norm(c->V, N, j + 1, h1, -1.0, c->w, N, c->part, c->GA, c->st));
        KL(K_DOTS, launch_reduce_partials(c->part, 1, c->GA, nrm, c->st));
        CK(cudaMemcpyAsync(c->hpin, h1, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(c->hpin + (m + 1), nrm, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int i = 0; i <= j; ++i) Hc(i, j) = c->hpin[i];
        const double wn0 = std::sqrt(c->hpin[j + 1]);
        hn = std::sqrt(c->hpin[m + 1]);
        if (c->opt.orth != 1 || hn < kReorthKappa * wn0) {
          if (dfk)
            KL(K_DOTS, launch_dots_partial_df(Vdf, N, j + 1, c->w, N, c->part, c->G, 0, c->st));
          else
            KL(K_DOTS, launch_dots_partial<double>(c->V, N, j + 1, c->w, N, c->part, c->G, c->st));
          KL(K_DOTS, launch_reduce_partials(c->part, j + 1, c->G, h2, c->st));
          if (dfk)
            KL(K_AXPY, launch_multi_axpy_norm_df(Vdf, N, j + 1, h2, -1.0, c->w, N, c->part, c->GA, c->st));
          else
            KL(K_AXPY, launch_multi_axpy_norm(c->V, N, j + 1, h2, -1.0, c->w, N, c->part, c->GA, c->st));
          KL(K_DOTS, launch_reduce_partials(c->part, 1, c->GA, nrm, c->st));
          CK(cudaMemcpyAsync(c->hpin, h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, c->st));
          CK(cudaMemcpyAsync(c->hpin + (m + 1), nrm, sizeof(double), cudaMemcpyDeviceToHost, c->st));
          CK(cudaStreamSynchronize(c->st));
          for (int i = 0; i <= j; ++i) Hc(i, j) += c->hpin[i];
          hn = std::sqrt(c->hpin[m + 1]);
        }
      }
      if (!std::isfinite(hn)) return fail(GS_EBREAKDOWN, "Arnoldi vector is not finite");
      Hc(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        const double tmp = cs[i] * Hc(i, j) + sn[i] * Hc(i + 1, j);
        Hc(i + 1, j) = -sn[i] * Hc(i, j) + cs[i] * Hc(i + 1, j);
        Hc(i, j) = tmp;
      }
      const double rr = std::hypot(Hc(j, j), Hc(j + 1, j));
      cs[j] = Hc(j, j) / rr;
      sn[j] = Hc(j + 1, j) / rr;
      Hc(j, j) = rr;
      Hc(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      it++;
      k = j + 1;
      if (std::fabs(g[j + 1]) / bnorm <= tol || hn == 0.0) { converged = true; break; }
      if (it >= c->opt.max_iter) break;
      if (dfk)
        KL(K_AXPY, launch_scale_by_rnorm_df(c->w, nrm, Vdf + (long long)(j + 1) * N, c->vcur, N, c->st));
      else
        KL(K_AXPY, launch_scale_by_rnorm(c->w, nrm, c->V + (long long)(j + 1) * N, N, c->st));
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= Hc(i, q) * y[q];
      y[i] = s / Hc(i, i);
    }
    CK(cudaMemcpyAsync(h1, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, c->st));
    KL(K_AXPY, launch_multi_axpy(c->Z, N, k, h1, 1.0, x, N, c->st));
    if (converged) {
      CKS(saddle(c, TILE_RESID, x, c->r, b));
      double r2;
      CKS(norm2_host(c, c->r, &r2));
      rel = std::sqrt(r2) / bnorm;
      if (!std::isfinite(rel)) return fail(GS_EBREAKDOWN, "residual is not finite");
      if (rel <= tol) break;
      if (extra >= 3) { result = GS_ENOCONV; break; }
      extra++;
    } else if (it >= c->opt.max_iter) {
      CKS(saddle(c, TILE_RESID, x, c->r, b));
      double r2;
      CKS(norm2_host(c, c->r, &r2));
      rel = std::sqrt(r2) / bnorm;
      result = rel <= tol ? GS_OK : GS_ENOCONV;
      break;
    }
  }
  CKS(project_pressure(c, x));
  CK(cudaStreamSynchronize(c->st));
  c->last_it = it;
  c->last_rel = rel;
  if (its) *its = it;
  if (relres) *relres = rel;
  if (result == GS_ENOCONV) g_err = "FGMRES did not reach the tolerance";
  return result;
}

template <typename T>
gs_status apply_level_T(gs_ctx* c, int l, gs_op op, const void* xv, void* yv, const void* auxv) {
  Level& lv = c->lv[l];
  const T* x = (const T*)xv;
  T* y = (T*)yv;
  const T* aux = (const T*)auxv;
  const bool finest = l == c->L - 1;
  const bool mgprec = (sizeof(T) == 4) == c->fp32;
  switch (op) {
    case GS_OP_A:
    case GS_OP_A_RAW: {
      TileArgs<T> a = tile_args<T>(lv);
      a.xu = x; a.yu = y; a.raw = op == GS_OP_A_RAW;
      CK(launch_tile<T>(c->dim, TILE_APPLY, OPS_A, a, c->st));
      return GS_OK;
    }
    case GS_OP_RESIDUAL_A: {
      if (!aux) return fail(GS_EINVAL, "residual needs aux = b");
      TileArgs<T> a = tile_args<T>(lv);
      a.xu = x; a.yu = y; a.bu = aux;
      CK(launch_tile<T>(c->dim, TILE_RESID, OPS_A, a, c->st));
      return GS_OK;
    }
    case GS_OP_DIAG_A:
      if (lv.conv) {  // corrector stage: diag(A_c) = diag(A) + diag(rho (C + S)), formed in FP64
        CK(launch_diagA<double>(lv.g, lv.c64, lv.eta64, lv.alpha64, c->t1, 0, c->st));
        CK(launch_diag_conv(lv.g, lv.vc64, lv.rk64, lv.rho, c->t1, c->st));
        CK(launch_cast<double, T>(c->t1, y, lv.nu, (T)1, c->st));
        return GS_OK;
      }
      CK(launch_diagA<T>(lv.g, coef<T>(lv), etap<T>(lv), alphap<T>(lv), y, 0, c->st));
      return GS_OK;
    case GS_OP_SMOOTH: {
      if (!mgprec || (l == 0 && c->opt.coarse_mode != 1))
        return fail(GS_EINVAL, "smoother: level >= 1 (or level 0 with coarse_mode 1), MG precision");
      if (aux) CK(cudaMemcpyAsync(lv.xA, aux, sizeof(T) * lv.nu, cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(lv.b, x, sizeof(T) * lv.nu, cudaMemcpyDeviceToDevice, c->st));
      for (int s = 0; s < c->opt.smooth_steps; ++s) CKS(cheb<T>(c, l, (const T*)lv.b, s == 0 && !aux));
      CK(cudaMemcpyAsync(y, lv.xA, sizeof(T) * lv.nu, cudaMemcpyDeviceToDevice, c->st));
      return GS_OK;
    }
    case GS_OP_CHEB_STEP: {
      // one fused step r = b - A x, d = c1 d + c2 D^-1 r, y = x + d with the coefficients of the
      // level's second Chebyshev step; aux = [b | d | D^-1] (3 d N_v,l entries, d updated in place)
      if (!aux) return fail(GS_EINVAL, "Chebyshev step needs aux = [b | d | D^-1]");
      if (!(lv.lam_hi > 0.0)) return fail(GS_EINVAL, "level has no Chebyshev bounds (level 0 with a dense coarse solve)");
      if ((const void*)x == (const void*)y) return fail(GS_EINVAL, "x and y must not alias");
      const double hi = lv.lam_hi, lo = hi / 15.0;
      const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
      const double rho = 1.0 / sigma, rn = 1.0 / (2.0 * sigma - rho);
      TileArgs<T> a = tile_args<T>(lv);
      a.xu = x; a.bu = aux; a.d = const_cast<T*>(aux) + lv.nu; a.dinv = aux + 2 * lv.nu; a.xout = y;
      a.c1 = (T)(rn * rho); a.c2 = (T)(2.0 * rn / delta); a.use_d = 1;
      CK(launch_tile<T>(c->dim, TILE_CHEB, OPS_A, a, c->st));
      return GS_OK;
    }
    case GS_OP_RESTRICT:
      if (l == 0) return fail(GS_EINVAL, "restriction needs level >= 1");
      CK(launch_restrict<T>(lv.g, c->lv[l - 1].g, x, y, c->st));
      return GS_OK;
    case GS_OP_PROLONGATE:
      if (l == 0) return fail(GS_EINVAL, "prolongation needs level >= 1");
      CK(launch_prolong_add<T>(lv.g, c->lv[l - 1].g, x, y, c->st));
      return GS_OK;
    case GS_OP_B:
    case GS_OP_BT: {
      if (!finest) return fail(GS_EINVAL, "B / B^T on the finest level only");
      TileArgs<T> a = tile_args<T>(lv);
      if (op == GS_OP_B) { a.xu = x; a.yp = y; } else { a.xp = x; a.yu = y; }
      CK(launch_tile<T>(c->dim, TILE_APPLY, op == GS_OP_B ? OPS_B : OPS_BT, a, c->st));
      return GS_OK;
    }
    case GS_OP_SCHUR_MASS: {
      if (!finest) return fail(GS_EINVAL, "Schur mass on the finest level only");
      PMassArgs<T> a{};
      a.g = lv.g; a.c = coef<T>(lv); a.eta = etap<T>(lv); a.x = x; a.y = y;
      CK(launch_pmass<T>(TILE_APPLY, a, c->st));
      return GS_OK;
    }
    case GS_OP_PLAP: {
      if (!c->cc) return fail(GS_EINVAL, "pressure Laplacian needs the Cahouet-Chabard Schur term");
      PLapArgs<T> a = plap_args<T>(lv);
      a.x = x; a.y = y;
      CK(launch_plap<T>(TILE_APPLY, a, c->st));
      return GS_OK;
    }
    case GS_OP_PLAP_INV: {
      if (!c->cc || !finest || !mgprec) return fail(GS_EINVAL, "pressure V-cycle: CC active, finest level, MG precision");
      CKS(plap_inverse<T>(c, x));
      CK(launch_mask_copy<T>((const T*)lv.pxA, lv.pcmask, y, lv.Np, c->st));
      return GS_OK;
    }
    case GS_OP_PRESTRICT:
    case GS_OP_PPROLONGATE: {
      if (!c->cc || l == 0) return fail(GS_EINVAL, "pressure transfer: CC active, level >= 1");
      const Level& cl = c->lv[l - 1];
      if (op == GS_OP_PRESTRICT)
        CK(launch_p_restrict<T>(lv.g, cl.g, lv.pcmask, cl.pcmask, x, y, c->st));
      else
        CK(launch_p_prolong_add<T>(lv.g, cl.g, lv.pcmask, cl.pcmask, x, y, c->st));
      return GS_OK;
    }
    case GS_OP_SCHUR_DIAG:
    case GS_OP_SADDLE_SMOOTH:
    case GS_OP_SADDLE_VCYCLE: {
      if (!c->mono || !mgprec) return fail(GS_EINVAL, "saddle-point multigrid operators: precond_kind 1, MG precision");
      if (op == GS_OP_SCHUR_DIAG) {
        CK(launch_schur_diag<T>(lv.g, lv.c64, (const T*)lv.dinv, y, 0, c->st));
        return GS_OK;
      }
      if (op == GS_OP_SADDLE_SMOOTH && l == 0 && c->opt.coarse_mode != 1)
        return fail(GS_EINVAL, "block smoother: level >= 1 (or level 0 with coarse_mode 1)");
      const long long n = lv.nu + lv.Np;
      CK(launch_cast<T, T>(x, (T*)lv.mr, n, (T)1, c->st));
      if (op == GS_OP_SADDLE_SMOOTH)
        CKS(mono_smooth_step<T>(c, l, true));
      else
        CKS(mono_vcycle<T>(c, l));
      CK(launch_cast<T, T>((const T*)lv.ms, y, n, (T)1, c->st));
      return GS_OK;
    }
    case GS_OP_SCHUR_INV: {
      if (!finest || !mgprec) return fail(GS_EINVAL, "Schur inverse: finest level, MG precision");
      CKS(schur_inv<T>(c, x));
      CK(cudaMemcpyAsync(y, c->p_xA, sizeof(T) * lv.Np, cudaMemcpyDeviceToDevice, c->st));
      return GS_OK;
    }
    default:
      return fail(GS_EINVAL, "unknown operator");
  }
}

}  // namespace

// ---- deflation space: E = Z^T A Z from FP64 applies of colour-batched modes -------------------
// Inclusions k and l interact when some cell has unconstrained nodes of both (then z_l^T A z_k
// may be nonzero).  With a distance-2 colouring of that graph, applying A to the sum of mode t
// over the inclusions of one colour gives, for every inclusion l, the entry of E in row (l, b)
// and column (k, t) for the single inclusion k of that colour that interacts with l (or is l).
gs_status setup_deflation(gs_ctx* c) {
  if (c->opt.deflate != 1) return GS_OK;
  const Level& F = c->lv[c->L - 1];
  c->defl = DeflArgs{};
  c->defl.g = F.g;
  c->defl.nodes = c->d_nodes;
  c->defl.off = c->d_off;
  c->defl.cen = c->d_cen;
  c->defl.ninc = c->defl_ninc;
  if (c->defl_ninc == 0) return GS_OK;
  const int dim = c->dim, nt = dim == 2 ? 3 : 6, ninc = c->defl_ninc, M = c->defl_M;
  CK(cudaMemcpyAsync(c->d_nodes, c->hd_nodes.data(), sizeof(int) * c->hd_nodes.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_off, c->hd_off.data(), sizeof(int) * c->hd_off.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->d_cen, c->hd_cen.data(), sizeof(double) * c->hd_cen.size(), cudaMemcpyHostToDevice, c->st));
  const int nv0 = F.g.nv[0], nv1 = F.g.nv[1];
  std::vector<std::vector<int>> nb(ninc);
  {
    std::vector<std::pair<long long, int>> touch;  // (cell, inclusion) through unconstrained nodes
    for (int k = 0; k < ninc; ++k)
      for (int i = c->hd_off[k]; i < c->hd_off[k + 1]; ++i) {
        const int nd = c->hd_nodes[i];
        const int idx[3] = {nd % nv0, (nd / nv0) % nv1, dim == 3 ? nd / (nv0 * nv1) : 0};
        int cl[3][2], cnt[3];
        for (int a = 0; a < 3; ++a) {
          cnt[a] = 0;
          if (a >= dim) { cl[a][cnt[a]++] = 0; continue; }
          const int v = idx[a];
          if (v & 1) { cl[a][cnt[a]++] = v >> 1; continue; }
          if ((v >> 1) - 1 >= 0) cl[a][cnt[a]++] = (v >> 1) - 1;
          if ((v >> 1) < F.n[a]) cl[a][cnt[a]++] = v >> 1;
        }
        for (int z = 0; z < cnt[2]; ++z)
          for (int y = 0; y < cnt[1]; ++y)
            for (int x = 0; x < cnt[0]; ++x)
              touch.push_back({cl[0][x] + (long long)F.n[0] * (cl[1][y] + (long long)F.n[1] * cl[2][z]), k});
      }
    std::sort(touch.begin(), touch.end());
    touch.erase(std::unique(touch.begin(), touch.end()), touch.end());
    for (size_t i = 0; i < touch.size();) {
      size_t j = i;
      while (j < touch.size() && touch[j].first == touch[i].first) ++j;
      for (size_t a = i; a < j; ++a)
        for (size_t b = i; b < j; ++b)
          if (touch[a].second != touch[b].second) nb[touch[a].second].push_back(touch[b].second);
      i = j;
    }
    for (auto& v : nb) {
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
  }
  std::vector<int> color(ninc, -1);
  int ncol = 0;
  for (int k = 0; k < ninc; ++k) {
    std::vector<char> used(ncol + 1, 0);
    for (int a : nb[k]) {
      if (color[a] >= 0) used[color[a]] = 1;
      for (int b : nb[a])
        if (b != k && color[b] >= 0) used[color[b]] = 1;
    }
    int col = 0;
    while (used[col]) ++col;
    color[k] = col;
    ncol = std::max(ncol, col + 1);
  }
  std::vector<double> E((size_t)M * M, 0.0), yh(M), ch(M);
  for (int col = 0; col < ncol; ++col)
    for (int t = 0; t < nt; ++t) {
      std::fill(yh.begin(), yh.end(), 0.0);
      bool any = false;
      for (int k = 0; k < ninc; ++k)
        if (color[k] == col && c->hd_keep[k * nt + t]) { yh[k * nt + t] = 1.0; any = true; }
      if (!any) continue;
      CK(cudaMemcpyAsync(c->d_y, yh.data(), sizeof(double) * M, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemsetAsync(c->w, 0, sizeof(double) * c->nu, c->st));
      CK(launch_defl_add<double>(c->defl, c->d_y, c->w, c->st));
      CKS(apply_level_T<double>(c, c->L - 1, GS_OP_A, c->w, c->r, nullptr));
      CK(launch_defl_dots<double>(c->defl, c->r, c->d_c, c->st));
      CK(cudaMemcpyAsync(ch.data(), c->d_c, sizeof(double) * M, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      for (int l = 0; l < ninc; ++l) {
        int src = color[l] == col ? l : -1;
        for (int k : nb[l])
          if (src < 0 && color[k] == col) src = k;
        if (src < 0 || !c->hd_keep[src * nt + t]) continue;
        for (int b = 0; b < nt; ++b)
          if (c->hd_keep[l * nt + b]) E[(size_t)(l * nt + b) * M + (src * nt + t)] = ch[l * nt + b];
      }
    }
  // invert E on the kept modes (Gauss-Jordan, partial pivoting), zero rows / columns elsewhere
  std::vector<int> kept;
  for (int q = 0; q < M; ++q)
    if (c->hd_keep[q]) kept.push_back(q);
  const int m = (int)kept.size();
  std::vector<double> A((size_t)m * 2 * m, 0.0);
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[(size_t)i * 2 * m + j] = E[(size_t)kept[i] * M + kept[j]];
    A[(size_t)i * 2 * m + m + i] = 1.0;
  }
  for (int p = 0; p < m; ++p) {
    int piv = p;
    for (int i = p + 1; i < m; ++i)
      if (std::fabs(A[(size_t)i * 2 * m + p]) > std::fabs(A[(size_t)piv * 2 * m + p])) piv = i;
    if (!(std::fabs(A[(size_t)piv * 2 * m + p]) > 0.0)) return fail(GS_EINVAL, "deflation: singular Z^T A Z");
    if (piv != p)
      for (int j = 0; j < 2 * m; ++j) std::swap(A[(size_t)p * 2 * m + j], A[(size_t)piv * 2 * m + j]);
    const double inv = 1.0 / A[(size_t)p * 2 * m + p];
    for (int j = 0; j < 2 * m; ++j) A[(size_t)p * 2 * m + j] *= inv;
    for (int i = 0; i < m; ++i) {
      if (i == p) continue;
      const double f = A[(size_t)i * 2 * m + p];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * m; ++j) A[(size_t)i * 2 * m + j] -= f * A[(size_t)p * 2 * m + j];
    }
  }
  std::fill(E.begin(), E.end(), 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) E[(size_t)kept[i] * M + kept[j]] = A[(size_t)i * 2 * m + m + j];
  CK(cudaMemcpyAsync(c->d_Einv, E.data(), sizeof(double) * E.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return GS_OK;
}

// ---- resumable FGMRES for the batching engine (gs_slot.h) ---------------------------------------
// Offsets in the context's scalar area dsc (4 (m + 4) doubles): h1 at 0, h2 at m + 4, the norm
// at 2 (m + 4), the pressure-mean sum at 3 (m + 4), then |r|^2 and |b|^2.
namespace gs {
namespace {
double* sl_nrm(gs_ctx* c) { return c->dsc + 2 * (c->opt.restart + 4); }
double* sl_beta2(gs_ctx* c) { return c->dsc + 3 * (c->opt.restart + 4) + 1; }
double* sl_bn2(gs_ctx* c) { return c->dsc + 3 * (c->opt.restart + 4) + 2; }

gs_status sl_fail(gs_ctx* c, gs_status s, const std::string& why) {
  c->ks.result = s;
  c->ks.err = why;
  c->ks.phase = KState::DONE;
  return GS_OK;  // a failed solve is a finished slot, not an engine error
}

// |v|^2 into dst with the kernels of dot_host (k = 1)
gs_status sl_norm2(gs_ctx* c, const double* v, double* dst) {
  KL(K_DOTS, launch_dots_partial<double>(v, c->N, 1, v, c->N, c->part, c->G, c->st));
  KL(K_DOTS, launch_reduce_partials(c->part, 1, c->G, dst, c->st));
  return GS_OK;
}

template <typename T>
gs_status sl_cast_in(gs_ctx* c, const double* v) {
  Level& F = c->lv[c->L - 1];
  KL(K_VEC, launch_precond_in<T>(v, (T*)body_in_u(c), (T*)body_in_p(c), F.nu, F.Np, c->st));
  return GS_OK;
}
template <typename T>
gs_status sl_cast_out(gs_ctx* c, const double* v, double* z) {
  Level& F = c->lv[c->L - 1];
  KL(K_VEC, launch_precond_out<T>((const T*)c->ks.zu, (const T*)c->ks.zp, v, z, F.g, c->st));
  CKS(project_pressure(c, z));
  return GS_OK;
}
}  // namespace

gs_status report(gs_status s, const std::string& why) { return fail(s, why); }

gs_status slot_begin(gs_ctx* c, const double* b, double* x, double tol) {
  if (!c || !b || !x) return fail(GS_EINVAL, "NULL argument");
  if (!(tol > 0.0)) return fail(GS_EINVAL, "tol must be > 0");
  if (c->opt.orth == 1) return fail(GS_EINVAL, "batched solves need a fixed number of Gram-Schmidt passes (orth != 1)");
  if (c->prof) return fail(GS_EINVAL, "kernel profiling is on for this context");
  KState& k = c->ks;
  const int m = c->opt.restart;
  k.phase = KState::INIT;
  k.pend = KState::P_NONE;
  k.b = b;
  k.x = x;
  k.tol = tol;
  k.from_conv = k.from_max = false;
  k.project_final = true;
  k.it = k.extra = k.j = k.kx = 0;
  k.bnorm = k.rel = 0.0;
  k.H.assign((size_t)(m + 1) * m, 0.0);
  k.cs.assign(m, 0.0);
  k.sn.assign(m, 0.0);
  k.g.assign(m + 1, 0.0);
  k.y.assign(m, 0.0);
  k.ydev = nullptr;
  k.result = GS_OK;
  k.err.clear();
  c->last_it = 0;
  c->last_rel = 0.0;
  return GS_OK;
}

const Recorder* slot_body(gs_ctx* c, gs_status* st) {
  KState& k = c->ks;
  *st = GS_OK;
  if (k.body_ok) return &k.body;
  k.body.clear();
  Recorder* prev = current_recorder();
  current_recorder() = &k.body;
  *st = c->fp32 ? precond_body<float>(c) : precond_body<double>(c);
  current_recorder() = prev;
  if (*st != GS_OK) return nullptr;
  k.zu = body_out_u(c);  // where the recorded launches leave z_u and z_p
  k.zp = body_out_p(c);
  k.body_ok = true;
  return &k.body;
}

bool slot_wants_body(const gs_ctx* c) { return c->ks.phase == KState::ITER; }

gs_status slot_record_pre(gs_ctx* c) {
  KState& k = c->ks;
  const long long N = c->N;
  const bool dfk = c->opt.krylov_fp64 == 0;
  float2* Vdf = reinterpret_cast<float2*>(c->V);
  switch (k.pend) {
    case KState::P_SCALE:  // v_{j+1} = w / |w|
      if (dfk)
        KL(K_AXPY, launch_scale_by_rnorm_df(c->w, sl_nrm(c), Vdf + (long long)k.j * N, c->vcur, N, c->st));
      else
        KL(K_AXPY, launch_scale_by_rnorm(c->w, sl_nrm(c), c->V + (long long)k.j * N, N, c->st));
      break;
    case KState::P_XUPDATE:  // x += Z y
      KL(K_AXPY, launch_multi_axpy(c->Z, N, k.kx, k.ydev, 1.0, k.x, N, c->st));
      break;
    case KState::P_ZERO_X:
      KL(K_VEC, launch_fill_zero<double>(k.x, N, c->st));
      break;
    default:
      break;
  }
  k.pend = KState::P_NONE;
  switch (k.phase) {
    case KState::INIT:
      CKS(sl_norm2(c, k.b, sl_bn2(c)));
      // fall through: the first residual
    case KState::RESID:
      CKS(saddle(c, TILE_RESID, k.x, c->r, k.b));
      CKS(sl_norm2(c, c->r, sl_beta2(c)));
      if (dfk)
        KL(K_AXPY, launch_scale_by_rnorm_df(c->r, sl_beta2(c), Vdf, c->vcur, N, c->st));
      else
        KL(K_AXPY, launch_scale_by_rnorm(c->r, sl_beta2(c), c->V, N, c->st));
      break;
    case KState::ITER: {
      const double* v = dfk ? c->vcur : c->V + (long long)k.j * N;
      CKS(c->fp32 ? sl_cast_in<float>(c, v) : sl_cast_in<double>(c, v));
      break;
    }
    case KState::FINAL:
      if (k.project_final) CKS(project_pressure(c, k.x));
      break;
    default:
      break;
  }
  return GS_OK;
}

gs_status slot_record_post(gs_ctx* c, double* gather_dev) {
  KState& k = c->ks;
  const long long N = c->N;
  const int m = c->opt.restart;
  const bool dfk = c->opt.krylov_fp64 == 0;
  float2* Vdf = reinterpret_cast<float2*>(c->V);
  switch (k.phase) {
    case KState::INIT:
      KL(K_VEC, launch_gather3(sl_bn2(c), 1, sl_beta2(c), 1, sl_beta2(c), 0, gather_dev, c->st));
      break;
    case KState::RESID:
      KL(K_VEC, launch_gather3(sl_beta2(c), 1, sl_beta2(c), 0, sl_beta2(c), 0, gather_dev, c->st));
      break;
    case KState::ITER: {
      const int j = k.j;
      const double* v = dfk ? c->vcur : c->V + (long long)j * N;
      double* Zj = c->Z + (long long)j * N;
      double* h1 = c->dsc;
      double* h2 = c->dsc + (m + 4);
      double* nrm = sl_nrm(c);
      CKS(c->fp32 ? sl_cast_out<float>(c, v, Zj) : sl_cast_out<double>(c, v, Zj));
      CKS(saddle(c, TILE_APPLY, Zj, c->w, nullptr));
      if (c->opt.orth == 2) {  // coefficients in h1, zeros in h2
        if (dfk)
          CKS(cgs_gram(c, (const float2*)Vdf, j, h1, nrm, h2));
        else
          CKS(cgs_gram(c, (const double*)c->V, j, h1, nrm, h2));
      } else if (j + 1 <= kFusedGsMax) {
        if (dfk)
          CKS(cgs2_fused(c, (const float2*)Vdf, j, h1, h2, nrm));
        else
          CKS(cgs2_fused(c, (const double*)c->V, j, h1, h2, nrm));
      } else {
        if (dfk)
          KL(K_DOTS, launch_dots_partial_df(Vdf, N, j + 1, c->w, N, c->part, c->G, 1, c->st));
        else
          KL(K_DOTS, launch_dots_norm_partial(c->V, N, j + 1, c->w, N, c->part, c->G, c->st));
        KL(K_DOTS, launch_reduce_partials(c->part, j + 2, c->G, h1, c->st));
        if (dfk)
          KL(K_AXPY, launch_multi_axpy_norm_df(Vdf, N, j + 1, h1, -1.0, c->w, N, c->part, c->GA, c->st));
        else
          KL(K_AXPY, launch_multi_axpy_norm(c->V, N, j + 1, h1, -1.0, c->w, N, c->part, c->GA, c->st));
        KL(K_DOTS, launch_reduce_partials(c->part, 1, c->GA, nrm, c->st));
        if (dfk)
          KL(K_DOTS, launch_dots_partial_df(Vdf, N, j + 1, c->w, N, c->part, c->G, 0, c->st));
        else
          KL(K_DOTS, launch_dots_partial<double>(c->V, N, j + 1, c->w, N, c->part, c->G, c->st));
        KL(K_DOTS, launch_reduce_partials(c->part, j + 1, c->G, h2, c->st));
        if (dfk)
          KL(K_AXPY, launch_multi_axpy_norm_df(Vdf, N, j + 1, h2, -1.0, c->w, N, c->part, c->GA, c->st));
        else
          KL(K_AXPY, launch_multi_axpy_norm(c->V, N, j + 1, h2, -1.0, c->w, N, c->part, c->GA, c->st));
        KL(K_DOTS, launch_reduce_partials(c->part, 1, c->GA, nrm, c->st));
      }
      KL(K_VEC, launch_gather3(h1, j + 1, h2, j + 1, nrm, 1, gather_dev, c->st));
      break;
    }
    default:
      break;
  }
  return GS_OK;
}

gs_status slot_update(gs_ctx* c, const double* gathered, double* y_host, const double* y_dev) {
  KState& k = c->ks;
  const int m = c->opt.restart;
  auto Hc = [&](int i, int j) -> double& { return k.H[(size_t)i * m + j]; };
  switch (k.phase) {
    case KState::INIT:
    case KState::RESID: {
      double beta2;
      if (k.phase == KState::INIT) {
        k.bnorm = std::sqrt(gathered[0]);
        if (!std::isfinite(k.bnorm)) return sl_fail(c, GS_EBREAKDOWN, "right-hand side is not finite");
        if (k.bnorm == 0.0) {  // x = 0, no iterations
          k.pend = KState::P_ZERO_X;
          k.project_final = false;
          k.rel = 0.0;
          k.phase = KState::FINAL;
          return GS_OK;
        }
        beta2 = gathered[1];
      } else {
        beta2 = gathered[0];
      }
      const double beta = std::sqrt(beta2);
      if (!std::isfinite(beta)) return sl_fail(c, GS_EBREAKDOWN, "residual is not finite");
      k.rel = beta / k.bnorm;
      if (k.from_conv) {  // explicit check after a cycle that converged on the implicit estimate
        k.from_conv = false;
        if (k.rel <= k.tol) { k.phase = KState::FINAL; return GS_OK; }
        if (k.extra >= 3) { k.result = GS_ENOCONV; k.phase = KState::FINAL; return GS_OK; }
        k.extra++;
      } else if (k.from_max) {
        k.from_max = false;
        k.result = k.rel <= k.tol ? GS_OK : GS_ENOCONV;
        k.phase = KState::FINAL;
        return GS_OK;
      }
      if (k.rel <= k.tol) { k.phase = KState::FINAL; return GS_OK; }
      if (k.it >= c->opt.max_iter) { k.result = GS_ENOCONV; k.phase = KState::FINAL; return GS_OK; }
      std::fill(k.g.begin(), k.g.end(), 0.0);
      k.g[0] = beta;
      k.j = 0;
      k.phase = KState::ITER;
      return GS_OK;
    }
    case KState::ITER: {
      const int j = k.j;
      for (int i = 0; i <= j; ++i) Hc(i, j) = gathered[i];
      for (int i = 0; i <= j; ++i) Hc(i, j) += gathered[j + 1 + i];
      const double hn = std::sqrt(gathered[2 * (j + 1)]);
      if (!std::isfinite(hn)) return sl_fail(c, GS_EBREAKDOWN, "Arnoldi vector is not finite");
      Hc(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        const double tmp = k.cs[i] * Hc(i, j) + k.sn[i] * Hc(i + 1, j);
        Hc(i + 1, j) = -k.sn[i] * Hc(i, j) + k.cs[i] * Hc(i + 1, j);
        Hc(i, j) = tmp;
      }
      const double rr = std::hypot(Hc(j, j), Hc(j + 1, j));
      k.cs[j] = Hc(j, j) / rr;
      k.sn[j] = Hc(j + 1, j) / rr;
      Hc(j, j) = rr;
      Hc(j + 1, j) = 0.0;
      k.g[j + 1] = -k.sn[j] * k.g[j];
      k.g[j] = k.cs[j] * k.g[j];
      k.it++;
      const bool converged = std::fabs(k.g[j + 1]) / k.bnorm <= k.tol || hn == 0.0;
      if (converged || k.it >= c->opt.max_iter || j + 1 == m) {
        const int kk = j + 1;
        for (int i = kk - 1; i >= 0; --i) {
          double s = k.g[i];
          for (int q = i + 1; q < kk; ++q) s -= Hc(i, q) * k.y[q];
          k.y[i] = s / Hc(i, i);
        }
        for (int i = 0; i < kk; ++i) y_host[i] = k.y[i];
        k.ydev = y_dev;
        k.kx = kk;
        k.pend = KState::P_XUPDATE;
        k.from_conv = converged;
        k.from_max = !converged && k.it >= c->opt.max_iter;
        k.phase = KState::RESID;
      } else {
        k.j = j + 1;
        k.pend = KState::P_SCALE;
      }
      return GS_OK;
    }
    case KState::FINAL:
      k.phase = KState::DONE;
      c->last_it = k.it;
      c->last_rel = k.rel;
      if (k.result == GS_ENOCONV) k.err = "FGMRES did not reach the tolerance";
      return GS_OK;
    default:
      return GS_OK;
  }
}

bool slot_done(const gs_ctx* c, gs_status* status, int* iterations, double* rel_residual) {
  const KState& k = c->ks;
  if (k.phase != KState::DONE) return false;
  if (status) *status = k.result;
  if (iterations) *iterations = k.it;
  if (rel_residual) *rel_residual = k.rel;
  return true;
}
const char* slot_error(const gs_ctx* c) { return c->ks.err.c_str(); }
int slot_restart(const gs_ctx* c) { return c->opt.restart; }
cudaStream_t slot_stream(const gs_ctx* c) { return c->st; }

}  // namespace gs



// =====================================================================================
extern "C" {

size_t gs_footprint_bytes(const gs_mesh* mesh, int levels, const gs_options* opts) {
  gs_ctx c;
  c.opt = normalize_opts(opts);
  c.fp32 = c.opt.mg_precision == 32;
  if (plan(mesh, levels, nullptr, &c) != GS_OK) return 0;
  Arena ar;
  layout(&c, ar);
  return c.footprint;
}

}  // extern "C"

namespace {
gs_status create_impl(const gs_mesh* mesh, int levels, const double* eta_per_cell, double alpha,
                      const double* alpha_per_cell, const gs_options* opts, void* stream, void* workspace,
                      size_t workspace_bytes, gs_ctx** out) {
  if (!out) return fail(GS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!eta_per_cell) return fail(GS_EINVAL, "eta_per_cell is NULL");
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) return fail(GS_EINVAL, "alpha must be finite and >= 0");
  if (!workspace) return fail(GS_EINVAL, "workspace is NULL");
  if (((uintptr_t)workspace & 255u) != 0) return fail(GS_EINVAL, "workspace must be 256-byte aligned");
  gs_ctx* c = new gs_ctx();
  c->opt = normalize_opts(opts);
  c->fp32 = c->opt.mg_precision == 32;
  c->alpha = alpha;
  c->alpha_cells = alpha_per_cell != nullptr;
  c->st = (cudaStream_t)stream;
  gs_status s = plan(mesh, levels, eta_per_cell, c, alpha_per_cell);
  if (s != GS_OK) { delete c; return s; }
  {
    Arena dry;
    layout(c, dry);
  }
  if (workspace_bytes < c->footprint) {
    delete c;
    return fail(GS_ENOMEM, "workspace smaller than gs_footprint_bytes()");
  }
  Arena ar;
  ar.base = (char*)workspace;
  layout(c, ar);
  c->cc = c->cc_alloc && (c->opt.schur_kind == 2 || c->alpha > 0.0);
  set_geom(c, mesh);
  cudaError_t e = cudaMallocHost(&c->hpin, sizeof(double) * (2 * c->opt.restart + 8));
  if (e != cudaSuccess) { delete c; return fail(GS_ECUDA, std::string("pinned buffer: ") + cudaGetErrorString(e)); }
  if (c->opt.graphs == 0 && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess)
    c->cap_st = nullptr;  // graphs stay off
  s = setup(c);
  if (s == GS_OK) s = setup_deflation(c);
  if (s != GS_OK) {
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    cudaFreeHost(c->hpin);
    delete c;
    return s;
  }
  *out = c;
  return GS_OK;
}
}  // namespace

extern "C" {

gs_status gs_create(const gs_mesh* mesh, int levels, const double* eta_per_cell, double alpha,
                    const gs_options* opts, void* stream, void* workspace, size_t workspace_bytes,
                    gs_ctx** out) {
  return create_impl(mesh, levels, eta_per_cell, alpha, nullptr, opts, stream, workspace, workspace_bytes, out);
}

gs_status gs_create_ex(const gs_mesh* mesh, int levels, const double* eta_per_cell, const double* alpha_per_cell,
                       const gs_options* opts, void* stream, void* workspace, size_t workspace_bytes, gs_ctx** out) {
  if (!alpha_per_cell) return fail(GS_EINVAL, "alpha_per_cell is NULL");
  return create_impl(mesh, levels, eta_per_cell, 0.0, alpha_per_cell, opts, stream, workspace, workspace_bytes,
                     out);
}

gs_status gs_vmult(gs_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return fail(GS_EINVAL, "NULL argument");
  if (x == y) return fail(GS_EINVAL, "x and y must not alias");
  return saddle(c, TILE_APPLY, x, y, nullptr);
}

gs_status gs_vmult_A(gs_ctx* c, const void* x, void* y, int fp32) {
  if (!c || !x || !y) return fail(GS_EINVAL, "NULL argument");
  if (x == y) return fail(GS_EINVAL, "x and y must not alias");
  return fp32 ? apply_level_T<float>(c, c->L - 1, GS_OP_A, x, y, nullptr)
              : apply_level_T<double>(c, c->L - 1, GS_OP_A, x, y, nullptr);
}

gs_status gs_vcycle(gs_ctx* c, const double* r, double* z) {
  if (!c || !r || !z) return fail(GS_EINVAL, "NULL argument");
  Level& F = c->lv[c->L - 1];
  if (c->fp32) {
    CK(launch_cast<double, float>(r, (float*)F.b, F.nu, 1.0f, c->st));
    CKS(vcycle<float>(c, c->L - 1));
    CK(launch_cast<float, double>((const float*)F.xA, z, F.nu, 1.0, c->st));
  } else {
    CK(cudaMemcpyAsync(F.b, r, sizeof(double) * F.nu, cudaMemcpyDeviceToDevice, c->st));
    CKS(vcycle<double>(c, c->L - 1));
    CK(cudaMemcpyAsync(z, F.xA, sizeof(double) * F.nu, cudaMemcpyDeviceToDevice, c->st));
  }
  return GS_OK;
}

// ---- mesh-extension solve (Eq. "extenstion", Sec. 5): flexible PCG on the velocity block ---------
namespace {
// z = V(r) on the finest level (FP64 in / out), z = r on constrained rows
gs_status ext_precond(gs_ctx* c, const double* r, double* z, const Geom& gu) {
  Level& F = c->lv[c->L - 1];
  if (c->fp32) {
    KL(K_VEC, launch_cast<double, float>(r, (float*)F.b, F.nu, 1.0f, c->st));
    CKS(vcycle<float>(c, c->L - 1));
    KL(K_VEC, launch_cast<float, double>((const float*)F.xA, z, F.nu, 1.0, c->st));
  } else {
    KL(K_VEC, launch_cast<double, double>(r, (double*)F.b, F.nu, 1.0, c->st));
    CKS(vcycle<double>(c, c->L - 1));
    KL(K_VEC, launch_cast<double, double>((const double*)F.xA, z, F.nu, 1.0, c->st));
  }
  KL(K_VEC, launch_copy_constrained(r, z, gu, c->st));
  return GS_OK;
}
// y = A x (APPLY) or y = b - A x (RESID), FP64, finest level
gs_status ext_apply(gs_ctx* c, int mode, const double* x, double* y, const double* b) {
  const Level& F = c->lv[c->L - 1];
  TileArgs<double> a = tile_args<double>(F);
  a.xu = x; a.yu = y; a.bu = b;
  KL(K_SADDLE64, launch_tile<double>(c->dim, mode, OPS_A, a, c->st));
  return GS_OK;
}
}  // namespace

// Flexible (Polak-Ribiere) PCG: beta = z_new . (r_new - r_old) / (z_old . r_old); x0 = rhs on the
// identity rows (Dirichlet data), the caller's guess elsewhere.  Vectors: r and r_old in the first
// two rows of the Krylov basis area (one fused pair of dot products), z, p, q in w, t1, t2.
gs_status gs_solve_A(gs_ctx* c, const double* rhs, double* x, double tol, int* iterations, double* rel_residual) {
  if (!c || !rhs || !x) return fail(GS_EINVAL, "NULL argument");
  if (!(tol > 0.0)) return fail(GS_EINVAL, "tol must be > 0");
  const Level& F = c->lv[c->L - 1];
  const long long n = F.nu;
  Geom gu = F.g;
  gu.Np = 0;  // velocity entries only
  double* r = c->V;
  double* rold = c->V + c->N;
  double *z = c->w, *p = c->t1, *q = c->t2;
  auto dots = [&](const double* V, int k, const double* w, double* out) { return dot_host<double>(c, V, c->N, k, w, n, out); };
  int it = 0;
  double bn2, rn2, rel = 0.0;
  CKS(dots(rhs, 1, rhs, &bn2));
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) return fail(GS_EBREAKDOWN, "right-hand side is not finite");
  KL(K_VEC, launch_copy_constrained(rhs, x, gu, c->st));
  if (bnorm == 0.0) {
    KL(K_VEC, launch_fill_zero<double>(x, n, c->st));
    if (iterations) *iterations = 0;
    if (rel_residual) *rel_residual = 0.0;
    return GS_OK;
  }
  CKS(ext_apply(c, TILE_RESID, x, r, rhs));
  CKS(dots(r, 1, r, &rn2));
  rel = std::sqrt(rn2) / bnorm;
  gs_status st = GS_OK;
  if (rel > tol) {
    CKS(ext_precond(c, r, z, gu));
    KL(K_VEC, launch_cast<double, double>(z, p, n, 1.0, c->st));
    double rz;
    CKS(dots(r, 1, z, &rz));
    const int max_it = c->opt.max_iter;
    while (true) {
      double pq;
      CKS(ext_apply(c, TILE_APPLY, p, q, nullptr));
      CKS(dots(p, 1, q, &pq));
      if (!(pq > 0.0) || !std::isfinite(pq)) { st = GS_EBREAKDOWN; break; }
      const double a = rz / pq;
      KL(K_VEC, launch_cast<double, double>(r, rold, n, 1.0, c->st));
      KL(K_AXPY, launch_axpby<double>(p, x, a, 1.0, n, c->st));
      KL(K_AXPY, launch_axpby<double>(q, r, -a, 1.0, n, c->st));
      ++it;
      CKS(dots(r, 1, r, &rn2));
      rel = std::sqrt(rn2) / bnorm;
      if (rel <= tol) break;
      if (it >= max_it) { st = GS_ENOCONV; break; }
      CKS(ext_precond(c, r, z, gu));
      double zr[2];
      CKS(dots(r, 2, z, zr));  // z . r_new, z . r_old
      const double beta = (zr[0] - zr[1]) / rz;
      rz = zr[0];
      KL(K_AXPY, launch_axpby<double>(z, p, 1.0, beta, n, c->st));
    }
  }
  // explicit residual of the returned iterate
  CKS(ext_apply(c, TILE_RESID, x, r, rhs));
  CKS(dots(r, 1, r, &rn2));
  rel = std::sqrt(rn2) / bnorm;
  c->last_it = it;
  c->last_rel = rel;
  if (iterations) *iterations = it;
  if (rel_residual) *rel_residual = rel;
  CKS(check_device_error(c));
  if (st == GS_EBREAKDOWN) return fail(st, "CG breakdown (p . A p <= 0)");
  if (st == GS_ENOCONV) return fail(st, "CG did not reach the tolerance");
  return GS_OK;
}

gs_status gs_solve(gs_ctx* c, const double* rhs, double* x, double tol, int* iterations, double* rel_residual) {
  if (!c || !rhs || !x) return fail(GS_EINVAL, "NULL argument");
  if (!(tol > 0.0)) return fail(GS_EINVAL, "tol must be > 0");
  const gs_status st = fgmres(c, rhs, x, tol, iterations, rel_residual);
  const gs_status dev = check_device_error(c);
  return dev != GS_OK ? dev : st;
}

gs_status gs_lift_rhs(gs_ctx* c, const double* f, const double* g, double* rhs) {
  if (!c || !f || !g || !rhs) return fail(GS_EINVAL, "NULL argument");
  if (rhs == f || rhs == g) return fail(GS_EINVAL, "rhs must not alias f or g");
  Level& F = c->lv[c->L - 1];
  // M f: velocity mass (alpha = 1, no viscous part) and plain Q1 pressure mass, unconstrained
  {
    TileArgs<double> a = tile_args<double>(F);
    a.c = make_coef<double>(c->dim, F.h, 1.0);
    a.c.eta_scale = 0.0;
    a.conv = 0;  // the load is the plain mass (the corrector terms belong to the operator)
    a.xu = f; a.yu = c->t1; a.raw = 1;
    CK(launch_tile<double>(c->dim, TILE_APPLY, OPS_A, a, c->st));
    PMassArgs<double> p{};
    p.g = F.g; p.c = F.c64; p.eta = F.eta64; p.x = f + c->nu; p.y = c->t1 + c->nu; p.raw = 1; p.unit = 1;
    CK(launch_pmass<double>(TILE_APPLY, p, c->st));
  }
  // K_raw applied to the Dirichlet data (g restricted to the constrained entries)
  CK(cudaMemsetAsync(c->w, 0, sizeof(double) * c->N, c->st));
  CK(launch_copy_constrained(g, c->w, F.g, c->st));
  CKS(saddle(c, TILE_APPLY, c->w, c->t2, nullptr, 1));
  CK(launch_combine_lift(c->t1, c->t2, g, F.vmask, F.pmask, F.g, rhs, c->st));
  return GS_OK;
}

}  // extern "C"

// ---- corrector stage (Sec. 3.1.2, Eq. "v_star" and Eq. "a_stab") ------------------------------
namespace {
// Brooks-Hughes streamline parameter r_K per cell: |v°| at the cell's centre node, h_K the cell
// diameter, Pe = rho |v°| h_K / (2 eta_K p1), r_K = h_K / (2 |v°| p1) (coth Pe - 1 / Pe), p1 = 2,
// and r_K = 0 where Pe < 1.
void streamline_parameters(Level& lv, int dim, double rho) {
  const long long nv0 = 2 * lv.n[0] + 1, nv1 = 2 * lv.n[1] + 1;
  double h2 = 0.0;
  for (int ax = 0; ax < dim; ++ax) h2 += lv.h[ax] * lv.h[ax];
  const double hK = std::sqrt(h2);  // the cell diameter
  lv.hrk.assign(lv.Nc, 0.0);
  for (int k = 0; k < lv.n[2]; ++k)
    for (int j = 0; j < lv.n[1]; ++j)
      for (int i = 0; i < lv.n[0]; ++i) {
        const long long cc = i + (long long)lv.n[0] * (j + (long long)lv.n[1] * k);
        const long long ctr = (2 * i + 1) + nv0 * ((2 * j + 1) + nv1 * (dim == 3 ? 2 * k + 1 : 0));
        double v2 = 0.0;
        for (int b = 0; b < dim; ++b) v2 += lv.hvc[b * lv.Nv + ctr] * lv.hvc[b * lv.Nv + ctr];
        const double vn = std::sqrt(v2);
        const double eta = lv.heta[cc];
        if (!(vn > 0.0) || !(eta > 0.0)) continue;
        const double pe = rho * vn * hK / (2.0 * eta * 2.0);
        if (pe >= 1.0) lv.hrk[cc] = hK / (2.0 * vn * 2.0) * (1.0 / std::tanh(pe) - 1.0 / pe);
      }
}

template <typename T>
gs_status corrector_setup_T(gs_ctx* c) {
  for (int l = 0; l < c->L; ++l) {
    Level& lv = c->lv[l];
    if (lv.conv) {
      CK(launch_diagA<double>(lv.g, lv.c64, lv.eta64, lv.alpha64, c->t1, 0, c->st));
      CK(launch_diag_conv(lv.g, lv.vc64, lv.rk64, lv.rho, c->t1, c->st));
      CK(launch_reciprocal<T>(c->t1, (T*)lv.dinv, lv.nu, c->st));
    } else {
      CK(launch_diagA<T>(lv.g, coef<T>(lv), etap<T>(lv), alphap<T>(lv), (T*)lv.dinv, 1, c->st));
    }
  }
  for (int l = (c->opt.coarse_mode == 1 ? 0 : 1); l < c->L; ++l) CKS(lanczos<T>(c, l));
  if (c->mono)  // diag(B diag(A_c)^{-1} B^T) of the saddle-point smoother
    for (int l = (c->opt.coarse_mode == 1 ? 0 : 1); l < c->L; ++l) {
      Level& lv = c->lv[l];
      CK(launch_schur_diag<T>(lv.g, lv.c64, (const T*)lv.dinv, (T*)lv.dsinv, 1, c->st));
    }
  return GS_OK;
}
}  // namespace

extern "C" {

gs_status gs_set_corrector(gs_ctx* c, const double* vcirc, double rho) {
  if (!c) return fail(GS_EINVAL, "NULL argument");
  if (!c->opt.corrector) return fail(GS_EINVAL, "the context was created without gs_options.corrector = 1");
  if (vcirc && !(rho >= 0.0 && std::isfinite(rho))) return fail(GS_EINVAL, "rho must be finite and >= 0");
  const int L = c->L;
  if (vcirc) {
    Level& F = c->lv[L - 1];
    for (long long i = 0; i < F.nu; ++i)
      if (!std::isfinite(vcirc[i])) return fail(GS_EINVAL, "v° is not finite");
    F.hvc.assign(vcirc, vcirc + F.nu);
    const int dim = c->dim;
    for (int l = L - 2; l >= 0; --l) {  // injection: coarse node (I, J, K) takes fine node (2 I, 2 J, 2 K)
      Level& cl = c->lv[l];
      const Level& fl = c->lv[l + 1];
      const long long cnv0 = 2 * cl.n[0] + 1, cnv1 = 2 * cl.n[1] + 1, cnv2 = dim == 3 ? 2 * cl.n[2] + 1 : 1;
      const long long fnv0 = 2 * fl.n[0] + 1, fnv1 = 2 * fl.n[1] + 1;
      cl.hvc.assign(cl.nu, 0.0);
      for (int a = 0; a < dim; ++a)
        for (long long K = 0; K < cnv2; ++K)
          for (long long J = 0; J < cnv1; ++J)
            for (long long I = 0; I < cnv0; ++I)
              cl.hvc[a * cl.Nv + I + cnv0 * (J + cnv1 * K)] = fl.hvc[a * fl.Nv + 2 * I + fnv0 * (2 * J + fnv1 * 2 * K)];
    }
    for (int l = 0; l < L; ++l) {
      Level& lv = c->lv[l];
      streamline_parameters(lv, dim, rho);
      lv.conv = 1;
      lv.rho = rho;
      CK(cudaMemcpyAsync(lv.vc64, lv.hvc.data(), sizeof(double) * lv.nu, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemcpyAsync(lv.rk64, lv.hrk.data(), sizeof(double) * lv.Nc, cudaMemcpyHostToDevice, c->st));
      {
        std::vector<float> v32(lv.hvc.begin(), lv.hvc.end()), r32(lv.hrk.begin(), lv.hrk.end());
        CK(cudaMemcpyAsync(lv.vc32, v32.data(), sizeof(float) * lv.nu, cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(lv.rk32, r32.data(), sizeof(float) * lv.Nc, cudaMemcpyHostToDevice, c->st));
        CK(cudaStreamSynchronize(c->st));  // the staging vectors go out of scope
      }
    }
  } else {
    for (int l = 0; l < L; ++l) c->lv[l].conv = 0;
  }
  // Jacobi diagonals and Chebyshev bounds (symmetric part) of every level, dense coarse inverse
  CKS(c->fp32 ? corrector_setup_T<float>(c) : corrector_setup_T<double>(c));
  if (c->nf > 0) {
    std::vector<double> A;
    assemble_coarse(c, A);
    CK(cudaMemcpyAsync(c->Ainv, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, c->st));
    for (int k = 0; k < c->nf; ++k) {
      CK(launch_gj_save(c->Ainv, c->nf, k, c->gjrow, c->gjcol, c->st));
      CK(launch_gj_update(c->Ainv, c->nf, k, c->gjrow, c->gjcol, c->st));
    }
  }
  if (c->mono && c->nmf > 0) {  // dense coarse saddle matrix with the corrector block
    std::vector<double> M;
    assemble_coarse_saddle(c, M);
    CK(cudaMemcpyAsync(c->MAinv, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice, c->st));
    for (int k = 0; k < c->nmf; ++k) {
      CK(launch_gj_save(c->MAinv, c->nmf, k, c->gjrow, c->gjcol, c->st));
      CK(launch_gj_update(c->MAinv, c->nmf, k, c->gjrow, c->gjcol, c->st));
    }
  }
  CK(cudaStreamSynchronize(c->st));
  // the captured preconditioner and the engine's recorded body hold the old operators
  if (c->pgraph) {
    cudaGraphExecDestroy(c->pgraph);
    c->pgraph = nullptr;
  }
  c->pcalls = 0;
  c->ks.body_ok = false;
  return GS_OK;
}

gs_status gs_batch_solve(gs_ctx* const* ctxs, int count, const double* const* rhs, double* const* x, double tol,
                         int* iterations, double* rel_residuals) {
  if (!ctxs || !rhs || !x || count < 0) return fail(GS_EINVAL, "NULL argument");
  gs_status first = GS_OK;
  bool engine_ok = count > 1;
  int max_restart = 1;
  for (int i = 0; i < count && engine_ok; ++i) {
    if (!ctxs[i] || ctxs[i]->opt.orth == 1 || ctxs[i]->prof) engine_ok = false;
    for (int q = 0; q < i && engine_ok; ++q) engine_ok = ctxs[q] != ctxs[i];
    if (engine_ok) max_restart = std::max(max_restart, ctxs[i]->opt.restart);
  }
  if (engine_ok) {  // all systems together, one launch per kernel per iteration
    gs_engine* eng = nullptr;
    CKS(gs_engine_create(count, max_restart, ctxs[0]->st, &eng));
    gs_status st = GS_OK;
    for (int i = 0; i < count && st == GS_OK; ++i) st = gs_engine_add(eng, ctxs[i], rhs[i], x[i], tol, i);
    int active = count;
    while (st == GS_OK && active > 0) st = gs_engine_step(eng, &active);
    std::vector<gs_engine_result> res(count);
    const int got = gs_engine_poll(eng, res.data(), count);
    gs_engine_destroy(eng);
    if (st != GS_OK) return st;
    for (int r = 0; r < got; ++r) {
      const int i = (int)res[r].tag;
      if (iterations) iterations[i] = res[r].iterations;
      if (rel_residuals) rel_residuals[i] = res[r].rel_residual;
      if (res[r].status != GS_OK && first == GS_OK) first = res[r].status;
    }
    return first;
  }
  for (int i = 0; i < count; ++i) {
    int it = 0;
    double rr = 0.0;
    gs_status s = gs_solve(ctxs[i], rhs[i], x[i], tol, &it, &rr);
    if (iterations) iterations[i] = it;
    if (rel_residuals) rel_residuals[i] = rr;
    if (s != GS_OK && first == GS_OK) first = s;
  }
  return first;
}

gs_status gs_apply_level(gs_ctx* c, int level, gs_op op, int prec, const void* x, void* y, const void* aux) {
  if (!c || !y) return fail(GS_EINVAL, "NULL argument");
  if (level < 0 || level >= c->L) return fail(GS_EINVAL, "level out of range");
  if (op == GS_OP_COARSE) {
    if (level != 0 || !x || c->nf == 0) return fail(GS_EINVAL, "coarse solve: level 0, x required, coarse_mode 0");
    CK(launch_coarse_solve<double>(c->Ainv, c->cfree, c->nf, (const double*)x, (double*)y, c->lv[0].nu, c->ctmp, c->st));
    return GS_OK;
  }
  if (op == GS_OP_SADDLE_COARSE) {
    if (level != 0 || !x || !c->mono || c->nmf == 0)
      return fail(GS_EINVAL, "coarse saddle solve: level 0, x required, precond_kind 1, coarse_mode 0");
    const Level& c0 = c->lv[0];
    CK(launch_coarse_solve<double>(c->MAinv, c->mcfree, c->nmf, (const double*)x, (double*)y, c0.nu + c0.Np, c->mctmp,
                                   c->st));
    return GS_OK;
  }
  if (op == GS_OP_WAIT_PROBE) {
    CK(launch_wait_probe(c->errw, c->st));
    return GS_OK;
  }
  if (op == GS_OP_PRECOND) {
    if (level != c->L - 1 || !x) return fail(GS_EINVAL, "preconditioner: finest level, x required");
    return precond(c, (const double*)x, (double*)y);
  }
  if (!x && op != GS_OP_DIAG_A) return fail(GS_EINVAL, "x is NULL");
  if (prec == 32) return apply_level_T<float>(c, level, op, x, y, aux);
  if (prec == 64) return apply_level_T<double>(c, level, op, x, y, aux);
  return fail(GS_EINVAL, "prec must be 32 or 64");
}

gs_status gs_get_info(const gs_ctx* c, gs_info* out) {
  if (!c || !out) return fail(GS_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->levels = c->L;
  out->dim = c->dim;
  out->n_total = c->N;
  out->n_u = c->nu;
  out->n_p = c->np;
  out->pressure_nullspace = c->nullspace ? 1 : 0;
  out->last_iterations = c->last_it;
  out->last_rel_residual = c->last_rel;
  for (int l = 0; l < c->L && l < 16; ++l) {
    out->lambda_max[l] = c->lv[l].lam_hi;
    out->level_n_u[l] = c->lv[l].nu;
  }
  out->coarse_free = c->nf;
  out->footprint_bytes = c->footprint;
  out->kernel_launches = launches_total();
  out->schur_cc = c->cc ? 1 : 0;
  out->pressure_coarse_free = c->nfp;
  for (int l = 0; l < c->L && l < 16; ++l) out->plambda_max[l] = c->lv[l].plam_hi;
  static const int rows[kTileShapes2D] = {16, 17, 8, 0};
  for (int l = 0; l < c->L && l < 16; ++l)
    out->tile_rows[l] = c->dim == 2 ? rows[c->lv[l].shape] : tile3d_depth(c->lv[l].shape);
  out->saddle_tile_rows = c->dim == 2 ? rows[c->saddle_shape] : tile3d_depth(c->saddle_shape);
  out->deflation_inclusions = c->defl_ninc;
  out->deflation_modes = c->defl_m;
  out->precond_kind = c->mono ? 1 : 0;
  out->saddle_coarse_free = c->nmf;
  return GS_OK;
}

int gs_profile_read_level(gs_ctx* c, int level, gs_kernel_stat* out, int max) {
  if (!c || !out || max <= 0) return 0;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return 0;
  double ms[K_NCLASS] = {0};
  long long cnt[K_NCLASS] = {0};
  for (auto& r : c->recs) {
    if (r.level != level) continue;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->evs[r.ev], c->evs[r.ev + 1]) == cudaSuccess) {
      ms[r.cls] += t;
      cnt[r.cls] += 1;
    }
  }
  int n = 0;
  for (int k = 0; k < K_NCLASS && n < max; ++k) {
    out[n].name = kclass_name[k];
    out[n].launches = cnt[k];
    out[n].total_ms = ms[k];
    ++n;
  }
  return n;
}

gs_status gs_profile(gs_ctx* c, int enable) {
  if (!c) return fail(GS_EINVAL, "NULL argument");
  if (enable) {
    CK(cudaStreamSynchronize(c->st));
    c->recs.clear();
    c->ev_used = 0;
  }
  c->prof = enable != 0;
  return GS_OK;
}

int gs_profile_read(gs_ctx* c, gs_kernel_stat* out, int max) {
  if (!c || !out || max <= 0) return 0;
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return 0;
  double ms[K_NCLASS] = {0};
  long long cnt[K_NCLASS] = {0};
  for (auto& r : c->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->evs[r.ev], c->evs[r.ev + 1]) == cudaSuccess) {
      ms[r.cls] += t;
      cnt[r.cls] += 1;
    }
  }
  int n = 0;
  for (int k = 0; k < K_NCLASS && n < max; ++k) {
    out[n].name = kclass_name[k];
    out[n].launches = cnt[k];
    out[n].total_ms = ms[k];
    ++n;
  }
  return n;
}

}  // extern "C"

// ---- coarse solve without workspace scratch (see gs_coarse_solve_noalloc in gs.h) ----------
// The gathered right-hand side of the dense coarse GEMV lives here instead of in the context
// workspace.  Host code must not use the symbol's host-side address: the device address is
// looked up once per device with cudaGetSymbolAddress and cached.
static __device__ __align__(256) double g_noalloc_coarse_rhs[GS_NOALLOC_COARSE_MAX];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[128] = {nullptr};

gs_status noalloc_scratch(double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(GS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_coarse_rhs));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return GS_OK;
}
}  // namespace

extern "C" {

gs_status gs_coarse_solve_noalloc(gs_ctx* c, const double* b, double* y) {
  if (!c || !b || !y) return fail(GS_EINVAL, "NULL argument");
  if (b == y) return fail(GS_EINVAL, "b and y must not alias");
  if (c->nf == 0) return fail(GS_EINVAL, "context has no dense coarse solve (coarse_mode 1)");
  if (c->nf > GS_NOALLOC_COARSE_MAX)
    return fail(GS_EINVAL, "coarse level has " + std::to_string(c->nf) + " free unknowns; the allocation-free "
                "coarse solve holds at most " + std::to_string(GS_NOALLOC_COARSE_MAX));
  double* scratch = nullptr;
  CKS(noalloc_scratch(&scratch));
  CK(launch_coarse_solve<double>(c->Ainv, c->cfree, c->nf, b, y, c->lv[0].nu, scratch, c->st));
  return GS_OK;
}

gs_status gs_set_stream(gs_ctx* c, void* stream) {
  if (!c) return fail(GS_EINVAL, "NULL argument");
  c->st = (cudaStream_t)stream;
  return GS_OK;
}

void gs_destroy(gs_ctx* c) {
  if (!c) return;
  if (c->pgraph) cudaGraphExecDestroy(c->pgraph);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  for (auto e : c->evs) cudaEventDestroy(e);
  if (c->hpin) cudaFreeHost(c->hpin);
  delete c;
}

const char* gs_strerror(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_EINVAL: return "invalid argument";
    case GS_ENOMEM: return "workspace too small";
    case GS_ECUDA: return "CUDA error";
    case GS_ENOCONV: return "no convergence";
    case GS_EBREAKDOWN: return "breakdown (non-finite values)";
    case GS_ETIMEOUT: return "timeout";
    case GS_EBUSY: return "busy (no free slot)";
  }
  return "unknown status";
}

const char* gs_last_error(void) { return g_err.c_str(); }

}  // extern "C"
