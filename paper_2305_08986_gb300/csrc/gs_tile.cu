// Cell-tile kernel for the blocks A, B^T (velocity rows) and B (pressure rows) of the saddle
// operator (Eq. "stokes-discrete-block"), matrix-free on Cartesian Q2-Q1 hexahedra (3D; the 2D
// path is gs_tile2d.cu).
//
// Work decomposition.  A CTA owns a box of TO_0 x TO_1 x TO_2 cells and the velocity / pressure
// nodes whose global index lies in [2 cs, 2 (cs + TO)) (resp. [cs, cs + TO)) per axis, plus the
// last node of the mesh when the box touches the upper boundary.  To complete the sums at its
// owned nodes it also evaluates the layer of cells just below the box (halo cells at local index
// -1), so no two CTAs write the same output and no atomics are needed.  Inside the CTA the
// evaluated cells are split in 8 classes by the parity of their global cell index along each
// axis; cells of one class share no node, so each phase adds its cell results into the
// shared-memory node tile with plain read-modify-writes.  The phases run in the order of the
// global parity class, so every node sums its cells' contributions in one order that depends on
// the node alone: tiles of any shape or position give the same bits, and the autotuner may pick
// the tile shape per level.  The owned nodes are then written once, coalesced, with the mode's
// epilogue (plain apply, residual, or a fused Chebyshev update).
#include "gs_cell.cuh"
#include "gs_kernels.h"

namespace gs {

// Tile shapes: TC0 x TC1 x TC2 evaluated cells ((TC - 1) owned per axis), one thread per
// (2 x 2 x 2 group, output component).  The skewed shared-memory layouts below assume TC0 = TC1 =
// 8; TC2 may be 8 or 4 (a warp then covers the same group pattern).
template <int C2>
struct TileShape3 {
  static_assert(C2 == 8 || C2 == 4, "3D tile depth");
  static constexpr int TC0 = 8, TC1 = 8, TC2 = C2;
  static constexpr int G0 = TC0 / 2, G1 = TC1 / 2, G2 = TC2 / 2;
  static constexpr int SPLIT = 3;
  static constexpr int NG = G0 * G1 * G2;
  static constexpr int THREADS = NG * SPLIT;
  static constexpr int VE0 = 2 * (TC0 - 1) + 1, VE1 = 2 * (TC1 - 1) + 1, VE2 = 2 * (TC2 - 1) + 1;
  static constexpr int PE0 = TC0, PE1 = TC1, PE2 = TC2;
  static constexpr int PSZ = PE0 * PE1 * PE2;
};
__device__ __forceinline__ int owned_v_ext(int cs, int TO, int n) {
  return (cs + TO >= n) ? (2 * n + 1 - 2 * cs) : 2 * TO;
}
__device__ __forceinline__ int owned_p_ext(int cs, int TO, int n) {
  return (cs + TO >= n) ? (n + 1 - cs) : TO;
}

// ---- 3D tile with a staged input window --------------------------------------------------------
// The CTA copies the velocity nodes of all its evaluated cells (a W^3 window per component, W =
// 2 TC0 + 1, with cp.async: zero fill outside the mesh and on constrained nodes) and, for B^T, the
// pressure nodes (PW^3), then runs the 8 parity-class phases (one cell and one output component
// per thread), every cell reading its nodes from the window, and writes the owned nodes with the
// mode's epilogue.
namespace {
template <typename T>
__device__ __forceinline__ void cp_async_3d(T* smem, const T* gmem, bool load) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(load ? 4 : 0));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(load ? 8 : 0));
}
}  // namespace

// Skewed layouts of the window and of the output tile: node (i0, i1, i2) of a W- (or VE-) wide
// box sits at i0 + W i1 + P i2 + A (i1 >> 2) + B (i2 >> 2), with the plane pitch P >= W^2 +
// A ((W - 1) >> 2) so that planes never overlap.  In one parity phase the cells of a warp start 4
// nodes apart along each axis, so in the plain layout all their accesses fall on 8 of the 32 banks
// (7-way conflicts); these (A, B, P) make them conflict-free (FP64 output tile: at most 2-way),
// found by enumerating every phase and local node over injective layouts.
template <typename T>
struct Skew3 {
  static constexpr bool F = sizeof(T) == 4;
  static constexpr int WA = 1, WB = 0, WP = F ? 300 : 294;       // window (W = 17)
  static constexpr int OA = 1, OB = F ? 0 : 3, OP = F ? 236 : 229;  // output tile (VE = 15)
};

template <typename T, int MODE, bool WA, bool WBT, bool WB, class S, int CONV = 0>
struct Smem3 {
  using K = Skew3<T>;
  static constexpr bool NEED_U = WA || WB, WU = WA || WBT;
  static constexpr int W0 = 2 * S::TC0 + 1, W1 = 2 * S::TC1 + 1, W2 = 2 * S::TC2 + 1;  // staged velocity window
  static constexpr int W = W0, WV = W0 * W1 * W2;
  static constexpr int WVA = (W0 - 1) + (W1 - 1) * W + (W2 - 1) * K::WP + K::WA * ((W1 - 1) >> 2) +
                             K::WB * ((W2 - 1) >> 2) + 1;  // skewed window
  static constexpr int VSZA = (S::VE0 - 1) + (S::VE1 - 1) * S::VE0 + (S::VE2 - 1) * K::OP +
                              K::OA * ((S::VE1 - 1) >> 2) + K::OB * ((S::VE2 - 1) >> 2) + 1;
  static constexpr int PW0 = S::TC0 + 1, PW1 = S::TC1 + 1, PW2 = S::TC2 + 1;
  static constexpr int PWV = PW0 * PW1 * PW2;               // staged pressure window
  static constexpr int SU = WU ? 3 * VSZA : 0;              // velocity outputs
  static constexpr int SP = WB ? S::PSZ : 0;                // pressure outputs
  static constexpr int SX = NEED_U ? 3 * WVA : 0;
  static constexpr int SPW = WBT ? PWV : 0;
  static constexpr int SV = CONV ? 3 * WVA : 0;              // v° window (corrector stage)
  static constexpr int TOTAL = SU + SP + SX + SPW + SV;      // elements of T
  static constexpr int FLAGS = NEED_U ? WV : 0;              // bytes
  static_assert(S::TC0 == 8 && S::TC1 == 8, "the skewed layouts assume 8 x 8 cells in x and y");
  static_assert(K::WP >= W * W1 + K::WA * ((W1 - 1) >> 2) && K::OP >= S::VE0 * S::VE1 + K::OA * ((S::VE1 - 1) >> 2),
                "planes of the skewed layouts must not overlap");
};

template <typename T, int MODE, bool WA, bool WBT, bool WB, class S, int CONV = 0>
__device__ __forceinline__ void tile3d_body(const TileArgs<T>& A, int bid) {
  using D = S;
  using SM = Smem3<T, MODE, WA, WBT, WB, S, CONV>;
  using K = Skew3<T>;
  constexpr bool NEED_U = SM::NEED_U, WU = SM::WU;
  constexpr int W = SM::W, WW = W * SM::W1, WV = SM::WV, WVA = SM::WVA, VSZA = SM::VSZA;
  constexpr int PW0 = SM::PW0, PW01 = SM::PW0 * SM::PW1;
  auto widx = [](int i0, int i1, int i2) { return i0 + W * i1 + K::WP * i2 + K::WA * (i1 >> 2) + K::WB * (i2 >> 2); };
  auto oidx = [](int i0, int i1, int i2) {
    return i0 + D::VE0 * i1 + K::OP * i2 + K::OA * (i1 >> 2) + K::OB * (i2 >> 2);
  };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* su = reinterpret_cast<T*>(smem_raw);
  T* sp = su + SM::SU;
  T* sx = sp + SM::SP;
  T* spw = sx + SM::SX;
  T* svc = spw + SM::SPW;  // v° window (CONV)
  uint8_t* sflag = reinterpret_cast<uint8_t*>(svc + SM::SV);
  const Geom& g = A.g;
  const OpCoef<T>& c = A.c;
  const bool raw = A.raw != 0;
  const bool vmasked = !raw && g.vmask != nullptr;
  const int tid = threadIdx.x;

  int tile = bid;
  const int t0 = tile % A.tiles[0];
  tile /= A.tiles[0];
  const int t1 = tile % A.tiles[1];
  const int t2 = tile / A.tiles[1];
  const int cs0 = t0 * (S::TC0 - 1), cs1 = t1 * (S::TC1 - 1), cs2 = t2 * (S::TC2 - 1);
  const int ve0 = owned_v_ext(cs0, S::TC0 - 1, g.n[0]);
  const int ve1 = owned_v_ext(cs1, S::TC1 - 1, g.n[1]);
  const int ve2 = owned_v_ext(cs2, S::TC2 - 1, g.n[2]);
  const int pe0 = owned_p_ext(cs0, S::TC0 - 1, g.n[0]);
  const int pe1 = owned_p_ext(cs1, S::TC1 - 1, g.n[1]);
  const int pe2 = owned_p_ext(cs2, S::TC2 - 1, g.n[2]);
  const long long Nv = g.Nv;

  // ---- stage the windows (all copies in flight together), zero the output tiles ----
  if (NEED_U) {
    const int I0 = 2 * (cs0 - 1), J0 = 2 * (cs1 - 1), K0 = 2 * (cs2 - 1);
    for (int i = tid; i < WV; i += D::THREADS) {
      const int a = i % W, b = (i / W) % SM::W1, k = i / WW;
      const int I = I0 + a, J = J0 + b, K = K0 + k;
      const bool inr = I >= 0 && I < g.nv[0] && J >= 0 && J < g.nv[1] && K >= 0 && K < g.nv[2];
      const long long node = inr ? I + (long long)g.nv[0] * (J + (long long)g.nv[1] * K) : 0;
      const bool fcon = !raw && inr && !vmasked && face_constrained(g, I, J, K);
      const int wi = widx(a, b, k);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) cp_async_3d(sx + cc * WVA + wi, A.xu + cc * Nv + node, inr && !fcon);
      if (CONV) {  // v° as given (constrained nodes included)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) cp_async_3d(svc + cc * WVA + wi, A.vc + cc * Nv + node, inr);
      }
      sflag[i] = (vmasked && inr) ? g.vmask[node] : 0;
    }
  }
  if (WBT) {
    const int P0 = cs0 - 1, Q0 = cs1 - 1, R0 = cs2 - 1;
    for (int i = tid; i < SM::PWV; i += D::THREADS) {
      const int P = P0 + i % PW0, Q = Q0 + (i / PW0) % SM::PW1, R = R0 + i / PW01;
      const bool inr = P >= 0 && P < g.npn[0] && Q >= 0 && Q < g.npn[1] && R >= 0 && R < g.npn[2];
      const long long q = inr ? P + (long long)g.npn[0] * (Q + (long long)g.npn[1] * R) : 0;
      const bool con = inr && !raw && pnode_constrained(g, q);
      cp_async_3d(spw + i, A.xp + q, inr && !con);
    }
  }
  for (int i = tid; i < SM::SU + SM::SP; i += D::THREADS) su[i] = T(0);
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (NEED_U && vmasked) {
    for (int i = tid; i < WV; i += D::THREADS)
      if (sflag[i]) {
        const int wi = widx(i % W, (i / W) % SM::W1, i / WW);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) sx[cc * WVA + wi] = T(0);
      }
  }
  __syncthreads();

  const int comp = tid / D::NG;  // warp-uniform component
  const int grp = tid % D::NG;
  const int g0 = grp % S::G0;
  const int g1 = (grp / S::G0) % S::G1;
  const int g2 = grp / (S::G0 * S::G1);
  // rotated frame of this thread's output component: logical axes (x, y, z) = physical
  // (comp, comp + 1, comp + 2) mod 3; coefficients and input components follow the rotation
  const int pa[3] = {comp, comp == 2 ? 0 : comp + 1, comp == 0 ? 2 : comp - 1};
  T km_l[3], ex_l[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    km_l[q] = c.km[pa[q]];
    ex_l[q] = c.ex[pa[q]];
  }
  const T bd_a = c.bd[comp];
  const int vext[3] = {ve0, ve1, ve2};
  auto fw = [](int ax, int i) { return ax == 0 ? i : (ax == 1 ? W * i + K::WA * (i >> 2) : K::WP * i + K::WB * (i >> 2)); };
  auto fo = [](int ax, int i) {
    return ax == 0 ? i : (ax == 1 ? D::VE0 * i + K::OA * (i >> 2) : K::OP * i + K::OB * (i >> 2));
  };
  auto fp = [](int ax, int i) { return ax == 0 ? i : (ax == 1 ? PW0 * i : PW01 * i); };
  // phase pc = the global parity class (c0 & 1) + 2 (c1 & 1) + 4 (c2 & 1) of its cells; the local
  // index of the first evaluated cell, cs - 1, fixes which local parity that is
  const int opar = ((cs0 - 1) & 1) | (((cs1 - 1) & 1) << 1) | (((cs2 - 1) & 1) << 2);
#pragma unroll 1
  for (int pc = 0; pc < 8; ++pc) {
    const int ph = pc ^ opar;
    const int lp[3] = {2 * g0 + (ph & 1), 2 * g1 + ((ph >> 1) & 1), 2 * g2 + ((ph >> 2) & 1)};
    const int c0 = cs0 - 1 + lp[0], c1 = cs1 - 1 + lp[1], c2 = cs2 - 1 + lp[2];
    bool active = c0 >= 0 && c0 < g.n[0] && c1 >= 0 && c1 < g.n[1] && c2 >= 0 && c2 < g.n[2];
    long long cell = 0;
    if (active) {
      cell = c0 + (long long)g.n[0] * (c1 + (long long)g.n[1] * c2);
      if (cell_void(g, cell)) active = false;
    }
    if (active) {
      const T eta = A.eta[cell] * c.eta_scale;
      const T mmK = A.alpha ? c.mm * A.alpha[cell] : c.mm;  // the cell's mass coefficient
      int o[3][3];  // window offsets of the cell's nodes along each logical axis
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int t = 0; t < 3; ++t) o[q][t] = fw(pa[q], 2 * lp[pa[q]] + t);
      if (WU) {
        T yl[27];
        if (WA)
          cell_A3p(sx + pa[0] * WVA, sx + pa[1] * WVA, sx + pa[2] * WVA, o[0], o[1], o[2], yl, eta, mmK, km_l, ex_l);
        if (CONV && WA) {  // corrector stage: rho (C + S) on the thread's own component
          const T* const vl[3] = {svc + pa[0] * WVA, svc + pa[1] * WVA, svc + pa[2] * WVA};
          const T ihl[3] = {pa[0] == 0 ? A.ihx : (pa[0] == 1 ? A.ihy : A.ihz),
                            pa[1] == 0 ? A.ihx : (pa[1] == 1 ? A.ihy : A.ihz),
                            pa[2] == 0 ? A.ihx : (pa[2] == 1 ? A.ihy : A.ihz)};
          cell_conv3<CONV>(sx + pa[0] * WVA, vl, o[0], o[1], o[2], A.rho, A.rk[cell], ihl, A.wq, yl);
        }
        if (WBT) {
          T pl[8];  // the cell's pressure nodes in the logical frame
#pragma unroll
          for (int lc = 0; lc < 2; ++lc)
#pragma unroll
            for (int lb = 0; lb < 2; ++lb)
#pragma unroll
              for (int la = 0; la < 2; ++la)
                pl[la + 2 * lb + 4 * lc] =
                    spw[fp(pa[0], lp[pa[0]] + la) + fp(pa[1], lp[pa[1]] + lb) + fp(pa[2], lp[pa[2]] + lc)];
          cell_BT3p(pl, yl, bd_a, WA);
        }
        int oo[3][3];
        bool ok[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int i = 2 * (lp[pa[q]] - 1) + t;
            ok[q][t] = i >= 0 && i < vext[pa[q]];
            oo[q][t] = fo(pa[q], i);
          }
        T* sc = su + comp * VSZA;
#pragma unroll
        for (int lc = 0; lc < 3; ++lc) {
          if (!ok[2][lc]) continue;
#pragma unroll
          for (int lb = 0; lb < 3; ++lb) {
            if (!ok[1][lb]) continue;
#pragma unroll
            for (int la = 0; la < 3; ++la) {
              if (!ok[0][la]) continue;
              sc[oo[0][la] + oo[1][lb] + oo[2][lc]] += yl[la + 3 * lb + 9 * lc];
            }
          }
        }
      }
      if (WB && comp == 0) {  // comp 0: the rotated frame is the physical one
        T ob[8];
        cell_B3w(sx + 2 * lp[0], sx + WVA + 2 * lp[0], sx + 2 * WVA + 2 * lp[0], o[1], o[2], ob, c);
#pragma unroll
        for (int lc = 0; lc < 2; ++lc) {
          const int i2 = (lp[2] - 1) + lc;
          if (i2 < 0 || i2 >= pe2) continue;
#pragma unroll
          for (int lb = 0; lb < 2; ++lb) {
            const int i1 = (lp[1] - 1) + lb;
            if (i1 < 0 || i1 >= pe1) continue;
#pragma unroll
            for (int la = 0; la < 2; ++la) {
              const int i0 = (lp[0] - 1) + la;
              if (i0 < 0 || i0 >= pe0) continue;
              sp[i0 + D::PE0 * (i1 + D::PE1 * i2)] += ob[la + 2 * lb + 4 * lc];
            }
          }
        }
      }
    }
    __syncthreads();
  }

  // ---- owned velocity nodes: epilogue ----
  if (WU) {
    const int nown = ve0 * ve1 * ve2;
    for (int i = tid; i < nown; i += D::THREADS) {
      const int i0 = i % ve0;
      const int i1 = (i / ve0) % ve1;
      const int i2 = i / (ve0 * ve1);
      const int I = 2 * cs0 + i0, J = 2 * cs1 + i1, K = 2 * cs2 + i2;
      const long long node = I + (long long)g.nv[0] * (J + (long long)g.nv[1] * K);
      const bool con = !raw && vnode_constrained(g, node, I, J, K);
      const int s = oidx(i0, i1, i2);
      const int w = widx(i0 + 2, i1 + 2, i2 + 2);  // the node in the staged window
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long gi = a * Nv + node;
        const T ax = con ? (WA ? A.xu[gi] : T(0)) : su[a * VSZA + s];
        if (MODE == TILE_APPLY) {
          A.yu[gi] = ax;
        } else if (MODE == TILE_RESID) {
          A.yu[gi] = A.bu[gi] - ax;
        } else {
          const T r = A.bu[gi] - ax;
          T dn = A.c2 * A.dinv[gi] * r;
          if (A.use_d) dn += A.c1 * A.d[gi];
          A.d[gi] = dn;
          const T xin = (con || !NEED_U) ? A.xu[gi] : sx[a * WVA + w];
          A.xout[gi] = xin + dn;
        }
      }
    }
  }
  if (WB) {
    const int nown = pe0 * pe1 * pe2;
    for (int i = tid; i < nown; i += D::THREADS) {
      const int i0 = i % pe0;
      const int i1 = (i / pe0) % pe1;
      const int i2 = i / (pe0 * pe1);
      const long long q = (cs0 + i0) + (long long)g.npn[0] * ((cs1 + i1) + (long long)g.npn[1] * (cs2 + i2));
      const bool con = !raw && pnode_constrained(g, q);
      const T bx = con ? (WBT ? A.xp[q] : T(0)) : sp[i0 + D::PE0 * (i1 + D::PE1 * i2)];
      if (MODE == TILE_RESID)
        A.yp[q] = A.bp[q] - bx;
      else
        A.yp[q] = bx;
    }
  }
}

// ---- 3D velocity block (A x, b - A x, Chebyshev step) without halo cells, FP32 ----------------------
// The tiles above evaluate one layer of halo cells per axis; on meshes of 2^k cells per axis a tile
// owning 7 cells per axis then evaluates ~1.95x the cells of the mesh.  Here a CTA owns and evaluates
// exactly the cells [cs, cs + TC) (8 x 8 x 4; the last tile along an axis may be cut by the mesh).
// Its cells touch the nodes [2 cs, 2 cs + 2 TC] per axis; the nodes strictly inside that box, and
// those on a face at the mesh boundary, are complete after the CTA's own cells and get the mode's
// epilogue at once.  A node on a face shared with a neighbouring tile receives contributions from
// up to 8 tiles: each tile writes its partial sum there to a per-tile slot of the partial buffer
// (TileArgs::part), and a second kernel (fix3nh_body) adds the partials of the sharing tiles in a
// fixed order (tiles lexicographic, x fastest) and applies the epilogue.  Inside a tile the cells are
// processed in 8 phases by their global parity class, as in the tiles above.  The sums are
// deterministic; they differ in rounding from the halo tiles' (a different association at the
// shared faces), so all FP32 applications of the 3D velocity block use this kernel, except in the
// corrector stage (the convection term runs in the 8 x 8 x 4 halo tiles).
struct NH3 {
  static constexpr int TC0 = kNH3Cells0, TC1 = kNH3Cells1, TC2 = kNH3Cells2;  // cells per tile
  static constexpr int G0 = TC0 / 2, G1 = TC1 / 2, G2 = TC2 / 2, NG = G0 * G1 * G2;  // 32 groups
  static constexpr int THREADS = NG * 3;                                // one warp per component
  static constexpr int W0 = 2 * TC0 + 1, W1 = 2 * TC1 + 1, W2 = 2 * TC2 + 1;  // node box 17 x 17 x 9
  static constexpr int NW = W0 * W1 * W2;                               // 2601 nodes
  static_assert(NW == kNH3Box, "node box of the partial-sum buffer");
  static constexpr int P0 = 2 * TC0, P1 = 2 * TC1, P2 = 2 * TC2;        // node spacing of tile faces
};

template <typename T>
struct SmemNH3 {
  using K = Skew3<T>;
  // node box in the skewed window layout (row pitch 17), used for the input window and the sums
  static constexpr int WVA = (NH3::W0 - 1) + (NH3::W1 - 1) * NH3::W0 + (NH3::W2 - 1) * K::WP +
                             K::WA * ((NH3::W1 - 1) >> 2) + K::WB * ((NH3::W2 - 1) >> 2) + 1;
  static constexpr int TOTAL = 6 * WVA;  // x window (3 components) + sums (3 components)
  static constexpr int FLAGS = NH3::NW;  // bytes
  static_assert(NH3::W0 == 17 && NH3::W1 == 17, "the skewed layout assumes a row pitch of 17");
  static_assert(K::WP >= NH3::W0 * NH3::W1 + K::WA * ((NH3::W1 - 1) >> 2), "planes must not overlap");
};

// number of tiles of the halo-free 3D kernel along each axis
__host__ __device__ inline int nh3_tiles(int n, int tc) { return (n + tc - 1) / tc; }

template <typename T, int MODE>
__device__ __forceinline__ void tile3nh_body(const TileArgs<T>& A, int bid) {
  using S = NH3;
  using SM = SmemNH3<T>;
  using K = Skew3<T>;
  constexpr int W = S::W0, WW = S::W0 * S::W1, WV = S::NW, WVA = SM::WVA;
  auto widx = [](int i0, int i1, int i2) { return i0 + W * i1 + K::WP * i2 + K::WA * (i1 >> 2) + K::WB * (i2 >> 2); };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);
  T* su = sx + 3 * WVA;
  uint8_t* sflag = reinterpret_cast<uint8_t*>(su + 3 * WVA);
  const Geom& g = A.g;
  const OpCoef<T>& c = A.c;
  const bool raw = A.raw != 0;
  const bool vmasked = !raw && g.vmask != nullptr;
  const int tid = threadIdx.x;
  int tile = bid;
  const int t0 = tile % A.tiles[0];
  tile /= A.tiles[0];
  const int t1 = tile % A.tiles[1];
  const int t2 = tile / A.tiles[1];
  const int cs0 = t0 * S::TC0, cs1 = t1 * S::TC1, cs2 = t2 * S::TC2;
  const int I0 = 2 * cs0, J0 = 2 * cs1, K0 = 2 * cs2;
  const long long Nv = g.Nv;

  // ---- stage the node box of x (all copies in flight together), zero the sums ----
  for (int i = tid; i < WV; i += S::THREADS) {
    const int a = i % W, b = (i / W) % S::W1, k = i / WW;
    const int I = I0 + a, J = J0 + b, Kz = K0 + k;
    const bool inr = I < g.nv[0] && J < g.nv[1] && Kz < g.nv[2];
    const long long node = inr ? I + (long long)g.nv[0] * (J + (long long)g.nv[1] * Kz) : 0;
    const bool fcon = !raw && inr && !vmasked && face_constrained(g, I, J, Kz);
    const int wi = widx(a, b, k);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) cp_async_3d(sx + cc * WVA + wi, A.xu + cc * Nv + node, inr && !fcon);
    sflag[i] = (vmasked && inr) ? g.vmask[node] : 0;
  }
  for (int i = tid; i < 3 * WVA; i += S::THREADS) su[i] = T(0);
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (vmasked) {
    for (int i = tid; i < WV; i += S::THREADS)
      if (sflag[i]) {
        const int wi = widx(i % W, (i / W) % S::W1, i / WW);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) sx[cc * WVA + wi] = T(0);
      }
  }
  __syncthreads();

  // ---- the tile's cells in 8 phases (cs is even on every axis: local parity = global parity) ----
  const int comp = tid / S::NG;  // warp-uniform component
  const int grp = tid % S::NG;
  const int g0 = grp % S::G0;
  const int g1 = (grp / S::G0) % S::G1;
  const int g2 = grp / (S::G0 * S::G1);
  const int pa[3] = {comp, comp == 2 ? 0 : comp + 1, comp == 0 ? 2 : comp - 1};
  T km_l[3], ex_l[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    km_l[q] = c.km[pa[q]];
    ex_l[q] = c.ex[pa[q]];
  }
  auto fw = [](int ax, int i) { return ax == 0 ? i : (ax == 1 ? W * i + K::WA * (i >> 2) : K::WP * i + K::WB * (i >> 2)); };
  T* sc = su + comp * WVA;
#pragma unroll 1
  for (int ph = 0; ph < 8; ++ph) {
    const int lp[3] = {2 * g0 + (ph & 1), 2 * g1 + ((ph >> 1) & 1), 2 * g2 + ((ph >> 2) & 1)};
    const int c0 = cs0 + lp[0], c1 = cs1 + lp[1], c2 = cs2 + lp[2];
    bool active = c0 < g.n[0] && c1 < g.n[1] && c2 < g.n[2];
    long long cell = 0;
    if (active) {
      cell = c0 + (long long)g.n[0] * (c1 + (long long)g.n[1] * c2);
      if (cell_void(g, cell)) active = false;
    }
    if (active) {
      const T eta = A.eta[cell] * c.eta_scale;
      const T mmK = A.alpha ? c.mm * A.alpha[cell] : c.mm;
      int o[3][3];  // box offsets of the cell's nodes along each logical axis (input and sums alike)
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int t = 0; t < 3; ++t) o[q][t] = fw(pa[q], 2 * lp[pa[q]] + t);
      T yl[27];
      cell_A3p(sx + pa[0] * WVA, sx + pa[1] * WVA, sx + pa[2] * WVA, o[0], o[1], o[2], yl, eta, mmK, km_l, ex_l);
#pragma unroll
      for (int lc = 0; lc < 3; ++lc)
#pragma unroll
        for (int lb = 0; lb < 3; ++lb)
#pragma unroll
          for (int la = 0; la < 3; ++la) sc[o[0][la] + o[1][lb] + o[2][lc]] += yl[la + 3 * lb + 9 * lc];
    }
    __syncthreads();
  }

  // ---- nodes of the box: epilogue, or the partial sum of a node on a shared face ----
  const int e0 = min(S::P0, 2 * g.n[0] - I0) + 1;
  const int e1 = min(S::P1, 2 * g.n[1] - J0) + 1;
  const int e2 = min(S::P2, 2 * g.n[2] - K0) + 1;
  const bool lo0 = cs0 > 0, lo1 = cs1 > 0, lo2 = cs2 > 0;
  const bool hi0 = cs0 + S::TC0 < g.n[0], hi1 = cs1 + S::TC1 < g.n[1], hi2 = cs2 + S::TC2 < g.n[2];
  T* part = A.part + (long long)bid * 3 * WV;
  const int nbox = e0 * e1 * e2;
  for (int i = tid; i < nbox; i += S::THREADS) {
    const int i0 = i % e0;
    const int i1 = (i / e0) % e1;
    const int i2 = i / (e0 * e1);
    const int s = widx(i0, i1, i2);
    const bool shared = (i0 == 0 && lo0) || (i0 == S::P0 && hi0) || (i1 == 0 && lo1) || (i1 == S::P1 && hi1) ||
                        (i2 == 0 && lo2) || (i2 == S::P2 && hi2);
    if (shared) {
      const int li = i0 + S::W0 * (i1 + S::W1 * i2);
#pragma unroll
      for (int a = 0; a < 3; ++a) part[a * WV + li] = su[a * WVA + s];
      continue;
    }
    const int I = I0 + i0, J = J0 + i1, Kz = K0 + i2;
    const long long node = I + (long long)g.nv[0] * (J + (long long)g.nv[1] * Kz);
    const bool con = !raw && vnode_constrained(g, node, I, J, Kz);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const long long gi = a * Nv + node;
      const T ax = con ? A.xu[gi] : su[a * WVA + s];
      if (MODE == TILE_APPLY) {
        A.yu[gi] = ax;
      } else if (MODE == TILE_RESID) {
        A.yu[gi] = A.bu[gi] - ax;
      } else {
        const T r = A.bu[gi] - ax;
        T dn = A.c2 * A.dinv[gi] * r;
        if (A.use_d) dn += A.c1 * A.d[gi];
        A.d[gi] = dn;
        const T xin = con ? A.xu[gi] : sx[a * WVA + s];
        A.xout[gi] = xin + dn;
      }
    }
  }
}

// The nodes on faces shared by tiles of tile3nh_body: one thread per node, all three components.
// Node families: planes x = 16 k (0 < k < tiles_x), then planes y = 16 k without the nodes of an
// x-plane, then planes z = 8 k without the nodes of an x- or y-plane, so each node is visited once.
template <typename T, int MODE>
__device__ __forceinline__ void fix3nh_body(const TileArgs<T>& A, int blk) {
  using S = NH3;
  const Geom& g = A.g;
  const int nv0 = g.nv[0], nv1 = g.nv[1], nv2 = g.nv[2];
  const int nb0 = A.tiles[0] - 1, nb1 = A.tiles[1] - 1, nb2 = A.tiles[2] - 1;
  const long long nX = (long long)nb0 * nv1 * nv2, nY = (long long)nb1 * nv0 * nv2, nZ = (long long)nb2 * nv0 * nv1;
  long long idx = (long long)blk * 256 + threadIdx.x;
  // an interior tile face along an axis: node coordinate P k with 0 < k < tiles
  auto face = [](int X, int P, int tiles) { return X % P == 0 && X > 0 && X / P < tiles; };
  // q = a / b and a - q b; every index and plane size here is below Nv, so 32-bit division serves
  // whenever Nv < 2^31 (a 64-bit division takes several times the instructions)
  const bool i32 = g.Nv < (1LL << 31);
  auto divmod = [i32](long long a, long long b, int& q) -> long long {
    if (i32) {
      const unsigned ua = (unsigned)a, ub = (unsigned)b, uq = ua / ub;
      q = (int)uq;
      return (long long)(ua - uq * ub);
    }
    const long long lq = a / b;
    q = (int)lq;
    return a - lq * b;
  };
  int I, J, Kz;
  if (idx < nX) {
    int p;
    const long long r = divmod(idx, (long long)nv1 * nv2, p);
    I = S::P0 * (p + 1);
    J = (int)divmod(r, nv1, Kz);
  } else if ((idx -= nX) < nY) {
    int p;
    const long long r = divmod(idx, (long long)nv0 * nv2, p);
    J = S::P1 * (p + 1);
    I = (int)divmod(r, nv0, Kz);
    if (face(I, S::P0, A.tiles[0])) return;
  } else if ((idx -= nY) < nZ) {
    int p;
    const long long r = divmod(idx, (long long)nv0 * nv1, p);
    Kz = S::P2 * (p + 1);
    I = (int)divmod(r, nv0, J);
    if (face(I, S::P0, A.tiles[0]) || face(J, S::P1, A.tiles[1])) return;
  } else {
    return;
  }
  // the tiles sharing the node and its local index in each (one or two per axis, lower tile first)
  int tl[3][2], ll[3][2], nt[3];
  const int X[3] = {I, J, Kz}, P[3] = {S::P0, S::P1, S::P2};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (face(X[ax], P[ax], A.tiles[ax])) {
      nt[ax] = 2;
      tl[ax][0] = X[ax] / P[ax] - 1;
      ll[ax][0] = P[ax];
      tl[ax][1] = X[ax] / P[ax];
      ll[ax][1] = 0;
    } else {
      nt[ax] = 1;
      tl[ax][0] = min(X[ax] / P[ax], A.tiles[ax] - 1);
      ll[ax][0] = X[ax] - P[ax] * tl[ax][0];
      tl[ax][1] = tl[ax][0];
      ll[ax][1] = ll[ax][0];
    }
  }
  const long long node = I + (long long)nv0 * (J + (long long)nv1 * Kz);
  const bool con = !A.raw && vnode_constrained(g, node, I, J, Kz);
  const long long Nv = g.Nv;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T acc = T(0);
    // unrolled to the maximum of two tiles per axis and predicated, so tl and ll stay in registers;
    // the sharing tiles are added in the same order (z, then y, then x outermost to innermost)
#pragma unroll
    for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
      for (int b1 = 0; b1 < 2; ++b1)
#pragma unroll
        for (int b0 = 0; b0 < 2; ++b0) {
          if (b2 >= nt[2] || b1 >= nt[1] || b0 >= nt[0]) continue;
          const long long t = tl[0][b0] + (long long)A.tiles[0] * (tl[1][b1] + (long long)A.tiles[1] * tl[2][b2]);
          const int li = ll[0][b0] + S::W0 * (ll[1][b1] + S::W1 * ll[2][b2]);
          acc += A.part[(t * 3 + a) * S::NW + li];
        }
    const long long gi = a * Nv + node;
    const T ax = con ? A.xu[gi] : acc;
    if (MODE == TILE_APPLY) {
      A.yu[gi] = ax;
    } else if (MODE == TILE_RESID) {
      A.yu[gi] = A.bu[gi] - ax;
    } else {
      const T r = A.bu[gi] - ax;
      T dn = A.c2 * A.dinv[gi] * r;
      if (A.use_d) dn += A.c1 * A.d[gi];
      A.d[gi] = dn;
      A.xout[gi] = A.xu[gi] + dn;
    }
  }
}

template <typename T, int MODE>
struct Tile3NHK {
  using Args = TileArgs<T>;
  static constexpr int THREADS = NH3::THREADS, MINB = 3;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) { tile3nh_body<T, MODE>(a, blk); }
};

template <typename T, int MODE>
struct Fix3NHK {
  using Args = TileArgs<T>;
  static constexpr int THREADS = 256, MINB = 4;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) { fix3nh_body<T, MODE>(a, blk); }
};

template <typename T, int MODE>
static cudaError_t launch_nh3(TileArgs<T> a, cudaStream_t st) {
  a.tiles[0] = nh3_tiles(a.g.n[0], NH3::TC0);
  a.tiles[1] = nh3_tiles(a.g.n[1], NH3::TC1);
  a.tiles[2] = nh3_tiles(a.g.n[2], NH3::TC2);
  const long long nblocks = (long long)a.tiles[0] * a.tiles[1] * a.tiles[2];
  cudaError_t e = submit<Tile3NHK<T, MODE>>(a, nblocks, sizeof(T) * SmemNH3<T>::TOTAL + SmemNH3<T>::FLAGS, st);
  if (e != cudaSuccess) return e;
  const long long nfix = (long long)(a.tiles[0] - 1) * a.g.nv[1] * a.g.nv[2] +
                         (long long)(a.tiles[1] - 1) * a.g.nv[0] * a.g.nv[2] +
                         (long long)(a.tiles[2] - 1) * a.g.nv[0] * a.g.nv[1];
  if (nfix == 0) return cudaSuccess;
  return submit<Fix3NHK<T, MODE>>(a, (nfix + 255) / 256, 0, st);
}

template <typename T, int MODE, bool WA, bool WBT, bool WB, int C2, int CONV = 0>
struct TileK {
  using Args = TileArgs<T>;
  using S = TileShape3<C2>;
  static constexpr int THREADS = S::THREADS, MINB = 1;
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    tile3d_body<T, MODE, WA, WBT, WB, S, CONV>(a, blk);
  }
};

template <typename T, int MODE, bool WA, bool WBT, bool WB, int C2, int CONV = 0>
static cudaError_t launch_shape(TileArgs<T> a, cudaStream_t st) {
  using S = TileShape3<C2>;
  using SM = Smem3<T, MODE, WA, WBT, WB, S, CONV>;
  a.tiles[0] = (a.g.n[0] + S::TC0 - 2) / (S::TC0 - 1);
  a.tiles[1] = (a.g.n[1] + S::TC1 - 2) / (S::TC1 - 1);
  a.tiles[2] = (a.g.n[2] + S::TC2 - 2) / (S::TC2 - 1);
  const size_t smem = sizeof(T) * SM::TOTAL + SM::FLAGS;
  const long long nblocks = (long long)a.tiles[0] * a.tiles[1] * a.tiles[2];
  return submit<TileK<T, MODE, WA, WBT, WB, C2, CONV>>(a, nblocks, smem, st);
}

template <typename T, int DIM, int MODE, bool WA, bool WBT, bool WB>
static cudaError_t launch_one(TileArgs<T> a, cudaStream_t st) {
  static_assert(DIM == 3, "2D launches use the kernels of gs_tile2d.cuh and gs_strip2d.cuh");
  if (a.shape == 1) return launch_shape<T, MODE, WA, WBT, WB, 4>(a, st);
  return launch_shape<T, MODE, WA, WBT, WB, 8>(a, st);
}

template <typename T, int DIM, int MODE>
static cudaError_t dispatch_ops(int ops, TileArgs<T> a, cudaStream_t st) {
  switch (ops) {
    case OPS_A: return launch_one<T, DIM, MODE, true, false, false>(a, st);
    case OPS_BT: return launch_one<T, DIM, MODE, false, true, false>(a, st);
    case OPS_B: return launch_one<T, DIM, MODE, false, false, true>(a, st);
    case OPS_A | OPS_BT | OPS_B: return launch_one<T, DIM, MODE, true, true, true>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_tile(int dim, int mode, int ops, TileArgs<T> a, cudaStream_t st) {
  if (mode == TILE_CHEB && ops != OPS_A) return cudaErrorInvalidValue;
  if (dim == 2) return launch_tile2d<T>(mode, ops, a, st);  // gs_tile2d.cu
  if (a.conv && (ops & OPS_A)) {  // corrector stage: 8 x 8 x 4 halo tiles with the convection term
    if (a.conv == 2) return mode == TILE_APPLY && ops == OPS_A ? launch_shape<T, TILE_APPLY, true, false, false, 4, 2>(a, st)
                                                               : cudaErrorInvalidValue;
    if (ops == OPS_A) {
      if (mode == TILE_APPLY) return launch_shape<T, TILE_APPLY, true, false, false, 4, 1>(a, st);
      if (mode == TILE_RESID) return launch_shape<T, TILE_RESID, true, false, false, 4, 1>(a, st);
      return launch_shape<T, TILE_CHEB, true, false, false, 4, 1>(a, st);
    }
    if (ops == (OPS_A | OPS_BT | OPS_B)) {
      if (mode == TILE_APPLY) return launch_shape<T, TILE_APPLY, true, true, true, 4, 1>(a, st);
      if (mode == TILE_RESID) return launch_shape<T, TILE_RESID, true, true, true, 4, 1>(a, st);
    }
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 4) {
    if (ops == OPS_A && a.part != nullptr) {  // FP32 velocity block: tiles without halo cells
      if (mode == TILE_APPLY) return launch_nh3<T, TILE_APPLY>(a, st);
      if (mode == TILE_RESID) return launch_nh3<T, TILE_RESID>(a, st);
      return launch_nh3<T, TILE_CHEB>(a, st);
    }
  }
  if (mode == TILE_APPLY) return dispatch_ops<T, 3, TILE_APPLY>(ops, a, st);
  if (mode == TILE_RESID) return dispatch_ops<T, 3, TILE_RESID>(ops, a, st);
  return launch_one<T, 3, TILE_CHEB, true, false, false>(a, st);
}

template cudaError_t launch_tile<float>(int, int, int, TileArgs<float>, cudaStream_t);
template cudaError_t launch_tile<double>(int, int, int, TileArgs<double>, cudaStream_t);

}  // namespace gs
