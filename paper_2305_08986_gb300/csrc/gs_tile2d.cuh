// 2D cell-tile kernel for the blocks A, B^T and B of the saddle operator (Eq.
// "stokes-discrete-block") on Cartesian Q2-Q1 quadrilaterals.
//
// A CTA owns TO0 x TO1 cells and the nodes [2 cs, 2 (cs + TO)) per axis (plus the last node of
// the mesh on the upper boundary); it evaluates (TO0 + 1) x (TO1 + 1) cells, including the layer
// just below its box, so that every owned node receives all of its cell contributions and each
// output is written by exactly one CTA.  Three phases, separated by block barriers:
//   1. the input nodes of all evaluated cells (a (2 E0 + 1) x (2 E1 + 1) node tile per
//      component), and the epilogue's b / d / D^-1 of the owned nodes, are copied to shared
//      memory with cp.async (zero fill for nodes outside the mesh and constrained columns), so
//      all global loads of the CTA are in flight together;
//   2. every evaluated cell is computed (sum-factorised, gs_cell.cuh) from shared memory and
//      its 18 velocity (and 4 pressure) results are stored cell-major in shared memory;
//   3. each owned node sums the <= 4 cell results that touch it, in a fixed order (so the
//      result does not depend on scheduling), and applies the mode's epilogue.
// Threads form a 32 x 8 grid.  In phases 1 and 3 thread (tx, ty) handles node columns 2 tx and
// 2 tx + 1 and node rows ty + 8 r, so the parity of its nodes is fixed (no per-node index
// arithmetic, uniform branches within a warp) and it consumes the epilogue operands it staged.
#pragma once
#include "gs_cell.cuh"
#include "gs_kernels.h"

namespace gs {

namespace tile2d {
constexpr int NT = 256;      // threads per CTA: 32 x 8
constexpr int TY = NT / 32;  // 8

// Tile shape: 32 x EY evaluated cells (EY = 16 by default; the per-level autotuner may pick
// another compiled height, see launch_tile2d).
template <int EY>
struct Shape2 {
  static constexpr int E0 = 32, E1 = EY;                  // evaluated cells per tile
  static constexpr int TO0 = E0 - 1, TO1 = E1 - 1;        // owned cells per tile
  static constexpr int NCELL = E0 * E1;
  static constexpr int IN0 = 2 * E0 + 1, IN1 = 2 * E1 + 1;  // velocity input node tile
  static constexpr int NIN = IN0 * IN1;
  static constexpr int PI0 = E0 + 1, PI1 = E1 + 1;        // pressure input node tile
  static constexpr int VP0 = 2 * TO0 + 1, VP1 = 2 * TO1 + 1;  // owned velocity node region
  static constexpr int OWN = VP0 * VP1;
  static constexpr int PP0 = TO0 + 1, PP1 = TO1 + 1;      // owned pressure node region
  static constexpr int POWN = PP0 * PP1;
  static constexpr int ROWS = (VP1 + TY - 1) / TY;        // owned node rows per thread
  static constexpr int IROWS = (IN1 + TY - 1) / TY;       // input tile rows per thread
  static constexpr int CROWS = (E1 + TY - 1) / TY;        // evaluated cell rows per thread
};

#define GS_SHAPE2_NAMES(EY)                                                                    \
  using S2__ = Shape2<EY>;                                                                     \
  constexpr int E0 = S2__::E0, E1 = S2__::E1, TO0 = S2__::TO0, TO1 = S2__::TO1;               \
  constexpr int NCELL = S2__::NCELL, IN0 = S2__::IN0, IN1 = S2__::IN1, NIN = S2__::NIN;        \
  constexpr int PI0 = S2__::PI0, PI1 = S2__::PI1, VP0 = S2__::VP0, VP1 = S2__::VP1;           \
  constexpr int OWN = S2__::OWN, PP0 = S2__::PP0, PP1 = S2__::PP1, POWN = S2__::POWN;         \
  constexpr int ROWS = S2__::ROWS, IROWS = S2__::IROWS, CROWS = S2__::CROWS;                  \
  (void)E0; (void)E1; (void)TO0; (void)TO1; (void)NCELL; (void)IN0; (void)IN1; (void)NIN;      \
  (void)PI0; (void)PI1; (void)VP0; (void)VP1; (void)OWN; (void)PP0; (void)PP1; (void)POWN;    \
  (void)ROWS; (void)IROWS; (void)CROWS

template <int EY, int MODE, bool NEED_U, bool WBT, bool WU, bool WB, int CONV = 0>
struct Smem2 {
  static constexpr int NIN = Shape2<EY>::NIN, PI0 = Shape2<EY>::PI0, PI1 = Shape2<EY>::PI1;
  static constexpr int NCELL = Shape2<EY>::NCELL, OWN = Shape2<EY>::OWN, POWN = Shape2<EY>::POWN;
  static constexpr int SX = NEED_U ? 2 * NIN : 0;
  static constexpr int SP = WBT ? PI0 * PI1 : 0;
  static constexpr int RU = WU ? 18 * NCELL : 0;
  static constexpr int RP = WB ? 4 * NCELL : 0;
  static constexpr int SB = (WU && MODE != TILE_APPLY) ? 2 * OWN : 0;   // b (residual / Chebyshev)
  static constexpr int SD = (WU && MODE == TILE_CHEB) ? 2 * OWN : 0;    // d and D^-1 (Chebyshev)
  static constexpr int SBP = (WB && MODE == TILE_RESID) ? POWN : 0;     // pressure b (residual)
  static constexpr int SV = CONV ? 2 * NIN : 0;                         // v° window (corrector stage)
  static constexpr int TOTAL = SX + SP + RU + RP + SB + 2 * SD + SBP + SV;  // elements of T
  static constexpr int FLAGS = NEED_U ? NIN : 0;                        // bytes: constrained nodes
};

// Asynchronous global -> shared copy of one element; src_bytes = 0 writes zero (used for nodes
// outside the mesh and constrained columns).  The source address is always a valid address.
template <typename T>
__device__ __forceinline__ void cp_async_el(T* smem, const T* gmem, bool load) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(load ? 4 : 0));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(load ? 8 : 0));
}
__device__ __forceinline__ void cp_async_commit_wait() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ int owned_ext(int cs, int TO, int n, int mult) {
  return (cs + TO >= n) ? (mult * (n - cs) + 1) : mult * TO;
}

// Sum of the cell results touching owned node (i0, i1), with the node's local positions fixed by
// its parities (even: local 0 in the next cell and local 2 in the previous one; odd: local 1).
// Evaluated cell index = cell + 1 - cs; indices beyond the evaluated range lie outside the mesh.
template <typename T, int EY, bool XODD, bool YODD>
__device__ __forceinline__ void gather2(const T* ru, int i0, int i1, T& s0, T& s1) {
  GS_SHAPE2_NAMES(EY);
  s0 = T(0);
  s1 = T(0);
  const int ey0 = YODD ? (i1 + 1) >> 1 : (i1 >> 1) + 1;
  const int ex0 = XODD ? (i0 + 1) >> 1 : (i0 >> 1) + 1;
#pragma unroll
  for (int b = 0; b < (YODD ? 1 : 2); ++b) {
    const int ey = ey0 - b;
    const int lb = YODD ? 1 : 2 * b;
    if (ey >= E1) continue;
#pragma unroll
    for (int a = 0; a < (XODD ? 1 : 2); ++a) {
      const int ex = ex0 - a;
      const int la = XODD ? 1 : 2 * a;
      if (ex >= E0) continue;
      const int e = ex + E0 * ey;
      const int li = la + 3 * lb;
      s0 += ru[li * NCELL + e];
      s1 += ru[(9 + li) * NCELL + e];
    }
  }
}
template <typename T, int EY, int MODE, bool WA, bool WBT, bool WB, int CONV = 0>
__device__ __forceinline__ void tile2d_body(const TileArgs<T>& A, int bid) {
  GS_SHAPE2_NAMES(EY);
  constexpr bool NEED_U = WA || WB;
  constexpr bool WU = WA || WBT;
  using SM = Smem2<EY, MODE, NEED_U, WBT, WU, WB, CONV>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sx = reinterpret_cast<T*>(smem_raw);
  T* sp = sx + SM::SX;
  T* ru = sp + SM::SP;
  T* rp = ru + SM::RU;
  T* sb = rp + SM::RP;
  T* sd = sb + SM::SB;
  T* sdi = sd + SM::SD;
  T* sbp = sdi + SM::SD;
  T* sv = sbp + SM::SBP;  // v° window (CONV)
  uint8_t* scon = reinterpret_cast<uint8_t*>(sv + SM::SV);
  const Geom& g = A.g;
  const OpCoef<T>& c = A.c;
  const bool raw = A.raw != 0;
  const int t0 = bid % A.tiles[0];
  const int t1 = bid / A.tiles[0];
  const int cs0 = t0 * TO0, cs1 = t1 * TO1;
  const long long Nv = g.Nv;
  const int tid = threadIdx.x;
  const int tx = tid & 31, ty = tid >> 5;
  const int ve0 = owned_ext(cs0, TO0, g.n[0], 2), ve1 = owned_ext(cs1, TO1, g.n[1], 2);
  const int pe0 = owned_ext(cs0, TO0, g.n[0], 1), pe1 = owned_ext(cs1, TO1, g.n[1], 1);
  const bool vmasked = !raw && g.vmask != nullptr;

  // ---- phase 1: stage inputs (all copies in flight together) ----
  uint8_t mk[3 * IROWS];  // constraint flags of the input nodes this thread stages
  if (NEED_U) {
    const int I0 = 2 * (cs0 - 1), J0 = 2 * (cs1 - 1);
#pragma unroll
    for (int r = 0; r < IROWS; ++r) {
      const int iy = ty + TY * r;
      const int J = J0 + iy;
      const bool rowok = iy < IN1 && J >= 0 && J < g.nv[1];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int ix = tx + 32 * q;
        mk[3 * r + q] = 0;
        if (iy < IN1 && ix < IN0) {
          const int I = I0 + ix;
          const bool inr = rowok && I >= 0 && I < g.nv[0];
          const long long node = inr ? I + (long long)g.nv[0] * J : 0;
          const bool fcon = !raw && inr && !vmasked && face_constrained(g, I, J, 0);
          const int s = ix + IN0 * iy;
          cp_async_el(sx + s, A.xu + node, inr && !fcon);
          cp_async_el(sx + NIN + s, A.xu + Nv + node, inr && !fcon);
          if (CONV) {
            cp_async_el(sv + s, A.vc + node, inr);
            cp_async_el(sv + NIN + s, A.vc + Nv + node, inr);
          }
          mk[3 * r + q] = (vmasked && inr) ? g.vmask[node] : (fcon ? 1 : 0);
        }
      }
    }
  }
  if (WBT) {
    const int P0 = cs0 - 1, Q0 = cs1 - 1;
    for (int i = tid; i < PI0 * PI1; i += NT) {
      const int P = P0 + i % PI0, Q = Q0 + i / PI0;
      const bool inr = P >= 0 && P < g.npn[0] && Q >= 0 && Q < g.npn[1];
      const long long q = inr ? P + (long long)g.npn[0] * Q : 0;
      const bool con = inr && !raw && pnode_constrained(g, q);
      cp_async_el(sp + i, A.xp + q, inr && !con);
    }
  }
  if (SM::SB) {
    // b, d, D^-1 of the owned nodes this thread finalises in phase 3
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int i1 = ty + TY * r;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i0 = 2 * tx + q;
        if (i1 < ve1 && i0 < ve0) {
          const long long node = (2 * cs0 + i0) + (long long)g.nv[0] * (2 * cs1 + i1);
          const int o = i0 + VP0 * i1;
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            cp_async_el(sb + a * OWN + o, A.bu + a * Nv + node, true);
            if (SM::SD) {
              cp_async_el(sd + a * OWN + o, A.d + a * Nv + node, A.use_d != 0);
              cp_async_el(sdi + a * OWN + o, A.dinv + a * Nv + node, true);
            }
          }
        }
      }
    }
  }
  if (SM::SBP) {
    for (int i = tid; i < pe0 * pe1; i += NT) {
      const int p0 = i % pe0, p1 = i / pe0;
      const long long q = (cs0 + p0) + (long long)g.npn[0] * (cs1 + p1);
      cp_async_el(sbp + p0 + PP0 * p1, A.bp + q, true);
    }
  }
  if (NEED_U) {
#pragma unroll
    for (int r = 0; r < IROWS; ++r) {
      const int iy = ty + TY * r;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int ix = tx + 32 * q;
        if (iy < IN1 && ix < IN0) scon[ix + IN0 * iy] = mk[3 * r + q];
      }
    }
  }
  cp_async_commit_wait();
  if (NEED_U && vmasked) {
    // obstacle meshes: zero the staged constrained columns this thread copied
#pragma unroll
    for (int r = 0; r < IROWS; ++r) {
      const int iy = ty + TY * r;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int ix = tx + 32 * q;
        if (iy < IN1 && ix < IN0 && mk[3 * r + q]) {
          sx[ix + IN0 * iy] = T(0);
          sx[NIN + ix + IN0 * iy] = T(0);
        }
      }
    }
  }
  __syncthreads();

  // ---- phase 2: evaluate cells; thread (tx, ty) -> cells (tx, ty) and (tx, ty + 8) ----
#pragma unroll 1
  for (int k = 0; k < CROWS; ++k) {
    const int e0 = tx, e1 = ty + TY * k;
    if (e1 >= E1) continue;
    const int e = e0 + E0 * e1;
    const int c0 = cs0 - 1 + e0, c1 = cs1 - 1 + e1;
    bool active = c0 >= 0 && c0 < g.n[0] && c1 >= 0 && c1 < g.n[1];
    long long cell = 0;
    if (active) {
      cell = c0 + (long long)g.n[0] * c1;
      if (cell_void(g, cell)) active = false;
    }
    T yl[2][9];
    T ob[4];
#pragma unroll
    for (int i = 0; i < 9; ++i) yl[0][i] = yl[1][i] = T(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) ob[i] = T(0);
    if (active) {
      const T eta = A.eta[cell] * c.eta_scale;
      OpCoef<T> cK = c;  // the cell's mass coefficient (alpha per cell)
      if (A.alpha) cK.mm = c.mm * A.alpha[cell];
      T xl[2][9];
      if (NEED_U) {
        const T* s0p = sx + 2 * e0 + IN0 * 2 * e1;
#pragma unroll
        for (int lb = 0; lb < 3; ++lb)
#pragma unroll
          for (int la = 0; la < 3; ++la) {
            xl[0][la + 3 * lb] = s0p[la + IN0 * lb];
            xl[1][la + 3 * lb] = s0p[NIN + la + IN0 * lb];
          }
      }
      if (WA) {
        cell_A2(xl, yl, eta, cK);
        if (CONV) {
          T vl[2][9];
          const T* v0p = sv + 2 * e0 + IN0 * 2 * e1;
#pragma unroll
          for (int lb = 0; lb < 3; ++lb)
#pragma unroll
            for (int la = 0; la < 3; ++la) {
              vl[0][la + 3 * lb] = v0p[la + IN0 * lb];
              vl[1][la + 3 * lb] = v0p[NIN + la + IN0 * lb];
            }
          cell_conv2<CONV>(xl, vl, A.rho, A.rk[cell], A.ihx, A.ihy, A.wq, yl);
        }
      }
      if (WBT) {
        T pl[4];
#pragma unroll
        for (int lb = 0; lb < 2; ++lb)
#pragma unroll
          for (int la = 0; la < 2; ++la) pl[la + 2 * lb] = sp[(e0 + la) + PI0 * (e1 + lb)];
        cell_BT2(pl, yl, c, WA);
      }
      if (WB) cell_B2(xl, ob, c);
    }
    if (WU) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        ru[i * NCELL + e] = yl[0][i];
        ru[(9 + i) * NCELL + e] = yl[1][i];
      }
    }
    if (WB) {
#pragma unroll
      for (int i = 0; i < 4; ++i) rp[i * NCELL + e] = ob[i];
    }
  }
  __syncthreads();

  // ---- phase 3: owned nodes gather their cell results, epilogue ----
  if (WU) {
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int i1 = ty + TY * r;
      if (i1 >= ve1) continue;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i0 = 2 * tx + q;
        if (i0 >= ve0) continue;
        T s0, s1;
        if (ty & 1) {
          if (q) gather2<T, EY, true, true>(ru, i0, i1, s0, s1);
          else gather2<T, EY, false, true>(ru, i0, i1, s0, s1);
        } else {
          if (q) gather2<T, EY, true, false>(ru, i0, i1, s0, s1);
          else gather2<T, EY, false, false>(ru, i0, i1, s0, s1);
        }
        const long long node = (2 * cs0 + i0) + (long long)g.nv[0] * (2 * cs1 + i1);
        const int sidx = (i0 + 2) + IN0 * (i1 + 2);  // the node in the staged input tile
        const bool con = NEED_U ? (scon[sidx] != 0)
                                : (!raw && vnode_constrained(g, node, 2 * cs0 + i0, 2 * cs1 + i1, 0));
        const int o = i0 + VP0 * i1;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const long long gi = a * Nv + node;
          const T ax = con ? (WA ? A.xu[gi] : T(0)) : (a == 0 ? s0 : s1);
          if (MODE == TILE_APPLY) {
            A.yu[gi] = ax;
          } else if (MODE == TILE_RESID) {
            A.yu[gi] = sb[a * OWN + o] - ax;
          } else {
            const T rr = sb[a * OWN + o] - ax;
            T dn = A.c2 * sdi[a * OWN + o] * rr;
            if (A.use_d) dn += A.c1 * sd[a * OWN + o];
            A.d[gi] = dn;
            const T xin = con ? A.xu[gi] : sx[a * NIN + sidx];
            A.xout[gi] = xin + dn;
          }
        }
      }
    }
  }
  if (WB) {
    for (int i = tid; i < pe0 * pe1; i += NT) {
      const int p0 = i % pe0, p1 = i / pe0;
      T s = T(0);
      // cells p (local node 0) and p - 1 (local node 1) along each axis; evaluated index = cell + 1
      for (int b = 0; b < 2; ++b) {
        const int ey = p1 + 1 - b, lyy = b;
        if (ey >= E1) continue;
        for (int a = 0; a < 2; ++a) {
          const int ex = p0 + 1 - a, lxx = a;
          if (ex >= E0) continue;
          s += rp[(lxx + 2 * lyy) * NCELL + ex + E0 * ey];
        }
      }
      const long long q = (cs0 + p0) + (long long)g.npn[0] * (cs1 + p1);
      const bool con = !raw && pnode_constrained(g, q);
      const T bx = con ? (WBT ? A.xp[q] : T(0)) : s;
      if (MODE == TILE_RESID)
        A.yp[q] = sbp[p0 + PP0 * p1] - bx;
      else
        A.yp[q] = bx;
    }
  }
}

template <typename T, int EY, int MODE, bool WA, bool WBT, bool WB, int CONV = 0>
struct Tile2dK {
  using Args = TileArgs<T>;
  // FP64 with B^T (the saddle operator): 3 CTAs per SM (85 registers, a few spills) measured 2.6 %
  // faster than 2 on the FP64-pipe-bound saddle operator; the FP32 variants stay at 2 (72 registers)
  static constexpr int THREADS = NT, MINB = CONV ? 1 : (sizeof(T) == 8 && WBT ? 3 : 2);
  static __device__ __forceinline__ void body(const Args& a, int blk, int) {
    tile2d_body<T, EY, MODE, WA, WBT, WB, CONV>(a, blk);
  }
};

template <typename T, int EY, int MODE, bool WA, bool WBT, bool WB, int CONV = 0>
cudaError_t launch2(TileArgs<T> a, cudaStream_t st) {
  using S2 = Shape2<EY>;
  using SM = Smem2<EY, MODE, WA || WB, WBT, WA || WBT, WB, CONV>;
  a.tiles[0] = (a.g.n[0] + S2::TO0 - 1) / S2::TO0;
  a.tiles[1] = (a.g.n[1] + S2::TO1 - 1) / S2::TO1;
  a.tiles[2] = 1;
  const size_t smem = sizeof(T) * SM::TOTAL + SM::FLAGS;
  return submit<Tile2dK<T, EY, MODE, WA, WBT, WB, CONV>>(a, (long long)a.tiles[0] * a.tiles[1], smem, st);
}

// Velocity block and saddle operator with the corrector-stage terms (cell_conv2): conv = 1 adds
// rho (C + S), conv = 2 the symmetric part rho (S + (C + C^T) / 2) (velocity block only).
template <typename T, int EY>
cudaError_t launch_conv_shape(int mode, int ops, const TileArgs<T>& a, cudaStream_t st) {
  if (ops == OPS_A) {
    if (a.conv == 2) {
      if (mode == TILE_APPLY) return launch2<T, EY, TILE_APPLY, true, false, false, 2>(a, st);
      return cudaErrorInvalidValue;
    }
    if (mode == TILE_APPLY) return launch2<T, EY, TILE_APPLY, true, false, false, 1>(a, st);
    if (mode == TILE_RESID) return launch2<T, EY, TILE_RESID, true, false, false, 1>(a, st);
    return launch2<T, EY, TILE_CHEB, true, false, false, 1>(a, st);
  }
  if (ops == (OPS_A | OPS_BT | OPS_B) && a.conv == 1) {
    return mode == TILE_APPLY ? launch2<T, EY, TILE_APPLY, true, true, true, 1>(a, st)
                              : launch2<T, EY, TILE_RESID, true, true, true, 1>(a, st);
  }
  return cudaErrorInvalidValue;
}

// Launch one tile height.  FULL: every mode / operator combination is compiled; otherwise only
// the velocity-block modes the multigrid uses on every level (apply, residual, Chebyshev).
template <typename T, int EY, bool FULL>
cudaError_t launch_shape(int mode, int ops, const TileArgs<T>& a, cudaStream_t st) {
  if (ops == OPS_A) {
    if (mode == TILE_APPLY) return launch2<T, EY, TILE_APPLY, true, false, false>(a, st);
    if (mode == TILE_RESID) return launch2<T, EY, TILE_RESID, true, false, false>(a, st);
    return launch2<T, EY, TILE_CHEB, true, false, false>(a, st);
  }
  if constexpr (FULL) {
    if (mode == TILE_CHEB) return cudaErrorInvalidValue;
    const bool ap = mode == TILE_APPLY;
    switch (ops) {
      case OPS_BT:
        return ap ? launch2<T, EY, TILE_APPLY, false, true, false>(a, st) : launch2<T, EY, TILE_RESID, false, true, false>(a, st);
      case OPS_B:
        return ap ? launch2<T, EY, TILE_APPLY, false, false, true>(a, st) : launch2<T, EY, TILE_RESID, false, false, true>(a, st);
      case OPS_A | OPS_BT | OPS_B:
        return ap ? launch2<T, EY, TILE_APPLY, true, true, true>(a, st) : launch2<T, EY, TILE_RESID, true, true, true>(a, st);
      default:
        return cudaErrorInvalidValue;
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace tile2d

// per-height launchers (one translation unit each, compiled in parallel)
template <typename T>
cudaError_t launch_tile2d_e16(int mode, int ops, const TileArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_tile2d_e17(int mode, int ops, const TileArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_tile2d_e8(int mode, int ops, const TileArgs<T>& a, cudaStream_t st);

}  // namespace gs
