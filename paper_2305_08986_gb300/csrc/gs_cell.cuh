// Cell-level operators of the Q2-Q1 generalized Stokes system on Cartesian cells.
//
// On a Cartesian cell every term of the bilinear forms a(u, v) (Sec. 3.1.2, Eq. "form_a_j",
// with the stress factor 2 eta eps) and b(u, q) (Eq. "form_b") is a Kronecker product of 1D
// matrices, so the cell operators are applied by sweeps of 3x3 (or 2x3) matrices along one
// axis at a time ("sum factorisation" of Kronbichler-Kormann matrix-free operators, Sec. 4).
// The 1D matrices are exact rationals; they are stored here as small integers, and the
// denominators and mesh widths live in the level coefficients OpCoef:
//
//   Mi/30  = int_0^1 phi_i phi_j          Mi = [4 2 -1; 2 16 2; -1 2 4]
//   Ki/3   = int_0^1 phi_i' phi_j'        Ki = [7 -8 1; -8 16 -8; 1 -8 7]
//   Ei/6   = int_0^1 phi_i' phi_j         Ei = [-3 -4 1; 4 0 -4; -1 4 3]   (test derivative)
//   Ni/6   = int_0^1 psi_a phi_b          Ni = [1 2 0; 0 2 1]
//   Gi/6   = int_0^1 psi_a phi_b'         Gi = [-5 4 1; -1 -4 5]
//   Pi/6   = int_0^1 psi_a psi_b          Pi = [2 1; 1 2]
//
// with phi the Q2 Lagrange basis on nodes {0, 1/2, 1} and psi the Q1 basis on {0, 1}.
// Local arrays are indexed a + 3 b (+ 9 c) (x fastest), Q1 arrays a + 2 b (+ 4 c).
#pragma once
#include "gs_common.cuh"

namespace gs {

// ---- 1D line operators ----------------------------------------------------------------------
struct OpM {
  static constexpr int NIN = 3, NOUT = 3;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = T(4) * a[0] + T(2) * a[1] - a[2];
    o[1] = T(2) * (a[0] + a[2]) + T(16) * a[1];
    o[2] = -a[0] + T(2) * a[1] + T(4) * a[2];
  }
};
struct OpK {
  static constexpr int NIN = 3, NOUT = 3;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = T(7) * a[0] - T(8) * a[1] + a[2];
    o[1] = T(-8) * (a[0] + a[2]) + T(16) * a[1];
    o[2] = a[0] - T(8) * a[1] + T(7) * a[2];
  }
};
struct OpE {  // Ei
  static constexpr int NIN = 3, NOUT = 3;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = T(-3) * a[0] - T(4) * a[1] + a[2];
    o[1] = T(4) * (a[0] - a[2]);
    o[2] = -a[0] + T(4) * a[1] + T(3) * a[2];
  }
};
struct OpET {  // Ei^T
  static constexpr int NIN = 3, NOUT = 3;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = T(-3) * a[0] + T(4) * a[1] - a[2];
    o[1] = T(-4) * (a[0] - a[2]);
    o[2] = a[0] - T(4) * a[1] + T(3) * a[2];
  }
};
struct OpN {  // Ni: 3 -> 2
  static constexpr int NIN = 3, NOUT = 2;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = a[0] + T(2) * a[1];
    o[1] = T(2) * a[1] + a[2];
  }
};
struct OpG {  // Gi: 3 -> 2
  static constexpr int NIN = 3, NOUT = 2;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = T(-5) * a[0] + T(4) * a[1] + a[2];
    o[1] = -a[0] - T(4) * a[1] + T(5) * a[2];
  }
};
struct OpNT {  // Ni^T: 2 -> 3
  static constexpr int NIN = 2, NOUT = 3;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = a[0];
    o[1] = T(2) * (a[0] + a[1]);
    o[2] = a[1];
  }
};
struct OpGT {  // Gi^T: 2 -> 3
  static constexpr int NIN = 2, NOUT = 3;
  template <typename T> __device__ __forceinline__ static void f(const T* a, T* o) {
    o[0] = T(-5) * a[0] - a[1];
    o[1] = T(4) * (a[0] - a[1]);
    o[2] = a[0] + T(5) * a[1];
  }
};

// Apply a line operator along axis AX of an array with extents (E0, E1, E2); the output has
// extent Op::NOUT along AX.  ACC: add into out instead of overwriting.
template <class Op, int AX, int E0, int E1, int E2, bool ACC, typename T>
__device__ __forceinline__ void sweep(const T* __restrict__ in, T* __restrict__ out) {
  constexpr int O0 = AX == 0 ? Op::NOUT : E0;
  constexpr int O1 = AX == 1 ? Op::NOUT : E1;
  constexpr int L0 = AX == 0 ? 1 : E0;
  constexpr int L1 = AX == 1 ? 1 : E1;
  constexpr int L2 = AX == 2 ? 1 : E2;
#pragma unroll
  for (int k = 0; k < L2; ++k) {
#pragma unroll
    for (int j = 0; j < L1; ++j) {
#pragma unroll
      for (int i = 0; i < L0; ++i) {
        T a[Op::NIN], o[Op::NOUT];
#pragma unroll
        for (int t = 0; t < Op::NIN; ++t) {
          const int ii = AX == 0 ? t : i, jj = AX == 1 ? t : j, kk = AX == 2 ? t : k;
          a[t] = in[ii + E0 * (jj + E1 * kk)];
        }
        Op::f(a, o);
#pragma unroll
        for (int t = 0; t < Op::NOUT; ++t) {
          const int ii = AX == 0 ? t : i, jj = AX == 1 ? t : j, kk = AX == 2 ? t : k;
          if (ACC)
            out[ii + O0 * (jj + O1 * kk)] += o[t];
          else
            out[ii + O0 * (jj + O1 * kk)] = o[t];
        }
      }
    }
  }
}

// ---- viscous + mass block -------------------------------------------------------------------
// y_a = sum_b A_ab^K x_b for both output components a of a 2D cell, with A^K the cell block of
// alpha (phi_i, phi_j) delta_ab + eta_K (2 eps(phi_j e_b), eps(phi_i e_a)).  Writes y (not +=).
//
// Diagonal block (true 1D matrices M, K):  alpha MM + eta (1+[a=x]) K_x M_y + eta (1+[a=y]) M_x K_y;
// off-diagonal blocks: eta (E^T along x)(E along y) x_y for a = x, eta (E along x)(E^T along y) x_x
// for a = y.  Evaluation, per input component (three node columns along y):
//   1. the three sweeps along y that the component feeds (M, K and E or E^T) from the symmetric and
//      antisymmetric parts s = x_0 + x_2, d = x_0 - x_2 of each column (M and K are centro-symmetric,
//      E and E^T centro-antisymmetric), e.g. (M x)_0 = 1.5 s + 2.5 d + 2 x_1;
//   2. per output node row, one fused combination along x, y_row = (mm M + cq K) a + ck M k + ce G r,
//      again from the symmetric / antisymmetric parts of the swept rows: y_0 = S + D, y_2 = S - D.
// This takes about 40 % fewer floating-point operations than sweeping each 1D operator separately;
// the exact 1D matrices are those of the header, only the association of the sums differs.
template <typename T>
__device__ __forceinline__ void ysweep_mk(T x0, T x1, T x2, T& s, T& d, T (&m)[3], T (&k)[3], T& q4) {
  s = x0 + x2;
  d = x0 - x2;
  const T q2 = T(2) * x1, q16 = T(16) * x1;
  q4 = T(4) * x1;
  const T u = fma(T(1.5), s, q2);          // M = [4 2 -1; 2 16 2; -1 2 4]
  m[0] = fma(T(2.5), d, u);
  m[2] = fma(T(-2.5), d, u);
  m[1] = fma(T(2), s, q16);
  const T v = fma(T(4), s, T(-2) * q4);    // K = [7 -8 1; -8 16 -8; 1 -8 7]
  k[0] = fma(T(3), d, v);
  k[2] = fma(T(-3), d, v);
  k[1] = fma(T(-8), s, q16);
}

// Output node row of component a from the swept rows a_ (M_y x_a), k_ (K_y x_a), r_ (the off-diagonal
// sweep); CA = 0: G = E^T along x (output x), CA = 1: G = E along x (output y).
template <int CA, typename T>
__device__ __forceinline__ void xrow_fused(const T* a_, const T* k_, const T* r_, T hs, T hd, T c01, T c11, T ck15,
                                           T ck2, T ck25, T ck16, T ce, T* y) {
  const T sa = a_[0] + a_[2], da = a_[0] - a_[2];
  const T sk = k_[0] + k_[2], dk = k_[0] - k_[2];
  const T sr = r_[0] + r_[2], dr = r_[0] - r_[2];
  // S = (y0 + y2) / 2, D = (y0 - y2) / 2
  T S = hs * sa + c01 * a_[1] + ck15 * sk + ck2 * k_[1];
  T D = hd * da + ck25 * dk;
  T y1 = c01 * sa + c11 * a_[1] + ck2 * sk + ck16 * k_[1];
  if (CA == 0) {  // E^T = [-3 4 -1; -4 0 4; 1 -4 3]
    S = fma(-ce, dr, S);
    D = fma(T(-2) * ce, sr, fma(T(4) * ce, r_[1], D));
    y1 = fma(T(-4) * ce, dr, y1);
  } else {        // E = [-3 -4 1; 4 0 -4; -1 4 3]
    S = fma(T(-2) * ce, dr, S);
    D = fma(-ce, sr, fma(T(-4) * ce, r_[1], D));
    y1 = fma(T(4) * ce, dr, y1);
  }
  y[0] = S + D;
  y[1] = y1;
  y[2] = S - D;
}

template <typename T>
__device__ __forceinline__ void cell_A2(const T (&x)[2][9], T (&y)[2][9], T eta, const OpCoef<T>& c) {
  // sweeps along y, column by column (column i = nodes i, i + 3, i + 6)
  T a[2][9], k[2][9], r[2][9];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T s0, d0, q40, m0[3], k0[3];
    ysweep_mk(x[0][i], x[0][i + 3], x[0][i + 6], s0, d0, m0, k0, q40);
    T s1, d1, q41, m1[3], k1[3];
    ysweep_mk(x[1][i], x[1][i + 3], x[1][i + 6], s1, d1, m1, k1, q41);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      a[0][i + 3 * j] = m0[j];
      k[0][i + 3 * j] = k0[j];
      a[1][i + 3 * j] = m1[j];
      k[1][i + 3 * j] = k1[j];
    }
    // output x takes E_y x_y: E = [-3 -4 1; 4 0 -4; -1 4 3]
    const T z = s1 + q41;
    r[0][i] = fma(T(-2), d1, -z);
    r[0][i + 3] = T(4) * d1;
    r[0][i + 6] = fma(T(-2), d1, z);
    // output y takes E^T_y x_x: E^T = [-3 4 -1; -4 0 4; 1 -4 3]
    r[1][i] = fma(T(-2), s0, q40 - d0);
    r[1][i + 3] = T(-4) * d0;
    r[1][i + 6] = fma(T(2), s0, -(d0 + q40));
  }
  const T mm = c.mm;
  const T ce = eta * c.ex[0];
#pragma unroll
  for (int comp = 0; comp < 2; ++comp) {
    const T ck = (comp == 1 ? T(2) : T(1)) * eta * c.km[1];   // stiffness along y
    const T cq = (comp == 0 ? T(2) : T(1)) * eta * c.km[0];   // stiffness along x
    // C = mm M + cq K: c00 = 4 mm + 7 cq, c01 = 2 mm - 8 cq, c02 = cq - mm, c11 = 16 (mm + cq)
    const T hs = fma(T(1.5), mm, T(4) * cq);   // (c00 + c02) / 2
    const T hd = fma(T(2.5), mm, T(3) * cq);   // (c00 - c02) / 2
    const T c01 = fma(T(2), mm, T(-8) * cq);
    const T c11 = T(16) * (mm + cq);
    const T ck15 = T(1.5) * ck, ck2 = T(2) * ck, ck25 = T(2.5) * ck, ck16 = T(16) * ck;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (comp == 0)
        xrow_fused<0>(a[0] + 3 * j, k[0] + 3 * j, r[0] + 3 * j, hs, hd, c01, c11, ck15, ck2, ck25, ck16, ce,
                      y[0] + 3 * j);
      else
        xrow_fused<1>(a[1] + 3 * j, k[1] + 3 * j, r[1] + 3 * j, hs, hd, c01, c11, ck15, ck2, ck25, ck16, ce,
                      y[1] + 3 * j);
    }
  }
}

// ---- corrector stage: convection by a given field and streamline diffusion (2D) -----------------
// In the corrector stage (Sec. 3.1.2, Eq. "v_star") the velocity block gains
//   rho ((v° . grad) u, w)                                   (convection by the given Q2 field v°)
//   rho r_K ((v° . grad) u, (v° . grad) w)_K                 (streamline diffusion, Eq. "a_stab")
// on every velocity component alike.  Both are evaluated at the 3 x 3 Gauss points of the cell
// (the rule of every other cell integral) by sum factorisation with the 1D matrices
//   Phi[q][j] = phi_j(g_q),  Dq[q][j] = phi_j'(g_q)  (g = 1/2 -+ sqrt(3/5)/2, 1/2 on [0, 1]),
// i.e. v° and grad u are interpolated to the Gauss points, combined pointwise, weighted and swept
// back with the transposed matrices.  With s = sqrt(3/5) / 2:
//   Phi = [0.3+s 0.4 0.3-s; 0 1 0; 0.3-s 0.4 0.3+s],
//   Dq  = [-1-4s 8s 1-4s; -1 0 1; -1+4s -8s 1+4s].
struct GaussQ2 {
  static constexpr double s = 0.38729833462074168852;   // sqrt(3/5) / 2
  __host__ __device__ static constexpr double phi(int q, int j) {
    return q == 1 ? (j == 1 ? 1.0 : 0.0) : (j == 1 ? 0.4 : (((q == 0) == (j == 0)) ? 0.3 + s : 0.3 - s));
  }
  __host__ __device__ static constexpr double dq(int q, int j) {
    return q == 1 ? (j == 0 ? -1.0 : (j == 1 ? 0.0 : 1.0))
                  : (j == 1 ? (q == 0 ? 8.0 * s : -8.0 * s) : (j == 0 ? -1.0 : 1.0) + (q == 0 ? -4.0 * s : 4.0 * s));
  }
  __host__ __device__ static constexpr double w(int q) { return q == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }
};

// out[along axis AX] = M in (TR: M^T in), M one of the 3 x 3 Gauss matrices; arrays 3 x 3, x fastest.
template <int AX, bool TR, bool DER, typename T>
__device__ __forceinline__ void gsweep(const T* __restrict__ in, T* __restrict__ out) {
#pragma unroll
  for (int o = 0; o < 3; ++o)      // the other axis
#pragma unroll
    for (int p = 0; p < 3; ++p) {  // output index along AX
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double m = TR ? (DER ? GaussQ2::dq(q, p) : GaussQ2::phi(q, p)) : (DER ? GaussQ2::dq(p, q) : GaussQ2::phi(p, q));
        if (m == 0.0) continue;
        const int ii = AX == 0 ? q : o, jj = AX == 0 ? o : q;
        acc += T(m) * in[ii + 3 * jj];
      }
      const int io = AX == 0 ? p : o, jo = AX == 0 ? o : p;
      out[io + 3 * jo] = acc;
    }
}

// y += rho (C + S) u   (CONV = 1)   or   y += rho (S + (C + C^T) / 2) u   (CONV = 2, the symmetric
// part, for the Chebyshev bounds of the non-symmetric block), for both components of u.
// vc: the cell's nodal v° (two components), rK: the cell's streamline parameter, ihx = 1 / h_x,
// ihy = 1 / h_y, wq = h_x h_y (the Jacobian of the Gauss weights).
template <int CONV, typename T>
__device__ __forceinline__ void cell_conv2(const T (&u)[2][9], const T (&vc)[2][9], T rho, T rK, T ihx, T ihy, T wq,
                                           T (&y)[2][9]) {
  T t[9], vx[9], vy[9], W[9];
  gsweep<0, false, false>(vc[0], t);
  gsweep<1, false, false>(t, vx);              // v°_x at the Gauss points
  gsweep<0, false, false>(vc[1], t);
  gsweep<1, false, false>(t, vy);              // v°_y at the Gauss points
#pragma unroll
  for (int qb = 0; qb < 3; ++qb)
#pragma unroll
    for (int qa = 0; qa < 3; ++qa) W[qa + 3 * qb] = T(GaussQ2::w(qa) * GaussQ2::w(qb)) * wq;
  const T kc = CONV == 1 ? rho : T(0.5) * rho;  // weight of C u
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    T px[9], gx[9], gy[9], c[9], g[9], back[9];
    gsweep<0, false, true>(u[a], t);
    gsweep<1, false, false>(t, gx);             // d u / d x (reference), / h_x below
    gsweep<0, false, false>(u[a], px);
    gsweep<1, false, true>(px, gy);             // d u / d y (reference), / h_y below
    T uq[9];
    if (CONV == 2) gsweep<1, false, false>(px, uq);  // u at the Gauss points
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const T adv = vx[q] * gx[q] * ihx + vy[q] * gy[q] * ihy;  // v° . grad u
      c[q] = kc * W[q] * adv;
      g[q] = rho * rK * W[q] * adv;                            // streamline source
      if (CONV == 2) g[q] += T(0.5) * rho * W[q] * uq[q];      // C^T u
    }
    // C u: (Phi^T x Phi^T) c
    gsweep<0, true, false>(c, t);
    gsweep<1, true, false>(t, back);
#pragma unroll
    for (int i = 0; i < 9; ++i) y[a][i] += back[i];
    // (v° . grad phi_i) terms: (Dq^T x Phi^T)(v°_x g) / h_x + (Phi^T x Dq^T)(v°_y g) / h_y
#pragma unroll
    for (int q = 0; q < 9; ++q) c[q] = vx[q] * g[q] * ihx;
    gsweep<0, true, true>(c, t);
    gsweep<1, true, false>(t, back);
#pragma unroll
    for (int i = 0; i < 9; ++i) y[a][i] += back[i];
#pragma unroll
    for (int q = 0; q < 9; ++q) c[q] = vy[q] * g[q] * ihy;
    gsweep<0, true, false>(c, t);
    gsweep<1, true, true>(t, back);
#pragma unroll
    for (int i = 0; i < 9; ++i) y[a][i] += back[i];
  }
}

// ---- corrector stage in 3D: the same terms at the 3 x 3 x 3 Gauss points ---------------------------
// out = (M along axis AX) in on a 3 x 3 x 3 array (x fastest); M = Phi or Dq (TR: transposed).
template <int AX, bool TR, bool DER, typename T>
__device__ __forceinline__ void gsweep3(const T* __restrict__ in, T* __restrict__ out) {
#pragma unroll
  for (int o2 = 0; o2 < 3; ++o2)
#pragma unroll
    for (int o1 = 0; o1 < 3; ++o1)
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const double m = TR ? (DER ? GaussQ2::dq(q, p) : GaussQ2::phi(q, p)) : (DER ? GaussQ2::dq(p, q) : GaussQ2::phi(p, q));
          if (m == 0.0) continue;
          const int a = AX == 0 ? q : o1, b = AX == 0 ? o1 : (AX == 1 ? q : o2), c = AX == 2 ? q : o2;
          acc += T(m) * in[a + 3 * b + 9 * c];
        }
        const int a = AX == 0 ? p : o1, b = AX == 0 ? o1 : (AX == 1 ? p : o2), c = AX == 2 ? p : o2;
        out[a + 3 * b + 9 * c] = acc;
      }
}

// (Phi or Dq along each axis) of a nodal 3 x 3 x 3 array: DX, DY, DZ select Dq on that axis
template <bool DX, bool DY, bool DZ, bool TR, typename T>
__device__ __forceinline__ void gsweep3_all(const T* __restrict__ in, T* __restrict__ out, T* __restrict__ tmp) {
  gsweep3<0, TR, DX>(in, out);
  gsweep3<1, TR, DY>(out, tmp);
  gsweep3<2, TR, DZ>(tmp, out);
}

// y += rho (C + S) u (CONV = 1) or rho (S + (C + C^T) / 2) u (CONV = 2) for one velocity component in
// the rotated frame of the caller: u, and v° component q (the component along logical axis q), are
// read from shared-memory windows at x[o0[i] + o1[j] + o2[k]]; ih[q] = 1 / h along logical axis q;
// jac = h_x h_y h_z.  Sum factorisation at the 3 x 3 x 3 Gauss points as in cell_conv2; the v°
// interpolation is redone for the back sweeps instead of keeping three Gauss-point arrays alive.
template <int CONV, typename T>
__device__ __forceinline__ void cell_conv3(const T* u_, const T* const (&v_)[3], const int* o0, const int* o1,
                                           const int* o2, T rho, T rK, const T (&ih)[3], T jac, T (&y)[27]) {
  T uu[27], f[27], g[27], t[27], adv[27];
  auto load = [&](const T* base, T (&dst)[27]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) dst[i + 3 * j + 9 * k] = base[o0[i] + o1[j] + o2[k]];
  };
  load(u_, uu);
#pragma unroll
  for (int q = 0; q < 27; ++q) adv[q] = T(0);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    T vv[27];
    load(v_[ax], vv);
    gsweep3_all<false, false, false, false>(vv, f, t);  // v°_ax at the Gauss points
    if (ax == 0) gsweep3_all<true, false, false, false>(uu, g, t);
    else if (ax == 1) gsweep3_all<false, true, false, false>(uu, g, t);
    else gsweep3_all<false, false, true, false>(uu, g, t);  // d u / d x_ax (reference)
#pragma unroll
    for (int q = 0; q < 27; ++q) adv[q] += f[q] * g[q] * ih[ax];
  }
  const T kc = CONV == 1 ? rho : T(0.5) * rho;
  if (CONV == 2) gsweep3_all<false, false, false, false>(uu, g, t);  // u at the Gauss points
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = a + 3 * b + 9 * c;
        const T W = T(GaussQ2::w(a) * GaussQ2::w(b) * GaussQ2::w(c)) * jac;
        f[q] = kc * W * adv[q];                                  // C u at the Gauss points
        T sq = rho * rK * W * adv[q];                             // streamline source
        if (CONV == 2) sq += T(0.5) * rho * W * g[q];             // C^T u
        adv[q] = sq;
      }
  gsweep3_all<false, false, false, true>(f, g, t);              // (Phi^T x Phi^T x Phi^T)
#pragma unroll
  for (int q = 0; q < 27; ++q) y[q] += g[q];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {  // (v° . grad phi_i) terms, axis by axis
    T vv[27];
    load(v_[ax], vv);
    gsweep3_all<false, false, false, false>(vv, f, t);
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q] = f[q] * adv[q] * ih[ax];
    if (ax == 0) gsweep3_all<true, false, false, true>(f, g, t);
    else if (ax == 1) gsweep3_all<false, true, false, true>(f, g, t);
    else gsweep3_all<false, false, true, true>(f, g, t);
#pragma unroll
    for (int q = 0; q < 27; ++q) y[q] += g[q];
  }
}

// ---- 3D cell operators reading their input nodes from a shared-memory window ----------------------
// x_a points to the cell's local node (0, 0, 0) of component a in the window; local node (i, j, k)
// sits at x_a[i + ro[j] + po[k]] (row and plane offsets of the cell, which absorb any skew of the
// window layout).  The first sweep over each input reads the window directly, so the inputs never
// sit in registers.
template <class Op, int AX, typename T>
__device__ __forceinline__ void sweep_w(const T* __restrict__ in, const int* ro, const int* po, T* __restrict__ out) {
  constexpr int O0 = AX == 0 ? Op::NOUT : 3;
  constexpr int O1 = AX == 1 ? Op::NOUT : 3;
  constexpr int L0 = AX == 0 ? 1 : 3;
  constexpr int L1 = AX == 1 ? 1 : 3;
  constexpr int L2 = AX == 2 ? 1 : 3;
#pragma unroll
  for (int k = 0; k < L2; ++k) {
#pragma unroll
    for (int j = 0; j < L1; ++j) {
#pragma unroll
      for (int i = 0; i < L0; ++i) {
        T a[Op::NIN], o[Op::NOUT];
#pragma unroll
        for (int t = 0; t < Op::NIN; ++t) {
          const int ii = AX == 0 ? t : i, jj = AX == 1 ? t : j, kk = AX == 2 ? t : k;
          a[t] = in[ii + ro[jj] + po[kk]];
        }
        Op::f(a, o);
#pragma unroll
        for (int t = 0; t < Op::NOUT; ++t) {
          const int ii = AX == 0 ? t : i, jj = AX == 1 ? t : j, kk = AX == 2 ? t : k;
          out[ii + O0 * (jj + O1 * kk)] = o[t];
        }
      }
    }
  }
}

// ---- divergence block B and its transpose -----------------------------------------------------
// (B u)_q = - sum_b int psi_q d phi_j/dx_b u_jb :  -sum_b (G in direction b, N elsewhere) u_b
template <typename T>
__device__ __forceinline__ void cell_B2(const T (&u)[2][9], T (&out)[4], const OpCoef<T>& c) {
  T t[6], s[4];
  sweep<OpN, 1, 3, 3, 1, false>(u[0], t);  // (3,2)
  sweep<OpG, 0, 3, 2, 1, false>(t, out);   // (2,2)
  sweep<OpG, 1, 3, 3, 1, false>(u[1], t);
  sweep<OpN, 0, 3, 2, 1, false>(t, s);
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = -(c.bd[0] * out[i] + c.bd[1] * s[i]);
}

template <typename T>
__device__ __forceinline__ void cell_BT2(const T (&p)[4], T (&u)[2][9], const OpCoef<T>& c, bool acc) {
  T t[6], v[9];
  sweep<OpNT, 1, 2, 2, 1, false>(p, t);  // (2,3)
  sweep<OpGT, 0, 2, 3, 1, false>(t, v);  // (3,3)
#pragma unroll
  for (int i = 0; i < 9; ++i) u[0][i] = (acc ? u[0][i] : T(0)) - c.bd[0] * v[i];
  sweep<OpGT, 1, 2, 2, 1, false>(p, t);
  sweep<OpNT, 0, 2, 3, 1, false>(t, v);
#pragma unroll
  for (int i = 0; i < 9; ++i) u[1][i] = (acc ? u[1][i] : T(0)) - c.bd[1] * v[i];
}

// ---- 3D operator in a rotated frame: one code path for every output component ------------------
// Local node (i, j, k) of the window sits at in[o0[i] + o1[j] + o2[k]]: the three offset tables map
// the logical axes to any physical axes.  A thread computing output component a uses the frame
// (a, a + 1, a + 2) (cyclic), rotated coefficients, and its own component as the logical x input,
// so one expression -- the one for output component 0 -- serves all three components (one
// instruction stream).  Diagonal block: alpha MMM + eta (1 + [a = x]) KMM + eta (1 + [a = y]) MKM +
// eta (1 + [a = z]) MMK; off-diagonal blocks: eta (E in direction b) (E^T in direction a) (M in
// the third direction).
template <class Op, int AX, typename T>
__device__ __forceinline__ void sweep_p(const T* __restrict__ in, const int* o0, const int* o1, const int* o2,
                                        T* __restrict__ out) {
  constexpr int O0 = AX == 0 ? Op::NOUT : 3;
  constexpr int O1 = AX == 1 ? Op::NOUT : 3;
  constexpr int L0 = AX == 0 ? 1 : 3;
  constexpr int L1 = AX == 1 ? 1 : 3;
  constexpr int L2 = AX == 2 ? 1 : 3;
#pragma unroll
  for (int k = 0; k < L2; ++k) {
#pragma unroll
    for (int j = 0; j < L1; ++j) {
#pragma unroll
      for (int i = 0; i < L0; ++i) {
        T a[Op::NIN], o[Op::NOUT];
#pragma unroll
        for (int t = 0; t < Op::NIN; ++t) {
          const int ii = AX == 0 ? t : i, jj = AX == 1 ? t : j, kk = AX == 2 ? t : k;
          a[t] = in[o0[ii] + o1[jj] + o2[kk]];
        }
        Op::f(a, o);
#pragma unroll
        for (int t = 0; t < Op::NOUT; ++t) {
          const int ii = AX == 0 ? t : i, jj = AX == 1 ? t : j, kk = AX == 2 ? t : k;
          out[ii + O0 * (jj + O1 * kk)] = o[t];
        }
      }
    }
  }
}

// y (logical layout, x fastest) = output component "logical x" of the cell operator; xc / x1 / x2:
// the input components along logical x / y / z; km, ex: coefficients of the logical axes
template <typename T>
__device__ __forceinline__ void cell_A3p(const T* xc, const T* x1, const T* x2, const int* o0, const int* o1,
                                         const int* o2, T (&y)[27], T eta, T mm, const T* km, const T* ex) {
  T a[27], k[27], b[27];
  sweep_p<OpM, 2>(xc, o0, o1, o2, a);
  sweep_p<OpK, 2>(xc, o0, o1, o2, k);
  {
    const T ckz = eta * km[2];
#pragma unroll
    for (int i = 0; i < 27; ++i) b[i] = mm * a[i] + ckz * k[i];
  }
  sweep<OpM, 1, 3, 3, 3, false>(b, k);
  sweep<OpK, 1, 3, 3, 3, false>(a, b);
  {
    const T cky = eta * km[1];
#pragma unroll
    for (int i = 0; i < 27; ++i) k[i] += cky * b[i];
  }
  sweep<OpM, 1, 3, 3, 3, false>(a, b);
  {
    const T ckx = T(2) * eta * km[0];
#pragma unroll
    for (int i = 0; i < 27; ++i) b[i] *= ckx;
  }
  sweep<OpM, 0, 3, 3, 3, false>(k, y);
  sweep<OpK, 0, 3, 3, 3, true>(b, y);
  sweep_p<OpM, 2>(x1, o0, o1, o2, a);
  sweep<OpE, 1, 3, 3, 3, false>(a, k);
  sweep_p<OpE, 2>(x2, o0, o1, o2, a);
  sweep<OpM, 1, 3, 3, 3, false>(a, b);
  const T c1 = eta * ex[2], c2 = eta * ex[1];
#pragma unroll
  for (int i = 0; i < 27; ++i) k[i] = c1 * k[i] + c2 * b[i];
  sweep<OpET, 0, 3, 3, 3, true>(k, y);
}

// B^T contribution to output component "logical x" in the rotated frame: -bd_a (Gi^T along x, Ni^T
// along y and z) applied to the cell's pressure nodes given in the logical frame
template <typename T>
__device__ __forceinline__ void cell_BT3p(const T (&p)[8], T (&u)[27], T bd_a, bool acc) {
  T a[12], b[18], v[27];
  sweep<OpNT, 2, 2, 2, 2, false>(p, a);  // (2,2,3)
  sweep<OpNT, 1, 2, 2, 3, false>(a, b);  // (2,3,3)
  sweep<OpGT, 0, 2, 3, 3, false>(b, v);  // (3,3,3)
#pragma unroll
  for (int i = 0; i < 27; ++i) u[i] = (acc ? u[i] : T(0)) - bd_a * v[i];
}

// (B u) of one 3D cell with the velocity read from a shared-memory window:
// (B u)_q = -sum_b bd[b] (Gi in direction b, Ni elsewhere) u_b
template <typename T>
__device__ __forceinline__ void cell_B3w(const T* u0, const T* u1, const T* u2, const int* ro, const int* po,
                                         T (&out)[8], const OpCoef<T>& c) {
  T t0[18], t1[18], s0[12], s1v[12], o[8];
  sweep_w<OpN, 2>(u0, ro, po, t0);        // (3,3,2)
  sweep_w<OpN, 2>(u1, ro, po, t1);
  sweep<OpN, 1, 3, 3, 2, false>(t0, s0);  // (3,2,2)
  sweep<OpG, 0, 3, 2, 2, false>(s0, out); // (2,2,2)
  sweep<OpG, 1, 3, 3, 2, false>(t1, s1v);
  sweep_w<OpG, 2>(u2, ro, po, t0);
  sweep<OpN, 1, 3, 3, 2, false>(t0, s0);
  const T c1 = c.bd[1], c2 = c.bd[2];
#pragma unroll
  for (int i = 0; i < 12; ++i) s1v[i] = c1 * s1v[i] + c2 * s0[i];
  sweep<OpN, 0, 3, 2, 2, false>(s1v, o);
#pragma unroll
  for (int i = 0; i < 8; ++i) out[i] = -(c.bd[0] * out[i] + o[i]);
}

// ---- diagonal of the viscous + mass block at one local node -------------------------------------
__host__ __device__ inline int mdiag(int a) { return a == 1 ? 16 : 4; }
__host__ __device__ inline int kdiag(int a) { return a == 1 ? 16 : 7; }

template <typename T>
__device__ __forceinline__ T cell_diagA(int dim, int comp, int la, int lb, int lc, T eta, const OpCoef<T>& c) {
  if (dim == 2) {
    const T Ma = T(mdiag(la)), Mb = T(mdiag(lb)), Ka = T(kdiag(la)), Kb = T(kdiag(lb));
    const T ck = (comp == 1 ? T(2) : T(1)) * eta * c.km[1];
    const T cq = (comp == 0 ? T(2) : T(1)) * eta * c.km[0];
    return Ma * (c.mm * Mb + ck * Kb) + Ka * (cq * Mb);
  }
  const T Ma = T(mdiag(la)), Mb = T(mdiag(lb)), Mc = T(mdiag(lc));
  const T Ka = T(kdiag(la)), Kb = T(kdiag(lb)), Kc = T(kdiag(lc));
  const T ckz = (comp == 2 ? T(2) : T(1)) * eta * c.km[2];
  const T cky = (comp == 1 ? T(2) : T(1)) * eta * c.km[1];
  const T ckx = (comp == 0 ? T(2) : T(1)) * eta * c.km[0];
  return Ma * (Mb * (c.mm * Mc + ckz * Kc) + cky * Kb * Mc) + Ka * (ckx * Mb * Mc);
}

}  // namespace gs
