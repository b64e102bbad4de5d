// Per-element arithmetic of the P1 operator (device functions).
//
//   geometry (App. A, explicit shape-function differentiation): D = [X_1-X_0 .. X_d-X_0],
//     dN_a/dX = row a-1 of D^-1 = c_a / det D (a >= 1) with c_a the rows of adj(D) (3-D:
//     c_1 = d_2 x d_3, c_2 = d_3 x d_1, c_3 = d_1 x d_2), dN_0/dX = -sum, V = |det D| / d!.
//     The kernels keep c_a unscaled and fold 1/det into one scale per element:
//     grad w = G'/det with G' = sum_a (w_a - w_0) (x) c_a, and for a stress T,
//     V T dN_a = T c_a * sgn(det)/d!  (and V (T(G'/det)) dN_a = T(G') c_a / (d! |det|) when T
//     is linear in the gradient).
//   linear (Sec. "Linear elastic plate with arbitrary holes"): eps = sym grad w, sigma = 2 mu eps + lam tr(eps) I, Psi = 1/2 sigma:eps;
//     force / tangent action  y_a = V sigma(w) dN_a  (f_int = K u for linear FEM, App. B)
//   Neo-Hookean (Sec. "Nonlinear hyperelasticity" energy; App. B total Lagrangian): F = I + grad u, J = det F,
//     H = F^-T = cof(F) / J, first Piola-Kirchhoff stress P = F S = mu (F - H) + lam ln J H
//     (S = mu (I - C^-1) + lam ln J C^-1), f_a = V P dN_a,
//     Psi = 1/2 lam ln^2 J - mu ln J + 1/2 mu (I1 - d);
//     tangent action = directional derivative of P along dF = grad v:
//       dP = mu dF + (mu - lam ln J) H dF^T H + lam (H : dF) H,  y_a = V dP dN_a
//     which is (K_geo + K_mat) v of App. B written in the two-point (P) form.
//   Jacobi diagonal: with dF = e_i (x) g_a the same derivative gives
//       K_(a i)(a i) = V [ mu |g_a|^2 + (mu + lam - lam ln J) (H g_a)_i^2 ]   (linear: H = I, ln J = 0).
#pragma once

#include <cuda_runtime.h>

namespace pfem {

template <typename T>
__device__ __forceinline__ T drcp(T x);
template <>
__device__ __forceinline__ float drcp<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double drcp<double>(double x) { return 1.0 / x; }

template <int DIM>
struct Factorial;
template <>
struct Factorial<2> {
  static constexpr double value = 2.0;
};
template <>
struct Factorial<3> {
  static constexpr double value = 6.0;
};

// c[a][j]: row a of adj(D) (gradient of N_{a+1} times det); det = det D; rdet = 1 / det;
// s = 1 / (d! |det|) (= V / det^2); kappa = sgn(det) / d! (= V / det).
template <int DIM, typename CT>
struct ElemGeo {
  CT c[DIM][DIM];
  CT det, rdet, s, kappa;
};

// Simplex i of a fan: corners (h_0, h_1, r_i, r_{i+1}) in 3-D, (h_0, r_i, r_{i+1}) in 2-D,
// from the edges Ei = r_i - h_0, En = r_{i+1} - h_0 and (3-D) H = h_1 - h_0 with
// Qj = H x Ej, each formed once per ring node: the adjugate rows are
//   3-D: c_1 = Ei x En, c_2 = En x H = -Qn, c_3 = H x Ei = Qi, det = H . c_1
//   2-D: c_1 = (En_y, -En_x), c_2 = (-Ei_y, Ei_x), det = Ei_x En_y - Ei_y En_x
template <int DIM, typename CT>
__device__ __forceinline__ void fan_geometry(const CT (&H)[3], const CT (&Ei)[3], const CT (&En)[3], const CT (&Qi)[3],
                                             const CT (&Qn)[3], ElemGeo<DIM, CT>& G) {
  if constexpr (DIM == 3) {
    G.c[0][0] = Ei[1] * En[2] - Ei[2] * En[1];
    G.c[0][1] = Ei[2] * En[0] - Ei[0] * En[2];
    G.c[0][2] = Ei[0] * En[1] - Ei[1] * En[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      G.c[1][j] = -Qn[j];
      G.c[2][j] = Qi[j];
    }
    G.det = H[0] * G.c[0][0] + H[1] * G.c[0][1] + H[2] * G.c[0][2];
  } else {
    G.c[0][0] = En[1];
    G.c[0][1] = -En[0];
    G.c[1][0] = -Ei[1];
    G.c[1][1] = Ei[0];
    G.det = Ei[0] * En[1] - Ei[1] * En[0];
  }
  G.rdet = drcp<CT>(G.det);
  const CT inv_fact = CT(1.0 / Factorial<DIM>::value);
  G.kappa = G.rdet > CT(0) ? inv_fact : -inv_fact;
  G.s = fabs(G.rdet) * inv_fact;
}

// G' from corner differences dw[a] = w_{a+1} - w_0 (a < DIM)
template <int DIM, typename CT>
__device__ __forceinline__ void grad_prime_d(const ElemGeo<DIM, CT>& G, const CT (&dw)[DIM][3], CT (&Gp)[DIM][DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      CT t = dw[0][i] * G.c[0][j];
#pragma unroll
      for (int a = 1; a < DIM; ++a) t = fma(dw[a][i], G.c[a][j], t);
      Gp[i][j] = t;
    }
}

// out_{a+1} = T c_a, out_0 = -sum (T already carries the element's scale)
template <int DIM, typename CT>
__device__ __forceinline__ void contract_c(const ElemGeo<DIM, CT>& G, const CT (&T)[DIM][DIM], CT (&out)[DIM + 1][DIM]) {
#pragma unroll
  for (int a = 0; a < DIM; ++a)
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      CT t = T[i][0] * G.c[a][0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) t = fma(T[i][j], G.c[a][j], t);
      out[a + 1][i] = t;
    }
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    CT t = out[1][i];
#pragma unroll
    for (int a = 2; a <= DIM; ++a) t += out[a][i];
    out[0][i] = -t;
  }
}

// V sigma(G'/det) dN_a for the linear law: sigma(G') scaled by s, contracted with c_a
template <int DIM, typename CT>
__device__ __forceinline__ void linear_force(const ElemGeo<DIM, CT>& G, const CT (&Gp)[DIM][DIM], CT mu, CT lam,
                                             CT (&out)[DIM + 1][DIM]) {
  const CT mus = mu * G.s, lams = lam * G.s;
  CT tr = Gp[0][0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) tr += Gp[i][i];
  const CT lt = lams * tr;
  CT S[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    S[i][i] = fma(CT(2) * mus, Gp[i][i], lt);
#pragma unroll
    for (int j = i + 1; j < DIM; ++j) {
      S[i][j] = mus * (Gp[i][j] + Gp[j][i]);
      S[j][i] = S[i][j];
    }
  }
  contract_c<DIM, CT>(G, S, out);
}

// V Psi for the linear law: s (mu eps':eps' + lam/2 tr'^2), eps' = sym G'
template <int DIM, typename CT>
__device__ __forceinline__ CT linear_energy(const ElemGeo<DIM, CT>& G, const CT (&Gp)[DIM][DIM], CT mu, CT lam) {
  CT tr = Gp[0][0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) tr += Gp[i][i];
  CT ee = CT(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const CT e = CT(0.5) * (Gp[i][j] + Gp[j][i]);
      ee = fma(e, e, ee);
    }
  return G.s * (mu * ee + CT(0.5) * lam * tr * tr);
}

// Neo-Hookean kinematics from G = grad u, arranged so that FP32 keeps its relative accuracy
// near the reference state (no quantity is formed as 1 + small and then differenced):
//   t = tr G, m2 = sum of principal 2x2 minors of G (3-D), det G,
//   J - 1 = t + m2 + det G (3-D) | t + det G (2-D)         (expansion of det(I + G))
//   cof(I + G) = (1 + t) I - G^T + cof(G) (3-D) | (1 + t) I - G^T (2-D)
//   Hm = H - I = [ -(J - 1 - t) I - G^T + cof(G) ] / J     with H = F^-T = cof(F) / J
//   ln J = log1p(J - 1),  I1 - d = 2 t + G:G
template <int DIM, typename CT>
struct NHState {
  CT G[DIM][DIM];
  CT Hm[DIM][DIM];  // H - I
  CT J, lnJ, t, GG;
};

template <typename T>
__device__ __forceinline__ T dlog1p(T x);
template <>
__device__ __forceinline__ float dlog1p<float>(float x) { return log1pf(x); }
template <>
__device__ __forceinline__ double dlog1p<double>(double x) { return log1p(x); }

template <int DIM, typename CT>
__device__ __forceinline__ void nh_state(const CT (&Gu)[DIM][DIM], NHState<DIM, CT>& s) {
  const auto& G = Gu;
  CT t = G[0][0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) t += G[i][i];
  CT GG = CT(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      s.G[i][j] = G[i][j];
      GG = fma(G[i][j], G[i][j], GG);
    }
  CT second;  // J - 1 - t
  CT cg[DIM][DIM];
  if constexpr (DIM == 3) {
    cg[0][0] = G[1][1] * G[2][2] - G[1][2] * G[2][1];
    cg[0][1] = G[1][2] * G[2][0] - G[1][0] * G[2][2];
    cg[0][2] = G[1][0] * G[2][1] - G[1][1] * G[2][0];
    cg[1][0] = G[0][2] * G[2][1] - G[0][1] * G[2][2];
    cg[1][1] = G[0][0] * G[2][2] - G[0][2] * G[2][0];
    cg[1][2] = G[0][1] * G[2][0] - G[0][0] * G[2][1];
    cg[2][0] = G[0][1] * G[1][2] - G[0][2] * G[1][1];
    cg[2][1] = G[0][2] * G[1][0] - G[0][0] * G[1][2];
    cg[2][2] = G[0][0] * G[1][1] - G[0][1] * G[1][0];
    const CT m2 = cg[0][0] + cg[1][1] + cg[2][2];
    const CT detG = G[0][0] * cg[0][0] + G[0][1] * cg[0][1] + G[0][2] * cg[0][2];
    second = m2 + detG;
  } else {
    second = G[0][0] * G[1][1] - G[0][1] * G[1][0];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) cg[i][j] = CT(0);
  }
  const CT jm1 = t + second;
  s.J = CT(1) + jm1;
  const CT rJ = CT(1) / s.J;
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) s.Hm[i][j] = (cg[i][j] - G[j][i] - (i == j ? second : CT(0))) * rJ;
  s.lnJ = dlog1p<CT>(jm1);
  s.t = t;
  s.GG = GG;
}

// P = mu (F - H) + lam lnJ H = mu (G - Hm) + lam lnJ (I + Hm)
template <int DIM, typename CT>
__device__ __forceinline__ void nh_pk1(const NHState<DIM, CT>& s, CT mu, CT lam, CT (&P)[DIM][DIM]) {
  const CT c = lam * s.lnJ;
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j)
      P[i][j] = fma(mu, s.G[i][j] - s.Hm[i][j], c * (s.Hm[i][j] + (i == j ? CT(1) : CT(0))));
}

// Psi = 1/2 lam ln^2 J - mu ln J + 1/2 mu (I1 - d) = 1/2 lam ln^2 J + mu (t - ln J) + 1/2 mu G:G
template <int DIM, typename CT>
__device__ __forceinline__ CT nh_psi(const NHState<DIM, CT>& s, CT mu, CT lam) {
  return CT(0.5) * lam * s.lnJ * s.lnJ + mu * (s.t - s.lnJ) + CT(0.5) * mu * s.GG;
}

// dP = mu dF + (mu - lam lnJ) H dF^T H + lam (H:dF) H,  H = I + Hm
template <int DIM, typename CT>
__device__ __forceinline__ void nh_dpk1(const NHState<DIM, CT>& s, CT mu, CT lam, const CT (&dF)[DIM][DIM],
                                        CT (&dP)[DIM][DIM]) {
  CT H[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) H[i][j] = s.Hm[i][j] + (i == j ? CT(1) : CT(0));
  CT M[DIM][DIM];  // M = dF^T H
  CT hd = CT(0);
#pragma unroll
  for (int k = 0; k < DIM; ++k)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      CT t = dF[0][k] * H[0][j];
#pragma unroll
      for (int l = 1; l < DIM; ++l) t = fma(dF[l][k], H[l][j], t);
      M[k][j] = t;
      hd = fma(H[k][j], dF[k][j], hd);
    }
  const CT c1 = mu - lam * s.lnJ;
  const CT c2 = lam * hd;
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      CT t = H[i][0] * M[0][j];
#pragma unroll
      for (int k = 1; k < DIM; ++k) t = fma(H[i][k], M[k][j], t);
      dP[i][j] = fma(mu, dF[i][j], fma(c1, t, c2 * H[i][j]));
    }
}

// Jacobi diagonal V [mu |g_a|^2 + (mu + lam - lam lnJ) (H g_a)_i^2] = s [mu |c_a|^2 + ... (H c_a)_i^2]
template <int DIM, typename CT>
__device__ __forceinline__ void nh_diag(const ElemGeo<DIM, CT>& Ge, const NHState<DIM, CT>* st, CT mu, CT lam,
                                        CT (&out)[DIM + 1][DIM]) {
  const CT lnJ = st ? st->lnJ : CT(0);
  const CT c = mu + lam - lam * lnJ;
#pragma unroll
  for (int a = 0; a <= DIM; ++a) {
    CT g[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      if (a > 0) {
        g[j] = Ge.c[a - 1][j];
      } else {
        CT t = Ge.c[0][j];
#pragma unroll
        for (int b = 1; b < DIM; ++b) t += Ge.c[b][j];
        g[j] = -t;
      }
    }
    CT gg = CT(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) gg = fma(g[j], g[j], gg);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      CT hg = g[i];
      if (st) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) hg = fma(st->Hm[i][j], g[j], hg);
      }
      out[a][i] = Ge.s * fma(c, hg * hg, mu * gg);
    }
  }
}

}  // namespace pfem
