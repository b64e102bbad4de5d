// Per-element arithmetic of the P1 operator (device functions).
//
//   geometry (App. A, explicit shape-function differentiation): D = [X_1-X_0 .. X_d-X_0],
//     dN_a/dX = row a-1 of D^-1 (a >= 1), dN_0/dX = -sum, V = |det D| / d!
//   linear (Sec. 3.1): eps = sym grad w, sigma = 2 mu eps + lam tr(eps) I, Psi = 1/2 sigma:eps;
//     force / tangent action  y_a = V sigma(w) dN_a  (f_int = K u for linear FEM, App. B)
//   Neo-Hookean (Sec. 3.2 energy; App. B total Lagrangian): F = I + grad u, J = det F,
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
__device__ __forceinline__ T dlog(T x);
template <>
__device__ __forceinline__ float dlog<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double dlog<double>(double x) { return log(x); }

template <int DIM, typename CT>
struct ElemGeo {
  CT g[DIM + 1][DIM];
  CT vol;
};

// DIM = 3: X[a][i], a = 0..3.
template <typename CT>
__device__ __forceinline__ void geometry3(const CT (&X)[4][3], ElemGeo<3, CT>& G) {
  CT d[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) d[i][a] = X[a + 1][i] - X[0][i];
  const CT c00 = d[1][1] * d[2][2] - d[1][2] * d[2][1];
  const CT c01 = d[1][2] * d[2][0] - d[1][0] * d[2][2];
  const CT c02 = d[1][0] * d[2][1] - d[1][1] * d[2][0];
  const CT det = d[0][0] * c00 + d[0][1] * c01 + d[0][2] * c02;
  const CT r = CT(1) / det;
  // inv[a][i] = cofactor(i, a) / det
  G.g[1][0] = c00 * r;
  G.g[1][1] = (d[0][2] * d[2][1] - d[0][1] * d[2][2]) * r;
  G.g[1][2] = (d[0][1] * d[1][2] - d[0][2] * d[1][1]) * r;
  G.g[2][0] = c01 * r;
  G.g[2][1] = (d[0][0] * d[2][2] - d[0][2] * d[2][0]) * r;
  G.g[2][2] = (d[0][2] * d[1][0] - d[0][0] * d[1][2]) * r;
  G.g[3][0] = c02 * r;
  G.g[3][1] = (d[0][1] * d[2][0] - d[0][0] * d[2][1]) * r;
  G.g[3][2] = (d[0][0] * d[1][1] - d[0][1] * d[1][0]) * r;
#pragma unroll
  for (int i = 0; i < 3; ++i) G.g[0][i] = -(G.g[1][i] + G.g[2][i] + G.g[3][i]);
  G.vol = fabs(det) * CT(1.0 / 6.0);
}

template <typename CT>
__device__ __forceinline__ void geometry2(const CT (&X)[3][3], ElemGeo<2, CT>& G) {
  const CT d00 = X[1][0] - X[0][0], d01 = X[2][0] - X[0][0];
  const CT d10 = X[1][1] - X[0][1], d11 = X[2][1] - X[0][1];
  const CT det = d00 * d11 - d01 * d10;
  const CT r = CT(1) / det;
  G.g[1][0] = d11 * r;
  G.g[1][1] = -d01 * r;
  G.g[2][0] = -d10 * r;
  G.g[2][1] = d00 * r;
  G.g[0][0] = -(G.g[1][0] + G.g[2][0]);
  G.g[0][1] = -(G.g[1][1] + G.g[2][1]);
  G.vol = fabs(det) * CT(0.5);
}

// grad w: Gw[i][j] = sum_a w_a,i g_a,j
template <int DIM, typename CT>
__device__ __forceinline__ void grad_of(const ElemGeo<DIM, CT>& G, const CT (&w)[DIM + 1][3], CT (&Gw)[DIM][DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      // sum_a w_a g_a = sum_{a>=1} (w_a - w_0) g_a since sum_a g_a = 0
      CT s = (w[1][i] - w[0][i]) * G.g[1][j];
#pragma unroll
      for (int a = 2; a <= DIM; ++a) s = fma(w[a][i] - w[0][i], G.g[a][j], s);
      Gw[i][j] = s;
    }
}

// out_a = V * T g_a (T: DIM x DIM stress-like tensor)
template <int DIM, typename CT>
__device__ __forceinline__ void contract(const ElemGeo<DIM, CT>& G, const CT (&T)[DIM][DIM], CT (&out)[DIM + 1][DIM]) {
  CT Tv[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) Tv[i][j] = T[i][j] * G.vol;
#pragma unroll
  for (int a = 1; a <= DIM; ++a)
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      CT s = Tv[i][0] * G.g[a][0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) s = fma(Tv[i][j], G.g[a][j], s);
      out[a][i] = s;
    }
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    CT s = out[1][i];
#pragma unroll
    for (int a = 2; a <= DIM; ++a) s += out[a][i];
    out[0][i] = -s;
  }
}

// linear stress sigma = 2 mu sym(Gw) + lam tr(Gw) I
template <int DIM, typename CT>
__device__ __forceinline__ void linear_stress(const CT (&Gw)[DIM][DIM], CT mu, CT lam, CT (&S)[DIM][DIM]) {
  CT tr = Gw[0][0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) tr += Gw[i][i];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) S[i][j] = mu * (Gw[i][j] + Gw[j][i]);
#pragma unroll
  for (int i = 0; i < DIM; ++i) S[i][i] = fma(lam, tr, S[i][i]);
}

template <int DIM, typename CT>
__device__ __forceinline__ CT linear_psi(const CT (&Gw)[DIM][DIM], CT mu, CT lam) {
  // Psi = mu eps:eps + lam/2 (tr eps)^2
  CT tr = Gw[0][0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) tr += Gw[i][i];
  CT ee = CT(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const CT e = CT(0.5) * (Gw[i][j] + Gw[j][i]);
      ee = fma(e, e, ee);
    }
  return mu * ee + CT(0.5) * lam * tr * tr;
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

// Jacobi diagonal entries V [mu |g_a|^2 + (mu + lam - lam lnJ) (H g_a)_i^2]
template <int DIM, typename CT>
__device__ __forceinline__ void nh_diag(const ElemGeo<DIM, CT>& Ge, const NHState<DIM, CT>* s, CT mu, CT lam,
                                        CT (&out)[DIM + 1][DIM]) {
  const CT lnJ = s ? s->lnJ : CT(0);
  const CT c = mu + lam - lam * lnJ;
#pragma unroll
  for (int a = 0; a <= DIM; ++a) {
    CT gg = CT(0);
#pragma unroll
    for (int j = 0; j < DIM; ++j) gg = fma(Ge.g[a][j], Ge.g[a][j], gg);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      CT hg = Ge.g[a][i];
      if (s) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) hg = fma(s->Hm[i][j], Ge.g[a][j], hg);
      }
      out[a][i] = Ge.vol * fma(c, hg * hg, mu * gg);
    }
  }
}

}  // namespace pfem
