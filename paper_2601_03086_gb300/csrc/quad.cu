// Bilinear (Q4) and serendipity (Q8) quadrilaterals in plane strain with Gauss quadrature
// (the element families of the beam and Cook-membrane results, Sec. "Nonlinear
// hyperelasticity"; App. B isoparametric interpolation, internal force and tangent).
//
// Element-major path: one thread per element loops over its Gauss points (2 x 2 for Q4,
// 3 x 3 for Q8), forms J = dX/dxi, grad N = J^-T dN/dxi and dV = w det J, evaluates the
// requested output with the same constitutive device functions as the simplex tiles
// (element.cuh: linear stress, Neo-Hookean P, dP, Psi) and writes one record per (element,
// local node). A node pass then sums each node's records in ascending (element, local) order
// through a CSR built at mesh creation: deterministic, no atomics. Energies and the PCG
// p_e . A_e p_e are summed per block of kQuadBlock elements in a fixed order.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "element.cuh"
#include "kernels_vec.cuh"
#include "pcg_state.cuh"
#include "tile.cuh"

namespace pfem {

// derivatives dN_a/dxi, dN_a/deta at (xi, eta); node order: corners (-1,-1), (1,-1), (1,1),
// (-1,1), then (Q8) mid-edge nodes (0,-1), (1,0), (0,1), (-1,0)
template <int NPE, typename CT>
__device__ __forceinline__ void qshape_d(CT xi, CT eta, CT (&dN)[NPE][2]) {
  const CT xa[4] = {CT(-1), CT(1), CT(1), CT(-1)}, ya[4] = {CT(-1), CT(-1), CT(1), CT(1)};
  if constexpr (NPE == 4) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      dN[a][0] = CT(0.25) * xa[a] * (CT(1) + eta * ya[a]);
      dN[a][1] = CT(0.25) * ya[a] * (CT(1) + xi * xa[a]);
    }
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      dN[a][0] = CT(0.25) * xa[a] * (CT(1) + eta * ya[a]) * (CT(2) * xi * xa[a] + eta * ya[a]);
      dN[a][1] = CT(0.25) * ya[a] * (CT(1) + xi * xa[a]) * (xi * xa[a] + CT(2) * eta * ya[a]);
    }
    dN[4][0] = -xi * (CT(1) - eta);
    dN[4][1] = CT(-0.5) * (CT(1) - xi * xi);
    dN[5][0] = CT(0.5) * (CT(1) - eta * eta);
    dN[5][1] = -eta * (CT(1) + xi);
    dN[6][0] = -xi * (CT(1) + eta);
    dN[6][1] = CT(0.5) * (CT(1) - xi * xi);
    dN[7][0] = CT(-0.5) * (CT(1) - eta * eta);
    dN[7][1] = -eta * (CT(1) - xi);
  }
}

template <typename CT>
__device__ __forceinline__ const CT* qmat_ptr(const DevPlan& P);
template <>
__device__ __forceinline__ const float* qmat_ptr<float>(const DevPlan& P) {
  return reinterpret_cast<const float*>(P.qmatf);
}
template <>
__device__ __forceinline__ const double* qmat_ptr<double>(const DevPlan& P) {
  return reinterpret_cast<const double*>(P.qmatd);
}
// Sum over the block's threads (warps in index order), valid in thread 0.
__device__ __forceinline__ double qblock_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// One element per thread. OUT: OUT_RES / OUT_TAN / OUT_DIAG, or -1 for the energy only.
template <int NPE, int KIND, int OUT, bool ENERGY, bool PCG, typename VT, typename CT>
__global__ void __launch_bounds__(kQuadBlock) quad_elem_kernel(DevPlan P, OpArgs A, int region) {
  __shared__ double red[kQuadBlock / 32];
  constexpr bool NEED_U = ENERGY || OUT == OUT_RES || (KIND == K_NH && (OUT == OUT_TAN || OUT == OUT_DIAG));
  constexpr bool NEED_V = OUT == OUT_TAN;
  const VT* vsrc = static_cast<const VT*>(A.v);
  if constexpr (PCG) {  // the direction formed by quad_dir_kernel for this iteration
    const PcgState* st = A.pcg.st;
    const int done = st->done, repl = st->repl, it = st->iter;
    if (done != 0 || repl != 0) return;  // uniform: written by earlier kernels
    vsrc = reinterpret_cast<const VT*>((it & 1) ? A.pcg.p[0] : A.pcg.p[1]);
  }
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = e < P.n_elems;
  CT x[NPE][2], u[NPE][2], v[NPE][2], acc[NPE][2];
  CT mu = CT(0), lam = CT(0);
  int inv = 0;
  double e_acc = 0.0;
  if (live) {
    // element-relative coordinates formed in FP64 (sum_a dN_a = 0 leaves J unchanged), so
    // that FP32 geometry keeps its relative accuracy far from the origin
    const double* X = reinterpret_cast<const double*>(P.qxd);
    const CT* M = qmat_ptr<CT>(P);
    const int64_t n0 = P.qconn[e * NPE];
    const double x00 = X[2 * n0], x01 = X[2 * n0 + 1];
    // fields likewise relative to node 0 (the element arithmetic only uses their gradients)
    const VT* usrc = static_cast<const VT*>(A.u);
    auto fld = [&](const VT* f, int64_t n, int i, bool masked) {
      return (masked && P.dmask[2 * n + i]) ? 0.0 : (double)f[2 * n + i];
    };
    double ua[2] = {0.0, 0.0}, va[2] = {0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (NEED_U) ua[i] = fld(usrc, n0, i, false);
      if (NEED_V) va[i] = fld(vsrc, n0, i, true);
    }
    mu = M[2 * e];
    lam = M[2 * e + 1];
#pragma unroll
    for (int a = 0; a < NPE; ++a) {
      const int64_t n = P.qconn[e * NPE + a];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        x[a][i] = CT(X[2 * n + i] - (i == 0 ? x00 : x01));
        u[a][i] = NEED_U ? CT(fld(usrc, n, i, false) - ua[i]) : CT(0);
        v[a][i] = NEED_V ? CT(fld(vsrc, n, i, true) - va[i]) : CT(0);
        acc[a][i] = CT(0);
      }
    }
    constexpr int NG = NPE == 4 ? 2 : 3;
    const CT gp4 = CT(0.57735026918962576451), gp8 = CT(0.77459666924148337704);
#pragma unroll
    for (int gb = 0; gb < NG; ++gb)
#pragma unroll
      for (int ga = 0; ga < NG; ++ga) {
        CT xi, eta, w;
        if constexpr (NPE == 4) {
          xi = ga == 0 ? -gp4 : gp4;
          eta = gb == 0 ? -gp4 : gp4;
          w = CT(1);
        } else {
          xi = ga == 0 ? -gp8 : (ga == 1 ? CT(0) : gp8);
          eta = gb == 0 ? -gp8 : (gb == 1 ? CT(0) : gp8);
          w = (ga == 1 ? CT(8.0 / 9.0) : CT(5.0 / 9.0)) * (gb == 1 ? CT(8.0 / 9.0) : CT(5.0 / 9.0));
        }
        CT dN[NPE][2];
        qshape_d<NPE, CT>(xi, eta, dN);
        CT J[2][2] = {{CT(0), CT(0)}, {CT(0), CT(0)}};
#pragma unroll
        for (int a = 0; a < NPE; ++a)
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) J[i][j] = fma(x[a][i], dN[a][j], J[i][j]);
        const CT det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const CT rd = CT(1) / det;
        const CT Ji[2][2] = {{J[1][1] * rd, -J[0][1] * rd}, {-J[1][0] * rd, J[0][0] * rd}};
        CT g[NPE][2];
#pragma unroll
        for (int a = 0; a < NPE; ++a)
#pragma unroll
          for (int i = 0; i < 2; ++i) g[a][i] = dN[a][0] * Ji[0][i] + dN[a][1] * Ji[1][i];
        const CT dv = w * det;
        auto grad = [&](const CT (&f)[NPE][2], CT (&G)[2][2]) {
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              CT t = CT(0);
#pragma unroll
              for (int a = 0; a < NPE; ++a) t = fma(f[a][i], g[a][j], t);
              G[i][j] = t;
            }
        };
        auto lin_stress = [&](const CT (&G)[2][2], CT (&S)[2][2]) {
          const CT tr = G[0][0] + G[1][1];
          S[0][0] = CT(2) * mu * G[0][0] + lam * tr;
          S[1][1] = CT(2) * mu * G[1][1] + lam * tr;
          S[0][1] = S[1][0] = mu * (G[0][1] + G[1][0]);
        };
        auto scatter = [&](const CT (&T)[2][2]) {  // acc_a += dV T grad N_a
#pragma unroll
          for (int a = 0; a < NPE; ++a)
#pragma unroll
            for (int i = 0; i < 2; ++i) acc[a][i] = fma(dv, T[i][0] * g[a][0] + T[i][1] * g[a][1], acc[a][i]);
        };
        if constexpr (KIND == K_LIN) {
          if constexpr (NEED_U) {
            CT Gu[2][2], S[2][2];
            grad(u, Gu);
            lin_stress(Gu, S);
            if constexpr (ENERGY) {
              const CT e01 = CT(0.5) * (Gu[0][1] + Gu[1][0]), tr = Gu[0][0] + Gu[1][1];
              const CT ee = Gu[0][0] * Gu[0][0] + Gu[1][1] * Gu[1][1] + CT(2) * e01 * e01;
              e_acc += (double)(dv * (mu * ee + CT(0.5) * lam * tr * tr));
            }
            if constexpr (OUT == OUT_RES) scatter(S);
          }
          if constexpr (OUT == OUT_TAN) {
            CT Gv[2][2], S[2][2];
            grad(v, Gv);
            lin_stress(Gv, S);
            scatter(S);
          } else if constexpr (OUT == OUT_DIAG) {
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
              const CT gg = g[a][0] * g[a][0] + g[a][1] * g[a][1];
#pragma unroll
              for (int i = 0; i < 2; ++i) acc[a][i] += dv * (mu * gg + (mu + lam) * g[a][i] * g[a][i]);
            }
          }
        } else {
          CT Gu[2][2];
          grad(u, Gu);
          NHState<2, CT> st;
          nh_state<2, CT>(Gu, st);
          if (!(st.J > CT(0))) ++inv;
          if constexpr (ENERGY) e_acc += (double)(dv * (st.J > CT(0) ? nh_psi<2, CT>(st, mu, lam) : CT(INFINITY)));
          if constexpr (OUT == OUT_RES) {
            CT T[2][2];
            nh_pk1<2, CT>(st, mu, lam, T);
            scatter(T);
          } else if constexpr (OUT == OUT_TAN) {
            CT Gv[2][2], T[2][2];
            grad(v, Gv);
            nh_dpk1<2, CT>(st, mu, lam, Gv, T);
            scatter(T);
          } else if constexpr (OUT == OUT_DIAG) {
            const CT c = mu + lam - lam * st.lnJ;
#pragma unroll
            for (int a = 0; a < NPE; ++a) {
              const CT gg = g[a][0] * g[a][0] + g[a][1] * g[a][1];
#pragma unroll
              for (int i = 0; i < 2; ++i) {
                const CT hg = g[a][i] + st.Hm[i][0] * g[a][0] + st.Hm[i][1] * g[a][1];
                acc[a][i] += dv * (mu * gg + c * hg * hg);
              }
            }
          }
        }
      }
    if constexpr (OUT >= 0) {
      CT* buf = static_cast<CT*>(P.qbuf) + ((size_t)region * P.n_elems + (size_t)e) * NPE * 2;
#pragma unroll
      for (int a = 0; a < NPE; ++a) {
        buf[2 * a] = acc[a][0];
        buf[2 * a + 1] = acc[a][1];
      }
    }
    if constexpr (PCG) {  // p_e . (A_e p_e) with the anchor added back
      CT d = CT(0);
#pragma unroll
      for (int a = 0; a < NPE; ++a)
        d = fma(v[a][0] + CT(va[0]), acc[a][0], fma(v[a][1] + CT(va[1]), acc[a][1], d));
      e_acc = (double)d;
    }
  }
  if constexpr (KIND == K_NH) {
    const int tot = __reduce_add_sync(0xffffffffu, inv);
    if ((threadIdx.x & 31) == 0 && tot > 0 && P.inverted) atomicAdd(P.inverted, tot);
  }
  if constexpr (ENERGY || PCG) {
    const double s = qblock_sum(e_acc, red);
    if (threadIdx.x == 0) {
      if constexpr (PCG) A.pcg.tile_part[blockIdx.x] = s;
      else P.tile_energy[blockIdx.x] = s;
    }
  }
}

// Node pass: each node sums its (element, local) records in CSR order, then the output rule
// of the simplex path (final_write: Dirichlet rows, f_ext, upstream scale, PCG directions).
template <int OUT, bool PCG, typename VT, typename CT>
__global__ void __launch_bounds__(256) quad_gather_kernel(DevPlan P, OpArgs A, int region) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= P.n_nodes) return;
  if constexpr (PCG) {
    const PcgState* st = A.pcg.st;
    if (st->done != 0 || st->repl != 0) return;
  }
  const CT* buf = static_cast<const CT*>(P.qbuf) + (size_t)region * P.n_elems * P.elem_npe * 2;
  CT acc[4] = {CT(0), CT(0), CT(0), CT(0)};
  for (int q = P.qptr[n]; q < P.qptr[n + 1]; ++q) {
    const int64_t r = P.qidx[q];
    acc[0] += buf[2 * r];
    acc[1] += buf[2 * r + 1];
  }
  const unsigned mask = (P.dmask[2 * n] ? 1u : 0u) | (P.dmask[2 * n + 1] ? 2u : 0u);
  const CT sc = A.out_scale ? CT(*static_cast<const VT*>(A.out_scale)) : CT(1);
  final_write<2, OUT, VT, CT, PCG>(P, A, n, mask, acc, sc);
}

// PCG direction of this iteration for every DOF: p = dinv r + beta p_old (0 on prescribed)
__global__ void quad_dir_kernel(DevPlan P, OpArgs A) {
  const PcgState* st = A.pcg.st;
  const int done = st->done, repl = st->repl, it = st->iter;
  const double beta = st->beta;
  if (done != 0 || repl != 0) return;
  const double* p_old = (it & 1) ? A.pcg.p[1] : A.pcg.p[0];
  double* p_new = (it & 1) ? A.pcg.p[0] : A.pcg.p[1];
  const int64_t nd = P.n_nodes * 2;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nd; k += (int64_t)gridDim.x * blockDim.x)
    p_new[k] = pcg_direction(A.pcg, p_old, beta, k, P.dmask[k] != 0);
}

}  // namespace pfem

namespace pfem {

template <int NPE, int KIND, int OUT, bool ENERGY, bool PCG, typename VT, typename CT>
static pfem_status quad_pass(const DevPlan& P, const OpArgs& A, int region, cudaStream_t s) {
  if (P.n_elems > 0) {
    quad_elem_kernel<NPE, KIND, OUT, ENERGY, PCG, VT, CT><<<P.n_tiles, kQuadBlock, 0, s>>>(P, A, region);
    PFEM_COUNT_LAUNCH();
    PFEM_CUDA(cudaGetLastError());
  }
  if constexpr (OUT >= 0) {
    quad_gather_kernel<OUT, PCG, VT, CT><<<(int)((P.n_nodes + 255) / 256), 256, 0, s>>>(P, A, region);
    PFEM_COUNT_LAUNCH();
    PFEM_CUDA(cudaGetLastError());
  }
  return PFEM_OK;
}

template <int NPE, int KIND, typename VT, typename CT>
static pfem_status quad_ops(const DevPlan& P, int ops, const OpArgs& a, cudaStream_t s) {
  switch (ops) {
    case OP_TANGENT: return quad_pass<NPE, KIND, OUT_TAN, false, false, VT, CT>(P, a, 0, s);
    case OP_RESIDUAL: return quad_pass<NPE, KIND, OUT_RES, false, false, VT, CT>(P, a, 0, s);
    case OP_ENERGY: return quad_pass<NPE, KIND, -1, true, false, VT, CT>(P, a, 0, s);
    case OP_DIAG: return quad_pass<NPE, KIND, OUT_DIAG, false, false, VT, CT>(P, a, 0, s);
    case OP_TANGENT | OP_PCG:
      if constexpr (sizeof(VT) == 8) {
        if (!a.pcg.alpha_by_update) break;  // the quadrilateral path leaves alpha to the update kernel
        quad_dir_kernel<<<(int)std::min<int64_t>((P.n_nodes * 2 + 255) / 256, 1216), 256, 0, s>>>(P, a);
        PFEM_COUNT_LAUNCH();
        PFEM_CUDA(cudaGetLastError());
        return quad_pass<NPE, KIND, OUT_TAN, false, true, VT, CT>(P, a, 0, s);
      }
      break;
    default: break;
  }
  set_error("quadrilateral meshes: unsupported op combination %d", ops);
  return PFEM_ERR_UNSUPPORTED;
}

template <typename VT, typename CT>
static pfem_status quad_dispatch(const DevPlan& P, int ops, const OpArgs& a, cudaStream_t s) {
  if (P.elem_npe == 4)
    return P.kind == PFEM_LINEAR ? quad_ops<4, K_LIN, VT, CT>(P, ops, a, s) : quad_ops<4, K_NH, VT, CT>(P, ops, a, s);
  return P.kind == PFEM_LINEAR ? quad_ops<8, K_LIN, VT, CT>(P, ops, a, s) : quad_ops<8, K_NH, VT, CT>(P, ops, a, s);
}

pfem_status launch_quad_op(const DevPlan& P, int ops, pfem_dtype vt, pfem_dtype ct, const OpArgs& a, cudaStream_t s) {
  if (vt == PFEM_F32 && ct == PFEM_F32) return quad_dispatch<float, float>(P, ops, a, s);
  if (vt == PFEM_F64 && ct == PFEM_F32) return quad_dispatch<double, float>(P, ops, a, s);
  if (vt == PFEM_F64 && ct == PFEM_F64) return quad_dispatch<double, double>(P, ops, a, s);
  set_error("unsupported dtype combination");
  return PFEM_ERR_UNSUPPORTED;
}

}  // namespace pfem

using namespace pfem;

// Reference geometry check on the host: det J > 0 at every Gauss point (counterclockwise
// elements); returns the element id of the first failure or -1.
static int64_t quad_bad_element(const pfem_mesh_desc* d, int npe) {
  const double g4 = 1.0 / std::sqrt(3.0), g8 = std::sqrt(0.6);
  const double xa[8] = {-1, 1, 1, -1, 0, 1, 0, -1}, ya[8] = {-1, -1, 1, 1, -1, 0, 1, 0};
  const int ng = npe == 4 ? 2 : 3;
  for (int64_t e = 0; e < d->n_elems; ++e)
    for (int gb = 0; gb < ng; ++gb)
      for (int ga = 0; ga < ng; ++ga) {
        const double xi = npe == 4 ? (ga ? g4 : -g4) : (ga == 0 ? -g8 : (ga == 1 ? 0.0 : g8));
        const double eta = npe == 4 ? (gb ? g4 : -g4) : (gb == 0 ? -g8 : (gb == 1 ? 0.0 : g8));
        double J[2][2] = {{0, 0}, {0, 0}};
        for (int a = 0; a < npe; ++a) {
          double dx, dy;
          if (npe == 4 || a < 4) {
            const double c = npe == 4 ? 1.0 : 0.0;
            dx = 0.25 * xa[a] * (1 + eta * ya[a]) * (npe == 4 ? 1.0 : (2 * xi * xa[a] + eta * ya[a]));
            dy = 0.25 * ya[a] * (1 + xi * xa[a]) * (npe == 4 ? 1.0 : (xi * xa[a] + 2 * eta * ya[a]));
            (void)c;
          } else if (xa[a] == 0) {
            dx = -xi * (1 + eta * ya[a]);
            dy = 0.5 * ya[a] * (1 - xi * xi);
          } else {
            dx = 0.5 * xa[a] * (1 - eta * eta);
            dy = -eta * (1 + xi * xa[a]);
          }
          const int32_t n = d->conn[e * npe + a];
          for (int i = 0; i < 2; ++i) {
            J[i][0] += d->coords[2 * n + i] * dx;
            J[i][1] += d->coords[2 * n + i] * dy;
          }
        }
        if (!(J[0][0] * J[1][1] - J[0][1] * J[1][0] > 0.0)) return e;
      }
  return -1;
}

extern "C" pfem_status pfem_mesh_create_quad(const pfem_mesh_desc* d, int32_t npe, void* cuda_stream,
                                             pfem_mesh_t* out) {
  if (!out || !d) {
    set_error("desc/out is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (d->dim != 2 || (npe != 4 && npe != 8) || d->n_nodes < 1 || d->n_elems < 0 || !d->coords ||
      (d->n_elems > 0 && (!d->conn || !d->mat_a || !d->mat_b)) || (d->kind != PFEM_LINEAR && d->kind != PFEM_NEOHOOKEAN) ||
      (d->n_facets > 0 && (!d->facets || !d->traction)) || d->n_facets < 0) {
    set_error("pfem_mesh_create_quad: needs dim 2, 4 or 8 nodes per element and valid arrays");
    return PFEM_ERR_INVALID_ARG;
  }
  const int64_t nn = d->n_nodes, ne = d->n_elems, nd = nn * 2;
  for (int64_t i = 0; i < nd; ++i)
    if (!std::isfinite(d->coords[i])) {
      set_error("non-finite coordinate");
      return PFEM_ERR_INVALID_ARG;
    }
  for (int64_t i = 0; i < ne * npe; ++i)
    if (d->conn[i] < 0 || d->conn[i] >= nn) {
      set_error("element node id out of range at %lld", (long long)i);
      return PFEM_ERR_INVALID_ARG;
    }
  std::vector<double> mat((size_t)ne * 2);
  for (int64_t e = 0; e < ne; ++e) {
    double a = d->mat_a[e], b = d->mat_b[e];
    if (d->kind == PFEM_LINEAR) {
      if (!(a > 0.0) || !(b > -1.0 && b < 0.5)) {
        set_error("element %lld: E must be > 0 and nu in (-1, 0.5)", (long long)e);
        return PFEM_ERR_INVALID_ARG;
      }
      const double mu = a / (2.0 * (1.0 + b)), lam = a * b / ((1.0 + b) * (1.0 - 2.0 * b));
      a = mu;
      b = lam;
    } else if (!(a > 0.0) || !(b >= 0.0) || !std::isfinite(a) || !std::isfinite(b)) {
      set_error("element %lld: mu must be > 0 and lambda >= 0", (long long)e);
      return PFEM_ERR_INVALID_ARG;
    }
    mat[(size_t)(2 * e)] = a;
    mat[(size_t)(2 * e + 1)] = b;
  }
  const int64_t bad = quad_bad_element(d, npe);
  if (bad >= 0) {
    set_error("element %lld has det J <= 0 at a Gauss point (nodes must run counterclockwise)", (long long)bad);
    return PFEM_ERR_DEGENERATE_ELEMENT;
  }
  // consistent edge loads of constant traction: Q4 edges (a, b) |e|/2 at each end, Q8 edges
  // (a, b, mid) |e| (1/6, 1/6, 2/3)
  const int fn = npe == 4 ? 2 : 3;
  std::vector<double> fext((size_t)nd, 0.0);
  for (int64_t f = 0; f < d->n_facets; ++f) {
    const int32_t* q = d->facets + f * fn;
    for (int k = 0; k < fn; ++k)
      if (q[k] < 0 || q[k] >= nn) {
        set_error("facet %lld node id out of range", (long long)f);
        return PFEM_ERR_INVALID_ARG;
      }
    const double L = std::hypot(d->coords[2 * q[1]] - d->coords[2 * q[0]], d->coords[2 * q[1] + 1] - d->coords[2 * q[0] + 1]);
    const double w[3] = {fn == 2 ? 0.5 : 1.0 / 6.0, fn == 2 ? 0.5 : 1.0 / 6.0, 2.0 / 3.0};
    for (int k = 0; k < fn; ++k)
      for (int i = 0; i < 2; ++i) fext[(size_t)(2 * q[k] + i)] += w[k] * L * d->traction[2 * f + i];
  }
  if (d->f_ext_extra)
    for (int64_t i = 0; i < nd; ++i) fext[(size_t)i] += d->f_ext_extra[i];
  // node -> (element, local) records, ascending
  std::vector<int32_t> ptr((size_t)nn + 1, 0), idx((size_t)(ne * npe));
  for (int64_t r = 0; r < ne * npe; ++r) ++ptr[(size_t)d->conn[r] + 1];
  for (int64_t i = 0; i < nn; ++i) ptr[(size_t)i + 1] += ptr[(size_t)i];
  {
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t r = 0; r < ne * npe; ++r) idx[(size_t)fill[(size_t)d->conn[r]]++] = (int32_t)r;
  }
  std::vector<double> vals((size_t)nd, 0.0);
  std::vector<uint8_t> mask((size_t)nd, 0);
  int64_t n_free = nd;
  for (int64_t i = 0; i < nd; ++i)
    if (d->dirichlet_mask && d->dirichlet_mask[i]) {
      mask[(size_t)i] = 1;
      --n_free;
      if (d->dirichlet_values) vals[(size_t)i] = d->dirichlet_values[i];
    }
  std::vector<float> xf((size_t)nd), matf((size_t)ne * 2), fextf((size_t)nd);
  for (int64_t i = 0; i < nd; ++i) {
    xf[(size_t)i] = (float)d->coords[i];
    fextf[(size_t)i] = (float)fext[(size_t)i];
  }
  for (int64_t i = 0; i < ne * 2; ++i) matf[(size_t)i] = (float)mat[(size_t)i];
  const int64_t nb = std::max<int64_t>((ne + kQuadBlock - 1) / kQuadBlock, 1);
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = (off + b + 255) & ~size_t(255);
    return o;
  };
  const size_t o_conn = take((size_t)ne * npe * 4), o_xd = take((size_t)nd * 8), o_xf = take((size_t)nd * 4);
  const size_t o_md = take((size_t)ne * 16), o_mf = take((size_t)ne * 8), o_ptr = take(((size_t)nn + 1) * 4);
  const size_t o_idx = take((size_t)ne * npe * 4), o_buf = take((size_t)std::max<int64_t>(ne, 1) * npe * 2 * 8 * kMaxRegions);
  const size_t o_te = take((size_t)nb * 8), o_inv = take(16), o_fe = take((size_t)nd * 8), o_ff = take((size_t)nd * 4);
  const size_t o_dv = take((size_t)nd * 8), o_dm = take((size_t)nd), o_rp = take((size_t)kReduceBlocks * 4 * 8);
  const size_t o_rc = take(64), o_ro = take(64);
  pfem_mesh_s* m = new (std::nothrow) pfem_mesh_s();
  if (!m) {
    set_error("host allocation failed");
    return PFEM_ERR_OUT_OF_MEMORY;
  }
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&m->device);
  cudaError_t ce = cudaMalloc(&m->arena, off);
  if (ce == cudaSuccess) ce = cudaMallocHost(&m->host_out, 8 * sizeof(double) + 4 * sizeof(int32_t));
  if (ce != cudaSuccess) {
    if (m->arena) cudaFree(m->arena);
    delete m;
    return cuda_fail(ce, "quadrilateral mesh allocation");
  }
  m->host_int = reinterpret_cast<int32_t*>(m->host_out + 8);
  m->arena_bytes = off;
  char* base = static_cast<char*>(m->arena);
  auto up = [&](size_t o, const void* src, size_t b) {
    return b == 0 ? cudaSuccess : cudaMemcpyAsync(base + o, src, b, cudaMemcpyHostToDevice, m->stream);
  };
  if (ce == cudaSuccess) ce = up(o_conn, d->conn, (size_t)ne * npe * 4);
  if (ce == cudaSuccess) ce = up(o_xd, d->coords, (size_t)nd * 8);
  if (ce == cudaSuccess) ce = up(o_xf, xf.data(), (size_t)nd * 4);
  if (ce == cudaSuccess) ce = up(o_md, mat.data(), (size_t)ne * 16);
  if (ce == cudaSuccess) ce = up(o_mf, matf.data(), (size_t)ne * 8);
  if (ce == cudaSuccess) ce = up(o_ptr, ptr.data(), ((size_t)nn + 1) * 4);
  if (ce == cudaSuccess) ce = up(o_idx, idx.data(), (size_t)ne * npe * 4);
  if (ce == cudaSuccess) ce = up(o_fe, fext.data(), (size_t)nd * 8);
  if (ce == cudaSuccess) ce = up(o_ff, fextf.data(), (size_t)nd * 4);
  if (ce == cudaSuccess) ce = up(o_dv, vals.data(), (size_t)nd * 8);
  if (ce == cudaSuccess) ce = up(o_dm, mask.data(), (size_t)nd);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + o_inv, 0, 16, m->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + o_rc, 0, 64, m->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(m->stream);
  if (ce != cudaSuccess) {
    cudaFree(m->arena);
    cudaFreeHost(m->host_out);
    delete m;
    return cuda_fail(ce, "quadrilateral mesh upload");
  }
  DevPlan& P = m->plan;
  std::memset(&P, 0, sizeof(P));
  P.dim = 2;
  P.kind = d->kind;
  P.n_tiles = (int)nb;
  P.n_nodes = nn;
  P.elem_npe = npe;
  P.n_elems = ne;
  P.qconn = reinterpret_cast<const int32_t*>(base + o_conn);
  P.qxd = reinterpret_cast<const double2*>(base + o_xd);
  P.qxf = reinterpret_cast<const float2*>(base + o_xf);
  P.qmatd = reinterpret_cast<const double2*>(base + o_md);
  P.qmatf = reinterpret_cast<const float2*>(base + o_mf);
  P.qptr = reinterpret_cast<const int32_t*>(base + o_ptr);
  P.qidx = reinterpret_cast<const int32_t*>(base + o_idx);
  P.qbuf = base + o_buf;
  P.tile_energy = reinterpret_cast<double*>(base + o_te);
  P.inverted = reinterpret_cast<int32_t*>(base + o_inv);
  P.f_ext = reinterpret_cast<const double*>(base + o_fe);
  P.f_ext_f = reinterpret_cast<const float*>(base + o_ff);
  P.dvalues = reinterpret_cast<const double*>(base + o_dv);
  P.dmask = reinterpret_cast<const uint8_t*>(base + o_dm);
  m->red_partials = reinterpret_cast<double*>(base + o_rp);
  m->red_counter = reinterpret_cast<unsigned int*>(base + o_rc);
  m->red_out = reinterpret_cast<double*>(base + o_ro);
  m->n_dofs = nd;
  m->n_free = n_free;
  pfem_mesh_stats& S = m->stats;
  S.n_nodes = nn;
  S.n_elems = ne;
  S.n_dofs = nd;
  S.n_free_dofs = n_free;
  S.n_tiles = nb;
  S.device_bytes = (int64_t)off;
  S.max_tile_elems = kQuadBlock;
  *out = m;
  return PFEM_OK;
}
