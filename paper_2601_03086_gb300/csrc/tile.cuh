// Element-tile kernel: one CTA per tile, shared-memory staging of the tile's nodes and
// element records, one thread per fan (a chain of simplices around a shared hinge, see
// pfem_internal.h), per-(fan, node) slots, fixed-order node sums, and halo nodes completed
// either in-kernel by the last tile to publish a partial (integer ticket per halo node) or
// by a separate pass over tile-ordered partials (large single-mesh launches).
//
// Passes of one tile CTA (every requested output op runs its own fan and node pass;
// element quantities are recomputed, never stored):
//   stage : step records and fan heads, tile node coordinates (tile-relative, FP32 or FP64)
//           and u and/or v gathered by node id
//   fans  : thread f walks fan f's ring: per simplex geometry, kinematics, stress / stress
//           derivative and V * T dN_a; a ring node's two contributions are summed in
//           registers and written once to its slot; optional V * Psi per thread
//   node  : each tile node sums its slots in rank order; a complete node writes its output;
//           a halo node publishes a partial, and the node is finished by summing all its
//           partials in ascending tile order. The summation order never depends on timing,
//           so the result is bitwise reproducible.
//
// Output conventions (Dirichlet DOFs eliminated): tangent y = v on prescribed DOFs and v is
// read as 0 there; residual r = 0 on prescribed DOFs; diagonal d = 1 on prescribed DOFs.

#pragma once

#include <cuda/atomic>
#include <type_traits>

#include "checked.cuh"
#include "element.cuh"
#include "pcg_state.cuh"
#include "pfem_internal.h"

namespace pfem {

enum : int { K_LIN = 0, K_NH = 1 };
enum : int { OUT_RES = 0, OUT_TAN = 1, OUT_DIAG = 2 };

template <typename CT>
struct SmemLayout {
  size_t slot, x, u, v, off, info, red, fb, head, smat, scode, total;
};

// Shared memory: 4-wide (x, y, z, pad) records for slots and staged node data; the tile's
// fan heads, step materials and step codes (step_cap >= fans and steps of any tile).
template <typename CT>
__host__ __device__ inline SmemLayout<CT> smem_layout(int max_local, int slot_cap, int step_cap, bool need_u,
                                                      bool need_v) {
  SmemLayout<CT> L;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 31) & ~size_t(31); };
  L.head = o;
  o = al(o + (size_t)step_cap * sizeof(ushort4));
  L.smat = o;
  o = al(o + (size_t)step_cap * 2 * sizeof(CT));
  L.scode = o;
  o = al(o + (size_t)step_cap * sizeof(uint16_t));
  L.slot = o;
  o = al(o + (size_t)slot_cap * 4 * sizeof(CT));
  L.x = o;
  o = al(o + (size_t)max_local * 4 * sizeof(CT));
  L.u = o;
  if (need_u) o = al(o + (size_t)max_local * 4 * sizeof(CT));
  L.v = o;
  if (need_v) o = al(o + (size_t)max_local * 4 * sizeof(CT));
  L.off = o;
  o = al(o + (size_t)(max_local + 1) * sizeof(int));
  L.info = o;
  o = al(o + (size_t)max_local * sizeof(int));
  L.red = o;
  o = al(o + 32 * sizeof(double));
  L.fb = o;
  o = al(o + kMaxFan * sizeof(int));
  L.total = o;
  return L;
}

// 4-wide loads/stores of compute-type records
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}
__device__ __forceinline__ void ldcg4(const float* p, float (&o)[4]) {
  const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
  o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
}
__device__ __forceinline__ void ldcg4(const double* p, double (&o)[4]) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}

template <typename CT>
__device__ __forceinline__ const CT* fext_ptr(const DevPlan& P);
template <>
__device__ __forceinline__ const float* fext_ptr<float>(const DevPlan& P) { return P.f_ext_f; }
template <>
__device__ __forceinline__ const double* fext_ptr<double>(const DevPlan& P) { return P.f_ext; }

// PCG direction of one DOF: p = dinv r + beta p_old (0 on prescribed DOFs)
__device__ __forceinline__ double pcg_direction(const PcgArgs& g, const double* p_old, double beta, int64_t k,
                                                bool fixed) {
  // r and p_old through L2 only: the persistent kernel rewrites them between grid barriers
  return fixed ? 0.0 : fma(g.dinv[k], __ldcg(g.r + k), beta * __ldcg(p_old + k));
}

template <int DIM, int OUT, typename VT, typename CT, bool PCG = false>
__device__ __forceinline__ void final_write(const DevPlan& P, const OpArgs& A, int64_t gid, unsigned mask,
                                            const CT (&acc)[4], CT sc) {
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    const int64_t k = gid * DIM + i;
    const bool fixed = (mask >> i) & 1u;
    if (OUT == OUT_RES) {
      const CT f = fext_ptr<CT>(P)[k];
      static_cast<VT*>(A.r)[k] = fixed ? VT(0) : VT(sc * (acc[i] - CT(A.load_scale) * f));
    } else if (OUT == OUT_TAN && PCG) {
      static_cast<VT*>(A.y)[k] = fixed ? VT(0) : VT(acc[i]);  // directions vanish on prescribed DOFs
    } else if (OUT == OUT_TAN) {
      // hess: energy Hessian on free DOFs (zero on prescribed); else the identity block
      static_cast<VT*>(A.y)[k] = fixed ? (A.hess ? VT(0) : static_cast<const VT*>(A.v)[k]) : VT(sc * acc[i]);
    } else {
      static_cast<VT*>(A.d)[k] = fixed ? VT(1) : VT(acc[i]);
    }
  }
}

// One fan pass for output OUT (or energy only when OUT < 0): thread f walks the ring of fan
// f once (see pfem_internal.h), evaluates its simplices in ring order and writes one slot per
// (fan, node).
template <int DIM, int KIND, int OUT, bool ENERGY, bool COUNT, typename CT>
__device__ __forceinline__ void fan_pass(unsigned char* smem, const SmemLayout<CT>& L, int nf, double& e_acc,
                                         int& n_inv) {
  constexpr int NV = DIM + 1;
  constexpr int HS = DIM - 1;  // hinge nodes
  constexpr bool NEED_GU = ENERGY || OUT == OUT_RES || (KIND == K_NH && (OUT == OUT_TAN || OUT == OUT_DIAG));
  constexpr bool NEED_GV = OUT == OUT_TAN;
  const CT* sx = reinterpret_cast<const CT*>(smem + L.x);
  const CT* su = reinterpret_cast<const CT*>(smem + L.u);
  const CT* sv = reinterpret_cast<const CT*>(smem + L.v);
  const int* soff = reinterpret_cast<const int*>(smem + L.off);
  const int* scnt = reinterpret_cast<const int*>(smem + L.fb);  // fans with more than i simplices
  const ushort4* shead = reinterpret_cast<const ushort4*>(smem + L.head);
  using M2 = typename std::conditional<sizeof(CT) == 4, float2, double2>::type;
  const M2* smat = reinterpret_cast<const M2*>(smem + L.smat);
  const uint16_t* scode = reinterpret_cast<const uint16_t*>(smem + L.scode);
  CT* slot = reinterpret_cast<CT*>(smem + L.slot);
  auto put = [&](unsigned code, const CT (&acc)[DIM]) {
    const int sl = soff[code & 1023u] + (int)(code >> 10);
    st4(slot + 4 * sl, acc[0], acc[1], DIM == 3 ? acc[DIM - 1] : CT(0), CT(0));
  };
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    const ushort4 hd = shead[f];
    const int k = hd.w;
    CT x0[4], u0[4] = {}, v0[4] = {};
    ld4(sx + 4 * (hd.x & 1023), x0);
    if constexpr (NEED_GU) ld4(su + 4 * (hd.x & 1023), u0);
    if constexpr (NEED_GV) ld4(sv + 4 * (hd.x & 1023), v0);
    CT H[3] = {CT(0), CT(0), CT(0)}, duH[3] = {CT(0), CT(0), CT(0)}, dvH[3] = {CT(0), CT(0), CT(0)};
    if constexpr (DIM == 3) {
      CT t[4];
      ld4(sx + 4 * (hd.y & 1023), t);
#pragma unroll
      for (int i = 0; i < 3; ++i) H[i] = t[i] - x0[i];
      if constexpr (NEED_GU) {
        ld4(su + 4 * (hd.y & 1023), t);
#pragma unroll
        for (int i = 0; i < 3; ++i) duH[i] = t[i] - u0[i];
      }
      if constexpr (NEED_GV) {
        ld4(sv + 4 * (hd.y & 1023), t);
#pragma unroll
        for (int i = 0; i < 3; ++i) dvH[i] = t[i] - v0[i];
      }
    }
    // ring node records (x, u, v) fetched one step ahead of their use
    struct Ring {
      CT x[4], u[4], v[4];
    };
    auto fetch_ring = [&](unsigned code, Ring& g) {
      const int l = (int)(code & 1023u);
      ld4(sx + 4 * l, g.x);
      if constexpr (NEED_GU) ld4(su + 4 * l, g.u);
      if constexpr (NEED_GV) ld4(sv + 4 * l, g.v);
    };
    // ring node state: edge from h_0, H x edge, field differences from h_0
    auto derive_ring = [&](const Ring& g, CT (&E)[3], CT (&Q)[3], CT (&du)[3], CT (&dv)[3]) {
#pragma unroll
      for (int i = 0; i < 3; ++i) E[i] = g.x[i] - x0[i];
      if constexpr (DIM == 3) {
        Q[0] = H[1] * E[2] - H[2] * E[1];
        Q[1] = H[2] * E[0] - H[0] * E[2];
        Q[2] = H[0] * E[1] - H[1] * E[0];
      }
      if constexpr (NEED_GU) {
#pragma unroll
        for (int i = 0; i < 3; ++i) du[i] = g.u[i] - u0[i];
      }
      if constexpr (NEED_GV) {
#pragma unroll
        for (int i = 0; i < 3; ++i) dv[i] = g.v[i] - v0[i];
      }
    };
    CT acc0[DIM], acc1[DIM], accc[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc0[i] = acc1[i] = accc[i] = CT(0);
    unsigned cc = hd.z;
    CT Ec[3], Qc[3] = {CT(0), CT(0), CT(0)}, duc[3] = {CT(0), CT(0), CT(0)}, dvc[3] = {CT(0), CT(0), CT(0)};
    Ring gnext;
    fetch_ring(cc, gnext);
    derive_ring(gnext, Ec, Qc, duc, dvc);
    int s = f;  // step record of the tile (step-major: step i of fan f at sum_{j<i} cnt_j + f)
    unsigned cnext = 0;
    M2 mnext{};
    if (k > 0) {
      cnext = scode[s];
      mnext = smat[s];
      fetch_ring(cnext, gnext);
    }
    for (int i = 0; i < k; ++i) {
      const unsigned cn = cnext;
      const CT mu = mnext.x, lam = mnext.y;
      CT En[3], Qn[3] = {CT(0), CT(0), CT(0)}, dun[3] = {CT(0), CT(0), CT(0)}, dvn[3] = {CT(0), CT(0), CT(0)};
      derive_ring(gnext, En, Qn, dun, dvn);
      s += scnt[i];
      if (i + 1 < k) {  // the next step's record and ring node, in flight during this simplex
        cnext = scode[s];
        mnext = smat[s];
        fetch_ring(cnext, gnext);
      }
      ElemGeo<DIM, CT> G;
      fan_geometry<DIM, CT>(H, Ec, En, Qc, Qn, G);
      // corner differences from h_0 of the simplex's fields
      auto diffs = [&](const CT (&dh)[3], const CT (&dci)[3], const CT (&dcn)[3], CT (&dw)[DIM][3]) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if constexpr (DIM == 3) {
            dw[0][j] = dh[j];
            dw[1][j] = dci[j];
            dw[2][j] = dcn[j];
          } else {
            dw[0][j] = dci[j];
            dw[1][j] = dcn[j];
          }
        }
      };
      CT out[NV][DIM];
      if constexpr (KIND == K_LIN) {
        if constexpr (NEED_GU) {
          CT dw[DIM][3], Gp[DIM][DIM];
          diffs(duH, duc, dun, dw);
          grad_prime_d<DIM, CT>(G, dw, Gp);
          if constexpr (ENERGY) e_acc += (double)linear_energy<DIM, CT>(G, Gp, mu, lam);
          if constexpr (OUT == OUT_RES) linear_force<DIM, CT>(G, Gp, mu, lam, out);
        }
        if constexpr (OUT == OUT_TAN) {
          CT dw[DIM][3], Gp[DIM][DIM];
          diffs(dvH, dvc, dvn, dw);
          grad_prime_d<DIM, CT>(G, dw, Gp);
          linear_force<DIM, CT>(G, Gp, mu, lam, out);
        } else if constexpr (OUT == OUT_DIAG) {
          nh_diag<DIM, CT>(G, static_cast<const NHState<DIM, CT>*>(nullptr), mu, lam, out);
        }
      } else {
        CT Gu[DIM][DIM];
        {
          CT dw[DIM][3];
          diffs(duH, duc, dun, dw);
          grad_prime_d<DIM, CT>(G, dw, Gu);
#pragma unroll
          for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) Gu[a][b] *= G.rdet;
        }
        NHState<DIM, CT> st;
        nh_state<DIM, CT>(Gu, st);
        if (COUNT && !(st.J > CT(0))) ++n_inv;
        if constexpr (ENERGY) {
          const CT psi = st.J > CT(0) ? nh_psi<DIM, CT>(st, mu, lam) : CT(INFINITY);
          e_acc += (double)(fabs(G.det) * CT(1.0 / Factorial<DIM>::value) * psi);
        }
        if constexpr (OUT == OUT_RES || OUT == OUT_TAN) {
          CT T[DIM][DIM];
          if constexpr (OUT == OUT_RES) {
            nh_pk1<DIM, CT>(st, mu, lam, T);
          } else {
            CT dw[DIM][3], Gv[DIM][DIM];
            diffs(dvH, dvc, dvn, dw);
            grad_prime_d<DIM, CT>(G, dw, Gv);
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
              for (int b = 0; b < DIM; ++b) Gv[a][b] *= G.rdet;
            nh_dpk1<DIM, CT>(st, mu, lam, Gv, T);
          }
#pragma unroll
          for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) T[a][b] *= G.kappa;  // V T dN_a = kappa T c_a
          contract_c<DIM, CT>(G, T, out);
        } else if constexpr (OUT == OUT_DIAG) {
          nh_diag<DIM, CT>(G, &st, mu, lam, out);
        }
      }
      if constexpr (OUT >= 0) {
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
          acc0[j] += out[0][j];
          if constexpr (DIM == 3) acc1[j] += out[1][j];
          accc[j] += out[HS][j];
        }
        put(cc, accc);  // ring node i is complete: it touches simplices i - 1 and i only
#pragma unroll
        for (int j = 0; j < DIM; ++j) accc[j] = out[HS + 1][j];
      }
      cc = cn;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Ec[j] = En[j];
        Qc[j] = Qn[j];
        duc[j] = dun[j];
        dvc[j] = dvn[j];
      }
    }
    if constexpr (OUT >= 0) {
      put(cc, accc);
      put(hd.x, acc0);
      if constexpr (DIM == 3) put(hd.y, acc1);
    }
  }
}

// p_l . (A_tile p)_l of one tile node in the element precision (summed in FP64 over the tile's
// nodes this is the tile's share of p . A p: every element contribution to node l sits in
// one of l's slots)
template <int DIM, typename CT>
__device__ __forceinline__ double pap_node(const CT* v, const CT (&acc)[4]) {
  CT d = v[0] * acc[0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) d = fma(v[i], acc[i], d);
  return (double)d;
}

template <int DIM, int OUT, typename VT, typename CT, bool PCG = false>
__device__ __forceinline__ void node_pass(const DevPlan& P, const OpArgs& A, unsigned char* smem,
                                          const SmemLayout<CT>& L, int nl, int ncomp, int pbeg, int region,
                                          const double* p_old = nullptr, double* p_new = nullptr, double beta = 0.0,
                                          double* e_pap = nullptr) {
  const int* soff = reinterpret_cast<const int*>(smem + L.off);
  const int* sinfo = reinterpret_cast<const int*>(smem + L.info);
  const CT* slot = reinterpret_cast<const CT*>(smem + L.slot);
  CT* part = static_cast<CT*>(P.partial) + (size_t)region * P.n_partials * 4;
  int32_t* count = P.halo_count + (size_t)region * P.n_partials;
  const CT sc = A.out_scale ? CT(*static_cast<const VT*>(A.out_scale)) : CT(1);  // upstream factor (autograd)
  const bool defer = A.defer_halo != 0;
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    int slot_i = pbeg + l - ncomp;  // deferred: tile order, no load on the way
    if (l >= ncomp && !defer) slot_i = P.halo_rec[slot_i].x;  // issued before the slot sums
    if (l >= ncomp && !checked_range(slot_i, 1, P.n_partials)) slot_i = 0;
    const int b = soff[l], e = soff[l + 1];
    CT acc[4] = {CT(0), CT(0), CT(0), CT(0)};
    for (int k = b; k < e; ++k) {
      CT t[4];
      ld4(slot + 4 * k, t);
#pragma unroll
      for (int i = 0; i < DIM; ++i) acc[i] += t[i];
    }
    if constexpr (PCG) *e_pap += pap_node<DIM, CT>(reinterpret_cast<const CT*>(smem + L.v) + 4 * l, acc);
    if (l < ncomp) {
      const unsigned info = (unsigned)sinfo[l];
      final_write<DIM, OUT, VT, CT, PCG>(P, A, checked_node((int64_t)(info & kInfoIdMask), P.n_nodes),
                                         info >> kInfoIdBits, acc, sc);
      continue;
    }
    // halo node: publish this tile's partial in the node's contiguous range
    st4(part + 4 * (size_t)slot_i, acc[0], acc[1], acc[2], CT(0));
  }
  if (defer) return;  // uniform: halo_finish_kernel completes the halo nodes
  // Release once per tile: every partial of this tile is visible device-wide before any of
  // its tickets; the tile whose ticket completes a halo node's set (acquire fence after the
  // ticket) sums that node's partials in ascending tile order and writes the output.
  __syncthreads();
  if (threadIdx.x == 0) __threadfence();
  __syncthreads();
  for (int l = ncomp + threadIdx.x; l < nl; l += blockDim.x) {
    const int4 rec = P.halo_rec[pbeg + l - ncomp];
    if (checked_range(rec.y, rec.z, P.n_partials) && atomicAdd(count + rec.y, 1) == rec.z - 1) {
      __threadfence();
      CT sum[4] = {CT(0), CT(0), CT(0), CT(0)};
      for (int k = rec.y; k < rec.y + rec.z; ++k) {
        CT t[4];
        ldcg4(part + 4 * (size_t)k, t);
#pragma unroll
        for (int i = 0; i < DIM; ++i) sum[i] += t[i];
      }
      const unsigned hinfo = (unsigned)rec.w;
      const int64_t hgid = checked_node((int64_t)(hinfo & kInfoIdMask), P.n_nodes);
      if constexpr (PCG) {  // the node's new direction, as every tile staged it
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int64_t k = hgid * DIM + i;
          p_new[k] = pcg_direction(A.pcg, p_old, beta, k, ((hinfo >> kInfoIdBits) >> i) & 1u);
        }
      }
      final_write<DIM, OUT, VT, CT, PCG>(P, A, hgid, hinfo >> kInfoIdBits, sum, sc);
      count[rec.y] = 0;
    }
  }
}

// All passes of tile t of plan P (one CTA). `lay` sizes the shared memory (it may come from
// a larger plan when several meshes share a launch).
template <int DIM, int KIND, int OPS, typename VT, typename CT>
__device__ __forceinline__ void process_tile(const DevPlan& P, const OpArgs& A, int t, unsigned char* smem,
                                             const SmemLayout<CT>& lay) {
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT>& L = lay;
  const int4 ta = P.tile_a[t];
  const int4 tb = P.tile_b[t];
  const int fbeg = ta.x, nf = ta.y, lbeg = ta.z, nl = ta.w;
  const int ncomp = tb.x, pbeg = tb.y, sbeg = tb.z, ns = tb.w;
  constexpr bool PCG = (OPS & OP_PCG) != 0;
  const double* p_old = nullptr;
  double* p_new = nullptr;
  double beta = 0.0;
  constexpr bool PERSIST = (OPS & OP_PERSIST) != 0;
  if constexpr (PCG) {
    bool odd;
    if constexpr (PERSIST) {  // the persistent kernel passes the state of this iteration
      beta = A.pcg.beta;
      odd = A.pcg.odd != 0;
    } else {
      // the state is written only by earlier kernels, so every CTA takes the same branch
      // (all four fields loaded before the branch: one round trip)
      const PcgState* st = A.pcg.st;
      const int done = st->done, repl = st->repl, it = st->iter;
      const double b = st->beta;
      if (done != 0 || repl != 0) return;
      beta = b;
      odd = (it & 1) != 0;
    }
    // select, not index: keeps the arguments out of local memory
    p_old = odd ? A.pcg.p[1] : A.pcg.p[0];
    p_new = odd ? A.pcg.p[0] : A.pcg.p[1];
  }

  // ---- stage the tile in shared memory; every round issues all its global loads before
  // its shared stores (the step records first: they depend on nothing)
  {
    CT* sx = reinterpret_cast<CT*>(smem + L.x);
    CT* su = reinterpret_cast<CT*>(smem + L.u);
    CT* sv = reinterpret_cast<CT*>(smem + L.v);
    int* soff = reinterpret_cast<int*>(smem + L.off);
    int* sinfo = reinterpret_cast<int*>(smem + L.info);
    const VT* u = static_cast<const VT*>(A.u);
    const VT* v = static_cast<const VT*>(A.v);
    // node records of this thread's first round (two nodes per thread and round), issued
    // before the step records so that their latency and the step loads overlap
    float4 rf[2];
    int so[2] = {0, 0};
    CT xc[2][3];
    auto load_records = [&](int l0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int l = l0 + q * (int)blockDim.x;
        if (l >= nl) continue;
        rf[q] = P.lnode_f[lbeg + l];
        so[q] = (int)P.slot_off[lbeg + l];
        if constexpr (sizeof(CT) == 4) {
          xc[q][0] = rf[q].x, xc[q][1] = rf[q].y, xc[q][2] = rf[q].z;
        } else {
          const PfemDouble4 rd = P.lnode_d[lbeg + l];
          xc[q][0] = rd.x, xc[q][1] = rd.y, xc[q][2] = rd.z;
        }
      }
    };
    if ((int)threadIdx.x < nl) load_records(threadIdx.x);
    {  // fan heads and step records (coalesced; read from shared memory by the fans)
      using M2 = typename std::conditional<sizeof(CT) == 4, float2, double2>::type;
      const M2* gmat = reinterpret_cast<const M2*>(sizeof(CT) == 4 ? static_cast<const void*>(P.step_mat_f)
                                                                   : static_cast<const void*>(P.step_mat_d));
      M2* smat = reinterpret_cast<M2*>(smem + L.smat);
      ushort4* shead = reinterpret_cast<ushort4*>(smem + L.head);
      uint16_t* scode = reinterpret_cast<uint16_t*>(smem + L.scode);
      for (int j0 = threadIdx.x; j0 < ns; j0 += 4 * blockDim.x) {
        uint16_t c[4];
        M2 m[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = j0 + q * (int)blockDim.x;
          if (j < ns) {
            c[q] = P.step_code[sbeg + j];
            m[q] = gmat[sbeg + j];
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = j0 + q * (int)blockDim.x;
          if (j < ns) {
            scode[j] = c[q];
            smat[j] = m[q];
          }
        }
      }
      for (int j = threadIdx.x; j < nf; j += blockDim.x) shead[j] = P.fan_head[fbeg + j];
    }
    // nodes, two per thread and round: records (the first round's are in flight already),
    // then the gathers their ids select
    for (int l0 = threadIdx.x; l0 < nl; l0 += 2 * blockDim.x) {
      const int ls[2] = {l0, l0 + (int)blockDim.x};
      if (l0 != (int)threadIdx.x) load_records(l0);
      CT wu[2][3], wv[2][3];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int i = 0; i < 3; ++i) wu[q][i] = wv[q][i] = CT(0);
        if (ls[q] >= nl) continue;
        const unsigned info = (unsigned)__float_as_int(rf[q].w);
        const int64_t gid = checked_node((int64_t)(info & kInfoIdMask), P.n_nodes);
        const unsigned mask = info >> kInfoIdBits;
        if constexpr (NEED_U) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) wu[q][i] = CT(u[gid * DIM + i]);
        }
        if constexpr (PCG) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            const int64_t k = gid * DIM + i;
            const double pn = pcg_direction(A.pcg, p_old, beta, k, (mask >> i) & 1u);
            if (ls[q] < ncomp) p_new[k] = pn;  // complete nodes: this tile owns the DOF
            wv[q][i] = CT(pn);
          }
        } else if constexpr (NEED_V) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) wv[q][i] = ((mask >> i) & 1u) ? CT(0) : CT(v[gid * DIM + i]);
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int l = ls[q];
        if (l >= nl) continue;
        st4(sx + 4 * l, xc[q][0], xc[q][1], xc[q][2], CT(0));
        sinfo[l] = __float_as_int(rf[q].w);
        soff[l] = so[q];
        if constexpr (NEED_U) st4(su + 4 * l, wu[q][0], wu[q][1], wu[q][2], CT(0));
        if constexpr (NEED_V) st4(sv + 4 * l, wv[q][0], wv[q][1], wv[q][2], CT(0));
      }
    }
    if (threadIdx.x == 0) soff[nl] = nf * DIM + ns;  // slots: DIM + k per fan
    if (threadIdx.x < kMaxFan) {  // fan counts per step (8 x uint16 in one uint4)
      const uint4 c = P.tile_cnt[t];
      const unsigned q = threadIdx.x >> 1;
      const unsigned word = q == 0 ? c.x : (q == 1 ? c.y : (q == 2 ? c.z : c.w));
      reinterpret_cast<int*>(smem + L.fb)[threadIdx.x] = (int)((word >> (16 * (threadIdx.x & 1))) & 0xffffu);
    }
  }
  __syncthreads();

  double e_acc = 0.0;
  int n_inv = 0;
  int region = 0;
  if constexpr ((OPS & OP_RESIDUAL) != 0) {
    fan_pass<DIM, KIND, OUT_RES, (OPS & OP_ENERGY) != 0, true, CT>(smem, L, nf, e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_RES, VT, CT>(P, A, smem, L, nl, ncomp, pbeg, region++);
    __syncthreads();
  } else if constexpr ((OPS & OP_ENERGY) != 0) {
    fan_pass<DIM, KIND, -1, true, true, CT>(smem, L, nf, e_acc, n_inv);
  }
  if constexpr ((OPS & OP_TANGENT) != 0) {
    fan_pass<DIM, KIND, OUT_TAN, false, (OPS & (OP_RESIDUAL | OP_ENERGY)) == 0, CT>(smem, L, nf, e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_TAN, VT, CT, PCG>(P, A, smem, L, nl, ncomp, pbeg, region++, p_old, p_new, beta, &e_acc);
    __syncthreads();
  }
  if constexpr ((OPS & OP_DIAG) != 0) {
    fan_pass<DIM, KIND, OUT_DIAG, false, (OPS & (OP_RESIDUAL | OP_ENERGY | OP_TANGENT)) == 0, CT>(
        smem, L, nf, e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_DIAG, VT, CT>(P, A, smem, L, nl, ncomp, pbeg, region++);
  }
  if constexpr (KIND == K_NH) {
    const int tot = __reduce_add_sync(0xffffffffu, n_inv);
    if ((threadIdx.x & 31) == 0 && tot > 0 && P.inverted) atomicAdd(P.inverted, tot);
  }
  if constexpr ((OPS & OP_ENERGY) != 0 || PCG) {
    // tile sum of the energy (or of p_e . A_e p_e): warp butterflies, warps in index order
    double* red = reinterpret_cast<double*>(smem + L.red);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      if constexpr (PCG) A.pcg.tile_part[t] = s;
      else P.tile_energy[t] = s;
    }
  }
  if constexpr (PCG) {
    // the last tile to finish sums the tile partials in tile order: alpha = rho / (p . A p)
    // (unless the update kernel forms alpha itself from the same partials)
    if (A.pcg.alpha_by_update) return;
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(A.pcg.ticket, 1u) == (unsigned)P.n_tiles - 1u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      // thread 0's state reads go out with the tile partials' loads
      PcgState* st = A.pcg.st;
      double rho = 0.0;
      int trunc = 0, it = 0;
      if (threadIdx.x == 0) {
        rho = __ldcg(&st->rho);
        trunc = __ldcg(&st->truncate);
        it = __ldcg(&st->iter);
      }
      const double pap = pcg_tile_total(A.pcg.tile_part, P.n_tiles, reinterpret_cast<double*>(smem + L.red));
      if (threadIdx.x == 0) {
        double alpha = 0.0;
        const int stop = pcg_alpha(pap, rho, trunc, it, &alpha);
        st->alpha = alpha;
        if (stop) st->done = stop;
        *A.pcg.ticket = 0u;
      }
    }
  }
}

// Opt a kernel into the largest dynamic shared memory its static shared memory leaves room
// for (227 KB per CTA in total), once; then check that `need` bytes fit.
template <typename Kernel>
static inline pfem_status allow_dynamic_smem(Kernel kernel, size_t need, int* max_dyn) {
  if (*max_dyn == 0) {
    cudaFuncAttributes fa;
    PFEM_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const int lim = 227 * 1024 - (int)fa.sharedSizeBytes;
    PFEM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    *max_dyn = lim;
  }
  if (need > (size_t)*max_dyn) {
    set_error("a tile needs %zu bytes of shared memory (at most %d)", need, *max_dyn);
    return PFEM_ERR_UNSUPPORTED;
  }
  return PFEM_OK;
}

}  // namespace pfem
