// Element-tile kernel: one CTA per tile, shared-memory staging of the tile's nodes, one
// thread per element (strided), per-incidence slots, fixed-order node sums, and halo nodes
// finished in-kernel by the last tile to publish its partial.
//
// Passes of one tile CTA (every requested output op runs its own element and node pass;
// element quantities are recomputed, never stored):
//   stage : tile node coordinates (tile-relative, FP32 or FP64) + u and/or v gathered by id
//   elem  : per element geometry, kinematics, stress / stress derivative, V * T dN_a into
//           slot (node, rank); optional V * Psi accumulated per thread
//   node  : each tile node sums its slots in rank order; a complete node writes its output;
//           a halo node publishes a partial, and the tile whose partial completes the set
//           (integer ticket per halo node) sums all partials of that node in ascending tile
//           order and writes the output. The summation order never depends on timing, so the
//           result is bitwise reproducible; the ticket is reset by that last tile.
//
// Output conventions (Dirichlet DOFs eliminated): tangent y = v on prescribed DOFs and v is
// read as 0 there; residual r = 0 on prescribed DOFs; diagonal d = 1 on prescribed DOFs.

#include <cuda/atomic>

#include "element.cuh"
#include "pcg_state.cuh"
#include "pfem_internal.h"

namespace pfem {

enum : int { K_LIN = 0, K_NH = 1 };
enum : int { OUT_RES = 0, OUT_TAN = 1, OUT_DIAG = 2 };

template <typename CT>
struct SmemLayout {
  size_t slot, x, u, v, off, info, red, total;
};

// Shared memory: 4-wide (x, y, z, pad) records for slots and staged node data.
template <typename CT>
__host__ __device__ inline SmemLayout<CT> smem_layout(int max_local, int slot_cap, bool need_u, bool need_v) {
  SmemLayout<CT> L;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 31) & ~size_t(31); };
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
  return fixed ? 0.0 : fma(g.dinv[k], g.r[k], beta * p_old[k]);
}

template <int DIM, int OUT, typename VT, typename CT, bool PCG = false>
__device__ __forceinline__ void final_write(const DevPlan& P, const OpArgs& A, int64_t gid, unsigned mask,
                                            const CT (&acc)[4]) {
  const CT sc = A.out_scale ? CT(*A.out_scale) : CT(1);  // upstream factor (batched autograd)
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

// v_e . y_e over the corners of one element (the element's share of v . A v)
template <int DIM, typename CT>
__device__ __forceinline__ double corner_dot(const CT (&w)[DIM + 1][3], const CT (&out)[DIM + 1][DIM]) {
  CT s = CT(0);
#pragma unroll
  for (int a = 0; a <= DIM; ++a)
#pragma unroll
    for (int i = 0; i < DIM; ++i) s = fma(w[a][i], out[a][i], s);
  return (double)s;
}

// One element pass for output OUT (or energy only when OUT < 0). PAP: accumulate v . A_e v
// into e_acc (tangent pass of the PCG-fused apply).
template <int DIM, int KIND, int OUT, bool ENERGY, bool COUNT, typename CT, bool PAP = false>
__device__ __forceinline__ void element_pass(const DevPlan& P, unsigned char* smem, const SmemLayout<CT>& L, int ebeg,
                                             int ne, double& e_acc, int& n_inv) {
  constexpr int NV = DIM + 1;
  const CT* sx = reinterpret_cast<const CT*>(smem + L.x);
  const CT* su = reinterpret_cast<const CT*>(smem + L.u);
  const CT* sv = reinterpret_cast<const CT*>(smem + L.v);
  const int* soff = reinterpret_cast<const int*>(smem + L.off);
  CT* slot = reinterpret_cast<CT*>(smem + L.slot);
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const ushort4 code = P.ecode[ebeg + e];
    const unsigned short cs[4] = {code.x, code.y, code.z, code.w};
    CT mu, lam;
    if constexpr (sizeof(CT) == 4) {
      const float2 m = P.emat_f[ebeg + e];
      mu = m.x;
      lam = m.y;
    } else {
      const double2 m = P.emat_d[ebeg + e];
      mu = m.x;
      lam = m.y;
    }
    int loc[NV];
    CT X[NV][4];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      loc[a] = cs[a] & 1023;
      ld4(sx + 4 * loc[a], X[a]);
    }
    ElemGeo<DIM, CT> G;
    if constexpr (DIM == 3) {
      CT X3[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) X3[a][i] = X[a][i];
      geometry3<CT>(X3, G);
    } else {
      CT X2[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) X2[a][i] = X[a][i];
      geometry2<CT>(X2, G);
    }
    constexpr bool NEED_GU = ENERGY || OUT == OUT_RES || (KIND == K_NH && (OUT == OUT_TAN || OUT == OUT_DIAG));
    CT Gu[DIM][DIM];
    if constexpr (NEED_GU) {
      CT w[NV][3];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        CT t[4];
        ld4(su + 4 * loc[a], t);
        w[a][0] = t[0], w[a][1] = t[1], w[a][2] = t[2];
      }
      grad_of<DIM, CT>(G, w, Gu);
    }
    CT out[NV][DIM];
    if constexpr (KIND == K_LIN) {
      if constexpr (ENERGY) e_acc += (double)(G.vol * linear_psi<DIM, CT>(Gu, mu, lam));
      if constexpr (OUT == OUT_RES) {
        CT S[DIM][DIM];
        linear_stress<DIM, CT>(Gu, mu, lam, S);
        contract<DIM, CT>(G, S, out);
      } else if constexpr (OUT == OUT_TAN) {
        CT w[NV][3];
#pragma unroll
        for (int a = 0; a < NV; ++a) {
          CT t[4];
          ld4(sv + 4 * loc[a], t);
          w[a][0] = t[0], w[a][1] = t[1], w[a][2] = t[2];
        }
        CT Gv[DIM][DIM], S[DIM][DIM];
        grad_of<DIM, CT>(G, w, Gv);
        linear_stress<DIM, CT>(Gv, mu, lam, S);
        contract<DIM, CT>(G, S, out);
        if constexpr (PAP) e_acc += corner_dot<DIM, CT>(w, out);
      } else if constexpr (OUT == OUT_DIAG) {
        nh_diag<DIM, CT>(G, static_cast<const NHState<DIM, CT>*>(nullptr), mu, lam, out);
      }
    } else {
      NHState<DIM, CT> s;
      nh_state<DIM, CT>(Gu, s);
      if (COUNT && !(s.J > CT(0))) ++n_inv;
      if constexpr (ENERGY) {
        const CT psi = s.J > CT(0) ? nh_psi<DIM, CT>(s, mu, lam) : CT(INFINITY);
        e_acc += (double)(G.vol * psi);
      }
      if constexpr (OUT == OUT_RES) {
        CT Pk[DIM][DIM];
        nh_pk1<DIM, CT>(s, mu, lam, Pk);
        contract<DIM, CT>(G, Pk, out);
      } else if constexpr (OUT == OUT_TAN) {
        CT w[NV][3];
#pragma unroll
        for (int a = 0; a < NV; ++a) {
          CT t[4];
          ld4(sv + 4 * loc[a], t);
          w[a][0] = t[0], w[a][1] = t[1], w[a][2] = t[2];
        }
        CT Gv[DIM][DIM], dP[DIM][DIM];
        grad_of<DIM, CT>(G, w, Gv);
        nh_dpk1<DIM, CT>(s, mu, lam, Gv, dP);
        contract<DIM, CT>(G, dP, out);
        if constexpr (PAP) e_acc += corner_dot<DIM, CT>(w, out);
      } else if constexpr (OUT == OUT_DIAG) {
        nh_diag<DIM, CT>(G, &s, mu, lam, out);
      }
    }
    if constexpr (OUT >= 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const int sl = soff[loc[a]] + (cs[a] >> 10);
        st4(slot + 4 * sl, out[a][0], out[a][1], DIM == 3 ? out[a][DIM - 1] : CT(0), CT(0));
      }
    }
  }
}

template <int DIM, int OUT, typename VT, typename CT, bool PCG = false>
__device__ __forceinline__ void node_pass(const DevPlan& P, const OpArgs& A, unsigned char* smem,
                                          const SmemLayout<CT>& L, int nl, int ncomp, int pbeg, int region,
                                          const double* p_old = nullptr, double* p_new = nullptr, double beta = 0.0) {
  const int* soff = reinterpret_cast<const int*>(smem + L.off);
  const int* sinfo = reinterpret_cast<const int*>(smem + L.info);
  const CT* slot = reinterpret_cast<const CT*>(smem + L.slot);
  CT* part = static_cast<CT*>(P.partial) + (size_t)region * P.n_partials * 4;
  int32_t* count = P.halo_count + (size_t)region * P.n_halo;
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int b = soff[l], e = soff[l + 1];
    CT acc[4] = {CT(0), CT(0), CT(0), CT(0)};
    for (int k = b; k < e; ++k) {
      CT t[4];
      ld4(slot + 4 * k, t);
#pragma unroll
      for (int i = 0; i < DIM; ++i) acc[i] += t[i];
    }
    if (l < ncomp) {
      const unsigned info = (unsigned)sinfo[l];
      final_write<DIM, OUT, VT, CT, PCG>(P, A, (int64_t)(info & kInfoIdMask), info >> kInfoIdBits, acc);
      continue;
    }
    // halo node: publish this tile's partial, the tile completing the set finishes the node
    const int pi = pbeg + l - ncomp;
    st4(part + 4 * (size_t)pi, acc[0], acc[1], acc[2], CT(0));
    const int h = P.partial_halo[pi];
    const int pb = P.halo_ptr[h], pe = P.halo_ptr[h + 1];
    // release: this partial is visible before the ticket; acquire: the last tile sees all
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> ticket(count[h]);
    if (ticket.fetch_add(1, cuda::memory_order_acq_rel) == pe - pb - 1) {
      CT sum[4] = {CT(0), CT(0), CT(0), CT(0)};
      for (int k = pb; k < pe; ++k) {
        CT t[4];
        ldcg4(part + 4 * (size_t)P.halo_src[k], t);
#pragma unroll
        for (int i = 0; i < DIM; ++i) sum[i] += t[i];
      }
      const unsigned hinfo = (unsigned)P.halo_info[h];
      const int64_t hgid = (int64_t)(hinfo & kInfoIdMask);
      if constexpr (PCG) {  // the node's new direction, as every tile staged it
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int64_t k = hgid * DIM + i;
          p_new[k] = pcg_direction(A.pcg, p_old, beta, k, ((hinfo >> kInfoIdBits) >> i) & 1u);
        }
      }
      final_write<DIM, OUT, VT, CT, PCG>(P, A, hgid, hinfo >> kInfoIdBits, sum);
      count[h] = 0;
    }
  }
}

// All passes of tile t of plan P (one CTA). `lay` sizes the shared memory (it may come from
// a larger plan when several meshes share a launch).
template <int DIM, int KIND, int OPS, typename VT, typename CT>
__device__ __forceinline__ void process_tile(const DevPlan& P, const OpArgs& A, int t, unsigned char* smem,
                                             const SmemLayout<CT>& lay) {
  constexpr int NV = DIM + 1;
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT>& L = lay;
  const int4 ta = P.tile_a[t];
  const int4 tb = P.tile_b[t];
  const int ebeg = ta.x, ne = ta.y, lbeg = ta.z, nl = ta.w;
  const int ncomp = tb.x, pbeg = tb.y;
  constexpr bool PCG = (OPS & OP_PCG) != 0;
  const double* p_old = nullptr;
  double* p_new = nullptr;
  double beta = 0.0;
  if constexpr (PCG) {
    // the state is written only by earlier kernels, so every CTA takes the same branch
    const PcgState* st = A.pcg.st;
    if (st->done != 0 || st->repl != 0) return;
    beta = st->beta;
    p_old = A.pcg.p[st->iter & 1];
    p_new = A.pcg.p[(st->iter + 1) & 1];
  }

  // ---- stage tile nodes
  {
    CT* sx = reinterpret_cast<CT*>(smem + L.x);
    CT* su = reinterpret_cast<CT*>(smem + L.u);
    CT* sv = reinterpret_cast<CT*>(smem + L.v);
    int* soff = reinterpret_cast<int*>(smem + L.off);
    int* sinfo = reinterpret_cast<int*>(smem + L.info);
    const VT* u = static_cast<const VT*>(A.u);
    const VT* v = static_cast<const VT*>(A.v);
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      const float4 rf = P.lnode_f[lbeg + l];
      const int info = __float_as_int(rf.w);
      if constexpr (sizeof(CT) == 4) {
        st4(sx + 4 * l, rf.x, rf.y, rf.z, 0.f);
      } else {
        const PfemDouble4 rd = P.lnode_d[lbeg + l];
        st4(sx + 4 * l, rd.x, rd.y, rd.z, 0.0);
      }
      sinfo[l] = info;
      soff[l] = (int)P.slot_off[lbeg + l];
      const int64_t gid = (int64_t)((unsigned)info & kInfoIdMask);
      const unsigned mask = (unsigned)info >> kInfoIdBits;
      if constexpr (NEED_U) {
        CT w[3] = {CT(0), CT(0), CT(0)};
#pragma unroll
        for (int i = 0; i < DIM; ++i) w[i] = CT(u[gid * DIM + i]);
        st4(su + 4 * l, w[0], w[1], w[2], CT(0));
      }
      if constexpr (PCG) {
        CT w[3] = {CT(0), CT(0), CT(0)};
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int64_t k = gid * DIM + i;
          const double pn = pcg_direction(A.pcg, p_old, beta, k, (mask >> i) & 1u);
          if (l < ncomp) p_new[k] = pn;  // complete nodes: this tile owns the DOF
          w[i] = CT(pn);
        }
        st4(sv + 4 * l, w[0], w[1], w[2], CT(0));
      } else if constexpr (NEED_V) {
        CT w[3] = {CT(0), CT(0), CT(0)};
#pragma unroll
        for (int i = 0; i < DIM; ++i) w[i] = ((mask >> i) & 1u) ? CT(0) : CT(v[gid * DIM + i]);
        st4(sv + 4 * l, w[0], w[1], w[2], CT(0));
      }
    }
    if (threadIdx.x == 0) soff[nl] = ne * NV;
  }
  __syncthreads();

  double e_acc = 0.0;
  int n_inv = 0;
  int region = 0;
  if constexpr ((OPS & OP_RESIDUAL) != 0) {
    element_pass<DIM, KIND, OUT_RES, (OPS & OP_ENERGY) != 0, true, CT>(P, smem, L, ebeg, ne, e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_RES, VT, CT>(P, A, smem, L, nl, ncomp, pbeg, region++);
    __syncthreads();
  } else if constexpr ((OPS & OP_ENERGY) != 0) {
    element_pass<DIM, KIND, -1, true, true, CT>(P, smem, L, ebeg, ne, e_acc, n_inv);
  }
  if constexpr ((OPS & OP_TANGENT) != 0) {
    element_pass<DIM, KIND, OUT_TAN, false, (OPS & (OP_RESIDUAL | OP_ENERGY)) == 0, CT, PCG>(P, smem, L, ebeg, ne,
                                                                                          e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_TAN, VT, CT, PCG>(P, A, smem, L, nl, ncomp, pbeg, region++, p_old, p_new, beta);
    __syncthreads();
  }
  if constexpr ((OPS & OP_DIAG) != 0) {
    element_pass<DIM, KIND, OUT_DIAG, false, (OPS & (OP_RESIDUAL | OP_ENERGY | OP_TANGENT)) == 0, CT>(
        P, smem, L, ebeg, ne, e_acc, n_inv);
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
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(A.pcg.ticket, 1u) == (unsigned)P.n_tiles - 1u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double s = 0.0;
      for (int i = threadIdx.x; i < P.n_tiles; i += blockDim.x) s += __ldcg(A.pcg.tile_part + i);
      double* red = reinterpret_cast<double*>(smem + L.red);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double pap = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pap += red[w];
        PcgState* st = A.pcg.st;
        // negative curvature does not stop plain CG; p.Ap = 0 or non-finite does
        if (pap == 0.0 || !isfinite(pap)) {
          st->alpha = 0.0;
          st->done = isfinite(pap) ? PCG_BREAKDOWN : PCG_NONFINITE;
        } else {
          st->alpha = st->rho / pap;
        }
        *A.pcg.ticket = 0u;
      }
    }
  }
}

template <int DIM, int KIND, int OPS, typename VT, typename CT>
__global__ void __launch_bounds__(kThreads) tile_kernel(DevPlan P, OpArgs A) {
  extern __shared__ __align__(32) unsigned char smem[];
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT> L = smem_layout<CT>(P.max_local, P.slot_cap, NEED_U, NEED_V);
  process_tile<DIM, KIND, OPS, VT, CT>(P, A, blockIdx.x, smem, L);
}

// Ragged batch of 3-D meshes in one launch: CTA b runs tile btile[b].y of mesh btile[b].x
// (FP32 vectors and arithmetic; linear or Neo-Hookean chosen per mesh, uniform per CTA).
template <int OPS>
__global__ void __launch_bounds__(kThreads) batch_kernel(BatchDev B, OpArgs A) {
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ DevPlan sP;
  const int2 bt = B.btile[blockIdx.x];
  if (threadIdx.x == 0) sP = B.plans[bt.x];
  __syncthreads();
  const int64_t off = B.dof_off[bt.x];
  OpArgs a = A;
  a.u = static_cast<const float*>(A.u) + off;
  if (A.v) a.v = static_cast<const float*>(A.v) + off;
  if (A.y) a.y = static_cast<float*>(A.y) + off;
  if (A.r) a.r = static_cast<float*>(A.r) + off;
  a.out_scale = B.mesh_scale ? B.mesh_scale + bt.x : nullptr;
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<float> L = smem_layout<float>(B.max_local, B.slot_cap, true, NEED_V);
  if (sP.kind == PFEM_LINEAR) process_tile<3, K_LIN, OPS, float, float>(sP, a, bt.y, smem, L);
  else process_tile<3, K_NH, OPS, float, float>(sP, a, bt.y, smem, L);
}

// Per mesh m (one CTA each): energy[m] = sum of its tile energies - f_ext . u_m.
__global__ void __launch_bounds__(256) batch_energy_kernel(BatchDev B, const float* u, double* energy) {
  __shared__ double red[16];
  const DevPlan& P = B.plans[blockIdx.x];
  const int64_t off = B.dof_off[blockIdx.x], nd = B.dof_off[blockIdx.x + 1] - off;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < P.n_tiles; i += blockDim.x) a += P.tile_energy[i];
  for (int64_t i = threadIdx.x; i < nd; i += blockDim.x) b += P.f_ext[i] * (double)u[off + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = a;
    red[2 * (threadIdx.x >> 5) + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += red[2 * w];
      sb += red[2 * w + 1];
    }
    energy[blockIdx.x] = sa - sb;
  }
}

// Opt a kernel into the largest dynamic shared memory its static shared memory leaves room
// for (227 KB per CTA in total), once; then check that `need` bytes fit.
template <typename Kernel>
static pfem_status allow_dynamic_smem(Kernel kernel, size_t need, int* max_dyn) {
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

template <int OPS>
static pfem_status run_batch(const BatchDev& B, const OpArgs& A, int n_blocks, cudaStream_t s) {
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<float> L = smem_layout<float>(B.max_local, B.slot_cap, true, NEED_V);
  static int max_dyn = 0;
  pfem_status st = allow_dynamic_smem(batch_kernel<OPS>, L.total, &max_dyn);
  if (st) return st;
  batch_kernel<OPS><<<n_blocks, kThreads, L.total, s>>>(B, A);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status launch_batch(const BatchDev& B, int n_blocks, int n_meshes, const float* u, const float* v, float* grad,
                         float* hvp, double* energy, cudaStream_t s) {
  OpArgs a{};
  a.u = u;
  a.v = v;
  a.y = hvp;
  a.r = grad;
  a.load_scale = 1.0;
  a.hess = 1;  // Hessian of the energy on free DOFs: zero rows and columns on prescribed DOFs
  pfem_status st;
  if (grad && hvp) st = run_batch<OP_ENERGY | OP_RESIDUAL | OP_TANGENT>(B, a, n_blocks, s);
  else if (grad) st = run_batch<OP_ENERGY | OP_RESIDUAL>(B, a, n_blocks, s);
  else if (hvp) st = run_batch<OP_ENERGY | OP_TANGENT>(B, a, n_blocks, s);
  else st = run_batch<OP_ENERGY>(B, a, n_blocks, s);
  if (st) return st;
  if (energy) {
    batch_energy_kernel<<<n_meshes, 256, 0, s>>>(B, u, energy);
    PFEM_COUNT_LAUNCH();
    PFEM_CUDA(cudaGetLastError());
  }
  return PFEM_OK;
}

// ---- serving: one shared PCG step over all resident solves ------------------------------

__global__ void __launch_bounds__(kThreads) serve_apply_kernel(const ReqDev* reqs, const int2* btile, int max_local,
                                                               int slot_cap) {
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ ReqDev sR;
  const int2 bt = btile[blockIdx.x];
  if (threadIdx.x == 0) sR = reqs[bt.x];
  __syncthreads();
  OpArgs a{};
  a.u = sR.u;
  a.y = sR.q;
  a.load_scale = 1.0;
  a.pcg = sR.pcg;
  const SmemLayout<float> L = smem_layout<float>(max_local, slot_cap, true, true);
  constexpr int OPS = OP_TANGENT | OP_PCG;
  if (sR.plan.kind == PFEM_LINEAR) process_tile<3, K_LIN, OPS, double, float>(sR.plan, a, bt.y, smem, L);
  else process_tile<3, K_NH, OPS, double, float>(sR.plan, a, bt.y, smem, L);
}

// x += alpha p; r -= alpha q; r.z and r.r reduced over the solve's own blocks (fixed order),
// then the shared iteration bookkeeping in the solve's last block.
__global__ void __launch_bounds__(256) serve_update_kernel(const ReqDev* reqs, const int* ublk) {
  __shared__ double scratch[16];
  __shared__ bool s_last;
  const ReqDev& R = reqs[ublk[blockIdx.x]];
  PcgState* st = R.pcg.st;
  if (st->done != 0 || st->repl != 0) return;  // uniform over the solve's blocks
  const int lb = blockIdx.x - R.ublk0;
  const double alpha = st->alpha;
  const double* p = R.pcg.p[(st->iter + 1) & 1];
  double* x = R.x;
  double* r = const_cast<double*>(R.pcg.r);
  const double* q = R.q;
  const double* dinv = R.pcg.dinv;
  double v0 = 0.0, v1 = 0.0;
  for (int64_t i = (int64_t)lb * blockDim.x + threadIdx.x; i < R.n; i += (int64_t)R.nublk * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    v0 += ri * (dinv[i] * ri);
    v1 += ri * ri;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    scratch[2 * (threadIdx.x >> 5)] = v0;
    scratch[2 * (threadIdx.x >> 5) + 1] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a0 += scratch[2 * w];
      a1 += scratch[2 * w + 1];
    }
    R.upart[2 * lb] = a0;
    R.upart[2 * lb + 1] = a1;
    __threadfence();
    s_last = atomicAdd(R.ucount, 1u) == (unsigned)R.nublk - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double rz = 0.0, rr = 0.0;
    for (int b = 0; b < R.nublk; ++b) {
      rz += __ldcg(R.upart + 2 * b);
      rr += __ldcg(R.upart + 2 * b + 1);
    }
    pcg_finish_update(st, rz, rr);
    *R.ucount = 0u;
  }
}

pfem_status launch_serve_step(const ReqDev* reqs, const int2* btile, int n_apply_blocks, const int* ublk,
                              int n_update_blocks, int max_local, int slot_cap, cudaStream_t s) {
  const SmemLayout<float> L = smem_layout<float>(max_local, slot_cap, true, true);
  static int max_dyn = 0;
  pfem_status st = allow_dynamic_smem(serve_apply_kernel, L.total, &max_dyn);
  if (st) return st;
  if (n_apply_blocks > 0) {
    serve_apply_kernel<<<n_apply_blocks, kThreads, L.total, s>>>(reqs, btile, max_local, slot_cap);
    PFEM_COUNT_LAUNCH();
  }
  if (n_update_blocks > 0) {
    serve_update_kernel<<<n_update_blocks, 256, 0, s>>>(reqs, ublk);
    PFEM_COUNT_LAUNCH();
  }
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

template <int DIM, int KIND, int OPS, typename VT, typename CT>
static pfem_status run(const DevPlan& P, const OpArgs& A, cudaStream_t s) {
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT> L = smem_layout<CT>(P.max_local, P.slot_cap, NEED_U, NEED_V);
  if (P.n_tiles <= 0) return PFEM_OK;
  static int max_dyn = 0;  // per instantiation
  pfem_status st = allow_dynamic_smem(tile_kernel<DIM, KIND, OPS, VT, CT>, L.total, &max_dyn);
  if (st) return st;
  tile_kernel<DIM, KIND, OPS, VT, CT><<<P.n_tiles, kThreads, L.total, s>>>(P, A);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

template <int DIM, int KIND, typename VT, typename CT>
static pfem_status dispatch_ops(const DevPlan& P, int ops, const OpArgs& A, cudaStream_t s) {
  switch (ops) {
    case OP_TANGENT: return run<DIM, KIND, OP_TANGENT, VT, CT>(P, A, s);
    case OP_RESIDUAL: return run<DIM, KIND, OP_RESIDUAL, VT, CT>(P, A, s);
    case OP_ENERGY: return run<DIM, KIND, OP_ENERGY, VT, CT>(P, A, s);
    case OP_DIAG: return run<DIM, KIND, OP_DIAG, VT, CT>(P, A, s);
    case OP_TANGENT | OP_PCG:
      if constexpr (sizeof(VT) == 8) return run<DIM, KIND, OP_TANGENT | OP_PCG, VT, CT>(P, A, s);
      break;
    default: break;
  }
  set_error("unsupported op combination %d", ops);
  return PFEM_ERR_UNSUPPORTED;
}

template <typename VT, typename CT>
static pfem_status dispatch_kind(const DevPlan& P, int ops, const OpArgs& A, cudaStream_t s) {
  if (P.dim == 3) {
    if (P.kind == PFEM_LINEAR) return dispatch_ops<3, K_LIN, VT, CT>(P, ops, A, s);
    return dispatch_ops<3, K_NH, VT, CT>(P, ops, A, s);
  }
  if (P.kind == PFEM_LINEAR) return dispatch_ops<2, K_LIN, VT, CT>(P, ops, A, s);
  return dispatch_ops<2, K_NH, VT, CT>(P, ops, A, s);
}

pfem_status launch_element_op(const DevPlan& P, int ops, pfem_dtype vt, pfem_dtype ct, const OpArgs& a,
                              cudaStream_t s) {
  if (vt == PFEM_F32 && ct == PFEM_F32) return dispatch_kind<float, float>(P, ops, a, s);
  if (vt == PFEM_F64 && ct == PFEM_F32) return dispatch_kind<double, float>(P, ops, a, s);
  if (vt == PFEM_F64 && ct == PFEM_F64) return dispatch_kind<double, double>(P, ops, a, s);
  set_error("unsupported dtype combination");
  return PFEM_ERR_UNSUPPORTED;
}

size_t element_op_smem(const DevPlan& P, int ops, pfem_dtype ct) {
  const bool need_u = (ops & (OP_RESIDUAL | OP_ENERGY)) || (P.kind == PFEM_NEOHOOKEAN && (ops & (OP_TANGENT | OP_DIAG)));
  const bool need_v = (ops & OP_TANGENT) != 0;
  if (ct == PFEM_F32) return smem_layout<float>(P.max_local, P.slot_cap, need_u, need_v).total;
  return smem_layout<double>(P.max_local, P.slot_cap, need_u, need_v).total;
}

}  // namespace pfem
