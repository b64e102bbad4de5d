// Element-tile kernels: one CTA per tile, shared-memory staging of the tile's nodes,
// one thread per element (strided), per-incidence slots, fixed-order node sums.
//
// Passes of one tile CTA (every requested output op runs its own element and node pass;
// element quantities are recomputed, never stored):
//   stage : tile node coordinates (tile-relative, FP32 or FP64) + u and/or v gathered by id
//   elem  : per element geometry, kinematics, stress / stress derivative, V * T dN_a into
//           slot (node, rank); optional V * Psi accumulated per thread
//   node  : each tile node sums its slots in rank order; complete nodes write the output,
//           halo nodes write a partial for the halo pass
// Halo pass: one thread per halo node sums its partials in ascending tile order.
//
// Output conventions (Dirichlet DOFs eliminated): tangent y = v on prescribed DOFs and v is
// read as 0 there; residual r = 0 on prescribed DOFs; diagonal d = 1 on prescribed DOFs.

#include "element.cuh"
#include "pfem_internal.h"

namespace pfem {

enum : int { K_LIN = 0, K_NH = 1 };
enum : int { OUT_RES = 0, OUT_TAN = 1, OUT_DIAG = 2 };

template <typename CT>
struct SmemLayout {
  size_t slot, x, u, v, off, info, red, total;
};

template <typename CT>
__host__ __device__ inline SmemLayout<CT> smem_layout(int dim, int max_local, int slot_cap, bool need_u,
                                                      bool need_v) {
  SmemLayout<CT> L;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  L.slot = o;
  o = al(o + (size_t)dim * slot_cap * sizeof(CT));
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

template <typename CT>
__device__ __forceinline__ const CT* fext_ptr(const DevPlan& P);
template <>
__device__ __forceinline__ const float* fext_ptr<float>(const DevPlan& P) { return P.f_ext_f; }
template <>
__device__ __forceinline__ const double* fext_ptr<double>(const DevPlan& P) { return P.f_ext; }

template <int DIM, int OUT, typename VT, typename CT>
__device__ __forceinline__ void final_write(const DevPlan& P, const OpArgs& A, int64_t gid, unsigned mask,
                                            const CT (&acc)[DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    const int64_t k = gid * DIM + i;
    const bool fixed = (mask >> i) & 1u;
    if (OUT == OUT_RES) {
      const CT f = fext_ptr<CT>(P)[k];
      static_cast<VT*>(A.r)[k] = fixed ? VT(0) : VT(acc[i] - CT(A.load_scale) * f);
    } else if (OUT == OUT_TAN) {
      static_cast<VT*>(A.y)[k] = fixed ? static_cast<const VT*>(A.v)[k] : VT(acc[i]);
    } else {
      static_cast<VT*>(A.d)[k] = fixed ? VT(1) : VT(acc[i]);
    }
  }
}

template <int DIM, typename CT>
__device__ __forceinline__ void load_corner(const unsigned char* smem, const SmemLayout<CT>& L, int l, CT (&x)[3]) {
  const CT* s = reinterpret_cast<const CT*>(smem + L.x) + 4 * l;
#pragma unroll
  for (int i = 0; i < 3; ++i) x[i] = s[i];
}

// One element pass for output OUT (or energy only when OUT < 0).
template <int DIM, int KIND, int OUT, bool ENERGY, bool COUNT, typename VT, typename CT>
__device__ __forceinline__ void element_pass(const DevPlan& P, unsigned char* smem, const SmemLayout<CT>& L, int ebeg,
                                             int ne, int slot_cap, double& e_acc, int& n_inv) {
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
    CT X[NV][3];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      loc[a] = cs[a] & 1023;
#pragma unroll
      for (int i = 0; i < 3; ++i) X[a][i] = sx[4 * loc[a] + i];
    }
    ElemGeo<DIM, CT> G;
    if constexpr (DIM == 3) geometry3<CT>(X, G);
    else {
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
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) w[a][i] = su[4 * loc[a] + i];
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
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int i = 0; i < 3; ++i) w[a][i] = sv[4 * loc[a] + i];
        CT Gv[DIM][DIM], S[DIM][DIM];
        grad_of<DIM, CT>(G, w, Gv);
        linear_stress<DIM, CT>(Gv, mu, lam, S);
        contract<DIM, CT>(G, S, out);
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
        for (int a = 0; a < NV; ++a)
#pragma unroll
          for (int i = 0; i < 3; ++i) w[a][i] = sv[4 * loc[a] + i];
        CT Gv[DIM][DIM], dP[DIM][DIM];
        grad_of<DIM, CT>(G, w, Gv);
        nh_dpk1<DIM, CT>(s, mu, lam, Gv, dP);
        contract<DIM, CT>(G, dP, out);
      } else if constexpr (OUT == OUT_DIAG) {
        nh_diag<DIM, CT>(G, &s, mu, lam, out);
      }
    }
    if constexpr (OUT >= 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const int sl = soff[loc[a]] + (cs[a] >> 10);
#pragma unroll
        for (int i = 0; i < DIM; ++i) slot[i * slot_cap + sl] = out[a][i];
      }
    }
  }
}

template <int DIM, int OUT, typename VT, typename CT>
__device__ __forceinline__ void node_pass(const DevPlan& P, const OpArgs& A, unsigned char* smem,
                                          const SmemLayout<CT>& L, int nl, int ncomp, int pbeg, int slot_cap,
                                          int region) {
  const int* soff = reinterpret_cast<const int*>(smem + L.off);
  const int* sinfo = reinterpret_cast<const int*>(smem + L.info);
  const CT* slot = reinterpret_cast<const CT*>(smem + L.slot);
  CT* part = static_cast<CT*>(P.partial) + (size_t)region * P.n_partials * DIM;
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int b = soff[l], e = soff[l + 1];
    CT acc[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc[i] = CT(0);
    for (int k = b; k < e; ++k)
#pragma unroll
      for (int i = 0; i < DIM; ++i) acc[i] += slot[i * slot_cap + k];
    const unsigned info = (unsigned)sinfo[l];
    if (l < ncomp) {
      final_write<DIM, OUT, VT, CT>(P, A, (int64_t)(info & kInfoIdMask), info >> kInfoIdBits, acc);
    } else {
      const int64_t pi = (int64_t)(pbeg + l - ncomp) * DIM;
#pragma unroll
      for (int i = 0; i < DIM; ++i) part[pi + i] = acc[i];
    }
  }
}

template <int DIM, int KIND, int OPS, typename VT, typename CT>
__global__ void __launch_bounds__(kThreads) tile_kernel(DevPlan P, OpArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NV = DIM + 1;
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT> L = smem_layout<CT>(DIM, P.max_local, P.slot_cap, NEED_U, NEED_V);
  const int t = blockIdx.x;
  const int4 ta = P.tile_a[t];
  const int4 tb = P.tile_b[t];
  const int ebeg = ta.x, ne = ta.y, lbeg = ta.z, nl = ta.w;
  const int ncomp = tb.x, pbeg = tb.y;
  const int slot_cap = P.slot_cap;

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
        sx[4 * l] = rf.x;
        sx[4 * l + 1] = rf.y;
        sx[4 * l + 2] = rf.z;
      } else {
        const PfemDouble4 rd = P.lnode_d[lbeg + l];
        sx[4 * l] = rd.x;
        sx[4 * l + 1] = rd.y;
        sx[4 * l + 2] = rd.z;
      }
      sinfo[l] = info;
      soff[l] = (int)P.slot_off[lbeg + l];
      const int64_t gid = (int64_t)((unsigned)info & kInfoIdMask);
      const unsigned mask = (unsigned)info >> kInfoIdBits;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if constexpr (NEED_U) su[4 * l + i] = i < DIM ? CT(u[gid * DIM + i]) : CT(0);
        if constexpr (NEED_V) sv[4 * l + i] = (i < DIM && !((mask >> i) & 1u)) ? CT(v[gid * DIM + i]) : CT(0);
      }
    }
    if (threadIdx.x == 0) soff[nl] = ne * NV;
  }
  __syncthreads();

  double e_acc = 0.0;
  int n_inv = 0;
  int region = 0;
  if constexpr ((OPS & OP_RESIDUAL) != 0) {
    element_pass<DIM, KIND, OUT_RES, (OPS & OP_ENERGY) != 0, true, VT, CT>(P, smem, L, ebeg, ne, slot_cap, e_acc,
                                                                         n_inv);
    __syncthreads();
    node_pass<DIM, OUT_RES, VT, CT>(P, A, smem, L, nl, ncomp, pbeg, slot_cap, region++);
    __syncthreads();
  } else if constexpr ((OPS & OP_ENERGY) != 0) {
    element_pass<DIM, KIND, -1, true, true, VT, CT>(P, smem, L, ebeg, ne, slot_cap, e_acc, n_inv);
  }
  if constexpr ((OPS & OP_TANGENT) != 0) {
    element_pass<DIM, KIND, OUT_TAN, false, (OPS & (OP_RESIDUAL | OP_ENERGY)) == 0, VT, CT>(P, smem, L, ebeg, ne,
                                                                                         slot_cap, e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_TAN, VT, CT>(P, A, smem, L, nl, ncomp, pbeg, slot_cap, region++);
    __syncthreads();
  }
  if constexpr ((OPS & OP_DIAG) != 0) {
    element_pass<DIM, KIND, OUT_DIAG, false, (OPS & (OP_RESIDUAL | OP_ENERGY | OP_TANGENT)) == 0, VT, CT>(
        P, smem, L, ebeg, ne, slot_cap, e_acc, n_inv);
    __syncthreads();
    node_pass<DIM, OUT_DIAG, VT, CT>(P, A, smem, L, nl, ncomp, pbeg, slot_cap, region++);
  }
  if constexpr (KIND == K_NH) {
    const int tot = __reduce_add_sync(0xffffffffu, n_inv);
    if ((threadIdx.x & 31) == 0 && tot > 0 && P.inverted) atomicAdd(P.inverted, tot);
  }
  if constexpr ((OPS & OP_ENERGY) != 0) {
    double* red = reinterpret_cast<double*>(smem + L.red);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      P.tile_energy[t] = s;
    }
  }
}

template <int DIM, int OPS, typename VT, typename CT>
__global__ void __launch_bounds__(256) halo_kernel(DevPlan P, OpArgs A) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= P.n_halo) return;
  const unsigned info = (unsigned)P.halo_info[h];
  const int64_t gid = (int64_t)(info & kInfoIdMask);
  const unsigned mask = info >> kInfoIdBits;
  const int b = P.halo_ptr[h], e = P.halo_ptr[h + 1];
  int region = 0;
  auto sum = [&](int reg, CT (&acc)[DIM]) {
    const CT* part = static_cast<const CT*>(P.partial) + (size_t)reg * P.n_partials * DIM;
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc[i] = CT(0);
    for (int k = b; k < e; ++k) {
      const int64_t s = (int64_t)P.halo_src[k] * DIM;
#pragma unroll
      for (int i = 0; i < DIM; ++i) acc[i] += part[s + i];
    }
  };
  if constexpr ((OPS & OP_RESIDUAL) != 0) {
    CT acc[DIM];
    sum(region++, acc);
    final_write<DIM, OUT_RES, VT, CT>(P, A, gid, mask, acc);
  }
  if constexpr ((OPS & OP_TANGENT) != 0) {
    CT acc[DIM];
    sum(region++, acc);
    final_write<DIM, OUT_TAN, VT, CT>(P, A, gid, mask, acc);
  }
  if constexpr ((OPS & OP_DIAG) != 0) {
    CT acc[DIM];
    sum(region++, acc);
    final_write<DIM, OUT_DIAG, VT, CT>(P, A, gid, mask, acc);
  }
}

template <int DIM, int KIND, int OPS, typename VT, typename CT>
static pfem_status run(const DevPlan& P, const OpArgs& A, cudaStream_t s) {
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT> L = smem_layout<CT>(DIM, P.max_local, P.slot_cap, NEED_U, NEED_V);
  if (P.n_tiles > 0) {
    static int attr_done = 0;  // per instantiation; allow the full 227 KB once
    if (!attr_done) {
      PFEM_CUDA(cudaFuncSetAttribute(tile_kernel<DIM, KIND, OPS, VT, CT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
      attr_done = 1;
    }
    if (L.total > 227 * 1024) {
      set_error("tile needs %zu bytes of shared memory", L.total);
      return PFEM_ERR_UNSUPPORTED;
    }
    tile_kernel<DIM, KIND, OPS, VT, CT><<<P.n_tiles, kThreads, L.total, s>>>(P, A); PFEM_COUNT_LAUNCH();
    PFEM_CUDA(cudaGetLastError());
  }
  constexpr int HOPS = OPS & (OP_RESIDUAL | OP_TANGENT | OP_DIAG);
  if constexpr (HOPS != 0) {
    if (P.n_halo > 0) {
      halo_kernel<DIM, HOPS, VT, CT><<<(P.n_halo + 255) / 256, 256, 0, s>>>(P, A); PFEM_COUNT_LAUNCH();
      PFEM_CUDA(cudaGetLastError());
    }
  }
  return PFEM_OK;
}

template <int DIM, int KIND, typename VT, typename CT>
static pfem_status dispatch_ops(const DevPlan& P, int ops, const OpArgs& A, cudaStream_t s) {
  switch (ops) {
    case OP_TANGENT: return run<DIM, KIND, OP_TANGENT, VT, CT>(P, A, s);
    case OP_RESIDUAL: return run<DIM, KIND, OP_RESIDUAL, VT, CT>(P, A, s);
    case OP_ENERGY: return run<DIM, KIND, OP_ENERGY, VT, CT>(P, A, s);
    case OP_DIAG: return run<DIM, KIND, OP_DIAG, VT, CT>(P, A, s);
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
  if (ct == PFEM_F32) return smem_layout<float>(P.dim, P.max_local, P.slot_cap, need_u, need_v).total;
  return smem_layout<double>(P.dim, P.max_local, P.slot_cap, need_u, need_v).total;
}

}  // namespace pfem
