// Multi-right-hand-side tangent action y_j = A v_j, j < k, of the linear element operator in
// one pass over the element data per group of up to kMultiPairs pairs (device code of the
// pairs in multi.cuh). Dirichlet DOFs as in pfem_tangent_apply: v read as 0 there, y = v.

#include "multi.cuh"
#include "solver.h"

namespace pfem {

constexpr int kMultiPairs = 3;  // pairs per launch: their halo partials fill the mesh's scratch

struct MultiArgs {
  const void* v;  // k vectors of n_dofs, vector j at j * n_dofs (VT)
  void* y;        // same layout
  int k;          // vectors in total
  int j0;         // first vector of this launch
  int n_pairs;    // pairs of this launch (<= kMultiPairs)
};

template <int DIM, typename VT>
__global__ void __launch_bounds__(kTileThreads, 2) multi_kernel(DevPlan P, MultiArgs M) {
  extern __shared__ __align__(32) unsigned char smem[];
  const MultiLayout L = multi_layout(P.max_local, P.slot_cap, P.step_cap);
  const int t = blockIdx.x;
  const int4 ta = P.tile_a[t];
  const int4 tb = P.tile_b[t];
  const int fbeg = ta.x, nf = ta.y, lbeg = ta.z, nl = ta.w;
  const int ncomp = tb.x, pbeg = tb.y, sbeg = tb.z, ns = tb.w;
  const int64_t nd = P.n_nodes * DIM;
  float* sx = reinterpret_cast<float*>(smem + L.x);
  int* soff = reinterpret_cast<int*>(smem + L.off);
  int* sinfo = reinterpret_cast<int*>(smem + L.info);
  // ---- static part of the tile, once for every pair
  {
    float2* smat = reinterpret_cast<float2*>(smem + L.smat);
    ushort4* shead = reinterpret_cast<ushort4*>(smem + L.head);
    uint16_t* scode = reinterpret_cast<uint16_t*>(smem + L.scode);
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
      scode[j] = P.step_code[sbeg + j];
      smat[j] = P.step_mat_f[sbeg + j];
    }
    for (int j = threadIdx.x; j < nf; j += blockDim.x) shead[j] = P.fan_head[fbeg + j];
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      const float4 rf = P.lnode_f[lbeg + l];
      st4(sx + 4 * l, rf.x, rf.y, rf.z, 0.f);
      sinfo[l] = __float_as_int(rf.w);
      soff[l] = (int)P.slot_off[lbeg + l];
    }
    if (threadIdx.x == 0) soff[nl] = nf * DIM + ns;
    if (threadIdx.x < kMaxFan) {
      const uint4 c = P.tile_cnt[t];
      const unsigned q = threadIdx.x >> 1;
      const unsigned word = q == 0 ? c.x : (q == 1 ? c.y : (q == 2 ? c.z : c.w));
      reinterpret_cast<int*>(smem + L.fb)[threadIdx.x] = (int)((word >> (16 * (threadIdx.x & 1))) & 0xffffu);
    }
  }
  const VT* v = static_cast<const VT*>(M.v);
  VT* y = static_cast<VT*>(M.y);
  for (int pr = 0; pr < M.n_pairs; ++pr) {
    const int ja = M.j0 + 2 * pr, jb = ja + 1;  // the pair's vectors (jb may be past k)
    const bool has_b = jb < M.k;
    __syncthreads();  // the previous pair's node pass has read its slots
    // ---- the pair's field on the tile's nodes (0 on prescribed DOFs)
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      const unsigned info = (unsigned)sinfo[l];
      const int64_t gid = checked_node((int64_t)(info & kInfoIdMask), P.n_nodes);
      const unsigned mask = info >> kInfoIdBits;
      F2 w[3] = {};
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        const int64_t k = gid * DIM + i;
        const bool fixed = (mask >> i) & 1u;
        w[i].x = fixed ? 0.f : (float)v[(int64_t)ja * nd + k];
        w[i].y = (fixed || !has_b) ? 0.f : (float)v[(int64_t)jb * nd + k];
      }
      st_pair(smem + L.v, l, w, DIM);
    }
    __syncthreads();
    fan_pass_pair<DIM>(smem, L, nf);
    __syncthreads();
    // ---- node sums in rank order; complete nodes written, halo partials in tile order
    unsigned char* part = static_cast<unsigned char*>(P.partial) + (size_t)pr * P.n_partials * 32;
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      F2 acc[3] = {};
      for (int s = soff[l]; s < soff[l + 1]; ++s) {
        F2 d[3];
        ld_pair(smem + L.slot, s, d);
#pragma unroll
        for (int i = 0; i < DIM; ++i) acc[i] = add2(acc[i], d[i]);
      }
      if (l < ncomp) {
        const unsigned info = (unsigned)sinfo[l];
        const int64_t gid = checked_node((int64_t)(info & kInfoIdMask), P.n_nodes);
        const unsigned mask = info >> kInfoIdBits;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int64_t k = gid * DIM + i;
          const bool fixed = (mask >> i) & 1u;
          y[(int64_t)ja * nd + k] = fixed ? v[(int64_t)ja * nd + k] : VT(acc[i].x);
          if (has_b) y[(int64_t)jb * nd + k] = fixed ? v[(int64_t)jb * nd + k] : VT(acc[i].y);
        }
      } else {
        st_pair(part, pbeg + l - ncomp, acc, DIM);
      }
    }
  }
}

// Halo nodes of every pair of a launch: the node's partials summed in ascending tile order.
template <int DIM, typename VT>
__global__ void __launch_bounds__(256) multi_halo_kernel(DevPlan P, MultiArgs M) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int pr = blockIdx.y;
  if (h >= P.n_halo) return;
  const int ja = M.j0 + 2 * pr, jb = ja + 1;
  const bool has_b = jb < M.k;
  const int64_t nd = P.n_nodes * DIM;
  const unsigned char* part = static_cast<const unsigned char*>(P.partial) + (size_t)pr * P.n_partials * 32;
  const int4 rec = P.halo_node[h];
  F2 acc[3] = {};
  for (int m = rec.x; m < rec.x + rec.y; ++m) {
    F2 d[3];
    ld_pair(part, P.halo_seq[m], d);
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc[i] = add2(acc[i], d[i]);
  }
  const unsigned info = (unsigned)rec.z;
  const int64_t gid = checked_node((int64_t)(info & kInfoIdMask), P.n_nodes);
  const unsigned mask = info >> kInfoIdBits;
  const VT* v = static_cast<const VT*>(M.v);
  VT* y = static_cast<VT*>(M.y);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    const int64_t k = gid * DIM + i;
    const bool fixed = (mask >> i) & 1u;
    y[(int64_t)ja * nd + k] = fixed ? v[(int64_t)ja * nd + k] : VT(acc[i].x);
    if (has_b) y[(int64_t)jb * nd + k] = fixed ? v[(int64_t)jb * nd + k] : VT(acc[i].y);
  }
}

template <int DIM, typename VT>
static pfem_status run_multi(const DevPlan& P, const void* v, void* y, int k, cudaStream_t s) {
  const size_t smem = multi_layout(P.max_local, P.slot_cap, P.step_cap).total;
  static int max_dyn = 0;
  pfem_status st = allow_dynamic_smem(multi_kernel<DIM, VT>, smem, &max_dyn);
  if (st) return st;
  for (int j0 = 0; j0 < k; j0 += 2 * kMultiPairs) {
    MultiArgs M{v, y, k, j0, std::min(kMultiPairs, (k - j0 + 1) / 2)};
    if (P.n_tiles > 0) {
      multi_kernel<DIM, VT><<<P.n_tiles, kTileThreads, smem, s>>>(P, M);
      PFEM_COUNT_LAUNCH();
      PFEM_CUDA(cudaGetLastError());
    }
    if (P.n_halo > 0) {
      multi_halo_kernel<DIM, VT><<<dim3((P.n_halo + 255) / 256, M.n_pairs), 256, 0, s>>>(P, M);
      PFEM_COUNT_LAUNCH();
      PFEM_CUDA(cudaGetLastError());
    }
  }
  return PFEM_OK;
}

pfem_status launch_multi_apply(const DevPlan& P, pfem_dtype vt, int k, const void* v, void* y, cudaStream_t s) {
  if (vt == PFEM_F32) return P.dim == 3 ? run_multi<3, float>(P, v, y, k, s) : run_multi<2, float>(P, v, y, k, s);
  return P.dim == 3 ? run_multi<3, double>(P, v, y, k, s) : run_multi<2, double>(P, v, y, k, s);
}

}  // namespace pfem

using namespace pfem;

extern "C" pfem_status pfem_tangent_apply_multi(pfem_mesh_t m, pfem_dtype dt, const void* u, int32_t k,
                                                const void* v, void* y) {
  (void)u;  // linear material: the tangent does not depend on u
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (dt != PFEM_F32 && dt != PFEM_F64_F32) {
    set_error("pfem_tangent_apply_multi: dtype must be PFEM_F32 or PFEM_F64_F32 (FP32 element arithmetic)");
    return PFEM_ERR_UNSUPPORTED;
  }
  if (m->plan.kind != PFEM_LINEAR || m->plan.elem_npe) {
    set_error("pfem_tangent_apply_multi: linear simplex meshes only (use pfem_tangent_apply per vector)");
    return PFEM_ERR_UNSUPPORTED;
  }
  if (k < 0 || (k > 0 && (!v || !y))) {
    set_error("pfem_tangent_apply_multi: k < 0 or v/y is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  if (k == 0) return PFEM_OK;
  const pfem_dtype vt = dt == PFEM_F32 ? PFEM_F32 : PFEM_F64;
  if ((st = launch_multi_apply(m->plan, vt, k, v, y, m->stream))) return st;
  return springs_apply(m, vt, k, v, y, m->stream);
}
