// Launchers of the element-tile kernels (single mesh, ragged batch, serving steps); the
// device code of a tile lives in tile.cuh.

#include "tile.cuh"

namespace pfem {

// Resident CTAs per SM the register allocation must allow: 4 for the FP32 linear operator
// (more tiles in flight hide the staging and halo latencies), fewer where the arithmetic
// needs more registers (Neo-Hookean, FP64).
template <int KIND, typename CT>
constexpr int tile_min_blocks() {
  return sizeof(CT) == 8 ? 1 : (KIND == K_LIN ? 4 : 3);
}

template <int DIM, int KIND, int OPS, typename VT, typename CT>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<KIND, CT>()) tile_kernel(DevPlan P, OpArgs A) {
  extern __shared__ __align__(32) unsigned char smem[];
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT> L = smem_layout<CT>(P.max_local, P.slot_cap, P.step_cap, NEED_U, NEED_V);
  process_tile<DIM, KIND, OPS, VT, CT>(P, A, blockIdx.x, smem, L);
}

// Ragged batch of 3-D meshes in one launch: CTA b runs tile btile[b].y of mesh btile[b].x
// (FP32 vectors and arithmetic; linear or Neo-Hookean chosen per mesh, uniform per CTA).
template <int OPS>
__global__ void __launch_bounds__(kTileThreads) batch_kernel(BatchDev B, OpArgs A) {
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
  const SmemLayout<float> L = smem_layout<float>(B.max_local, B.slot_cap, B.step_cap, true, NEED_V);
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

template <int OPS>
static pfem_status run_batch(const BatchDev& B, const OpArgs& A, int n_blocks, cudaStream_t s) {
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<float> L = smem_layout<float>(B.max_local, B.slot_cap, B.step_cap, true, NEED_V);
  static int max_dyn = 0;
  pfem_status st = allow_dynamic_smem(batch_kernel<OPS>, L.total, &max_dyn);
  if (st) return st;
  batch_kernel<OPS><<<n_blocks, kTileThreads, L.total, s>>>(B, A);
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

// One kernel per material kind, so that each gets the register budget (and resident CTAs
// per SM) of its own arithmetic, as the single-solve tile kernels do.
template <int KIND>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<KIND, float>())
    serve_apply_kernel(const ReqDev* reqs, const int2* btile, int max_local, int slot_cap, int step_cap) {
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
  const SmemLayout<float> L = smem_layout<float>(max_local, slot_cap, step_cap, KIND == K_NH, true);
  process_tile<3, KIND, OP_TANGENT | OP_PCG, double, float>(sR.plan, a, bt.y, smem, L);
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

pfem_status launch_serve_step(const ReqDev* reqs, const int2* btile, const ServeTiles (&tiles)[2], const int* ublk,
                              int n_update_blocks, cudaStream_t s) {
  static int max_dyn[2] = {0, 0};
  const int2* bt = btile;
  for (int kind = 0; kind < 2; ++kind) {
    const ServeTiles& T = tiles[kind];
    const SmemLayout<float> L = smem_layout<float>(T.max_local, T.slot_cap, T.step_cap, kind == K_NH, true);
    pfem_status st = kind == K_LIN ? allow_dynamic_smem(serve_apply_kernel<K_LIN>, L.total, &max_dyn[0])
                                   : allow_dynamic_smem(serve_apply_kernel<K_NH>, L.total, &max_dyn[1]);
    if (st) return st;
    if (T.n_blocks > 0) {
      if (kind == K_LIN)
        serve_apply_kernel<K_LIN><<<T.n_blocks, kTileThreads, L.total, s>>>(reqs, bt, T.max_local, T.slot_cap,
                                                                             T.step_cap);
      else
        serve_apply_kernel<K_NH><<<T.n_blocks, kTileThreads, L.total, s>>>(reqs, bt, T.max_local, T.slot_cap,
                                                                            T.step_cap);
      PFEM_COUNT_LAUNCH();
    }
    bt += T.n_blocks;
  }
  if (n_update_blocks > 0) {
    serve_update_kernel<<<n_update_blocks, 256, 0, s>>>(reqs, ublk);
    PFEM_COUNT_LAUNCH();
  }
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

// Halo nodes of region `region` after a tile launch with defer_halo: each thread sums one
// node's partials in ascending tile order (the order the in-tile completion uses, so the
// result is the same bit for bit) and writes the output.
template <int DIM, int OUT, typename VT, typename CT>
__global__ void __launch_bounds__(256) halo_finish_kernel(DevPlan P, OpArgs A, int region) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= P.n_halo) return;
  const CT* part = static_cast<const CT*>(P.partial) + (size_t)region * P.n_partials * 4;
  const CT sc = A.out_scale ? CT(*static_cast<const VT*>(A.out_scale)) : CT(1);
  const int4 rec = P.halo_node[h];
  CT sum[4] = {CT(0), CT(0), CT(0), CT(0)};
  const int n_seq = checked_range(rec.x, rec.y, P.n_partials) ? rec.y : 0;
  for (int k = rec.x; k < rec.x + n_seq; ++k) {
    CT t[4];
    int64_t q = P.halo_seq[k];
    if (!checked_range(q, 1, P.n_partials)) q = 0;
    ld4(part + 4 * (size_t)q, t);
#pragma unroll
    for (int i = 0; i < DIM; ++i) sum[i] += t[i];
  }
  const unsigned info = (unsigned)rec.z;
  final_write<DIM, OUT, VT, CT>(P, A, checked_node((int64_t)(info & kInfoIdMask), P.n_nodes), info >> kInfoIdBits,
                                sum, sc);
}

template <int DIM, int OUT, typename VT, typename CT>
static pfem_status finish_halo(const DevPlan& P, const OpArgs& A, int region, cudaStream_t s) {
  if (P.n_halo <= 0) return PFEM_OK;
  halo_finish_kernel<DIM, OUT, VT, CT><<<(P.n_halo + 255) / 256, 256, 0, s>>>(P, A, region);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

template <int DIM, int KIND, int OPS, typename VT, typename CT>
static pfem_status run(const DevPlan& P, const OpArgs& A, cudaStream_t s) {
  constexpr bool NEED_U = (OPS & (OP_RESIDUAL | OP_ENERGY)) || (KIND == K_NH && (OPS & (OP_TANGENT | OP_DIAG)));
  constexpr bool NEED_V = (OPS & OP_TANGENT) != 0;
  const SmemLayout<CT> L = smem_layout<CT>(P.max_local, P.slot_cap, P.step_cap, NEED_U, NEED_V);
  if (P.n_tiles <= 0) return PFEM_OK;
  static int max_dyn = 0;  // per instantiation
  pfem_status st = allow_dynamic_smem(tile_kernel<DIM, KIND, OPS, VT, CT>, L.total, &max_dyn);
  if (st) return st;
  OpArgs a = A;
  a.defer_halo = ((OPS & OP_PCG) == 0 && P.n_partials >= kDeferHaloPartials) ? 1 : 0;
  tile_kernel<DIM, KIND, OPS, VT, CT><<<P.n_tiles, kTileThreads, L.total, s>>>(P, a);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  if (!a.defer_halo) return PFEM_OK;
  int region = 0;  // regions in the order the tile kernel fills them
  if constexpr ((OPS & OP_RESIDUAL) != 0)
    if ((st = finish_halo<DIM, OUT_RES, VT, CT>(P, a, region++, s))) return st;
  if constexpr ((OPS & OP_TANGENT) != 0)
    if ((st = finish_halo<DIM, OUT_TAN, VT, CT>(P, a, region++, s))) return st;
  if constexpr ((OPS & OP_DIAG) != 0)
    if ((st = finish_halo<DIM, OUT_DIAG, VT, CT>(P, a, region++, s))) return st;
  (void)region;
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
  if (P.elem_npe) return launch_quad_op(P, ops, vt, ct, a, s);
  if (vt == PFEM_F32 && ct == PFEM_F32) return dispatch_kind<float, float>(P, ops, a, s);
  if (vt == PFEM_F64 && ct == PFEM_F32) return dispatch_kind<double, float>(P, ops, a, s);
  if (vt == PFEM_F64 && ct == PFEM_F64) return dispatch_kind<double, double>(P, ops, a, s);
  set_error("unsupported dtype combination");
  return PFEM_ERR_UNSUPPORTED;
}

size_t element_op_smem(const DevPlan& P, int ops, pfem_dtype ct) {
  const bool need_u = (ops & (OP_RESIDUAL | OP_ENERGY)) || (P.kind == PFEM_NEOHOOKEAN && (ops & (OP_TANGENT | OP_DIAG)));
  const bool need_v = (ops & OP_TANGENT) != 0;
  if (ct == PFEM_F32) return smem_layout<float>(P.max_local, P.slot_cap, P.step_cap, need_u, need_v).total;
  return smem_layout<double>(P.max_local, P.slot_cap, P.step_cap, need_u, need_v).total;
}

}  // namespace pfem
