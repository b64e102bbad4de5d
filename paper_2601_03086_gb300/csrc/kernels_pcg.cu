// Persistent Jacobi-PCG kernel (App. B linear system, Sec. 2.3.2 warm start): one cooperative
// launch keeps every CTA resident and runs whole iterations of the two-kernel body
//
//   A  tiles (round robin over CTAs): p = dinv r + beta p_old on the fly, q = A p,
//      per-tile p_e . A_e p_e                                    -> grid barrier
//   B  alpha = rho / sum(tile sums); x += alpha p, r -= alpha q, partial r.z and r.r per
//      virtual reduction block                                   -> grid barrier
//   C  every CTA sums the partials in the same order and takes the same decision
//      (beta, relative residual, replacement request, termination)
//
// until the state asks for an FP64 residual replacement or terminates; the host then does
// the replacement and launches again. The arithmetic and every summation order are those of
// the two-kernel body (the same tile partial sum, the same kReduceBlocks x 256 partition of
// the update reduction), so the iterates are bitwise identical to the graph and plain modes.
//
// Vectors written inside the launch by one CTA and read by another (r, p, q, the partial
// sums) are read through L2 only (ld.global.cg). The barrier waits are bounded: a CTA that
// waits longer than the limit flags the barrier, and the solve ends with
// PCG_BARRIER_TIMEOUT instead of hanging.

#include "reduce.cuh"
#include "tile.cuh"

namespace pfem {

constexpr long long kBarrierSpinLimit = 1ll << 25;  // x >= 32 ns sleep: more than a second

// Grid-wide barrier among co-resident CTAs; returns false (in every thread) once any CTA has
// given up waiting. `gen` is thread 0's count of completed barriers.
__device__ __forceinline__ bool grid_barrier(GridBar* b, unsigned int& gen, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(b->count);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> g(b->gen);
    cuda::atomic_ref<int, cuda::thread_scope_device> err(b->err);
    __threadfence();
    int bad = 0;
    if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      g.store(gen + 1u, cuda::memory_order_release);
    } else {
      long long spins = 0;
      while (g.load(cuda::memory_order_acquire) == gen) {
        if (err.load(cuda::memory_order_relaxed) != 0 || ++spins > kBarrierSpinLimit) {
          err.store(1, cuda::memory_order_relaxed);
          bad = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen += 1u;
    *s_flag = bad | err.load(cuda::memory_order_relaxed);
  }
  __syncthreads();
  return *s_flag == 0;
}

template <int DIM, int KIND>
__global__ void __launch_bounds__(kThreads) pcg_persistent_kernel(DevPlan P, PersistArgs A) {
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ PcgState s_st;
  __shared__ double scratch[16];
  __shared__ int s_flag;
  constexpr int OPS = OP_TANGENT | OP_PCG | OP_PERSIST;
  const SmemLayout<float> L = smem_layout<float>(P.max_local, P.slot_cap, KIND == K_NH, true);
  unsigned int gen = 0;
  if (threadIdx.x == 0) {
    s_st = *A.st;
    gen = cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(A.bar->gen).load(cuda::memory_order_acquire);
  }
  __syncthreads();
  if (s_st.done != 0 || s_st.repl != 0) return;  // uniform: written before the launch

  OpArgs oa{};
  oa.u = A.u;
  oa.y = A.q;
  oa.load_scale = 1.0;
  oa.pcg.r = A.r;
  oa.pcg.dinv = A.dinv;
  oa.pcg.p[0] = A.p[0];
  oa.pcg.p[1] = A.p[1];
  oa.pcg.st = A.st;
  oa.pcg.tile_part = A.tile_part;
  bool ok = true;
  for (;;) {
    // ---- A: direction, q = A p, tile sums of p_e . A_e p_e
    oa.pcg.beta = s_st.beta;
    oa.pcg.odd = s_st.iter & 1;
    for (int t = blockIdx.x; t < P.n_tiles; t += gridDim.x) {
      process_tile<DIM, KIND, OPS, double, float>(P, oa, t, smem, L);
      __syncthreads();
    }
    if (!(ok = grid_barrier(A.bar, gen, &s_flag))) break;

    // ---- alpha = rho / p.Ap (the fused apply's last-tile sum, in every CTA)
    {
      double s = 0.0;
      for (int i = threadIdx.x; i < P.n_tiles; i += blockDim.x) s += __ldcg(A.tile_part + i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double pap = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pap += scratch[w];
        if (pap == 0.0 || !isfinite(pap)) {
          s_st.alpha = 0.0;
          s_st.done = isfinite(pap) ? PCG_BREAKDOWN : PCG_NONFINITE;
        } else {
          s_st.alpha = s_st.rho / pap;
        }
      }
      __syncthreads();
      if (s_st.done != 0) break;
    }

    // ---- B: x += alpha p, r -= alpha q; r.z and r.r partials of virtual block vb
    {
      const double alpha = s_st.alpha;
      const double* p = oa.pcg.odd ? A.p[0] : A.p[1];  // the direction just formed
      for (int vb = blockIdx.x; vb < kReduceBlocks; vb += gridDim.x) {
        double v[2] = {0.0, 0.0};
        for (int64_t i = (int64_t)vb * kReduceThreads + threadIdx.x; i < A.n;
             i += (int64_t)kReduceBlocks * kReduceThreads) {
          A.x[i] += alpha * __ldcg(p + i);
          const double ri = __ldcg(A.r + i) - alpha * __ldcg(A.q + i);
          A.r[i] = ri;
          v[0] += ri * (A.dinv[i] * ri);
          v[1] += ri * ri;
        }
        block_sum<2>(v, scratch);
        if (threadIdx.x == 0) {
          A.red_part[vb * 2] = v[0];
          A.red_part[vb * 2 + 1] = v[1];
        }
      }
    }
    if (!(ok = grid_barrier(A.bar, gen, &s_flag))) break;

    // ---- C: totals in block order, then the iteration's bookkeeping (same in every CTA)
    {
      double acc[2] = {0.0, 0.0};
      for (int b = threadIdx.x; b < kReduceBlocks; b += blockDim.x) {
        acc[0] += __ldcg(A.red_part + b * 2);
        acc[1] += __ldcg(A.red_part + b * 2 + 1);
      }
      block_sum<2>(acc, scratch);
      if (threadIdx.x == 0) pcg_finish_update(&s_st, acc[0], acc[1]);
      __syncthreads();
      if (s_st.done != 0 || s_st.repl != 0) break;
    }
  }
  if (threadIdx.x == 0) {
    if (!ok && s_st.done == 0) s_st.done = PCG_BARRIER_TIMEOUT;
    if (blockIdx.x == 0) *A.st = s_st;
    if (!ok) cuda::atomic_ref<int, cuda::thread_scope_device>(A.st->done).store(PCG_BARRIER_TIMEOUT);
  }
}

template <int DIM, int KIND>
static pfem_status run_persistent(const DevPlan& P, const PersistArgs& a, cudaStream_t s) {
  static int max_dyn = 0;  // per instantiation
  auto kern = pcg_persistent_kernel<DIM, KIND>;
  const size_t smem = smem_layout<float>(P.max_local, P.slot_cap, KIND == K_NH, true).total;
  pfem_status st = allow_dynamic_smem(kern, smem, &max_dyn);
  if (st) return st;
  int dev = 0, n_sm = 0, nb = 0;
  PFEM_CUDA(cudaGetDevice(&dev));
  PFEM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  PFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem));
  if (nb < 1) {
    set_error("persistent PCG kernel: no co-resident grid");
    return PFEM_ERR_UNSUPPORTED;
  }
  const int grid = nb * n_sm;
  PFEM_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(GridBar), s));
  DevPlan pc = P;
  PersistArgs ac = a;
  void* args[2] = {&pc, &ac};
  PFEM_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kThreads), args, smem, s));
  PFEM_COUNT_LAUNCH();
  return PFEM_OK;
}

pfem_status launch_pcg_persistent(const DevPlan& P, pfem_dtype ct, const PersistArgs& a, cudaStream_t s) {
  if (ct == PFEM_F64) {
    set_error("persistent PCG kernel runs FP32 element arithmetic only");
    return PFEM_ERR_UNSUPPORTED;
  }
  if (P.n_tiles < 1) {
    set_error("persistent PCG kernel: empty plan");
    return PFEM_ERR_UNSUPPORTED;
  }
  if (P.dim == 3) {
    if (P.kind == PFEM_LINEAR) return run_persistent<3, K_LIN>(P, a, s);
    return run_persistent<3, K_NH>(P, a, s);
  }
  if (P.kind == PFEM_LINEAR) return run_persistent<2, K_LIN>(P, a, s);
  return run_persistent<2, K_NH>(P, a, s);
}

}  // namespace pfem
