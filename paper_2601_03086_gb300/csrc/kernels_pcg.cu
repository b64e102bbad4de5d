// Persistent Jacobi-PCG kernel (App. B linear system, Sec. "Warm-start"): one cooperative
// launch keeps every CTA resident and runs whole iterations of the two-kernel body of the
// graph mode, with grid barriers where the graph has kernel boundaries:
//
//   A  tiles (round robin over CTAs): p = dinv r + beta p_old on the fly, q = A p, per-tile
//      p_e . A_e p_e; the last tile to finish forms alpha = rho / p.Ap     -> grid barrier
//   B  x += alpha p, r -= alpha q with r.z and r.r per reduction block; the last block to
//      finish sums the blocks in order and updates the state (beta, relative residual,
//      replacement request, termination)                                  -> grid barrier
//
// until the state asks for an FP64 residual replacement or terminates; the host then does
// the replacement and launches again. The arithmetic and every summation order are those of
// the graph body (same tile sum, same kReduceBlocks x 256 update partition), so the iterates
// are bitwise identical to the graph and plain modes.
//
// Data written inside the launch by one CTA and read by another (r, p, q, partial sums, the
// state) is read through L2 only (ld.global.cg). The barrier waits are bounded: a CTA that
// waits longer than the limit flags the barrier, and the solve ends with
// PCG_BARRIER_TIMEOUT instead of hanging.

#include "reduce.cuh"
#include "tile.cuh"

namespace pfem {

// Grid-wide barrier among co-resident CTAs; returns false (in every thread) once any CTA has
// given up waiting. `gen` is thread 0's count of completed barriers.
__device__ __forceinline__ bool grid_barrier(GridBar* b, unsigned int& gen, int* s_flag, long long limit) {
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
        if (err.load(cuda::memory_order_relaxed) != 0 || ++spins > limit) {
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
__global__ void __launch_bounds__(kThreads, 2) pcg_persistent_kernel(DevPlan P, PersistArgs A) {
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ double scratch[16];
  __shared__ double s_beta, s_alpha;
  __shared__ int s_stop, s_iter, s_flag;
  constexpr int OPS = OP_TANGENT | OP_PCG | OP_PERSIST;
  const SmemLayout<float> L = smem_layout<float>(P.max_local, P.slot_cap, P.step_cap, KIND == K_NH, true);
  PcgState* st = A.st;
  unsigned int gen = 0;
  auto read_state = [&]() {  // thread 0; the state was last written by another CTA
    s_stop = (__ldcg(&st->done) != 0 || __ldcg(&st->repl) != 0) ? 1 : 0;
    s_iter = __ldcg(&st->iter);
    s_beta = __ldcg(&st->beta);
  };
  if (threadIdx.x == 0) {
    read_state();
    gen = cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(A.bar->gen).load(cuda::memory_order_acquire);
  }
  __syncthreads();
  if (s_stop) return;  // uniform: written before the launch

  // the apply's arguments live in shared memory (read by every thread, kept out of registers)
  __shared__ OpArgs oa;
  if (threadIdx.x == 0) {
    oa = OpArgs{};
    oa.u = A.u;
    oa.y = A.q;
    oa.load_scale = 1.0;
    oa.pcg.r = A.r;
    oa.pcg.dinv = A.dinv;
    oa.pcg.p[0] = A.p[0];
    oa.pcg.p[1] = A.p[1];
    oa.pcg.st = st;
    oa.pcg.tile_part = A.tile_part;
    oa.pcg.ticket = A.ticket;
  }
  bool ok = true;
  for (;;) {
    // ---- A: direction, q = A p, tile sums of p_e . A_e p_e, alpha by the last tile
    const int odd = s_iter & 1;
    if (threadIdx.x == 0) {
      oa.pcg.beta = s_beta;
      oa.pcg.odd = odd;
    }
    __syncthreads();
    for (int t = blockIdx.x; t < P.n_tiles; t += gridDim.x) {
      process_tile<DIM, KIND, OPS, double, float>(P, oa, t, smem, L);
      __syncthreads();
    }
    // failure-detection test: one CTA leaves without arriving (after its tiles, so the
    // apply's tile ticket is complete); every other CTA's wait runs out
    if ((int)blockIdx.x == A.absent_cta) return;
    if (!(ok = grid_barrier(A.bar, gen, &s_flag, A.spin_limit))) break;
    if (threadIdx.x == 0) {
      s_stop = __ldcg(&st->done) != 0 ? 1 : 0;
      s_alpha = __ldcg(&st->alpha);
    }
    __syncthreads();
    if (s_stop) break;

    // ---- B: x += alpha p, r -= alpha q; the last reduction block updates the state
    {
      const double alpha = s_alpha;
      const double* p = odd ? A.p[0] : A.p[1];  // the direction just formed
      for (int vb = blockIdx.x; vb < kReduceBlocks; vb += gridDim.x) {
        double v[2] = {0.0, 0.0};
        pcg_update_range<2>(A.n, A.x, A.r, p, A.q, A.dinv, alpha, vb, v);
        if (grid_sum_v<2>(v, A.red_part, A.red_counter, scratch, vb, kReduceBlocks) && threadIdx.x == 0)
          pcg_finish_update(st, v[0], v[1]);
      }
    }
    if (!(ok = grid_barrier(A.bar, gen, &s_flag, A.spin_limit))) break;
    if (threadIdx.x == 0) read_state();
    __syncthreads();
    if (s_stop) break;
  }
  if (!ok && threadIdx.x == 0)
    cuda::atomic_ref<int, cuda::thread_scope_device>(st->done).store(PCG_BARRIER_TIMEOUT);
}

template <int DIM, int KIND>
static pfem_status run_persistent(const DevPlan& P, const PersistArgs& a, cudaStream_t s) {
  static int max_dyn = 0;  // per instantiation
  auto kern = pcg_persistent_kernel<DIM, KIND>;
  const size_t smem = smem_layout<float>(P.max_local, P.slot_cap, P.step_cap, KIND == K_NH, true).total;
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
