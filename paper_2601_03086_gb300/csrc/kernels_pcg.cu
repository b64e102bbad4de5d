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

// Grid barrier whose last CTA to arrive runs last() with all its threads (it has seen every
// other CTA's writes) and publishes scalars before it releases the others; thread 0 of every
// other CTA runs receive() once released (the scalars share the released word's line).
// Returns false (in every thread) once any CTA has given up waiting.
template <typename Last, typename Receive>
__device__ __forceinline__ bool grid_barrier_last(GridBar* b, unsigned int& gen, int* s_flag, int* s_last,
                                                  long long limit, Last&& last, Receive&& receive) {
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(b->count);
  cuda::atomic_ref<unsigned int, cuda::thread_scope_device> g(b->gen);
  cuda::atomic_ref<int, cuda::thread_scope_device> err(b->err);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *s_last = cnt.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (*s_last) {
    last();
    __syncthreads();
    if (threadIdx.x == 0) {
      cnt.store(0u, cuda::memory_order_relaxed);
      g.store(gen + 1u, cuda::memory_order_release);
      gen += 1u;
      *s_flag = err.load(cuda::memory_order_relaxed);
    }
  } else if (threadIdx.x == 0) {
    int bad = 0;
    long long spins = 0;
    while (g.load(cuda::memory_order_acquire) == gen) {
      if (err.load(cuda::memory_order_relaxed) != 0 || ++spins > limit) {
        err.store(1, cuda::memory_order_relaxed);
        bad = 1;
        break;
      }
      __nanosleep(32);
    }
    gen += 1u;
    *s_flag = bad | err.load(cuda::memory_order_relaxed);
    if (!*s_flag) receive();
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

// ---- tile-resident persistent kernel ----------------------------------------------------
//
// When every tile of the mesh fits on the GPU at once (one CTA per tile, all co-resident),
// each CTA keeps its tile's static data in shared memory for the whole launch: step records,
// fan heads, node coordinates, ids and slot offsets (and u for a Newton inner solve) are
// staged once, and an iteration only gathers the new direction of the tile's nodes. Halo
// nodes are not finished inside the apply: tiles publish their partials (no fences, no
// tickets; the grid barrier orders them) and the update phase sums a halo DOF's partials in
// ascending tile order when it reaches that DOF, forming its direction from the same formula
// the tiles used. Every value and every summation order are those of the two-kernel body
// (same tile sums, same 296 x 256 update partition, same partial order), so the iterates
// stay bitwise identical to the graph and plain modes.

// Shared memory of the resident kernel: the tile layout plus one partial index per tile node.
template <int KIND>
__host__ __device__ inline size_t resident_smem(const DevPlan& P, size_t* hslot_off) {
  const SmemLayout<float> L = smem_layout<float>(P.max_local, P.slot_cap, P.step_cap, KIND == K_NH, true);
  *hslot_off = L.total;
  return L.total + (((size_t)P.max_local * sizeof(int) + 31) & ~size_t(31));
}

template <int DIM, int KIND>
__device__ __forceinline__ void resident_stage_static(const DevPlan& P, const double* u, int t, unsigned char* smem,
                                                      const SmemLayout<float>& L, int* hslot) {
  const int4 ta = P.tile_a[t];
  const int4 tb = P.tile_b[t];
  const int fbeg = ta.x, nf = ta.y, lbeg = ta.z, nl = ta.w;
  const int ncomp = tb.x, pbeg = tb.y, sbeg = tb.z, ns = tb.w;
  float* sx = reinterpret_cast<float*>(smem + L.x);
  float* su = reinterpret_cast<float*>(smem + L.u);
  int* soff = reinterpret_cast<int*>(smem + L.off);
  int* sinfo = reinterpret_cast<int*>(smem + L.info);
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
    hslot[l] = l >= ncomp ? P.halo_rec[pbeg + l - ncomp].x : -1;
    if constexpr (KIND == K_NH) {
      const int64_t gid = checked_node((int64_t)((unsigned)__float_as_int(rf.w) & kInfoIdMask), P.n_nodes);
      float w[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < DIM; ++i) w[i] = (float)u[gid * DIM + i];
      st4(su + 4 * l, w[0], w[1], w[2], 0.f);
    }
  }
  if (threadIdx.x == 0) soff[nl] = nf * DIM + ns;
  if (threadIdx.x < kMaxFan) {
    const uint4 c = P.tile_cnt[t];
    const unsigned q = threadIdx.x >> 1;
    const unsigned word = q == 0 ? c.x : (q == 1 ? c.y : (q == 2 ? c.z : c.w));
    reinterpret_cast<int*>(smem + L.fb)[threadIdx.x] = (int)((word >> (16 * (threadIdx.x & 1))) & 0xffffu);
  }
}

template <int DIM, int KIND>
__global__ void __launch_bounds__(kTileThreads, KIND == K_LIN ? 4 : 3)
    pcg_resident_kernel(DevPlan P, PersistArgs A) {
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ double scratch[16];
  // the solve's scalars, kept per CTA (every CTA takes the same decisions from the same
  // totals; CTA 0 writes them back to the state for the host)
  __shared__ double s_beta, s_alpha, s_rho, s_ref, s_tol, s_thr;
  __shared__ int s_stop, s_iter, s_trunc, s_maxit, s_flag, s_last;
  __shared__ int s_nf, s_nl, s_ncomp;  // tile shape (kept in shared memory, out of registers)
  __shared__ SmemLayout<float> L;      // shared-memory layout (likewise)
  __shared__ size_t s_hoff;
  // the launch arguments, read from shared memory inside the iteration loop: kernel
  // parameters used in the loop would otherwise be held in registers across the fan pass
  __shared__ PersistArgs sA;
  __shared__ DevPlan sP;
  PcgState* st = A.st;
  const int t = blockIdx.x;
  unsigned int gen = 0;
  if (threadIdx.x == 0) {
    sA = A;
    sP = P;
    L = smem_layout<float>(P.max_local, P.slot_cap, P.step_cap, KIND == K_NH, true);
    resident_smem<KIND>(P, &s_hoff);
    s_nf = P.tile_a[t].y;
    s_nl = P.tile_a[t].w;
    s_ncomp = P.tile_b[t].x;
    s_stop = (st->done != 0 || st->repl != 0) ? 1 : 0;  // written before the launch
    s_iter = st->iter;
    s_beta = st->beta;
    s_rho = st->rho;
    s_trunc = st->truncate;
    s_maxit = st->max_iter;
    s_ref = st->ref;
    s_tol = st->tol;
    s_thr = st->repl_threshold;
    gen = cuda::atomic_ref<unsigned int, cuda::thread_scope_device>(A.bar->gen).load(cuda::memory_order_acquire);
  }
  __syncthreads();
  resident_stage_static<DIM, KIND>(P, A.u, t, smem, L, reinterpret_cast<int*>(smem + s_hoff));
  __syncthreads();
  if (s_stop) return;  // uniform
  bool ok = true;
  for (;;) {
    // ---- A: this iteration's direction on the tile's nodes, q = A p, tile sum of p_e.A_e p_e
    {
      const int* sinfo = reinterpret_cast<const int*>(smem + L.info);
      float* sv = reinterpret_cast<float*>(smem + L.v);
      const bool odd = (s_iter & 1) != 0;
      const double beta = s_beta;
      const double* p_old = odd ? sA.p[1] : sA.p[0];
      double* p_new = odd ? sA.p[0] : sA.p[1];
      for (int l = threadIdx.x, nl = s_nl, ncomp = s_ncomp; l < nl; l += blockDim.x) {
        const unsigned info = (unsigned)sinfo[l];
        const int64_t gid = checked_node((int64_t)(info & kInfoIdMask), P.n_nodes);
        const unsigned mask = info >> kInfoIdBits;
        float w[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          const int64_t k = gid * DIM + i;
          const bool fixed = (mask >> i) & 1u;
          const double pn = fixed ? 0.0 : fma(sA.dinv[k], __ldcg(sA.r + k), beta * __ldcg(p_old + k));
          if (l < ncomp) p_new[k] = pn;  // complete nodes: this tile owns the DOF
          w[i] = (float)pn;
        }
        st4(sv + 4 * l, w[0], w[1], w[2], 0.f);
      }
    }
    __syncthreads();
    double e_acc = 0.0;
    {
      int n_inv = 0;
      fan_pass<DIM, KIND, OUT_TAN, false, false, float>(smem, L, s_nf, e_acc, n_inv);
    }
    __syncthreads();
    {
      const int* sinfo = reinterpret_cast<const int*>(smem + L.info);
      const int* soff = reinterpret_cast<const int*>(smem + L.off);
      const int* hslot = reinterpret_cast<const int*>(smem + s_hoff);
      const float* slot = reinterpret_cast<const float*>(smem + L.slot);
      const float* sv = reinterpret_cast<const float*>(smem + L.v);
      float* part = static_cast<float*>(sP.partial);
      for (int l = threadIdx.x, nl = s_nl, ncomp = s_ncomp; l < nl; l += blockDim.x) {
        const int b = soff[l], e = soff[l + 1];
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = b; k < e; ++k) {
          float tt[4];
          ld4(slot + 4 * k, tt);
#pragma unroll
          for (int i = 0; i < DIM; ++i) acc[i] += tt[i];
        }
        e_acc += pap_node<DIM, float>(sv + 4 * l, acc);  // as node_pass
        if (l < ncomp) {
          const unsigned info = (unsigned)sinfo[l];
          const int64_t gid = checked_node((int64_t)(info & kInfoIdMask), P.n_nodes);
#pragma unroll
          for (int i = 0; i < DIM; ++i)
            sA.q[gid * DIM + i] = ((info >> (kInfoIdBits + i)) & 1u) ? 0.0 : (double)acc[i];
        } else {
          st4(part + 4 * (size_t)hslot[l], acc[0], acc[1], acc[2], 0.f);
        }
      }
    }
    // tile sum of p_e . A_e p_e: warp butterflies, warps in index order (as process_tile)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = e_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += scratch[w];
      sA.tile_part[t] = s;
    }
    if (t == sA.absent_cta) return;  // failure-detection test (see PersistArgs)
    // barrier; the last CTA forms alpha = rho / p.Ap from the tile sums (the order of the
    // other modes) and publishes it
    ok = grid_barrier_last(
        sA.bar, gen, &s_flag, &s_last, sA.spin_limit,
        [&] {
          const double pap = pcg_tile_total(sA.tile_part, sP.n_tiles, scratch);
          if (threadIdx.x == 0) {
            double a = 0.0;
            const int stop = pcg_alpha(pap, s_rho, s_trunc, s_iter, &a);
            s_alpha = a;
            s_stop = stop != 0;
            sA.bar->b_alpha = a;
            sA.bar->b_stop = stop;
            st->alpha = a;
            if (stop) st->done = stop;
          }
        },
        [&] {
          s_alpha = __ldcg(&sA.bar->b_alpha);
          s_stop = __ldcg(&sA.bar->b_stop) != 0;
        });
    if (!ok || s_stop) break;

    // ---- B: for each update block of this CTA: halo DOFs summed from their partials,
    // x += alpha p, r -= alpha q and the block's r.z, r.r
    {
      const bool odd = (s_iter & 1) != 0;
      const double beta = s_beta;
      const double* p_old = odd ? sA.p[1] : sA.p[0];
      double* p_new = odd ? sA.p[0] : sA.p[1];
      const float* part = static_cast<const float*>(sP.partial);
      const int64_t S = (int64_t)kReduceBlocks * kReduceThreads;
      constexpr int U = 2;  // DOFs per thread whose loads go out together (register budget)
      double rr[U], dd[U], xx[U], pp[U], qq[U];
      int2 np[U];
      bool fx[U];
      auto load = [&](int64_t i0) {  // every load of a chunk, independent of one another
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const int64_t k = i0 + j * S;
          if (k < sA.n) {
            np[j] = sP.node_part[k / DIM];
            rr[j] = __ldcg(sA.r + k);
            dd[j] = sA.dinv[k];
            xx[j] = sA.x[k];
            pp[j] = __ldcg(p_new + k);
            qq[j] = __ldcg(sA.q + k);
            fx[j] = sP.dmask[k] != 0;
          }
        }
      };
      auto finish = [&](int64_t i0, double alpha, double (&v)[2]) {
#pragma unroll
        for (int j = 0; j < U; ++j) {  // halo DOFs: direction and A p from the partials
          const int64_t k = i0 + j * S;
          if (k < sA.n && np[j].y != 0) {
            if (fx[j]) {
              pp[j] = 0.0;
              qq[j] = 0.0;
            } else {
              const float* pk = part + 4 * (size_t)np[j].x + (int)(k % DIM);
              float pt[4];
#pragma unroll
              for (int m = 0; m < 4; ++m) pt[m] = m < np[j].y ? __ldcg(pk + 4 * m) : 0.f;
              const double po = __ldcg(p_old + k);
              float qs = 0.f;
#pragma unroll
              for (int m = 0; m < 4; ++m)
                if (m < np[j].y) qs += pt[m];
              for (int m = 4; m < np[j].y; ++m) qs += __ldcg(pk + 4 * m);
              qq[j] = (double)qs;
              pp[j] = fma(dd[j], rr[j], beta * po);
            }
            p_new[k] = pp[j];
          }
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {  // same arithmetic and order as pcg_update_range
          const int64_t k = i0 + j * S;
          if (k < sA.n) {
            sA.x[k] = xx[j] + alpha * pp[j];
            const double ri = rr[j] - alpha * qq[j];
            sA.r[k] = ri;
            v[0] += ri * (dd[j] * ri);
            v[1] += ri * ri;
          }
        }
      };
      const double alpha = s_alpha;
      for (int vb = t; vb < kReduceBlocks; vb += gridDim.x) {
        double v[2] = {0.0, 0.0};
        for (int64_t i0 = (int64_t)vb * kReduceThreads + threadIdx.x; i0 < sA.n; i0 += U * S) {
          load(i0);
          finish(i0, alpha, v);
        }
        block_sum<2>(v, scratch);
        if (threadIdx.x == 0) {
          sA.red_part[2 * vb] = v[0];
          sA.red_part[2 * vb + 1] = v[1];
        }
      }
    }
    // barrier; the last CTA sums the update blocks' partials in block order (the order of the
    // last block in the other modes), takes the iteration's decision, writes the state for the
    // host and publishes the next iteration's scalars
    ok = grid_barrier_last(
        sA.bar, gen, &s_flag, &s_last, sA.spin_limit,
        [&] {
          double acc[2] = {0.0, 0.0};
          for (int b = threadIdx.x; b < kReduceBlocks; b += blockDim.x) {
            acc[0] += __ldcg(sA.red_part + 2 * b);
            acc[1] += __ldcg(sA.red_part + 2 * b + 1);
          }
          block_sum<2>(acc, scratch);
          if (threadIdx.x == 0) {
            const PcgStep s = pcg_decide(s_iter, 0, s_maxit, s_ref, s_tol, s_thr, s_rho, acc[0], acc[1]);
            s_iter = s.iter;
            if (s.next) {
              s_beta = s.beta;
              s_rho = s.rho;
            }
            s_stop = (s.done != 0 || s.repl != 0) ? 1 : 0;
            st->iter = s.iter;
            st->rel = s.rel;
            if (s.done) st->done = s.done;
            if (s.repl) st->repl = 1;
            if (s.next) {
              st->beta = s.beta;
              st->rho = s.rho;
            }
            sA.bar->b_iter = s_iter;
            sA.bar->b_beta = s_beta;
            sA.bar->b_rho = s_rho;
            sA.bar->b_stop = s_stop;
          }
        },
        [&] {
          s_iter = __ldcg(&sA.bar->b_iter);
          s_beta = __ldcg(&sA.bar->b_beta);
          s_rho = __ldcg(&sA.bar->b_rho);
          s_stop = __ldcg(&sA.bar->b_stop);
        });
    if (!ok || s_stop) break;
  }
  if (!ok && threadIdx.x == 0)
    cuda::atomic_ref<int, cuda::thread_scope_device>(st->done).store(PCG_BARRIER_TIMEOUT);
}

// Launches the resident kernel if every tile fits co-resident; PFEM_ERR_UNSUPPORTED (no side
// effects) otherwise.
template <int DIM, int KIND>
static pfem_status run_resident(const DevPlan& P, const PersistArgs& a, cudaStream_t s) {
  static int max_dyn = 0;  // per instantiation
  auto kern = pcg_resident_kernel<DIM, KIND>;
  size_t hoff;
  const size_t smem = resident_smem<KIND>(P, &hoff);
  pfem_status st = allow_dynamic_smem(kern, smem, &max_dyn);
  if (st) return st;
  int dev = 0, n_sm = 0, nb = 0;
  PFEM_CUDA(cudaGetDevice(&dev));
  PFEM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  PFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kTileThreads, smem));
  if ((int64_t)nb * n_sm < P.n_tiles) {
    set_error("resident PCG kernel: %d tiles exceed the %d co-resident CTAs", P.n_tiles, nb * n_sm);
    return PFEM_ERR_UNSUPPORTED;
  }
  PFEM_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(GridBar), s));
  DevPlan pc = P;
  PersistArgs ac = a;
  void* args[2] = {&pc, &ac};
  PFEM_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(P.n_tiles), dim3(kTileThreads), args, smem, s));
  PFEM_COUNT_LAUNCH();
  return PFEM_OK;
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
  if (P.n_tiles < 1 || P.elem_npe) {
    set_error("persistent PCG kernel: empty plan or quadrilateral mesh");
    return PFEM_ERR_UNSUPPORTED;
  }
  // one resident CTA per tile where the whole mesh fits on the GPU at once, else CTAs that
  // loop over tiles and stage each tile in every iteration
  pfem_status st;
  if (P.dim == 3) {
    st = P.kind == PFEM_LINEAR ? run_resident<3, K_LIN>(P, a, s) : run_resident<3, K_NH>(P, a, s);
    if (st != PFEM_ERR_UNSUPPORTED) return st;
    if (P.kind == PFEM_LINEAR) return run_persistent<3, K_LIN>(P, a, s);
    return run_persistent<3, K_NH>(P, a, s);
  }
  st = P.kind == PFEM_LINEAR ? run_resident<2, K_LIN>(P, a, s) : run_resident<2, K_NH>(P, a, s);
  if (st != PFEM_ERR_UNSUPPORTED) return st;
  if (P.kind == PFEM_LINEAR) return run_persistent<2, K_LIN>(P, a, s);
  return run_persistent<2, K_NH>(P, a, s);
}

}  // namespace pfem
