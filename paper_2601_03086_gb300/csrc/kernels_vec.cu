// Vector kernels: energy finalisation and the Jacobi-PCG recurrences (FP64 vectors, FP64
// dots and norms, deterministic reductions).

#include "kernels_vec.cuh"
#include "pcg_state.cuh"
#include "reduce.cuh"

namespace pfem {

// ---- energy ------------------------------------------------------------------------------

template <typename VT>
__global__ void __launch_bounds__(kReduceThreads)
    energy_finalize_kernel(int n_tiles, const double* tile_energy, int64_t n_dofs, const double* f_ext, const VT* u,
                           double s, double* partials, unsigned int* counter, double* out) {
  __shared__ double scratch[16];
  double v[2] = {0.0, 0.0};
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tiles; i += stride) v[0] += tile_energy[i];
  for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_dofs; i += stride) v[1] += f_ext[i] * (double)u[i];
  if (grid_sum<2>(v, partials, counter, scratch) && threadIdx.x == 0) {
    out[1] = v[0];
    out[0] = v[0] - s * v[1];
  }
}

pfem_status launch_energy_finalize(const DevPlan& P, pfem_dtype vt, const void* u, double s, double* partials,
                                   unsigned int* counter, double* out, cudaStream_t st) {
  const int64_t nd = P.n_nodes * P.dim;
  if (vt == PFEM_F32)
    energy_finalize_kernel<float><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        P.n_tiles, P.tile_energy, nd, P.f_ext, static_cast<const float*>(u), s, partials, counter, out);
  else
    energy_finalize_kernel<double><<<kReduceBlocks, kReduceThreads, 0, st>>>(
        P.n_tiles, P.tile_energy, nd, P.f_ext, static_cast<const double*>(u), s, partials, counter, out);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

// ---- PCG ---------------------------------------------------------------------------------

// x = u0 (or 0) with x = s * values on prescribed DOFs
__global__ void lift_kernel(int64_t n, const double* u0, const double* values, const uint8_t* mask, double s,
                            double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = mask[i] ? s * values[i] : (u0 ? u0[i] : 0.0);
}

// dinv = 1 / d (1 where d is not positive: orphan free DOFs keep a unit scaling)
template <typename T>
__global__ void invert_diag_kernel(int64_t n, const T* d, double* dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)d[i];
    dinv[i] = v > 0.0 ? 1.0 / v : 1.0;
  }
}

// alpha = rho / p.Ap from the fused apply's tile sums (every block forms it, in the same
// order: same bits), then x += alpha p; r -= alpha q; (r.z, r.r) with z = dinv r; flags and
// beta in the last block. p is this iteration's direction, p_buf[(iter + 1) & 1]. The first
// chunk's vector loads are issued before the tile sum, so the two latencies overlap.
__global__ void __launch_bounds__(kReduceThreads)
    pcg_update_kernel(int64_t n, double* x, double* r, const double* p0, const double* p1, const double* q,
                      const double* dinv, PcgState* st, const double* tile_part, int n_tiles, double* partials,
                      unsigned int* counter, cudaGraphConditionalHandle cond, int set_cond) {
  __shared__ double scratch[16];
  __shared__ double s_alpha;
  __shared__ int s_stop;
  // every state field this kernel reads, loaded before the branch (one round trip); rho is
  // rewritten only by the last block, after every block has read it
  const int done = st->done, repl = st->repl, it = st->iter, trunc = st->truncate;
  const double rho = st->rho;
  if (done != 0 || repl != 0) {  // nothing to do (uniform: written by earlier kernels)
    if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      st->bodies += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  const double* p = ((it + 1) & 1) ? p1 : p0;
  constexpr int U = 4;
  const int64_t S = (int64_t)kReduceBlocks * kReduceThreads;
  const int64_t i0 = (int64_t)blockIdx.x * kReduceThreads + threadIdx.x;
  double pp[U], qq[U], rr[U], dd[U], xx[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int64_t k = i0 + j * S;
    if (k < n) {
      pp[j] = __ldcg(p + k);
      qq[j] = __ldcg(q + k);
      rr[j] = __ldcg(r + k);
      dd[j] = dinv[k];
      xx[j] = x[k];
    }
  }
  const double pap = pcg_tile_total(tile_part, n_tiles, scratch);
  if (threadIdx.x == 0) {
    double a = 0.0;
    s_stop = pcg_alpha(pap, rho, trunc, it, &a);
    s_alpha = a;
    if (blockIdx.x == 0) {  // for the host; nothing in this launch reads it back
      st->alpha = a;
      if (s_stop) {
        st->done = s_stop;
        if (set_cond) {
          st->bodies += 1;
          cudaGraphSetConditional(cond, 0u);
        }
      }
    }
  }
  __syncthreads();
  if (s_stop) return;  // uniform: every block formed the same p.Ap
  const double alpha = s_alpha;
  double v[2] = {0.0, 0.0};
#pragma unroll
  for (int j = 0; j < U; ++j) {  // same arithmetic and order as pcg_update_range
    const int64_t k = i0 + j * S;
    if (k < n) {
      x[k] = xx[j] + alpha * pp[j];
      const double ri = rr[j] - alpha * qq[j];
      r[k] = ri;
      v[0] += ri * (dd[j] * ri);
      v[1] += ri * ri;
    }
  }
  if (i0 + U * S < n)  // the rest (meshes of more than U x 296 x 256 DOFs)
    pcg_update_range_from<U>(n, x, r, p, q, dinv, alpha, i0 + U * S, v);
  if (grid_sum<2>(v, partials, counter, scratch) && threadIdx.x == 0) {
    pcg_finish_update(st, v[0], v[1]);
    if (set_cond) {
      st->bodies += 1;
      cudaGraphSetConditional(cond, (st->done == 0 && st->repl == 0) ? 1u : 0u);
    }
  }
}

// Residual replacement / (re)start: r = -res (res = P (f_int(x) - f), FP64 operator),
// rz = r.dinv r, rr = r.r; last block decides convergence and the new beta.
// restart != 0: beta = 0 (p = z) and rho = rz.
__global__ void __launch_bounds__(kReduceThreads)
    pcg_replace_kernel(int64_t n, const double* res, double* r, const double* dinv, PcgState* st, int restart,
                       double* partials, unsigned int* counter) {
  __shared__ double scratch[16];
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = -res[i];
    r[i] = ri;
    v[0] += ri * (dinv[i] * ri);
    v[1] += ri * ri;
  }
  if (grid_sum<2>(v, partials, counter, scratch) && threadIdx.x == 0) {
    const double rel = sqrt(v[1]) / st->ref;
    st->rel_true = rel;
    st->rel = rel;
    st->repl = 0;
    st->replacements += restart ? 0 : 1;
    if (!isfinite(v[1]) || !isfinite(v[0])) {
      st->done = PCG_NONFINITE;
    } else if (rel < st->tol) {
      st->done = PCG_CONVERGED;
    } else if (st->iter >= st->max_iter) {
      st->done = PCG_MAXITER;
    } else {
      st->beta = restart ? 0.0 : v[0] / st->rho;
      st->rho = v[0];
      st->repl_threshold = rel * st->repl_factor;
    }
  }
}

// ||v||_2 of a double vector into out (device)
__global__ void __launch_bounds__(kReduceThreads)
    norm2_kernel(int64_t n, const double* v, double* out, double* partials, unsigned int* counter) {
  __shared__ double scratch[8];
  double a[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[0] += v[i] * v[i];
  if (grid_sum<1>(a, partials, counter, scratch) && threadIdx.x == 0) *out = sqrt(a[0]);
}

// a . b over n entries (FP64 sums of the products), written to out in the vector type
template <typename VT>
__global__ void __launch_bounds__(kReduceThreads)
    dot_kernel(int64_t n, const VT* a, const VT* b, VT* out, double* partials, unsigned int* counter) {
  __shared__ double scratch[8];
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[0] += (double)a[i] * (double)b[i];
  if (grid_sum<1>(s, partials, counter, scratch) && threadIdx.x == 0) *out = VT(s[0]);
}

__global__ void axpy_kernel(int64_t n, double a, const double* x, double* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

static inline int vec_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

pfem_status vk_lift(int64_t n, const double* u0, const double* values, const uint8_t* mask, double s, double* x,
                    cudaStream_t st) {
  lift_kernel<<<vec_grid(n), 256, 0, st>>>(n, u0, values, mask, s, x); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_invert_diag(int64_t n, const void* d, pfem_dtype dt, double* dinv, cudaStream_t st) {
  if (dt == PFEM_F32) invert_diag_kernel<float><<<vec_grid(n), 256, 0, st>>>(n, static_cast<const float*>(d), dinv);
  else invert_diag_kernel<double><<<vec_grid(n), 256, 0, st>>>(n, static_cast<const double*>(d), dinv);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_update(int64_t n, double* x, double* r, const double* p0, const double* p1, const double* q,
                      const double* dinv, PcgState* st, const double* tile_part, int n_tiles, double* partials,
                      unsigned int* counter, cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s) {
  pcg_update_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, x, r, p0, p1, q, dinv, st, tile_part, n_tiles,
                                                            partials, counter, cond, set_cond);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_replace(int64_t n, const double* res, double* r, const double* dinv, PcgState* st, int restart,
                       double* partials, unsigned int* counter, cudaStream_t s) {
  pcg_replace_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, res, r, dinv, st, restart, partials, counter); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_norm2(int64_t n, const double* v, double* out, double* partials, unsigned int* counter,
                     cudaStream_t s) {
  norm2_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, v, out, partials, counter); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_dot(int64_t n, pfem_dtype vt, const void* a, const void* b, void* out, double* partials,
                   unsigned int* counter, cudaStream_t s) {
  if (vt == PFEM_F32)
    dot_kernel<float><<<kReduceBlocks, kReduceThreads, 0, s>>>(n, static_cast<const float*>(a),
                                                              static_cast<const float*>(b), static_cast<float*>(out),
                                                              partials, counter);
  else
    dot_kernel<double><<<kReduceBlocks, kReduceThreads, 0, s>>>(n, static_cast<const double*>(a),
                                                               static_cast<const double*>(b), static_cast<double*>(out),
                                                               partials, counter);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  axpy_kernel<<<vec_grid(n), 256, 0, s>>>(n, a, x, y); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

}  // namespace pfem
