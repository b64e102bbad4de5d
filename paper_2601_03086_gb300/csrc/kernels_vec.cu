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

// alpha = rho / (p . q)
__global__ void __launch_bounds__(kReduceThreads)
    pcg_alpha_kernel(int64_t n, const double* p, const double* q, PcgState* st, double* partials,
                     unsigned int* counter) {
  __shared__ double scratch[8];
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += p[i] * q[i];
  if (grid_sum<1>(v, partials, counter, scratch) && threadIdx.x == 0) {
    // Negative curvature (an indefinite tangent far from equilibrium) does not stop the
    // iteration, as in plain CG; only p.q = 0 or a non-finite value does.
    const double pq = v[0];
    if (pq == 0.0 || !isfinite(pq)) {
      st->alpha = 0.0;
      st->done = isfinite(pq) ? PCG_BREAKDOWN : PCG_NONFINITE;
    } else {
      st->alpha = st->rho / pq;
    }
  }
}

// x += alpha p; r -= alpha q; (r.z, r.r) with z = dinv r; flags and beta in the last block.
// p is this iteration's direction, p_buf[(iter + 1) & 1] (written by the fused apply).
__global__ void __launch_bounds__(kReduceThreads)
    pcg_update_kernel(int64_t n, double* x, double* r, const double* p0, const double* p1, const double* q,
                      const double* dinv, PcgState* st, double* partials, unsigned int* counter,
                      cudaGraphConditionalHandle cond, int set_cond) {
  __shared__ double scratch[16];
  if (st->done != 0 || st->repl != 0) {  // nothing to do (uniform: written by earlier kernels)
    if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) {
      st->bodies += 1;
      cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  const double alpha = st->alpha;
  const double* p = ((st->iter + 1) & 1) ? p1 : p0;
  double v[2] = {0.0, 0.0};
  pcg_update_range<4>(n, x, r, p, q, dinv, alpha, blockIdx.x, v);  // launched as kReduceBlocks x kReduceThreads
  if (grid_sum<2>(v, partials, counter, scratch) && threadIdx.x == 0) {
    pcg_finish_update(st, v[0], v[1]);
    if (set_cond) {
      st->bodies += 1;
      cudaGraphSetConditional(cond, (st->done == 0 && st->repl == 0) ? 1u : 0u);
    }
  }
}

// p = dinv r + beta p (skipped while a replacement is pending or after termination)
__global__ void pcg_direction_kernel(int64_t n, const double* r, const double* dinv, double* p, const PcgState* st) {
  if (st->done != 0 || st->repl != 0) return;
  const double beta = st->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = dinv[i] * r[i] + beta * p[i];
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

pfem_status vk_alpha(int64_t n, const double* p, const double* q, PcgState* st, double* partials,
                     unsigned int* counter, cudaStream_t s) {
  pcg_alpha_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, p, q, st, partials, counter); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_update(int64_t n, double* x, double* r, const double* p0, const double* p1, const double* q,
                      const double* dinv, PcgState* st, double* partials, unsigned int* counter,
                      cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s) {
  pcg_update_kernel<<<kReduceBlocks, kReduceThreads, 0, s>>>(n, x, r, p0, p1, q, dinv, st, partials, counter, cond,
                                                            set_cond);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status vk_direction(int64_t n, const double* r, const double* dinv, double* p, const PcgState* st,
                         cudaStream_t s) {
  pcg_direction_kernel<<<vec_grid(n), 256, 0, s>>>(n, r, dinv, p, st); PFEM_COUNT_LAUNCH();
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

pfem_status vk_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  axpy_kernel<<<vec_grid(n), 256, 0, s>>>(n, a, x, y); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

}  // namespace pfem
