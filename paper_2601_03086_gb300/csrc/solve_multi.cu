// k independent Jacobi-PCG solves on one mesh that share every operator application
// (App. B linear system K u = f for several load cases; the six unit-strain cases of the
// homogenisation appendix): one multi-right-hand-side element pass q_j = A p_j per
// iteration for all running solves, then per-solve FP64 dots, updates and decisions.
//
//   per iteration: direction p_j = dinv r_j + beta_j p_j, q = A p (FP32 element arithmetic,
//   FP64 vectors), alpha_j = rho_j / p_j.q_j, x_j += alpha_j p_j, r_j -= alpha_j q_j,
//   (r_j.z_j, r_j.r_j) and the state of solve j (the single solver's decision code).
// Every reduction is deterministic (fixed grid, per-solve block partials summed in block
// order by the last block). Each solve's recursive residual is replaced by its FP64 true
// residual P (b_j - A x_j) (FP64 element operator) every two decades and before it is
// declared converged, as in pfem_solve_linear.

#include <cmath>
#include <cstring>
#include <vector>

#include "kernels_vec.cuh"
#include "pcg_state.cuh"
#include "pfem_internal.h"
#include "reduce.cuh"
#include "solver.h"

namespace pfem {

namespace {

// p_j = dinv r_j + beta_j p_j (0 on prescribed DOFs) for every running solve j (blockIdx.y)
__global__ void mdir_kernel(int64_t n, const double* r, const double* dinv, const uint8_t* mask, double* p,
                            const PcgState* st, int first) {
  const int j = blockIdx.y;
  const PcgState& s = st[j];
  if (s.done != 0 || s.repl != 0) return;
  const double beta = first ? 0.0 : s.beta;
  const double* rj = r + (int64_t)j * n;
  double* pj = p + (int64_t)j * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pj[i] = mask[i] ? 0.0 : fma(dinv[i], rj[i], beta * pj[i]);
}

// alpha_j = rho_j / (p_j . q_j): block partials of p_j.q_j, the last block of solve j sums them
__global__ void __launch_bounds__(kReduceThreads)
    mdot_kernel(int64_t n, const double* p, const double* q, PcgState* st, double* partials, unsigned int* counters) {
  __shared__ double scratch[8];
  const int j = blockIdx.y;
  PcgState* s = st + j;
  if (s->done != 0 || s->repl != 0) return;  // uniform over the solve's blocks
  const double* pj = p + (int64_t)j * n;
  const double* qj = q + (int64_t)j * n;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += pj[i] * qj[i];
  if (grid_sum_v<1>(v, partials + (size_t)j * kReduceBlocks * 2, counters + j, scratch, blockIdx.x, gridDim.x) &&
      threadIdx.x == 0) {
    double a = 0.0;
    const int stop = pcg_alpha(v[0], s->rho, s->truncate, s->iter, &a);
    s->alpha = a;
    if (stop) s->done = stop;
  }
}

// x_j += alpha_j p_j, r_j -= alpha_j q_j, (r.z, r.r); the last block of solve j decides
__global__ void __launch_bounds__(kReduceThreads)
    mupdate_kernel(int64_t n, double* x, double* r, const double* p, const double* q, const double* dinv,
                   PcgState* st, double* partials, unsigned int* counters) {
  __shared__ double scratch[16];
  const int j = blockIdx.y;
  PcgState* s = st + j;
  if (s->done != 0 || s->repl != 0) return;
  const double alpha = s->alpha;
  double* xj = x + (int64_t)j * n;
  double* rj = r + (int64_t)j * n;
  const double* pj = p + (int64_t)j * n;
  const double* qj = q + (int64_t)j * n;
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    xj[i] += alpha * pj[i];
    const double ri = rj[i] - alpha * qj[i];
    rj[i] = ri;
    v[0] += ri * (dinv[i] * ri);
    v[1] += ri * ri;
  }
  if (grid_sum_v<2>(v, partials + (size_t)j * kReduceBlocks * 2, counters + j, scratch, blockIdx.x, gridDim.x) &&
      threadIdx.x == 0)
    pcg_finish_update(s, v[0], v[1]);
}

// res = P (A x - b) from y = A x (A's identity rows give y = x on prescribed DOFs)
__global__ void res_kernel(int64_t n, const double* y, const double* b, const uint8_t* mask, double* res) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    res[i] = mask[i] ? 0.0 : y[i] - b[i];
}

// b projected on the free DOFs (its norm is the reference of the stopping rule)
__global__ void project_kernel(int64_t n, const double* b, const uint8_t* mask, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mask[i] ? 0.0 : b[i];
}

__global__ void set_ref_kernel(const double* nrm, PcgState* st) { st->ref = *nrm > 0.0 ? *nrm : 1.0; }

inline int vgrid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

}  // namespace

}  // namespace pfem

namespace pfem {

// The k solves; b, u0, u_out: k vectors of n_dofs (device FP64). Fills infos[0..k).
pfem_status solve_multi_core(pfem_mesh_t m, pfem_dtype dt, int k, const double* b, const double* u0, double tol,
                             int max_iter, double* u_out, pfem_solve_info* infos) {
  const int64_t n = m->n_dofs;
  const int64_t launches0 = g_kernel_launches;
  cudaStream_t s = m->stream;
  const size_t vb = ((size_t)n * sizeof(double) + 255) & ~size_t(255);
  const size_t sb = ((size_t)k * sizeof(PcgState) + 255) & ~size_t(255);
  const size_t pb = ((size_t)k * kReduceBlocks * 2 * sizeof(double) + 255) & ~size_t(255);
  const size_t cb = ((size_t)k * sizeof(unsigned int) + 255) & ~size_t(255);
  const size_t bytes = 4 * (size_t)k * vb + 4 * vb + sb + pb + cb + 256;
  char* blk = nullptr;
  PcgState* hst = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&blk), bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(multi-solve workspace)");
  e = cudaMallocHost(reinterpret_cast<void**>(&hst), (size_t)k * sizeof(PcgState));
  if (e != cudaSuccess) {
    cudaFree(blk);
    return cuda_fail(e, "cudaMallocHost(multi-solve states)");
  }
  struct Free {
    char* b;
    PcgState* h;
    ~Free() {
      cudaFree(b);
      cudaFreeHost(h);
    }
  } guard{blk, hst};
  // vectors of solve j at j * n inside x, r, p, q (vb-aligned blocks)
  double* x = reinterpret_cast<double*>(blk);
  double* r = reinterpret_cast<double*>(blk + (size_t)k * vb);
  double* p = reinterpret_cast<double*>(blk + 2 * (size_t)k * vb);
  double* q = reinterpret_cast<double*>(blk + 3 * (size_t)k * vb);
  char* tail = blk + 4 * (size_t)k * vb;
  double* dinv = reinterpret_cast<double*>(tail);
  double* y = reinterpret_cast<double*>(tail + vb);
  double* res = reinterpret_cast<double*>(tail + 2 * vb);
  double* tmp = reinterpret_cast<double*>(tail + 3 * vb);
  PcgState* st = reinterpret_cast<PcgState*>(tail + 4 * vb);
  double* partials = reinterpret_cast<double*>(tail + 4 * vb + sb);
  unsigned int* counters = reinterpret_cast<unsigned int*>(tail + 4 * vb + sb + pb);
  double* dnorm = reinterpret_cast<double*>(tail + 4 * vb + sb + pb + cb);
  // vectors of solve j are n apart (the vb padding is only between the four families)
  PFEM_CUDA(cudaMemsetAsync(p, 0, (size_t)k * vb, s));
  PFEM_CUDA(cudaMemsetAsync(counters, 0, (size_t)k * sizeof(unsigned int), s));
  pfem_status stt;
  // Jacobi diagonal of A (with the springs), inverted
  {
    OpArgs a{nullptr, nullptr, nullptr, nullptr, tmp, 1.0};
    if ((stt = launch_element_op(m->plan, OP_DIAG, PFEM_F64, dt == PFEM_F64 ? PFEM_F64 : PFEM_F32, a, s))) return stt;
    if ((stt = springs_diag(m, PFEM_F64, tmp, s))) return stt;
    if ((stt = vk_invert_diag(n, tmp, PFEM_F64, dinv, s))) return stt;
  }
  std::vector<PcgState> init((size_t)k);
  for (auto& h : init) {
    std::memset(&h, 0, sizeof(h));
    h.tol = tol;
    h.max_iter = max_iter;
    h.repl_factor = 1e-2;
    h.ref = 1.0;
  }
  PFEM_CUDA(cudaMemcpyAsync(st, init.data(), (size_t)k * sizeof(PcgState), cudaMemcpyHostToDevice, s));
  PFEM_CUDA(cudaStreamSynchronize(s));
  const int g = vgrid(n);
  // FP64 true residual of solve j into its r (restart = 1: beta = 0, first direction p = z)
  auto true_residual = [&](int j, int restart) -> pfem_status {
    OpArgs a{nullptr, x + (size_t)j * n, y, nullptr, nullptr, 1.0};
    pfem_status e2 = launch_element_op(m->plan, OP_TANGENT, PFEM_F64, PFEM_F64, a, s);
    if (e2) return e2;
    if ((e2 = springs_apply(m, PFEM_F64, 1, x + (size_t)j * n, y, s))) return e2;
    res_kernel<<<g, 256, 0, s>>>(n, y, b + (size_t)j * n, m->plan.dmask, res);
    PFEM_COUNT_LAUNCH();
    return vk_replace(n, res, r + (size_t)j * n, dinv, st + j, restart, partials + (size_t)j * kReduceBlocks * 2,
                      counters + j, s);
  };
  for (int j = 0; j < k; ++j) {
    project_kernel<<<g, 256, 0, s>>>(n, b + (size_t)j * n, m->plan.dmask, tmp);
    PFEM_COUNT_LAUNCH();
    if ((stt = vk_norm2(n, tmp, dnorm, partials, counters, s))) return stt;
    set_ref_kernel<<<1, 1, 0, s>>>(dnorm, st + j);
    PFEM_COUNT_LAUNCH();
    if (u0) project_kernel<<<g, 256, 0, s>>>(n, u0 + (size_t)j * n, m->plan.dmask, x + (size_t)j * n);
    else PFEM_CUDA(cudaMemsetAsync(x + (size_t)j * n, 0, (size_t)n * sizeof(double), s));
    if (u0) PFEM_COUNT_LAUNCH();
    if ((stt = true_residual(j, 1))) return stt;
  }
  PFEM_CUDA(cudaGetLastError());
  std::vector<double> prev((size_t)k, -1.0);
  std::vector<int> stalls((size_t)k, 0), replaced((size_t)k, 1);
  const dim3 vg(kReduceBlocks, k);
  const pfem_dtype vt_apply = PFEM_F64;  // the solver's vectors are FP64
  for (;;) {
    PFEM_CUDA(cudaMemcpyAsync(hst, st, (size_t)k * sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    PFEM_CUDA(cudaStreamSynchronize(s));
    bool running = false, again = false;
    for (int j = 0; j < k; ++j) {
      PcgState& h = hst[j];
      if (replaced[(size_t)j]) {  // stagnation of the FP32 operator: two weak replacements
        replaced[(size_t)j] = 0;
        const double rt = h.rel_true;
        stalls[(size_t)j] = (prev[(size_t)j] > 0.0 && !(rt < 0.5 * prev[(size_t)j])) ? stalls[(size_t)j] + 1 : 0;
        prev[(size_t)j] = rt;
        if (stalls[(size_t)j] >= 2 && h.done == 0) {
          static const int kStag = PCG_STAGNATED;
          PFEM_CUDA(cudaMemcpyAsync(&st[j].done, &kStag, sizeof(int), cudaMemcpyHostToDevice, s));
          h.done = PCG_STAGNATED;
        }
      }
      if (h.done != 0) continue;
      if (h.repl != 0) {
        if ((stt = true_residual(j, 0))) return stt;
        replaced[(size_t)j] = 1;
        again = true;  // re-read the states before iterating
        continue;
      }
      running = true;
    }
    if (again) continue;
    if (!running) break;
    for (int it = 0; it < 16; ++it) {
      mdir_kernel<<<dim3(g, k), 256, 0, s>>>(n, r, dinv, m->plan.dmask, p, st, 0);
      PFEM_COUNT_LAUNCH();
      if (dt == PFEM_F64) {
        for (int j = 0; j < k; ++j) {
          OpArgs a{nullptr, p + (size_t)j * n, q + (size_t)j * n, nullptr, nullptr, 1.0};
          if ((stt = launch_element_op(m->plan, OP_TANGENT, PFEM_F64, PFEM_F64, a, s))) return stt;
        }
      } else if ((stt = launch_multi_apply(m->plan, vt_apply, k, p, q, s))) {
        return stt;
      }
      if ((stt = springs_apply(m, PFEM_F64, k, p, q, s))) return stt;
      mdot_kernel<<<vg, kReduceThreads, 0, s>>>(n, p, q, st, partials, counters);
      PFEM_COUNT_LAUNCH();
      mupdate_kernel<<<vg, kReduceThreads, 0, s>>>(n, x, r, p, q, dinv, st, partials, counters);
      PFEM_COUNT_LAUNCH();
    }
    PFEM_CUDA(cudaGetLastError());
  }
  for (int j = 0; j < k; ++j)
    PFEM_CUDA(cudaMemcpyAsync(u_out + (size_t)j * n, x + (size_t)j * n, (size_t)n * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
  PFEM_CUDA(cudaMemcpyAsync(hst, st, (size_t)k * sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  PFEM_CUDA(cudaStreamSynchronize(s));
  pfem_status worst = PFEM_OK;
  for (int j = 0; j < k; ++j) {
    const PcgState& h = hst[j];
    pfem_status sj = PFEM_OK;
    switch (h.done) {
      case PCG_CONVERGED: sj = PFEM_OK; break;
      case PCG_NONFINITE: sj = PFEM_ERR_NONFINITE; break;
      default: sj = PFEM_ERR_NOT_CONVERGED; break;
    }
    if (sj != PFEM_OK && worst == PFEM_OK) worst = sj;
    if (infos) {
      pfem_solve_info& in = infos[j];
      std::memset(&in, 0, sizeof(in));
      in.iterations = h.iter;
      in.replacements = h.replacements;
      in.rel_residual_recursive = h.rel;
      in.rel_residual_true_f64 = h.rel_true;
      in.reference_norm = h.ref;
      in.status = sj;
      in.kernel_launches = g_kernel_launches - launches0;
    }
  }
  if (worst != PFEM_OK) set_error("pfem_solve_linear_multi: a solve did not converge");
  return worst;
}

}  // namespace pfem

using namespace pfem;

extern "C" pfem_status pfem_solve_linear_multi(pfem_mesh_t m, pfem_dtype dt, int32_t k, const double* b,
                                               const double* u0, double tol, int32_t max_iter, double* u_out,
                                               pfem_solve_info* infos) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (m->plan.kind != PFEM_LINEAR || m->plan.elem_npe) {
    set_error("pfem_solve_linear_multi needs a linear-elastic simplex mesh");
    return PFEM_ERR_INVALID_ARG;
  }
  if (k < 1 || !b || !u_out || !(tol > 0.0) || max_iter < 0 || (dt != PFEM_F32 && dt != PFEM_F64)) {
    set_error("invalid multi-solve arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  return solve_multi_core(m, dt, k, b, u0, tol, max_iter, u_out, infos);
}
