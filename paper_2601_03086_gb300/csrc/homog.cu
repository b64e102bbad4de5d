// Numerical homogenisation of a periodic cell (appendix "Numerical homogenization theory"),
// every step on the device:
//   1. the six affine fields X^0(IJ) = eps0^(IJ) X of the unit strains (both off-diagonal
//      entries 1 for the shear cases, as printed);
//   2. their load vectors F^(IJ) = K X^0(IJ) (for P1 elements K applied to an affine field is
//      exactly int B^T E eps0), FP64 element arithmetic;
//   3. the fluctuations from (K + S) X^v = F with S the penalty springs that couple opposite
//      faces: six Jacobi-PCG solves sharing each operator pass (pfem_solve_linear_multi),
//      optionally warm-started from a prediction of X^v (the PFEM warm start);
//   4. the total fields X = X^0 - X^v and E^H_(IJ)(KL) = X^(IJ) . K X^(KL) / |Omega|, which is
//      the appendix's element integral of (eps0 - eps^v) : E : (eps0 - eps^v) written with the
//      stiffness matrix (P1 strains are constant per element); FP64 element arithmetic,
//      deterministic FP64 dots.

#include <cmath>
#include <cstring>
#include <vector>

#include "kernels_vec.cuh"
#include "pfem_internal.h"
#include "solver.h"

namespace pfem {

pfem_status solve_multi_core(pfem_mesh_t m, pfem_dtype dt, int k, const double* b, const double* u0, double tol,
                             int max_iter, double* u_out, pfem_solve_info* infos);

namespace {

// X^0(c)_i = eps0^(c) X_i for the six cases (c = blockIdx.y), node-major coordinates
__global__ void affine_kernel(int64_t n_nodes, const double* X, double* u0) {
  const int c = blockIdx.y;
  const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
  const int a = ci[c], b = cj[c];
  double* u = u0 + (int64_t)c * n_nodes * 3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
    double w[3] = {0.0, 0.0, 0.0};
    w[a] += X[i * 3 + b];
    if (a != b) w[b] += X[i * 3 + a];
    u[i * 3] = w[0];
    u[i * 3 + 1] = w[1];
    u[i * 3 + 2] = w[2];
  }
}

// x = a - b, element by element over n
__global__ void sub_kernel(int64_t n, const double* a, const double* b, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = a[i] - b[i];
}

}  // namespace
}  // namespace pfem

using namespace pfem;

extern "C" pfem_status pfem_homogenize(pfem_mesh_t m, pfem_dtype dt, const double* coords, const double* xv0,
                                       double tol, int32_t max_iter, double* eh, double* xv_out,
                                       pfem_solve_info* infos) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (m->plan.dim != 3 || m->plan.kind != PFEM_LINEAR) {
    set_error("pfem_homogenize needs a 3-D linear-elastic mesh");
    return PFEM_ERR_INVALID_ARG;
  }
  if (!coords || !eh || !(tol > 0.0) || max_iter < 0 || (dt != PFEM_F32 && dt != PFEM_F64)) {
    set_error("invalid homogenisation arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  const int64_t nn = m->plan.n_nodes, n = m->n_dofs;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) lo[d] = hi[d] = coords[d];
  for (int64_t i = 0; i < nn; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], coords[i * 3 + d]);
      hi[d] = std::max(hi[d], coords[i * 3 + d]);
    }
  const double omega = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  if (!(omega > 0.0)) {
    set_error("pfem_homogenize: the cell has no volume");
    return PFEM_ERR_INVALID_ARG;
  }
  cudaStream_t s = m->stream;
  const size_t vb = (size_t)n * sizeof(double);
  char* blk = nullptr;
  // X (coords), X0, F, Xv, Xt, Y: six vectors each (coords: one), 36 dots
  const size_t bytes = vb + 5 * 6 * vb + 64 * sizeof(double);
  PFEM_CUDA(cudaMalloc(reinterpret_cast<void**>(&blk), bytes));
  struct Free {
    char* b;
    ~Free() { cudaFree(b); }
  } guard{blk};
  double* X = reinterpret_cast<double*>(blk);
  double* X0 = X + n;
  double* F = X0 + 6 * n;
  double* Xv = F + 6 * n;
  double* Xt = Xv + 6 * n;
  double* Y = Xt + 6 * n;
  double* dots = Y + 6 * n;
  // affine fields vanish at the cell's minimum corner, where the fixed node sits
  std::vector<double> xs((size_t)n);
  for (int64_t i = 0; i < nn; ++i)
    for (int d = 0; d < 3; ++d) xs[(size_t)(i * 3 + d)] = coords[i * 3 + d] - lo[d];
  PFEM_CUDA(cudaMemcpyAsync(X, xs.data(), vb, cudaMemcpyHostToDevice, s));
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nn + 255) / 256, 1216));
  affine_kernel<<<dim3(g, 6), 256, 0, s>>>(nn, X, X0);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  auto apply_k = [&](const double* v, double* y) -> pfem_status {  // y_c = K v_c (no springs)
    for (int c = 0; c < 6; ++c) {
      OpArgs a{nullptr, v + (size_t)c * n, y + (size_t)c * n, nullptr, nullptr, 1.0};
      pfem_status e = launch_element_op(m->plan, OP_TANGENT, PFEM_F64, PFEM_F64, a, s);
      if (e) return e;
    }
    return PFEM_OK;
  };
  if ((st = apply_k(X0, F))) return st;
  pfem_solve_info local[6];
  pfem_solve_info* inf = infos ? infos : local;
  st = solve_multi_core(m, dt, 6, F, xv0, tol, max_iter, Xv, inf);
  if (st != PFEM_OK && st != PFEM_ERR_NOT_CONVERGED) return st;
  const pfem_status solve_status = st;
  const int gv = (int)std::max<int64_t>(1, std::min<int64_t>((6 * n + 255) / 256, 1216));
  sub_kernel<<<gv, 256, 0, s>>>(6 * n, X0, Xv, Xt);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  if ((st = apply_k(Xt, Y))) return st;
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b)
      if ((st = vk_dot(n, PFEM_F64, Xt + (size_t)a * n, Y + (size_t)b * n, dots + a * 6 + b, m->red_partials,
                       m->red_counter, s)))
        return st;
  double h[36];
  PFEM_CUDA(cudaMemcpyAsync(h, dots, sizeof(h), cudaMemcpyDeviceToHost, s));  // synchronised below
  if (xv_out) PFEM_CUDA(cudaMemcpyAsync(xv_out, Xv, 6 * vb, cudaMemcpyDeviceToDevice, s));
  PFEM_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < 36; ++i) eh[i] = h[i] / omega;
  return solve_status;
}
