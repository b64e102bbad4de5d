// Penalty springs between node pairs: the "virtual elements" with which the homogenisation
// appendix couples corresponding nodes of opposite faces of a periodic unit cell (ring-type
// coupling). A spring (a, b) of stiffness kappa adds the energy 1/2 kappa |u_a - u_b|^2, i.e.
// kappa (u_a - u_b) to the force at a (and the opposite at b), kappa to the diagonal of each
// of its DOFs. Each node keeps its partners in ascending order and one thread sums one DOF's
// terms in that order, so the result is deterministic (no atomics).

#include <algorithm>
#include <cmath>
#include <vector>

#include "pfem_internal.h"
#include "solver.h"

namespace pfem {

template <typename VT>
__global__ void springs_apply_kernel(int n_sn, const int32_t* node, const int32_t* ptr, const int32_t* partner,
                                     double kappa, const uint8_t* mask, int dim, int k, int64_t nd, const VT* v,
                                     VT* y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)n_sn * dim;
  if (t >= per * k) return;
  const int j = (int)(t / per);
  const int64_t r = t - (int64_t)j * per;
  const int i = (int)(r / dim), c = (int)(r - (int64_t)i * dim);
  const int64_t a = (int64_t)node[i] * dim + c;
  if (mask[a]) return;  // prescribed rows keep the identity block
  const VT* vj = v + (int64_t)j * nd;
  const double va = (double)vj[a];
  double s = 0.0;
  for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
    const int64_t b = (int64_t)partner[q] * dim + c;
    s += va - (mask[b] ? 0.0 : (double)vj[b]);
  }
  y[(int64_t)j * nd + a] += VT(kappa * s);
}

template <typename VT>
__global__ void springs_diag_kernel(int n_sn, const int32_t* node, const int32_t* ptr, double kappa,
                                    const uint8_t* mask, int dim, VT* d) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_sn * dim) return;
  const int i = (int)(t / dim), c = (int)(t - (int64_t)(t / dim) * dim);
  const int64_t a = (int64_t)node[i] * dim + c;
  if (mask[a]) return;
  d[a] += VT(kappa * (double)(ptr[i + 1] - ptr[i]));
}

pfem_status springs_apply(pfem_mesh_t m, pfem_dtype vt, int k, const void* v, void* y, cudaStream_t s) {
  if (!m->n_spring_nodes || k <= 0) return PFEM_OK;
  const int dim = m->plan.dim;
  const int64_t total = (int64_t)m->n_spring_nodes * dim * k;
  const int grid = (int)((total + 255) / 256);
  if (vt == PFEM_F32)
    springs_apply_kernel<float><<<grid, 256, 0, s>>>(m->n_spring_nodes, m->spring_node, m->spring_ptr,
                                                     m->spring_partner, m->spring_k, m->plan.dmask, dim, k,
                                                     m->n_dofs, static_cast<const float*>(v), static_cast<float*>(y));
  else
    springs_apply_kernel<double><<<grid, 256, 0, s>>>(m->n_spring_nodes, m->spring_node, m->spring_ptr,
                                                      m->spring_partner, m->spring_k, m->plan.dmask, dim, k,
                                                      m->n_dofs, static_cast<const double*>(v),
                                                      static_cast<double*>(y));
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

pfem_status springs_diag(pfem_mesh_t m, pfem_dtype vt, void* d, cudaStream_t s) {
  if (!m->n_spring_nodes) return PFEM_OK;
  const int dim = m->plan.dim;
  const int grid = (int)(((int64_t)m->n_spring_nodes * dim + 255) / 256);
  if (vt == PFEM_F32)
    springs_diag_kernel<float><<<grid, 256, 0, s>>>(m->n_spring_nodes, m->spring_node, m->spring_ptr, m->spring_k,
                                                    m->plan.dmask, dim, static_cast<float*>(d));
  else
    springs_diag_kernel<double><<<grid, 256, 0, s>>>(m->n_spring_nodes, m->spring_node, m->spring_ptr, m->spring_k,
                                                     m->plan.dmask, dim, static_cast<double*>(d));
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

void springs_release(pfem_mesh_t m) {
  if (m->spring_block) cudaFree(m->spring_block);
  m->spring_block = nullptr;
  m->spring_node = m->spring_ptr = m->spring_partner = nullptr;
  m->n_spring_nodes = 0;
  m->spring_k = 0.0;
}

}  // namespace pfem

using namespace pfem;

extern "C" pfem_status pfem_mesh_set_springs(pfem_mesh_t m, int64_t n_pairs, const int32_t* pairs, double stiffness) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (n_pairs < 0 || (n_pairs > 0 && !pairs) || !(stiffness >= 0.0) || !std::isfinite(stiffness)) {
    set_error("pfem_mesh_set_springs: bad pair count, pairs pointer or stiffness");
    return PFEM_ERR_INVALID_ARG;
  }
  const int64_t nn = m->plan.n_nodes;
  std::vector<std::vector<int32_t>> adj;
  std::vector<int32_t> nodes, ptr(1, 0), partner;
  if (n_pairs > 0) {
    adj.resize((size_t)nn);
    for (int64_t q = 0; q < n_pairs; ++q) {
      const int32_t a = pairs[2 * q], b = pairs[2 * q + 1];
      if (a < 0 || b < 0 || a >= nn || b >= nn || a == b) {
        set_error("pfem_mesh_set_springs: pair %lld (%d, %d) is not two distinct node ids", (long long)q, a, b);
        return PFEM_ERR_INVALID_ARG;
      }
      adj[(size_t)a].push_back(b);
      adj[(size_t)b].push_back(a);
    }
    for (int64_t i = 0; i < nn; ++i) {
      auto& l = adj[(size_t)i];
      if (l.empty()) continue;
      std::sort(l.begin(), l.end());
      nodes.push_back((int32_t)i);
      partner.insert(partner.end(), l.begin(), l.end());
      ptr.push_back((int32_t)partner.size());
    }
  }
  PFEM_CUDA(cudaStreamSynchronize(m->stream));  // earlier calls may still read the old springs
  springs_release(m);
  if (nodes.empty()) return PFEM_OK;
  const size_t bn = nodes.size() * 4, bp = ptr.size() * 4, bq = partner.size() * 4;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  char* blk = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&blk), al(bn) + al(bp) + al(bq));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(springs)");
  m->spring_block = blk;
  m->spring_node = reinterpret_cast<int32_t*>(blk);
  m->spring_ptr = reinterpret_cast<int32_t*>(blk + al(bn));
  m->spring_partner = reinterpret_cast<int32_t*>(blk + al(bn) + al(bp));
  e = cudaMemcpy(m->spring_node, nodes.data(), bn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->spring_ptr, ptr.data(), bp, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->spring_partner, partner.data(), bq, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    springs_release(m);
    return cuda_fail(e, "uploading springs");
  }
  m->n_spring_nodes = (int32_t)nodes.size();
  m->spring_k = stiffness;
  return PFEM_OK;
}
