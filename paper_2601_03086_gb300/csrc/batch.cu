// Ragged batches: several meshes' energies, gradients and Hessian-vector products in one
// element launch (the differentiable FE energy loss of the plate and
// hyperelasticity results, Secs. "Linear elastic plate with arbitrary holes" and "Nonlinear
// hyperelasticity", over a batch).

#include <cstring>
#include <new>
#include <vector>

#include "pfem_internal.h"

struct pfem_batch_s {
  std::vector<pfem_mesh_t> meshes;
  std::vector<int64_t> off;  // DOF offsets (host copy)
  pfem::BatchDev dev{};
  void* block = nullptr;
  int32_t* inverted = nullptr;
  int n_blocks = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
};

using namespace pfem;

extern "C" {

pfem_status pfem_batch_create(const pfem_mesh_t* meshes, int32_t n, pfem_batch_t* out) {
  if (!out || !meshes || n < 1) {
    set_error("invalid batch arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) {
      set_error("mesh %d is NULL", i);
      return PFEM_ERR_INVALID_ARG;
    }
    if (meshes[i]->n_spring_nodes || meshes[i]->plan.elem_npe) {
      set_error("mesh %d has penalty springs or quadrilaterals, which batches do not evaluate", i);
      return PFEM_ERR_UNSUPPORTED;
    }
    if (meshes[i]->plan.dim != 3) {
      set_error("batches hold 3-D meshes only (mesh %d has dim %d)", i, meshes[i]->plan.dim);
      return PFEM_ERR_UNSUPPORTED;
    }
    if (meshes[i]->device != meshes[0]->device) {
      set_error("all meshes of a batch must live on one device");
      return PFEM_ERR_INVALID_ARG;
    }
  }
  pfem_batch_s* b = new (std::nothrow) pfem_batch_s();
  if (!b) {
    set_error("host allocation failed");
    return PFEM_ERR_OUT_OF_MEMORY;
  }
  b->meshes.assign(meshes, meshes + n);
  b->stream = meshes[0]->stream;
  b->device = meshes[0]->device;
  b->off.assign((size_t)n + 1, 0);
  std::vector<int2> btile;
  int max_local = 0, slot_cap = 0, step_cap = 0;
  for (int i = 0; i < n; ++i) {
    const DevPlan& P = meshes[i]->plan;
    b->off[(size_t)i + 1] = b->off[(size_t)i] + meshes[i]->n_dofs;
    for (int t = 0; t < P.n_tiles; ++t) btile.push_back(make_int2(i, t));
    max_local = std::max(max_local, P.max_local);
    slot_cap = std::max(slot_cap, P.slot_cap);
    step_cap = std::max(step_cap, P.step_cap);
  }
  b->n_blocks = (int)btile.size();
  const size_t o_plans = 0;
  const size_t o_bt = (o_plans + (size_t)n * sizeof(DevPlan) + 255) & ~size_t(255);
  const size_t o_off = (o_bt + btile.size() * sizeof(int2) + 255) & ~size_t(255);
  const size_t o_inv = (o_off + ((size_t)n + 1) * sizeof(int64_t) + 255) & ~size_t(255);
  const size_t total = o_inv + 256;
  cudaError_t e = cudaMalloc(&b->block, total);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaMalloc(batch)");
  }
  char* base = static_cast<char*>(b->block);
  b->inverted = reinterpret_cast<int32_t*>(base + o_inv);
  std::vector<DevPlan> plans((size_t)n);
  for (int i = 0; i < n; ++i) {
    plans[(size_t)i] = meshes[i]->plan;
    plans[(size_t)i].inverted = b->inverted;
  }
  e = cudaMemcpy(base + o_plans, plans.data(), plans.size() * sizeof(DevPlan), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !btile.empty())
    e = cudaMemcpy(base + o_bt, btile.data(), btile.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + o_off, b->off.data(), b->off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->inverted, 0, sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaFree(b->block);
    delete b;
    return cuda_fail(e, "batch upload");
  }
  b->dev.plans = reinterpret_cast<const DevPlan*>(base + o_plans);
  b->dev.btile = reinterpret_cast<const int2*>(base + o_bt);
  b->dev.dof_off = reinterpret_cast<const int64_t*>(base + o_off);
  b->dev.mesh_scale = nullptr;
  b->dev.max_local = max_local;
  b->dev.slot_cap = slot_cap;
  b->dev.step_cap = step_cap;
  *out = b;
  return PFEM_OK;
}

void pfem_batch_destroy(pfem_batch_t b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  cudaFree(b->block);
  delete b;
}

pfem_status pfem_batch_offsets(pfem_batch_t b, int64_t* offsets) {
  if (!b || !offsets) {
    set_error("invalid arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  std::memcpy(offsets, b->off.data(), b->off.size() * sizeof(int64_t));
  return PFEM_OK;
}

pfem_status pfem_batch_eval(pfem_batch_t b, const float* u, const float* v, const float* mesh_scale,
                            double* energy_dev, float* grad, float* hvp, int32_t* inverted_dev) {
  if (!b || !u || (hvp && !v)) {
    set_error("invalid batch evaluation arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  BatchDev d = b->dev;
  d.mesh_scale = mesh_scale;
  PFEM_CUDA(cudaMemsetAsync(b->inverted, 0, sizeof(int32_t), b->stream));
  pfem_status st = launch_batch(d, b->n_blocks, (int)b->meshes.size(), u, v, grad, hvp, energy_dev, b->stream);
  if (st) return st;
  if (inverted_dev)
    PFEM_CUDA(cudaMemcpyAsync(inverted_dev, b->inverted, sizeof(int32_t), cudaMemcpyDeviceToDevice, b->stream));
  return PFEM_OK;
}

}  // extern "C"
