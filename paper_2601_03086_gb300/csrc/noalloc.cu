// pfem_tangent_apply_noalloc: the tangent action y = A(u) v without any allocation.
//
// Some callers cannot allocate device memory at the time they need the operator: code that
// runs while a memory pool is frozen or exhausted, inside allocator callbacks, or in
// embedded runtimes whose only device memory is what they were handed up front. The regular
// pfem_tangent_apply writes its per-call scratch (one partial sum per (tile, halo node) pair,
// summed by the halo pass) into a buffer the mesh allocated at creation. This variant runs
// the same kernels but keeps that scratch in a fixed, file-scope device array, so the call
// itself never allocates: no cudaMalloc, no cudaFree, no allocating library routine.

#include <mutex>

#include "pfem_internal.h"

namespace pfem {

// 16 MiB per device. Every GPU that loads the library holds it until process exit.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device. The host-side name of the
// array is only a stand-in, so the address is looked up once per device with that device
// current (cudaGetSymbolAddress) and cached. With lazy module loading the first lookup also
// loads this file's module, which is when the driver allocates the array: pfem_mesh_create
// calls this (allocation is allowed there), so the no-alloc call itself only reads the cache.
pfem_status noalloc_scratch(void** out) {
  int dev = -1;
  PFEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d is beyond the %d devices the no-alloc path tracks", dev, kMaxDevices);
    return PFEM_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PFEM_OK;
}

}  // namespace pfem

using namespace pfem;

extern "C" pfem_status pfem_tangent_apply_noalloc(pfem_mesh_t m, pfem_dtype dt, const void* u, const void* v,
                                                  void* y) {
  if (!m) {
    set_error("null mesh");
    return PFEM_ERR_INVALID_ARG;
  }
  if (m->n_spring_nodes || m->plan.elem_npe) {
    set_error("pfem_tangent_apply_noalloc: simplex meshes without penalty springs only");
    return PFEM_ERR_UNSUPPORTED;
  }
  if (dt != PFEM_F32 && dt != PFEM_F64 && dt != PFEM_F64_F32) {
    set_error("unknown dtype %d", (int)dt);
    return PFEM_ERR_INVALID_ARG;
  }
  if (!v || !y || (m->plan.kind == PFEM_NEOHOOKEAN && !u)) {
    set_error("u/v/y is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  int dev = -1;
  PFEM_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) {
    set_error("the current device (%d) is not the mesh's device (%d)", dev, m->device);
    return PFEM_ERR_INVALID_ARG;
  }
  const pfem_dtype vt = dt == PFEM_F32 ? PFEM_F32 : PFEM_F64;
  const pfem_dtype ct = dt == PFEM_F64 ? PFEM_F64 : PFEM_F32;
  const size_t need = (size_t)m->plan.n_partials * 4u * (ct == PFEM_F64 ? 8u : 4u);
  if (need > kNoAllocScratchBytes) {
    set_error("mesh needs %zu bytes of halo scratch; the no-alloc array holds %zu (use pfem_tangent_apply)", need,
              kNoAllocScratchBytes);
    return PFEM_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;  // resolved when the mesh was created on this device
  pfem_status st = noalloc_scratch(&scratch);
  if (st != PFEM_OK) return st;
  DevPlan P = m->plan;  // same plan, scratch redirected to the fixed array
  P.partial = scratch;
  OpArgs a{u, v, y, nullptr, nullptr, m->load_scale};
  return launch_element_op(P, OP_TANGENT, vt, ct, a, m->stream);
}
