// Bounds-checked build (nvcc -DPFEM_CHECKED, built as libpfem_checked.so): the global node
// indices and halo-partial ranges through which the element tiles gather and scatter are
// checked against the mesh before use. An index out of range is replaced by 0, a valid
// address, and recorded in a device word, so a corrupted plan shows up as a status instead
// of an illegal memory access (the role a memory checker would play). pfem_check_status
// reads and clears the words of every module. In the regular build the checks compile to
// nothing.
#pragma once

#include <cstdint>

#include "pfem_internal.h"

namespace pfem {

#ifdef PFEM_CHECKED
namespace {
__device__ unsigned int g_bad_index;  // one word per translation unit (internal linkage)

unsigned read_and_clear_bad_index() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bad_index, sizeof(v)) != cudaSuccess) return 0x80000000u;
  const unsigned zero = 0;
  if (cudaMemcpyToSymbol(g_bad_index, &zero, sizeof(zero)) != cudaSuccess) return v | 0x80000000u;
  return v;
}

const bool g_bad_index_registered = register_check_word(&read_and_clear_bad_index);
}  // namespace

// id if 0 <= id < n; else records bit 1 and returns 0
__device__ __forceinline__ int64_t checked_node(int64_t id, int64_t n) {
  if (static_cast<uint64_t>(id) >= static_cast<uint64_t>(n)) {
    atomicOr(&g_bad_index, 1u);
    return 0;
  }
  return id;
}

// [first, first + count) inside [0, n); else records bit 2 and returns false
__device__ __forceinline__ bool checked_range(int64_t first, int64_t count, int64_t n) {
  if (first < 0 || count < 0 || first + count > n) {
    atomicOr(&g_bad_index, 2u);
    return false;
  }
  return true;
}
#else
__device__ __forceinline__ int64_t checked_node(int64_t id, int64_t) { return id; }
__device__ __forceinline__ bool checked_range(int64_t, int64_t, int64_t) { return true; }
#endif

}  // namespace pfem
