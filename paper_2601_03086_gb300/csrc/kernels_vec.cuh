// Declarations of the PCG vector kernels (kernels_vec.cu) and the device-resident solver state.
#pragma once

#include <cuda_runtime.h>

#include "pfem_internal.h"

namespace pfem {

pfem_status vk_lift(int64_t n, const double* u0, const double* values, const uint8_t* mask, double s, double* x,
                    cudaStream_t st);
pfem_status vk_invert_diag(int64_t n, const void* d, pfem_dtype dt, double* dinv, cudaStream_t st);
pfem_status vk_update(int64_t n, double* x, double* r, const double* p0, const double* p1, const double* q,
                      const double* dinv, PcgState* st, const double* tile_part, int n_tiles, double* partials,
                      unsigned int* counter, cudaGraphConditionalHandle cond, int set_cond, cudaStream_t s);
pfem_status vk_replace(int64_t n, const double* res, double* r, const double* dinv, PcgState* st, int restart,
                       double* partials, unsigned int* counter, cudaStream_t s);
pfem_status vk_norm2(int64_t n, const double* v, double* out, double* partials, unsigned int* counter,
                     cudaStream_t s);
pfem_status vk_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t s);
// out = a . b (vector type vt, FP64 sums), deterministic
pfem_status vk_dot(int64_t n, pfem_dtype vt, const void* a, const void* b, void* out, double* partials,
                   unsigned int* counter, cudaStream_t s);

}  // namespace pfem
