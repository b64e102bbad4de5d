// Solver workspace management (solve.cu).
#pragma once

#include "pfem_internal.h"

namespace pfem {
void solver_release(pfem_mesh_t m);
size_t solver_bytes(pfem_mesh_t m);
pfem_status check_mesh(pfem_mesh_t m);
}  // namespace pfem
