// Scalar bookkeeping of one Jacobi-PCG iteration (device), shared by the single-solve and the
// serving update kernels so both make identical decisions.
#pragma once

#include "pfem_internal.h"

namespace pfem {

// After x += alpha p, r -= alpha q with rz = r . dinv r and rr = r . r of the new residual:
// count the iteration, record the recursive relative residual and decide what comes next
// (FP64 replacement / convergence check by the host, iteration cap, or the next beta).
__device__ __forceinline__ void pcg_finish_update(PcgState* st, double rz, double rr) {
  st->iter += 1;
  const double rel = sqrt(rr) / st->ref;
  st->rel = rel;
  if (!isfinite(rz) || !isfinite(rr)) {
    if (st->done == 0) st->done = PCG_NONFINITE;
  } else if (st->done == 0) {
    if (rel < st->tol || rel < st->repl_threshold) {
      st->repl = 1;  // the host verifies / replaces with the FP64 true residual
    } else if (st->iter >= st->max_iter) {
      st->done = PCG_MAXITER;
    } else {
      st->beta = rz / st->rho;
      st->rho = rz;
    }
  }
}

}  // namespace pfem
