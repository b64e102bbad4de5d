// Scalar bookkeeping of one Jacobi-PCG iteration (device), shared by the single-solve and the
// serving update kernels so both make identical decisions.
#pragma once

#include "pfem_internal.h"
#include "reduce.cuh"

namespace pfem {

// After x += alpha p, r -= alpha q with rz = r . dinv r and rr = r . r of the new residual:
// count the iteration, record the recursive relative residual and decide what comes next
// (FP64 replacement / convergence check by the host, iteration cap, or the next beta).
// The state is read through L2 only: inside a persistent launch another CTA may have
// written it since this one last looked.
__device__ __forceinline__ void pcg_finish_update(PcgState* st, double rz, double rr) {
  const int iter = __ldcg(&st->iter) + 1;
  const int done = __ldcg(&st->done);
  st->iter = iter;
  const double rel = sqrt(rr) / __ldcg(&st->ref);
  st->rel = rel;
  if (!isfinite(rz) || !isfinite(rr)) {
    if (done == 0) st->done = PCG_NONFINITE;
  } else if (done == 0) {
    if (rel < __ldcg(&st->tol) || rel < __ldcg(&st->repl_threshold)) {
      st->repl = 1;  // the host verifies / replaces with the FP64 true residual
    } else if (iter >= __ldcg(&st->max_iter)) {
      st->done = PCG_MAXITER;
    } else {
      st->beta = rz / __ldcg(&st->rho);
      st->rho = rz;
    }
  }
}

// The vector part of the update for the DOFs of reduction block vb (of kReduceBlocks x
// kReduceThreads; thread t takes i = vb * 256 + t + k * S, S = 296 * 256, in k order):
// x += alpha p, r -= alpha q, and r.z, r.r of the new residual accumulated into v. Loads of
// U consecutive k are issued before their arithmetic; the arithmetic and its order are those
// of the plain loop (any U gives the same bits). r, p, q go through L2 only (other CTAs of a
// persistent launch write them).
template <int U>
__device__ __forceinline__ void pcg_update_range(int64_t n, double* x, double* r, const double* p, const double* q,
                                                 const double* dinv, double alpha, int vb, double (&v)[2]) {
  const int64_t S = (int64_t)kReduceBlocks * kReduceThreads;
  for (int64_t i = (int64_t)vb * kReduceThreads + threadIdx.x; i < n; i += U * S) {
    double pp[U], qq[U], rr[U], dd[U], xx[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int64_t k = i + j * S;
      if (k < n) {
        pp[j] = __ldcg(p + k);
        qq[j] = __ldcg(q + k);
        rr[j] = __ldcg(r + k);
        dd[j] = dinv[k];
        xx[j] = x[k];
      }
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int64_t k = i + j * S;
      if (k < n) {
        x[k] = xx[j] + alpha * pp[j];
        const double ri = rr[j] - alpha * qq[j];
        r[k] = ri;
        v[0] += ri * (dd[j] * ri);
        v[1] += ri * ri;
      }
    }
  }
}

}  // namespace pfem
