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
// The decision itself, on values (so that a kernel can take it from local copies of the
// state): the new iteration count and relative residual, then a non-finite stop, a request
// for an FP64 replacement, the iteration cap, or the next beta and rho (next = 1).
struct PcgStep {
  int iter, done, repl, next;
  double rel, beta, rho;
};
__device__ __forceinline__ PcgStep pcg_decide(int iter0, int done, int max_iter, double ref, double tol, double thr,
                                              double rho, double rz, double rr) {
  PcgStep s{iter0 + 1, done, 0, 0, sqrt(rr) / ref, 0.0, rho};
  if (!isfinite(rz) || !isfinite(rr)) {
    if (done == 0) s.done = PCG_NONFINITE;
  } else if (done == 0) {
    if (s.rel < tol || s.rel < thr) {
      s.repl = 1;  // the host verifies / replaces with the FP64 true residual
    } else if (s.iter >= max_iter) {
      s.done = PCG_MAXITER;
    } else {
      s.next = 1;
      s.beta = rz / rho;
      s.rho = rz;
    }
  }
  return s;
}

__device__ __forceinline__ void pcg_finish_update(PcgState* st, double rz, double rr) {
  // every field this needs, loaded before the first store (one round trip)
  const int iter = __ldcg(&st->iter);
  const int done = __ldcg(&st->done);
  const int max_iter = __ldcg(&st->max_iter);
  const double ref = __ldcg(&st->ref), tol = __ldcg(&st->tol), thr = __ldcg(&st->repl_threshold);
  const double rho = __ldcg(&st->rho);
  const PcgStep s = pcg_decide(iter, done, max_iter, ref, tol, thr, rho, rz, rr);
  st->iter = s.iter;
  st->rel = s.rel;
  if (s.done != done) st->done = s.done;
  if (s.repl) st->repl = 1;
  if (s.next) {
    st->beta = s.beta;
    st->rho = s.rho;
  }
}

// p . A p from the per-tile sums, in one fixed order (thread t sums tiles t, t + 256, ...;
// warp butterflies; warps in index order): every block that calls it, and the last tile of
// the fused apply, get the same bits. Valid in thread 0; needs 256 threads and red[8].
__device__ __forceinline__ double pcg_tile_total(const double* tile_part, int n_tiles, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) s += __ldcg(tile_part + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double pap = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pap += red[w];
  return pap;
}

// alpha from p . A p, or the reason to stop: p.Ap = 0 or non-finite ends the solve; negative
// curvature ends a truncated (Newton inner) solve after its first iteration, and does not
// stop plain CG. Returns 0 (go on, *alpha set) or a PCG_* code.
__device__ __forceinline__ int pcg_alpha(double pap, double rho, int truncate, int iter, double* alpha) {
  if (pap == 0.0 || !isfinite(pap)) return isfinite(pap) ? PCG_BREAKDOWN : PCG_NONFINITE;
  if (pap < 0.0 && truncate != 0 && iter > 0) return PCG_NEGCURV;
  *alpha = rho / pap;
  return 0;
}

// The vector part of the update for the DOFs of reduction block vb (of kReduceBlocks x
// kReduceThreads; thread t takes i = vb * 256 + t + k * S, S = 296 * 256, in k order):
// x += alpha p, r -= alpha q, and r.z, r.r of the new residual accumulated into v. Loads of
// U consecutive k are issued before their arithmetic; the arithmetic and its order are those
// of the plain loop (any U gives the same bits). r, p, q go through L2 only (other CTAs of a
// persistent launch write them).
template <int U>
__device__ __forceinline__ void pcg_update_range_from(int64_t n, double* x, double* r, const double* p,
                                                      const double* q, const double* dinv, double alpha, int64_t i0,
                                                      double (&v)[2]) {
  const int64_t S = (int64_t)kReduceBlocks * kReduceThreads;
  for (int64_t i = i0; i < n; i += U * S) {
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

template <int U>
__device__ __forceinline__ void pcg_update_range(int64_t n, double* x, double* r, const double* p, const double* q,
                                                 const double* dinv, double alpha, int vb, double (&v)[2]) {
  pcg_update_range_from<U>(n, x, r, p, q, dinv, alpha, (int64_t)vb * kReduceThreads + threadIdx.x, v);
}

}  // namespace pfem
