// Warm-started solvers on the device (Sec. "Warm-start"; App. B linear system and
// Newton-Raphson with load steps).
//
// Jacobi-PCG keeps every vector, dot and norm in FP64 on the GPU; the operator applications
// inside the iteration run in the requested element precision. With the FP32 operator the
// recursive residual drifts from the true one at the 1e-7 level, so the iteration stops for
// an FP64 residual replacement (true residual with the FP64 operator swapped in for the
// recursive one, search direction kept) whenever the recursive residual has dropped by
// repl_factor since the last replacement, and before declaring convergence: the stopping
// rule ||f - K u|| / ref < tol is always confirmed with the FP64 operator.
//
// Solver modes (pfem_set_solver_mode), all giving bitwise identical iterates:
//   0  persistent: one cooperative launch runs iterations until the state asks for a
//      replacement or terminates (kernels_pcg.cu); FP32 element arithmetic. Where it cannot
//      run (FP64 arithmetic, no co-resident grid) mode 2 takes over.
//   1  plain: the two kernels of one iteration at a time, host-synchronised check after each.
//   2  graph (default): the iteration body (fused apply + update) captured once per mesh into
//      a CUDA graph whose while-conditional node repeats it on the device. On GB300 it beats
//      the persistent kernel, whose register footprint halves the resident tiles per SM.
// In modes 0 and 2 the host synchronises only a handful of times per solve.

#include <cmath>
#include <cstring>
#include <vector>

#include "kernels_vec.cuh"
#include "pfem_internal.h"
#include "solver.h"

namespace pfem {

static int g_solver_mode = 2;  // 0 = persistent kernel, 1 = plain host loop, 2 = while-loop graph (default)

struct SolverWS {
  int64_t n = 0;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *dinv = nullptr, *res = nullptr;
  double *u = nullptr, *rn = nullptr, *tmp = nullptr, *p2 = nullptr;
  double* uc = nullptr;              // Newton: state at the last converged load level
  double* tile_part = nullptr;       // per-tile p . A p partials of the fused apply
  unsigned int* ticket = nullptr;    // last-tile ticket of the fused apply
  GridBar* bar = nullptr;            // grid barrier of the persistent kernel
  PcgState* st = nullptr;    // device
  PcgState* hst = nullptr;   // pinned host mirror
  double* dnorm = nullptr;   // device scalar
  void* block = nullptr;
  size_t bytes = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [ct][use_u]
  int64_t body_kernels[2][2] = {{0, 0}, {0, 0}};  // kernels per captured iteration
  bool graph_failed = false;
  bool persist_failed[2] = {false, false};  // [use_u]
  // kernel timing (plain loop): events around the apply and the update of an iteration
  cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};
  bool t_pending = false;
  double t_apply_ms = 0.0, t_update_ms = 0.0;
  int t_n = 0;
};

static int g_kernel_timing = 0;
static long long g_barrier_spin_limit = kBarrierSpinLimit;  // persistent kernel's barrier waits
static int g_absent_cta = -1;                               // failure-detection test hook

__global__ void set_cond_kernel(cudaGraphConditionalHandle h, const PcgState* st) {
  cudaGraphSetConditional(h, (st->done == 0 && st->repl == 0) ? 1u : 0u);
}

__global__ void norm_to_ref_kernel(const double* nrm, PcgState* st) {
  const double v = *nrm;
  st->ref = v > 0.0 ? v : 1.0;
}

static SolverWS* ws_of(pfem_mesh_t m) { return static_cast<SolverWS*>(m->solver); }

size_t solver_bytes(pfem_mesh_t m) { return m && m->solver ? ws_of(m)->bytes : 0; }

void solver_release(pfem_mesh_t m) {
  SolverWS* w = ws_of(m);
  if (!w) return;
  for (auto& row : w->exec)
    for (auto& e : row)
      if (e) cudaGraphExecDestroy(e);
  if (w->cap) cudaStreamDestroy(w->cap);
  for (cudaEvent_t e : w->tev)
    if (e) cudaEventDestroy(e);
  if (w->block) cudaFree(w->block);
  if (w->hst) cudaFreeHost(w->hst);
  delete w;
  m->solver = nullptr;
}

static pfem_status ws_get(pfem_mesh_t m, SolverWS** out) {
  if (m->solver) {
    *out = ws_of(m);
    return PFEM_OK;
  }
  SolverWS* w = new SolverWS();
  w->n = m->n_dofs;
  const size_t vb = ((size_t)w->n * sizeof(double) + 255) & ~size_t(255);
  const size_t tb = ((size_t)std::max(m->plan.n_tiles, 1) * sizeof(double) + 255) & ~size_t(255);
  w->bytes = 11 * vb + tb + 1024;
  cudaError_t e = cudaMalloc(&w->block, w->bytes);
  if (e != cudaSuccess) {
    delete w;
    return cuda_fail(e, "cudaMalloc(solver workspace)");
  }
  char* b = static_cast<char*>(w->block);
  double** vecs[11] = {&w->x, &w->r, &w->p, &w->q, &w->dinv, &w->res, &w->u, &w->rn, &w->tmp, &w->p2, &w->uc};
  for (int i = 0; i < 11; ++i) *vecs[i] = reinterpret_cast<double*>(b + i * vb);
  w->tile_part = reinterpret_cast<double*>(b + 11 * vb);
  w->st = reinterpret_cast<PcgState*>(b + 11 * vb + tb);
  w->dnorm = reinterpret_cast<double*>(b + 11 * vb + tb + 256);
  w->ticket = reinterpret_cast<unsigned int*>(b + 11 * vb + tb + 512);
  w->bar = reinterpret_cast<GridBar*>(b + 11 * vb + tb + 640);
  e = cudaMemset(w->ticket, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMallocHost(&w->hst, sizeof(PcgState));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(w->block);
    if (w->hst) cudaFreeHost(w->hst);
    delete w;
    return cuda_fail(e, "solver workspace");
  }
  m->solver = w;
  *out = w;
  return PFEM_OK;
}

// One PCG iteration in two kernels: the fused apply (p = dinv r + beta p_old, q = A p,
// alpha = rho / p.Ap) and the update (x += alpha p, r -= alpha q, rho, beta, flags).
// ev (plain loop, kernel timing): three events recorded before, between and after the kernels.
static pfem_status pcg_body(pfem_mesh_t m, SolverWS* w, pfem_dtype ct, bool use_u, cudaStream_t s,
                            cudaGraphConditionalHandle h, int set_cond, cudaEvent_t* ev = nullptr) {
  OpArgs a{use_u ? w->u : nullptr, nullptr, w->q, nullptr, nullptr, 1.0};
  a.pcg.r = w->r;
  a.pcg.dinv = w->dinv;
  a.pcg.p[0] = w->p;
  a.pcg.p[1] = w->p2;
  a.pcg.st = w->st;
  a.pcg.tile_part = w->tile_part;
  a.pcg.ticket = w->ticket;
  a.pcg.alpha_by_update = 1;  // the update kernel forms alpha from the tile sums
  if (ev) PFEM_CUDA(cudaEventRecord(ev[0], s));
  pfem_status st = launch_element_op(m->plan, OP_TANGENT | OP_PCG, PFEM_F64, ct, a, s);
  if (st) return st;
  if (ev) PFEM_CUDA(cudaEventRecord(ev[1], s));
  st = vk_update(w->n, w->x, w->r, w->p, w->p2, w->q, w->dinv, w->st, w->tile_part, (int)m->plan.n_tiles,
                 m->red_partials, m->red_counter, h, set_cond, s);
  if (st) return st;
  if (ev) PFEM_CUDA(cudaEventRecord(ev[2], s));
  return PFEM_OK;
}

// PCG iterations per replay of the graph's while-loop body (fewer conditional-node
// evaluations per iteration; the iterates do not depend on it).
constexpr int kGraphUnroll = 8;

static pfem_status build_graph(pfem_mesh_t m, SolverWS* w, pfem_dtype ct, bool use_u, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  PFEM_CUDA(cudaGraphCreate(&g, 0));
  auto fail = [&](cudaError_t e) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return cuda_fail(e, "building the PCG while-loop graph");
  };
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e);
  // pre-node: condition = state still running (so a finished state runs the body zero times)
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  void* args[2] = {&h, &w->st};
  kp.func = (void*)set_cond_kernel;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = args;
  cudaGraphNode_t pre, cn;
  e = cudaGraphAddKernelNode(&pre, g, nullptr, 0, &kp);
  if (e != cudaSuccess) return fail(e);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(&cn, g, &pre, nullptr, 1, &cp);
  if (e != cudaSuccess) return fail(e);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(w->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(e);
  const int64_t before = g_kernel_launches;
  // kGraphUnroll iterations per replay of the body; the kernels of an iteration after the
  // state stops return at once, and only the body's last update sets the condition
  pfem_status st = PFEM_OK;
  for (int j = 0; j < kGraphUnroll && st == PFEM_OK; ++j)
    st = pcg_body(m, w, ct, use_u, w->cap, h, j == kGraphUnroll - 1 ? 1 : 0);
  w->body_kernels[ct == PFEM_F64][use_u ? 1 : 0] = g_kernel_launches - before;
  g_kernel_launches = before;  // captured, not run: replays are counted per launch
  e = cudaStreamEndCapture(w->cap, &body);
  if (st != PFEM_OK) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(e);
  e = cudaGraphInstantiate(out, g, 0);
  if (e != cudaSuccess) return fail(e);
  cudaGraphDestroy(g);
  return PFEM_OK;
}

// Residual for a replacement: linear solve -> res = P (f_int(x) - s f) with the FP64
// operator; Newton inner solve (A d = -rn) -> res = rn + A64(u) x.
static pfem_status true_residual(pfem_mesh_t m, SolverWS* w, bool newton_inner, cudaStream_t s) {
  if (!newton_inner) {
    OpArgs a{w->x, nullptr, nullptr, w->res, nullptr, m->load_scale};
    return launch_element_op(m->plan, OP_RESIDUAL, PFEM_F64, PFEM_F64, a, s);
  }
  OpArgs a{w->u, w->x, w->res, nullptr, nullptr, 1.0};
  pfem_status st = launch_element_op(m->plan, OP_TANGENT, PFEM_F64, PFEM_F64, a, s);
  if (st) return st;
  return vk_axpy(w->n, 1.0, w->rn, w->res, s);
}

static pfem_status read_state(pfem_mesh_t m, SolverWS* w) {
  PFEM_CUDA(cudaMemcpyAsync(w->hst, w->st, sizeof(PcgState), cudaMemcpyDeviceToHost, m->stream));
  PFEM_CUDA(cudaStreamSynchronize(m->stream));
  return PFEM_OK;
}

// Runs PCG from the current x (dinv, ref, tol, max_iter already set in the device state).
//
// Stagnation: an FP32 operator limits how far the true residual can fall (its rounding is a
// fixed fraction of ||A|| ||x||). When two consecutive FP64 replacements improve the true
// residual by less than 2x, a Newton inner solve stops with PCG_STAGNATED (its direction is
// as accurate as the arithmetic allows, and Newton checks progress in FP64 anyway); a linear
// solve continues with the FP64 element operator.
static pfem_status pcg_run(pfem_mesh_t m, SolverWS* w, pfem_dtype ct, bool use_u, bool newton_inner) {
  static const int kStagnated = PCG_STAGNATED;
  cudaStream_t s = m->stream;
  pfem_status st;
  const int ui = use_u ? 1 : 0;
  // both direction buffers start at zero (the first direction is p = dinv r with beta = 0)
  PFEM_CUDA(cudaMemsetAsync(w->p, 0, (size_t)w->n * sizeof(double), s));
  PFEM_CUDA(cudaMemsetAsync(w->p2, 0, (size_t)w->n * sizeof(double), s));
  if ((st = true_residual(m, w, newton_inner, s))) return st;
  if ((st = vk_replace(w->n, w->res, w->r, w->dinv, w->st, 1, m->red_partials, m->red_counter, s))) return st;
  bool replaced = true;  // the start is an FP64 true residual too
  double prev_true = -1.0;
  int stalls = 0;
  int pending_bodies0 = -1;  // body replays counted before the last graph launch
  int64_t pending_body = 0;
  for (;;) {
    if ((st = read_state(m, w))) return st;
    if (w->t_pending) {  // the timed iteration has completed (read_state synchronised)
      float a = 0.f, b = 0.f;
      PFEM_CUDA(cudaEventElapsedTime(&a, w->tev[0], w->tev[1]));
      PFEM_CUDA(cudaEventElapsedTime(&b, w->tev[1], w->tev[2]));
      w->t_apply_ms += a;
      w->t_update_ms += b;
      ++w->t_n;
      w->t_pending = false;
    }
    if (pending_bodies0 >= 0) {  // a graph launch ran (body replays x body) + the pre-node
      g_kernel_launches += (int64_t)(w->hst->bodies - pending_bodies0) * pending_body + 1;
      pending_bodies0 = -1;
    }
    if (replaced) {
      replaced = false;
      const double rt = w->hst->rel_true;
      stalls = (prev_true > 0.0 && !(rt < 0.5 * prev_true)) ? stalls + 1 : 0;
      prev_true = rt;
      if (stalls >= 2 && w->hst->done == 0) {
        if (newton_inner) {
          PFEM_CUDA(cudaMemcpyAsync(&w->st->done, &kStagnated, sizeof(int), cudaMemcpyHostToDevice, s));
          PFEM_CUDA(cudaStreamSynchronize(s));
          w->hst->done = PCG_STAGNATED;
          break;
        }
        if (ct != PFEM_F64) {
          ct = PFEM_F64;
          stalls = 0;
        }
      }
    }
    if (w->hst->done != 0) break;
    if (w->hst->repl != 0) {
      if ((st = true_residual(m, w, newton_inner, s))) return st;
      if ((st = vk_replace(w->n, w->res, w->r, w->dinv, w->st, 0, m->red_partials, m->red_counter, s))) return st;
      replaced = true;
      continue;
    }
    if (g_solver_mode == 0 && ct != PFEM_F64 && !w->persist_failed[ui]) {
      PersistArgs pa{use_u ? w->u : nullptr, w->x, w->r, w->dinv, {w->p, w->p2}, w->q, w->st, w->tile_part,
                     w->ticket, m->red_partials, m->red_counter, w->bar, w->n, g_barrier_spin_limit, g_absent_cta};
      st = launch_pcg_persistent(m->plan, ct, pa, s);
      if (st == PFEM_OK) continue;
      if (st != PFEM_ERR_UNSUPPORTED) return st;
      w->persist_failed[ui] = true;  // falls back to the graph (or plain) loop
    }
    cudaGraphExec_t* ex = &w->exec[ct == PFEM_F64][ui];
    if (g_solver_mode != 1 && !w->graph_failed && !*ex && build_graph(m, w, ct, use_u, ex) != PFEM_OK) {
      w->graph_failed = true;
      *ex = nullptr;
    }
    if (g_solver_mode != 1 && !w->graph_failed && *ex) {
      pending_bodies0 = w->hst->bodies;
      pending_body = w->body_kernels[ct == PFEM_F64][ui];
      PFEM_CUDA(cudaGraphLaunch(*ex, s));
    } else {
      const bool timed = g_kernel_timing != 0;
      if (timed && !w->tev[0])
        for (cudaEvent_t& e : w->tev) PFEM_CUDA(cudaEventCreate(&e));
      if ((st = pcg_body(m, w, ct, use_u, s, cudaGraphConditionalHandle(), 0, timed ? w->tev : nullptr))) return st;
      w->t_pending = timed;
    }
  }
  return PFEM_OK;
}

static void timing_reset(SolverWS* w) {
  w->t_pending = false;
  w->t_apply_ms = w->t_update_ms = 0.0;
  w->t_n = 0;
}

static void timing_report(const SolverWS* w, pfem_solve_info* info) {
  info->apply_ms = w->t_apply_ms;
  info->update_ms = w->t_update_ms;
  info->timed_iterations = w->t_n;
}

static pfem_status set_state(pfem_mesh_t m, SolverWS* w, double tol, int max_iter, int truncate = 0) {
  PcgState h;
  std::memset(&h, 0, sizeof(h));
  h.tol = tol;
  h.max_iter = max_iter;
  h.truncate = truncate;
  h.repl_factor = 1e-2;
  h.repl_threshold = 0.0;
  h.ref = 1.0;
  *w->hst = h;
  PFEM_CUDA(cudaMemcpyAsync(w->st, w->hst, sizeof(PcgState), cudaMemcpyHostToDevice, m->stream));
  PFEM_CUDA(cudaStreamSynchronize(m->stream));  // the pinned mirror is reused right away
  return PFEM_OK;
}

// ref = ||P (f_int(u_lift) - s f)||, u_lift = prescribed values (x s) with zero free DOFs.
static pfem_status reference_norm(pfem_mesh_t m, SolverWS* w, double scale) {
  cudaStream_t s = m->stream;
  pfem_status st;
  if ((st = vk_lift(w->n, nullptr, m->plan.dvalues, m->plan.dmask, scale, w->tmp, s))) return st;
  OpArgs a{w->tmp, nullptr, nullptr, w->res, nullptr, scale};
  if ((st = launch_element_op(m->plan, OP_RESIDUAL, PFEM_F64, PFEM_F64, a, s))) return st;
  if ((st = vk_norm2(w->n, w->res, w->dnorm, m->red_partials, m->red_counter, s))) return st;
  norm_to_ref_kernel<<<1, 1, 0, s>>>(w->dnorm, w->st); PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  return PFEM_OK;
}

static pfem_status jacobi(pfem_mesh_t m, SolverWS* w, pfem_dtype ct, const double* u) {
  // the diagonal lands in q (FP64), then dinv = 1 / d
  OpArgs a{u, nullptr, nullptr, nullptr, w->q, 1.0};
  pfem_status st = launch_element_op(m->plan, OP_DIAG, PFEM_F64, ct, a, m->stream);
  if (st) return st;
  return vk_invert_diag(w->n, w->q, PFEM_F64, w->dinv, m->stream);
}

static pfem_status status_of(int done) {
  switch (done) {
    case PCG_CONVERGED: return PFEM_OK;
    case PCG_MAXITER: return PFEM_ERR_NOT_CONVERGED;
    case PCG_NONFINITE: return PFEM_ERR_NONFINITE;
    case PCG_STAGNATED: set_error("PCG stagnated above the tolerance with the FP64 operator"); return PFEM_ERR_NOT_CONVERGED;
    case PCG_BARRIER_TIMEOUT: set_error("a grid barrier of the persistent PCG kernel timed out"); return PFEM_ERR_TIMEOUT;
    default: return PFEM_ERR_NOT_CONVERGED;
  }
}

pfem_status solve_multi_core(pfem_mesh_t m, pfem_dtype dt, int k, const double* b, const double* u0, double tol,
                             int max_iter, double* u_out, pfem_solve_info* infos);

// A linear solve on a mesh with penalty springs: the multi-solve path with one right-hand
// side b = s f_ext (prescribed values must be zero there: no lifting of nonzero values).
static pfem_status solve_with_springs(pfem_mesh_t m, pfem_dtype dt, const double* u0, double tol, int max_iter,
                                      double* u_out, pfem_solve_info* info) {
  if (m->load_scale != 1.0) {
    set_error("meshes with penalty springs solve at load scale 1 only");
    return PFEM_ERR_UNSUPPORTED;
  }
  std::vector<double> v((size_t)m->n_dofs);
  PFEM_CUDA(cudaMemcpy(v.data(), m->plan.dvalues, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (double x : v)
    if (x != 0.0) {
      set_error("meshes with penalty springs need zero prescribed values");
      return PFEM_ERR_UNSUPPORTED;
    }
  pfem_solve_info tmp;
  return solve_multi_core(m, dt, 1, m->plan.f_ext, u0, tol, max_iter, u_out, info ? info : &tmp);
}

}  // namespace pfem

using namespace pfem;

extern "C" {

pfem_status pfem_set_solver_mode(int32_t mode) {
  if (mode < 0 || mode > 2) {
    set_error("solver mode must be 0 (persistent), 1 (plain) or 2 (graph)");
    return PFEM_ERR_INVALID_ARG;
  }
  g_solver_mode = mode;
  return PFEM_OK;
}

pfem_status pfem_set_barrier_test(int64_t spin_limit, int32_t absent_cta) {
  if (absent_cta < -1) {
    set_error("absent_cta must be -1 (none) or a CTA index");
    return PFEM_ERR_INVALID_ARG;
  }
  g_barrier_spin_limit = spin_limit > 0 ? (long long)spin_limit : kBarrierSpinLimit;
  g_absent_cta = absent_cta;
  return PFEM_OK;
}

pfem_status pfem_set_kernel_timing(int32_t on) {
  if (on != 0 && on != 1) {
    set_error("kernel timing must be 0 (off) or 1 (on)");
    return PFEM_ERR_INVALID_ARG;
  }
  g_kernel_timing = on;
  return PFEM_OK;
}

pfem_status pfem_solve_linear(pfem_mesh_t m, pfem_dtype dt, const double* u0, double tol, int32_t max_iter,
                              double* u_out, pfem_solve_info* info) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (m->plan.kind != PFEM_LINEAR) {
    set_error("pfem_solve_linear needs a linear-elastic mesh (use pfem_solve_newton)");
    return PFEM_ERR_INVALID_ARG;
  }
  if (!u_out || !(tol > 0.0) || max_iter < 0 || (dt != PFEM_F32 && dt != PFEM_F64)) {
    set_error("invalid solve arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  if (m->n_spring_nodes) return solve_with_springs(m, dt, u0, tol, max_iter, u_out, info);
  SolverWS* w;
  const int64_t launches0 = g_kernel_launches;
  if ((st = ws_get(m, &w))) return st;
  timing_reset(w);
  cudaStream_t s = m->stream;
  if ((st = set_state(m, w, tol, max_iter))) return st;
  if ((st = reference_norm(m, w, m->load_scale))) return st;
  if ((st = jacobi(m, w, dt, nullptr))) return st;
  if ((st = vk_lift(w->n, u0, m->plan.dvalues, m->plan.dmask, m->load_scale, w->x, s))) return st;
  if ((st = pcg_run(m, w, dt, false, false))) return st;
  PFEM_CUDA(cudaMemcpyAsync(u_out, w->x, (size_t)w->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if ((st = read_state(m, w))) return st;
  const PcgState& h = *w->hst;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iterations = h.iter;
    info->replacements = h.replacements;
    info->rel_residual_recursive = h.rel;
    info->rel_residual_true_f64 = h.rel_true;
    info->reference_norm = h.ref;
  }
  st = status_of(h.done);
  if (info) {
    info->status = st;
    info->kernel_launches = g_kernel_launches - launches0;
    timing_report(w, info);
  }
  if (st) set_error("PCG stopped with state %d after %d iterations (rel %g)", h.done, h.iter, h.rel_true);
  return st;
}

pfem_status pfem_solve_newton(pfem_mesh_t m, pfem_dtype dt, const double* u0, double tol, int32_t n_load_steps,
                              int32_t max_newton, double inner_tol, double* u_out, pfem_solve_info* info) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (!u_out || !(tol > 0.0) || !(inner_tol > 0.0) || n_load_steps < 1 || max_newton < 1 ||
      (dt != PFEM_F32 && dt != PFEM_F64)) {
    set_error("invalid Newton arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  if (m->n_spring_nodes) {
    set_error("pfem_solve_newton does not include penalty springs");
    return PFEM_ERR_UNSUPPORTED;
  }
  SolverWS* w;
  const int64_t launches0 = g_kernel_launches;
  if ((st = ws_get(m, &w))) return st;
  timing_reset(w);
  cudaStream_t s = m->stream;
  const double saved_scale = m->load_scale;
  struct ScaleRestore {  // the caller's load scale comes back on every return path
    pfem_mesh_t m;
    double v;
    ~ScaleRestore() { m->load_scale = v; }
  } restore{m, saved_scale};
  const int64_t n = w->n;
  int total_inner = 0, n_newton = 0, n_repl = 0, n_back = 0;
  double init_rel = -1.0, final_rel = 0.0, ref = 1.0;
  pfem_status result = PFEM_OK;
  if (u0) PFEM_CUDA(cudaMemcpyAsync(w->u, u0, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else PFEM_CUDA(cudaMemsetAsync(w->u, 0, (size_t)n * sizeof(double), s));
  const int inner_max = (int)std::min<int64_t>(10 * n + 100, kInnerMaxIter);
  LoadSchedule ls;
  ls.start(n_load_steps);
  PFEM_CUDA(cudaMemcpyAsync(w->uc, w->u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (;;) {
    const double scale = saved_scale * ls.fraction();
    m->load_scale = scale;
    if ((st = vk_lift(n, w->u, m->plan.dvalues, m->plan.dmask, scale, w->u, s))) break;
    if ((st = set_state(m, w, inner_tol, inner_max))) break;
    if ((st = reference_norm(m, w, scale))) break;
    if ((st = read_state(m, w))) break;
    ref = w->hst->ref;
    for (int it = 0;; ++it) {
      OpArgs a{w->u, nullptr, nullptr, w->rn, nullptr, scale};
      if ((st = launch_element_op(m->plan, OP_RESIDUAL, PFEM_F64, PFEM_F64, a, s))) break;
      if ((st = vk_norm2(n, w->rn, w->dnorm, m->red_partials, m->red_counter, s))) break;
      PFEM_CUDA(cudaMemcpyAsync(m->host_out, w->dnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
      PFEM_CUDA(cudaStreamSynchronize(s));
      const double rel = m->host_out[0] / ref;
      if (init_rel < 0) init_rel = rel;
      final_rel = rel;
      if (!std::isfinite(rel)) {
        result = PFEM_ERR_NONFINITE;
        break;
      }
      if (rel <= tol) break;
      if (it >= max_newton) {
        result = PFEM_ERR_NOT_CONVERGED;
        set_error("Newton: %d iterations at load fraction %g, rel residual %g", it, ls.fraction(), rel);
        break;
      }
      // inner solve A(u) d = -rn from d = 0 to inner_tol relative to ||rn||
      if ((st = set_state(m, w, inner_tol, inner_max, 1))) break;
      PFEM_CUDA(cudaMemcpyAsync(&w->st->ref, w->dnorm, sizeof(double), cudaMemcpyDeviceToDevice, s));
      if ((st = jacobi(m, w, dt, w->u))) break;
      PFEM_CUDA(cudaMemsetAsync(w->x, 0, (size_t)n * sizeof(double), s));
      if ((st = pcg_run(m, w, dt, true, true))) break;
      if ((st = read_state(m, w))) break;
      total_inner += w->hst->iter;
      n_repl += w->hst->replacements;
      if (w->hst->done != PCG_CONVERGED && w->hst->done != PCG_MAXITER && w->hst->done != PCG_STAGNATED &&
          w->hst->done != PCG_NEGCURV) {
        result = status_of(w->hst->done);
        set_error("inner PCG failed with state %d", w->hst->done);
        break;
      }
      // step with halving while any element would invert
      double t = 1.0;
      bool ok = false;
      for (int k = 0; k <= 10; ++k) {
        PFEM_CUDA(cudaMemcpyAsync(w->tmp, w->u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if ((st = vk_axpy(n, t, w->x, w->tmp, s))) break;
        PFEM_CUDA(cudaMemsetAsync(m->plan.inverted, 0, sizeof(int32_t), s));
        OpArgs ea{w->tmp, nullptr, nullptr, nullptr, nullptr, scale};
        if ((st = launch_element_op(m->plan, OP_ENERGY, PFEM_F64, PFEM_F64, ea, s))) break;
        PFEM_CUDA(cudaMemcpyAsync(m->host_int, m->plan.inverted, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PFEM_CUDA(cudaStreamSynchronize(s));
        if (m->host_int[0] == 0) {
          ok = true;
          break;
        }
        ++n_back;
        t *= 0.5;
      }
      if (st) break;
      if (!ok) {
        result = PFEM_ERR_INVERTED;
        set_error("Newton: every trial step inverts an element");
        break;
      }
      PFEM_CUDA(cudaMemcpyAsync(w->u, w->tmp, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      ++n_newton;
    }
    if (st) break;
    if (result == PFEM_OK) {  // this level converged
      if (ls.last()) break;
      ls.converged();
      PFEM_CUDA(cudaMemcpyAsync(w->uc, w->u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      continue;
    }
    const bool retry = result == PFEM_ERR_INVERTED || result == PFEM_ERR_NOT_CONVERGED || result == PFEM_ERR_NONFINITE;
    if (!retry || !ls.cut()) break;
    result = PFEM_OK;  // again from the last converged state with half the increment
    PFEM_CUDA(cudaMemcpyAsync(w->u, w->uc, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (st) return st;
  PFEM_CUDA(cudaMemcpyAsync(u_out, w->u, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PFEM_CUDA(cudaStreamSynchronize(s));
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iterations = total_inner;
    info->newton_iterations = n_newton;
    info->replacements = n_repl;
    info->inverted_backtracks = n_back;
    info->rel_residual_recursive = final_rel;
    info->rel_residual_true_f64 = final_rel;
    info->initial_rel_residual = init_rel;
    info->reference_norm = ref;
    info->status = result;
    info->kernel_launches = g_kernel_launches - launches0;
    info->load_step_cuts = ls.cuts;
    timing_report(w, info);
  }
  return result;
}

}  // extern "C"
