// Serving: continuous batching of warm-started solves (Sec. "Warm-start": a platform receives
// problems and refines the pretrained prediction by FE iterations).
//
// Requests arrive through pfem_serve_submit. Planner threads validate and tile their meshes
// on the host while the GPU works. A single worker thread owns the GPU stream: it admits
// planned requests while a slot is free and their device footprint fits the HBM budget,
// uploads them, and then advances every resident solve together. One "step" is two
// launches shared by all resident solves: the PCG-fused element apply (one CTA per
// (solve, tile), linear or Neo-Hookean per solve) and the update (a fixed block range per
// solve). Chunks of steps run back to back; between chunks the worker reads every solve's
// scalar state in one copy and drives each solve's own state machine: FP64 residual
// replacements and convergence checks for PCG; residual, tangent set-up and step-halving
// line search for Newton. Solves finish independently and free their slot and memory, and
// waiting requests are admitted, while the others keep iterating.
//
// Each solve's arithmetic (tiles, reduction partitioning, decisions) depends only on the
// solve itself, so its result is bitwise the same alone and in any mix.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels_vec.cuh"
#include "pfem_internal.h"

namespace pfem {

namespace {

constexpr int PCG_PAUSED = 5;  // a solve not in a PCG phase: skipped by the shared steps
constexpr int kAux = 4;        // per-solve scalar results read back each chunk

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

__global__ void init_state_kernel(PcgState* st, double tol, int max_iter, const double* ref_src, int done,
                                  int truncate) {
  PcgState s;
  memset(&s, 0, sizeof(s));
  s.tol = tol;
  s.max_iter = max_iter;
  s.truncate = truncate;
  s.repl_factor = 1e-2;
  s.ref = 1.0;
  if (ref_src) s.ref = *ref_src > 0.0 ? *ref_src : 1.0;
  s.done = done;
  *st = s;
}

// keep the start's relative residual (the Sec. "Warm-start" skip-test quantity) for the report
__global__ void save_init_rel_kernel(const PcgState* st, double* dst) { *dst = st->rel_true; }

struct StateSlot {
  PcgState st;
  double aux[kAux];
  int32_t inverted;
  int32_t pad;
};

__global__ void gather_states_kernel(PcgState* const* st, double* const* aux, int32_t* const* inv, int n,
                                     StateSlot* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i].st = *st[i];
  for (int k = 0; k < kAux; ++k) out[i].aux[k] = aux[i][k];
  out[i].inverted = *inv[i];
}

enum Phase {
  PH_LIN_RUN,    // linear PCG in the shared steps
  PH_NT_REF,     // waiting for the load step's reference norm
  PH_NT_CHECK,   // waiting for the Newton residual norm
  PH_NT_INNER,   // inner PCG in the shared steps
  PH_NT_LS,      // waiting for the inverted-element count of a trial step
  PH_FINISHED,
};

struct Request {
  uint64_t ticket = 0;
  int solve_kind = PFEM_SOLVE_LINEAR;
  // owned copy of the description
  pfem_mesh_desc desc{};
  std::vector<double> coords, mat_a, mat_b, values, traction, f_extra, u0;
  std::vector<int32_t> conn, facets;
  std::vector<uint8_t> mask;
  double tol = 1e-8;
  int n_load_steps = 1;
  // planning
  HostPlan plan;
  std::vector<double> fext;
  pfem_status plan_status = PFEM_OK;
  bool planned = false;
  size_t footprint = 0;
  // device
  pfem_mesh_t mesh = nullptr;
  void* block = nullptr;
  double *x = nullptr, *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr, *dinv = nullptr;
  double *res = nullptr, *u = nullptr, *rn = nullptr, *tmp = nullptr, *tile_part = nullptr, *upart = nullptr;
  double* uc = nullptr;  // Newton: state at the last converged load level
  double* aux = nullptr;
  unsigned *ticket_dev = nullptr, *ucount = nullptr;
  PcgState* st = nullptr;
  int nublk = 1;
  int64_t n = 0;
  // state machine
  Phase phase = PH_LIN_RUN;
  LoadSchedule load;
  int level_newton = 0;  // Newton steps at the current load level
  double ref = 1.0, t_ls = 1.0;
  int newton = 0, inner_iters = 0, repl = 0, backtracks = 0, ls_tries = 0;
  double init_rel = -1.0, last_rel = 0.0;
  // FP64 replacements of the current PCG solve: a true residual that improves by less than
  // 2x twice in a row ends a Newton inner solve as stagnated (the FP32 operator's limit)
  bool replaced = false;
  double prev_true = -1.0;
  int stalls = 0;
  // result
  std::vector<double> result;
  pfem_solve_info info{};
  pfem_status status = PFEM_PENDING;
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool done = false;
};

}  // namespace
}  // namespace pfem

using namespace pfem;

struct pfem_server_s {
  size_t budget = 0;
  int max_slots = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;    // stream-ordered allocations of resident solves
  std::mutex mu;
  std::condition_variable cv_work, cv_plan, cv_done;
  std::deque<Request*> queue;      // submitted, in arrival order (planned or not)
  std::deque<Request*> to_plan;
  std::unordered_map<uint64_t, Request*> tickets;
  std::vector<Request*> active;
  std::atomic<bool> stop{false};
  std::thread worker;
  std::vector<std::thread> planners;
  uint64_t next_ticket = 1;
  size_t used = 0;
  int pending = 0;                 // submitted and not finished
  pfem_status fatal = PFEM_OK;
  // device tables of the active set
  bool dirty = true;
  ReqDev* d_reqs = nullptr;
  int2* d_btile = nullptr;
  int* d_ublk = nullptr;
  PcgState** d_stp = nullptr;
  double** d_auxp = nullptr;
  int32_t** d_invp = nullptr;
  StateSlot* d_slots = nullptr;
  StateSlot* h_slots = nullptr;
  size_t cap_reqs = 0, cap_btile = 0, cap_ublk = 0;
  ServeTiles tiles[2];  // linear, Neo-Hookean apply blocks
  int n_update = 0;
  std::vector<int> active_index;   // position of each active request in the tables
  // one chunk (kChunk shared steps, the state gather and its read-back) captured as a CUDA
  // graph for the current tables; captured again whenever the tables change
  cudaGraphExec_t chunk_exec = nullptr;
  int64_t chunk_kernels = 0;       // kernels per replay of the chunk graph
  bool graph_failed = false;       // capture unavailable: plain launches
  // worker-thread wall time by activity (s) and counts, for pfem_serve_stats
  std::atomic<double> t_wait{0.0}, t_admit{0.0}, t_tables{0.0}, t_advance{0.0};
  std::atomic<int64_t> n_chunks{0}, n_rebuilds{0}, n_admitted{0};
};

namespace pfem {
namespace {

pfem_status grow(void** p, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap && *p) return PFEM_OK;
  size_t c = std::max<size_t>(need, 2 * *cap + 16);
  if (*p) cudaFree(*p);
  *p = nullptr;
  PFEM_CUDA(cudaMalloc(p, c * elem));
  *cap = c;
  return PFEM_OK;
}

size_t request_bytes(const HostPlan& hp) {
  const int64_t n = hp.n_nodes * hp.dim;
  const size_t vb = ((size_t)n * 8 + 255) & ~size_t(255);
  return mesh_arena_bytes(hp) + 11 * vb + (size_t)hp.n_tiles() * 8 + 296 * 16 + 4096;
}

pfem_status admit(pfem_server_s* S, Request* R) {
  pfem_status st = mesh_upload(R->plan, R->fext, &R->desc, S->stream, &R->mesh, S->pool);
  if (st) return st;
  R->n = R->mesh->n_dofs;
  R->nublk = serve_update_blocks(R->n);
  const size_t vb = ((size_t)R->n * 8 + 255) & ~size_t(255);
  const size_t tb = ((size_t)std::max(R->mesh->plan.n_tiles, 1) * 8 + 255) & ~size_t(255);
  const size_t ub = ((size_t)R->nublk * 16 + 255) & ~size_t(255);
  const size_t bytes = 11 * vb + tb + ub + 1024;
  cudaError_t e = cudaMallocFromPoolAsync(&R->block, bytes, S->pool, S->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device allocation (serving workspace)");
  char* b = static_cast<char*>(R->block);
  double** v[11] = {&R->x, &R->r, &R->p0, &R->p1, &R->q, &R->dinv, &R->res, &R->u, &R->rn, &R->tmp, &R->uc};
  for (int i = 0; i < 11; ++i) *v[i] = reinterpret_cast<double*>(b + i * vb);
  R->tile_part = reinterpret_cast<double*>(b + 11 * vb);
  R->upart = reinterpret_cast<double*>(b + 11 * vb + tb);
  char* tail = b + 11 * vb + tb + ub;
  R->st = reinterpret_cast<PcgState*>(tail);
  R->aux = reinterpret_cast<double*>(tail + 256);
  R->ticket_dev = reinterpret_cast<unsigned*>(tail + 512);
  R->ucount = reinterpret_cast<unsigned*>(tail + 576);
  PFEM_CUDA(cudaMemsetAsync(tail, 0, 1024, S->stream));
  // start vector: u0 (host) or zero
  if (!R->u0.empty())
    PFEM_CUDA(cudaMemcpyAsync(R->u, R->u0.data(), (size_t)R->n * 8, cudaMemcpyHostToDevice, S->stream));
  else
    PFEM_CUDA(cudaMemsetAsync(R->u, 0, (size_t)R->n * 8, S->stream));
  PFEM_CUDA(cudaStreamSynchronize(S->stream));  // host copies of the request may be released
  R->t_admit = now_s();
  return PFEM_OK;
}

// ---- per-solve enqueue helpers (all on the server stream) ---------------------------------

pfem_status enq_residual64(Request* R, const double* u, double* out, double scale, cudaStream_t s) {
  OpArgs a{u, nullptr, nullptr, out, nullptr, scale};
  return launch_element_op(R->mesh->plan, OP_RESIDUAL, PFEM_F64, PFEM_F64, a, s);
}

pfem_status enq_norm(Request* R, const double* v, double* out, cudaStream_t s) {
  return vk_norm2(R->n, v, out, R->mesh->red_partials, R->mesh->red_counter, s);
}

// (Re)start PCG on A d = b from the current x: res = residual of the system at x, then
// r = -res, rho, beta = 0 (replace kernel, restart) and both directions zero.
pfem_status enq_pcg_start(Request* R, bool newton, double tol, const double* ref_src, cudaStream_t s) {
  const int max_iter = (int)std::min<int64_t>(10 * R->n + 100, newton ? kInnerMaxIter : 1000000);
  init_state_kernel<<<1, 1, 0, s>>>(R->st, tol, max_iter, ref_src, 0, newton ? 1 : 0);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaMemsetAsync(R->p0, 0, (size_t)R->n * 8, s));
  PFEM_CUDA(cudaMemsetAsync(R->p1, 0, (size_t)R->n * 8, s));
  pfem_status st;
  if (!newton) {
    if ((st = enq_residual64(R, R->x, R->res, 1.0, s))) return st;
  } else {  // res = rn + A64(u) x
    OpArgs a{R->u, R->x, R->res, nullptr, nullptr, 1.0};
    if ((st = launch_element_op(R->mesh->plan, OP_TANGENT, PFEM_F64, PFEM_F64, a, s))) return st;
    if ((st = vk_axpy(R->n, 1.0, R->rn, R->res, s))) return st;
  }
  R->replaced = true;
  R->prev_true = -1.0;
  R->stalls = 0;
  return vk_replace(R->n, R->res, R->r, R->dinv, R->st, 1, R->mesh->red_partials, R->mesh->red_counter, s);
}

pfem_status enq_replacement(Request* R, bool newton, cudaStream_t s) {
  R->replaced = true;
  pfem_status st;
  if (!newton) {
    if ((st = enq_residual64(R, R->x, R->res, 1.0, s))) return st;
  } else {
    OpArgs a{R->u, R->x, R->res, nullptr, nullptr, 1.0};
    if ((st = launch_element_op(R->mesh->plan, OP_TANGENT, PFEM_F64, PFEM_F64, a, s))) return st;
    if ((st = vk_axpy(R->n, 1.0, R->rn, R->res, s))) return st;
  }
  return vk_replace(R->n, R->res, R->r, R->dinv, R->st, 0, R->mesh->red_partials, R->mesh->red_counter, s);
}

pfem_status enq_jacobi(Request* R, const double* u, cudaStream_t s) {
  OpArgs a{u, nullptr, nullptr, nullptr, R->q, 1.0};
  pfem_status st = launch_element_op(R->mesh->plan, OP_DIAG, PFEM_F64, PFEM_F32, a, s);
  if (st) return st;
  return vk_invert_diag(R->n, R->q, PFEM_F64, R->dinv, s);
}

double load_scale_of(const Request* R) { return R->load.fraction(); }

// Newton: reference norm of this load step (lift the prescribed values first)
pfem_status enq_newton_step(Request* R, cudaStream_t s) {
  const double sc = load_scale_of(R);
  pfem_status st;
  if ((st = vk_lift(R->n, R->u, R->mesh->plan.dvalues, R->mesh->plan.dmask, sc, R->u, s))) return st;
  if ((st = vk_lift(R->n, nullptr, R->mesh->plan.dvalues, R->mesh->plan.dmask, sc, R->tmp, s))) return st;
  if ((st = enq_residual64(R, R->tmp, R->res, sc, s))) return st;
  if ((st = enq_norm(R, R->res, R->aux + 0, s))) return st;
  init_state_kernel<<<1, 1, 0, s>>>(R->st, R->tol, 1, nullptr, PCG_PAUSED, 0);
  PFEM_COUNT_LAUNCH();
  R->phase = PH_NT_REF;
  return PFEM_OK;
}

pfem_status enq_newton_check(Request* R, cudaStream_t s) {
  pfem_status st;
  if ((st = enq_residual64(R, R->u, R->rn, load_scale_of(R), s))) return st;
  if ((st = enq_norm(R, R->rn, R->aux + 1, s))) return st;
  R->phase = PH_NT_CHECK;
  return PFEM_OK;
}

pfem_status enq_line_search(Request* R, cudaStream_t s) {
  PFEM_CUDA(cudaMemcpyAsync(R->tmp, R->u, (size_t)R->n * 8, cudaMemcpyDeviceToDevice, s));
  pfem_status st;
  if ((st = vk_axpy(R->n, R->t_ls, R->x, R->tmp, s))) return st;
  PFEM_CUDA(cudaMemsetAsync(R->mesh->plan.inverted, 0, sizeof(int32_t), s));
  OpArgs a{R->tmp, nullptr, nullptr, nullptr, nullptr, load_scale_of(R)};
  if ((st = launch_element_op(R->mesh->plan, OP_ENERGY, PFEM_F64, PFEM_F64, a, s))) return st;
  R->phase = PH_NT_LS;
  return PFEM_OK;
}

pfem_status start_solve(Request* R, cudaStream_t s) {
  if (R->solve_kind == PFEM_SOLVE_LINEAR) {
    pfem_status st;
    // reference norm ||r(u_lift)||, Jacobi diagonal, lifted start, PCG start (skip test included)
    if ((st = vk_lift(R->n, nullptr, R->mesh->plan.dvalues, R->mesh->plan.dmask, 1.0, R->tmp, s))) return st;
    if ((st = enq_residual64(R, R->tmp, R->res, 1.0, s))) return st;
    if ((st = enq_norm(R, R->res, R->aux + 0, s))) return st;
    if ((st = enq_jacobi(R, nullptr, s))) return st;
    if ((st = vk_lift(R->n, R->u, R->mesh->plan.dvalues, R->mesh->plan.dmask, 1.0, R->x, s))) return st;
    if ((st = enq_pcg_start(R, false, R->tol, R->aux + 0, s))) return st;
    save_init_rel_kernel<<<1, 1, 0, s>>>(R->st, R->aux + 2);
    PFEM_COUNT_LAUNCH();
    R->phase = PH_LIN_RUN;
    return PFEM_OK;
  }
  R->load.start(R->n_load_steps);
  R->level_newton = 0;
  PFEM_CUDA(cudaMemcpyAsync(R->uc, R->u, (size_t)R->n * 8, cudaMemcpyDeviceToDevice, s));
  return enq_newton_step(R, s);
}

void finish(pfem_server_s* S, Request* R, pfem_status status) {
  if (R->mesh && status == PFEM_OK) {
    R->result.resize((size_t)R->n);
    const double* src = R->solve_kind == PFEM_SOLVE_LINEAR ? R->x : R->u;
    cudaMemcpyAsync(R->result.data(), src, (size_t)R->n * 8, cudaMemcpyDeviceToHost, S->stream);
  }
  cudaStreamSynchronize(S->stream);
  R->status = status;
  R->info.status = status;
  R->t_done = now_s();
  if (R->block) cudaFreeAsync(R->block, S->stream);  // stream-ordered: no device synchronisation
  R->block = nullptr;
  if (R->mesh) pfem_mesh_destroy(R->mesh);
  R->mesh = nullptr;
  R->phase = PH_FINISHED;
  std::lock_guard<std::mutex> lock(S->mu);
  S->used -= std::min(S->used, R->footprint);
  R->done = true;
  S->pending--;
  S->cv_done.notify_all();
}

// React to the state read after a chunk; returns false when the solve finished.
bool advance(pfem_server_s* S, Request* R, const StateSlot& sl) {
  cudaStream_t s = S->stream;
  const PcgState& ps = sl.st;
  pfem_status st = PFEM_OK;
  auto fail = [&](pfem_status e) {
    if (e != PFEM_OK && R->solve_kind != PFEM_SOLVE_LINEAR) {  // the work done before the failure
      R->info.iterations = R->inner_iters;
      R->info.newton_iterations = R->newton;
      R->info.replacements = R->repl;
      R->info.inverted_backtracks = R->backtracks;
      R->info.rel_residual_recursive = R->last_rel;
      R->info.initial_rel_residual = R->init_rel;
      R->info.reference_norm = R->ref;
    }
    R->info.load_step_cuts = R->load.cuts;
    finish(S, R, e);
    return false;
  };
  // a failed Newton load level: again from the last converged state with half the
  // increment, or the failure when the cuts are used up
  auto retry_level = [&](pfem_status e) {
    if (!R->load.cut()) return fail(e);
    if (cudaMemcpyAsync(R->u, R->uc, (size_t)R->n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail(PFEM_ERR_CUDA);
    R->level_newton = 0;
    const pfem_status st2 = enq_newton_step(R, s);
    if (st2) return fail(st2);
    return true;
  };
  switch (R->phase) {
    case PH_LIN_RUN:
      if (R->init_rel < 0) R->init_rel = sl.aux[2];
      if (ps.done == PCG_CONVERGED) {
        R->info.iterations = ps.iter;
        R->info.replacements = ps.replacements;
        R->info.rel_residual_recursive = ps.rel;
        R->info.rel_residual_true_f64 = ps.rel_true;
        R->info.reference_norm = ps.ref;
        R->info.initial_rel_residual = R->init_rel;
        return fail(PFEM_OK);
      }
      if (ps.done != 0) {
        R->info.iterations = ps.iter;
        return fail(ps.done == PCG_NONFINITE ? PFEM_ERR_NONFINITE : PFEM_ERR_NOT_CONVERGED);
      }
      if (ps.repl) st = enq_replacement(R, false, s);
      break;
    case PH_NT_REF:
      R->ref = sl.aux[0] > 0.0 ? sl.aux[0] : 1.0;
      st = enq_newton_check(R, s);
      break;
    case PH_NT_CHECK: {
      const double rel = sl.aux[1] / R->ref;
      if (R->init_rel < 0) R->init_rel = rel;
      R->last_rel = rel;
      if (!std::isfinite(rel)) return retry_level(PFEM_ERR_NONFINITE);
      if (rel <= R->tol) {
        if (!R->load.last()) {  // next load level from this converged state
          R->load.converged();
          R->level_newton = 0;
          if (cudaMemcpyAsync(R->uc, R->u, (size_t)R->n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            st = PFEM_ERR_CUDA;
            break;
          }
          st = enq_newton_step(R, s);
          break;
        }
        R->info.iterations = R->inner_iters;
        R->info.newton_iterations = R->newton;
        R->info.replacements = R->repl;
        R->info.inverted_backtracks = R->backtracks;
        R->info.rel_residual_recursive = rel;
        R->info.rel_residual_true_f64 = rel;
        R->info.initial_rel_residual = R->init_rel;
        R->info.reference_norm = R->ref;
        return fail(PFEM_OK);
      }
      if (R->level_newton >= 50) return retry_level(PFEM_ERR_NOT_CONVERGED);
      // inner solve A(u) d = -rn from d = 0 to 1e-8 relative to ||rn||
      if ((st = enq_jacobi(R, R->u, s))) break;
      if (cudaMemsetAsync(R->x, 0, (size_t)R->n * 8, s) != cudaSuccess) {
        st = PFEM_ERR_CUDA;
        break;
      }
      if ((st = enq_pcg_start(R, true, 1e-8, R->aux + 1, s))) break;
      R->phase = PH_NT_INNER;
      break;
    }
    case PH_NT_INNER: {
      bool stagnated = false;
      if (R->replaced) {
        R->replaced = false;
        R->stalls = (R->prev_true > 0.0 && !(ps.rel_true < 0.5 * R->prev_true)) ? R->stalls + 1 : 0;
        R->prev_true = ps.rel_true;
        stagnated = R->stalls >= 2 && ps.done == 0;
      }
      if (stagnated) {  // take the solve out of the shared steps before the line search
        static const int kStagnated = PCG_STAGNATED;
        if (cudaMemcpyAsync(&R->st->done, &kStagnated, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
          st = PFEM_ERR_CUDA;
          break;
        }
      }
      if (ps.done == PCG_CONVERGED || ps.done == PCG_MAXITER || ps.done == PCG_NEGCURV || stagnated) {
        R->inner_iters += ps.iter;
        R->repl += ps.replacements;
        R->t_ls = 1.0;
        R->ls_tries = 0;
        st = enq_line_search(R, s);
      } else if (ps.done != 0) {
        return retry_level(ps.done == PCG_NONFINITE ? PFEM_ERR_NONFINITE : PFEM_ERR_NOT_CONVERGED);
      } else if (ps.repl) {
        st = enq_replacement(R, true, s);
      }
      break;
    }
    case PH_NT_LS:
      if (sl.inverted == 0) {
        cudaMemcpyAsync(R->u, R->tmp, (size_t)R->n * 8, cudaMemcpyDeviceToDevice, s);
        R->newton++;
        R->level_newton++;
        st = enq_newton_check(R, s);
      } else if (++R->ls_tries <= 10) {
        R->backtracks++;
        R->t_ls *= 0.5;
        st = enq_line_search(R, s);
      } else {
        return retry_level(PFEM_ERR_INVERTED);
      }
      break;
    default:
      break;
  }
  if (st) return fail(st);
  return true;
}

pfem_status rebuild_tables(pfem_server_s* S) {
  const int na = (int)S->active.size();
  std::vector<ReqDev> reqs((size_t)na);
  std::vector<int2> btile_k[2];
  std::vector<int> ublk;
  ServeTiles tiles[2];
  std::vector<PcgState*> stp((size_t)na);
  std::vector<double*> auxp((size_t)na);
  std::vector<int32_t*> invp((size_t)na);
  for (int i = 0; i < na; ++i) {
    Request* R = S->active[(size_t)i];
    ReqDev& d = reqs[(size_t)i];
    d.plan = R->mesh->plan;
    d.pcg.r = R->r;
    d.pcg.dinv = R->dinv;
    d.pcg.p[0] = R->p0;
    d.pcg.p[1] = R->p1;
    d.pcg.st = R->st;
    d.pcg.tile_part = R->tile_part;
    d.pcg.ticket = R->ticket_dev;
    d.pcg.alpha_by_update = 0;  // alpha by each solve's last tile
    d.q = R->q;
    d.x = R->x;
    d.u = R->solve_kind == PFEM_SOLVE_NEWTON ? R->u : nullptr;
    d.n = R->n;
    d.ublk0 = (int)ublk.size();
    d.nublk = R->nublk;
    d.upart = R->upart;
    d.ucount = R->ucount;
    const int kind = d.plan.kind == PFEM_LINEAR ? 0 : 1;
    for (int t = 0; t < d.plan.n_tiles; ++t) btile_k[kind].push_back(make_int2(i, t));
    for (int k = 0; k < R->nublk; ++k) ublk.push_back(i);
    ServeTiles& T = tiles[kind];
    T.max_local = std::max(T.max_local, d.plan.max_local);
    T.slot_cap = std::max(T.slot_cap, d.plan.slot_cap);
    T.step_cap = std::max(T.step_cap, d.plan.step_cap);
    stp[(size_t)i] = R->st;
    auxp[(size_t)i] = R->aux;
    invp[(size_t)i] = R->mesh->plan.inverted;
  }
  tiles[0].n_blocks = (int)btile_k[0].size();
  tiles[1].n_blocks = (int)btile_k[1].size();
  std::vector<int2> btile(btile_k[0]);  // linear blocks first
  btile.insert(btile.end(), btile_k[1].begin(), btile_k[1].end());
  PFEM_CUDA(cudaStreamSynchronize(S->stream));  // the old tables are no longer read
  pfem_status st;
  size_t cap_r = S->cap_reqs, cap_bt = S->cap_btile, cap_u = S->cap_ublk;
  if ((st = grow(reinterpret_cast<void**>(&S->d_reqs), &cap_r, (size_t)std::max(na, 1), sizeof(ReqDev)))) return st;
  size_t cap_tmp = cap_r;
  if (cap_r != S->cap_reqs) {  // per-solve pointer tables follow the solve capacity
    if (S->d_stp) cudaFree(S->d_stp);
    if (S->d_auxp) cudaFree(S->d_auxp);
    if (S->d_invp) cudaFree(S->d_invp);
    if (S->d_slots) cudaFree(S->d_slots);
    if (S->h_slots) cudaFreeHost(S->h_slots);
    PFEM_CUDA(cudaMalloc(&S->d_stp, cap_tmp * sizeof(PcgState*)));
    PFEM_CUDA(cudaMalloc(&S->d_auxp, cap_tmp * sizeof(double*)));
    PFEM_CUDA(cudaMalloc(&S->d_invp, cap_tmp * sizeof(int32_t*)));
    PFEM_CUDA(cudaMalloc(&S->d_slots, cap_tmp * sizeof(StateSlot)));
    PFEM_CUDA(cudaMallocHost(&S->h_slots, cap_tmp * sizeof(StateSlot)));
  }
  S->cap_reqs = cap_r;
  if ((st = grow(reinterpret_cast<void**>(&S->d_btile), &cap_bt, std::max<size_t>(btile.size(), 1), sizeof(int2))))
    return st;
  S->cap_btile = cap_bt;
  if ((st = grow(reinterpret_cast<void**>(&S->d_ublk), &cap_u, std::max<size_t>(ublk.size(), 1), sizeof(int))))
    return st;
  S->cap_ublk = cap_u;
  if (na > 0) {
    PFEM_CUDA(cudaMemcpy(S->d_reqs, reqs.data(), (size_t)na * sizeof(ReqDev), cudaMemcpyHostToDevice));
    PFEM_CUDA(cudaMemcpy(S->d_stp, stp.data(), (size_t)na * sizeof(PcgState*), cudaMemcpyHostToDevice));
    PFEM_CUDA(cudaMemcpy(S->d_auxp, auxp.data(), (size_t)na * sizeof(double*), cudaMemcpyHostToDevice));
    PFEM_CUDA(cudaMemcpy(S->d_invp, invp.data(), (size_t)na * sizeof(int32_t*), cudaMemcpyHostToDevice));
  }
  if (!btile.empty())
    PFEM_CUDA(cudaMemcpy(S->d_btile, btile.data(), btile.size() * sizeof(int2), cudaMemcpyHostToDevice));
  if (!ublk.empty()) PFEM_CUDA(cudaMemcpy(S->d_ublk, ublk.data(), ublk.size() * sizeof(int), cudaMemcpyHostToDevice));
  S->tiles[0] = tiles[0];
  S->tiles[1] = tiles[1];
  S->n_update = (int)ublk.size();
  S->dirty = false;
  return PFEM_OK;
}

void plan_worker(pfem_server_s* S) {
  for (;;) {
    Request* R = nullptr;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_plan.wait(lock, [&] { return S->stop.load() || !S->to_plan.empty(); });
      if (S->stop.load() && S->to_plan.empty()) return;
      R = S->to_plan.front();
      S->to_plan.pop_front();
    }
    pfem_status st = build_plan(&R->desc, &R->plan, &R->fext, 0);
    if (st == PFEM_OK && R->desc.dim != 3) st = PFEM_ERR_UNSUPPORTED;
    if (st == PFEM_OK && !R->u0.empty() && (int64_t)R->u0.size() != R->desc.n_nodes * R->desc.dim)
      st = PFEM_ERR_INVALID_ARG;
    {
      std::lock_guard<std::mutex> lock(S->mu);
      R->plan_status = st;
      R->footprint = st == PFEM_OK ? request_bytes(R->plan) : 0;
      R->planned = true;
    }
    S->cv_work.notify_all();
  }
}

constexpr int kChunk = 8;  // shared steps between two read-backs of the solves' scalars

// The work of one chunk, enqueued on s: kChunk shared steps, then every active solve's state
// gathered into one table and copied to the pinned host mirror.
pfem_status enqueue_chunk(pfem_server_s* S, cudaStream_t s) {
  pfem_status st;
  for (int k = 0; k < kChunk; ++k)
    if ((st = launch_serve_step(S->d_reqs, S->d_btile, S->tiles, S->d_ublk, S->n_update, s)))
      return st;
  const int na = (int)S->active.size();
  gather_states_kernel<<<(na + 127) / 128, 128, 0, s>>>(S->d_stp, S->d_auxp, S->d_invp, na, S->d_slots);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  PFEM_CUDA(cudaMemcpyAsync(S->h_slots, S->d_slots, (size_t)na * sizeof(StateSlot), cudaMemcpyDeviceToHost, s));
  return PFEM_OK;
}

// Captures the chunk for the current tables into S->chunk_exec (replacing the old graph).
pfem_status capture_chunk(pfem_server_s* S) {
  if (S->chunk_exec) {
    cudaGraphExecDestroy(S->chunk_exec);
    S->chunk_exec = nullptr;
  }
  // a step with no blocks launches nothing but sets the apply kernel's shared-memory limit,
  // which is a function attribute and stays outside the capture
  ServeTiles none[2] = {S->tiles[0], S->tiles[1]};
  none[0].n_blocks = none[1].n_blocks = 0;
  pfem_status pre = launch_serve_step(S->d_reqs, S->d_btile, none, S->d_ublk, 0, S->stream);
  if (pre != PFEM_OK) return pre;
  const int64_t before = g_kernel_launches;
  PFEM_CUDA(cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal));
  const pfem_status st = enqueue_chunk(S, S->stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(S->stream, &g);
  S->chunk_kernels = g_kernel_launches - before;
  g_kernel_launches = before;  // captured, not run: each replay is counted when launched
  if (st != PFEM_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != PFEM_OK ? st : cuda_fail(e, "capturing the serving chunk");
  }
  const cudaError_t ei = cudaGraphInstantiate(&S->chunk_exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    S->chunk_exec = nullptr;
    return cuda_fail(ei, "instantiating the serving chunk");
  }
  return PFEM_OK;
}

void worker_loop(pfem_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    // ---- admission (FIFO: a request waits for the one ahead of it)
    std::vector<Request*> admitted, rejected;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      if (S->active.empty())
        S->cv_work.wait_for(lock, std::chrono::milliseconds(2),
                            [&] { return S->stop.load() || (!S->queue.empty() && S->queue.front()->planned); });
      if (S->stop.load()) {  // destroy: abandon what is left (reported as timed out)
        lock.unlock();
        for (Request* R : S->active) finish(S, R, PFEM_ERR_TIMEOUT);
        S->active.clear();
        return;
      }
      while (!S->queue.empty() && S->queue.front()->planned &&
             (int)(S->active.size() + admitted.size()) < S->max_slots) {
        Request* R = S->queue.front();
        if (R->plan_status != PFEM_OK || R->footprint > S->budget) {
          if (R->plan_status == PFEM_OK) R->plan_status = PFEM_ERR_OVER_BUDGET;
          rejected.push_back(R);
          S->queue.pop_front();
          continue;
        }
        if (S->used + R->footprint > S->budget) break;
        S->used += R->footprint;
        admitted.push_back(R);
        S->queue.pop_front();
      }
    }
    for (Request* R : rejected) finish(S, R, R->plan_status);
    const auto t_a0 = std::chrono::steady_clock::now();
    for (Request* R : admitted) {
      pfem_status st = admit(S, R);
      if (st == PFEM_OK) st = start_solve(R, S->stream);
      R->plan = HostPlan();  // host copies are no longer needed
      R->fext = std::vector<double>();
      R->coords = std::vector<double>();
      R->conn = std::vector<int32_t>();
      R->u0 = std::vector<double>();
      if (st != PFEM_OK) {
        finish(S, R, st);
        continue;
      }
      S->active.push_back(R);
      S->dirty = true;
    }
    const auto t_a1 = std::chrono::steady_clock::now();
    S->t_admit = S->t_admit + std::chrono::duration<double>(t_a1 - t_a0).count();
    S->n_admitted += (int64_t)admitted.size();
    if (S->active.empty()) continue;
    if (S->dirty) {
      S->n_rebuilds++;
      if (rebuild_tables(S) != PFEM_OK) {
        for (Request* R : S->active) finish(S, R, PFEM_ERR_CUDA);
        S->active.clear();
        S->dirty = true;
        continue;
      }
      if (!S->graph_failed && capture_chunk(S) != PFEM_OK) S->graph_failed = true;  // plain launches from now on
    }
    const auto t_c0 = std::chrono::steady_clock::now();
    S->t_tables = S->t_tables + std::chrono::duration<double>(t_c0 - t_a1).count();
    // ---- a chunk of shared steps, then one read-back of every solve's scalars
    const int na = (int)S->active.size();
    bool launched = false;
    if (S->chunk_exec && !S->graph_failed) {
      launched = cudaGraphLaunch(S->chunk_exec, S->stream) == cudaSuccess;
      if (launched) g_kernel_launches += S->chunk_kernels;
    }
    if (!launched) enqueue_chunk(S, S->stream);
    S->n_chunks++;
    const bool synced = cudaStreamSynchronize(S->stream) == cudaSuccess;
    const auto t_c1 = std::chrono::steady_clock::now();
    S->t_wait = S->t_wait + std::chrono::duration<double>(t_c1 - t_c0).count();
    if (!synced) {
      for (Request* R : S->active) finish(S, R, PFEM_ERR_CUDA);
      S->active.clear();
      continue;
    }
    std::vector<Request*> still;
    for (int i = 0; i < na; ++i) {
      Request* R = S->active[(size_t)i];
      if (advance(S, R, S->h_slots[i])) still.push_back(R);
      else S->dirty = true;
    }
    S->active.swap(still);
    S->t_advance = S->t_advance + std::chrono::duration<double>(std::chrono::steady_clock::now() - t_c1).count();
  }
}

}  // namespace
}  // namespace pfem

extern "C" {

pfem_status pfem_serve_create(size_t hbm_budget_bytes, int32_t max_slots, pfem_server_t* out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1) {
    set_error("invalid server arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  pfem_server_s* S = new (std::nothrow) pfem_server_s();
  if (!S) {
    set_error("host allocation failed");
    return PFEM_ERR_OUT_OF_MEMORY;
  }
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  cudaGetDevice(&S->device);
  cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "cudaStreamCreate");
  }
  // resident solves allocate and free through a pool that keeps its memory (up to the
  // admission budget) instead of synchronising the device on every admission and release
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S->device;
  e = cudaMemPoolCreate(&S->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = (uint64_t)hbm_budget_bytes;
    e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e != cudaSuccess) {
    if (S->pool) cudaMemPoolDestroy(S->pool);
    cudaStreamDestroy(S->stream);
    delete S;
    return cuda_fail(e, "memory pool");
  }
  unsigned hc = std::thread::hardware_concurrency();
  const int np = (int)std::max(1u, std::min(8u, hc > 2 ? hc / 2 : 1u));
  for (int i = 0; i < np; ++i) S->planners.emplace_back(plan_worker, S);
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return PFEM_OK;
}

pfem_status pfem_serve_submit(pfem_server_t S, const pfem_mesh_desc* d, int32_t kind, const double* u0_host,
                              double tol, int32_t n_load_steps, uint64_t* ticket) {
  if (!S || !d || !ticket || !(tol > 0.0) || n_load_steps < 1 || (kind != PFEM_SOLVE_LINEAR && kind != PFEM_SOLVE_NEWTON)) {
    set_error("invalid submit arguments");
    return PFEM_ERR_INVALID_ARG;
  }
  if (d->dim != 2 && d->dim != 3) {
    set_error("dim must be 2 or 3");
    return PFEM_ERR_INVALID_ARG;
  }
  if (kind == PFEM_SOLVE_LINEAR && d->kind != PFEM_LINEAR) {
    set_error("linear solves need a linear-elastic mesh");
    return PFEM_ERR_INVALID_ARG;
  }
  Request* R = new (std::nothrow) Request();
  if (!R) {
    set_error("host allocation failed");
    return PFEM_ERR_OUT_OF_MEMORY;
  }
  const int dim = d->dim, nv = dim + 1;
  const int64_t N = d->n_nodes, E = d->n_elems, F = d->n_facets;
  if (N < 1 || E < 0 || F < 0 || !d->coords || (E > 0 && (!d->conn || !d->mat_a || !d->mat_b)) ||
      (F > 0 && (!d->facets || !d->traction))) {
    delete R;
    set_error("invalid mesh description");
    return PFEM_ERR_INVALID_ARG;
  }
  R->coords.assign(d->coords, d->coords + N * dim);
  R->conn.assign(d->conn, d->conn + E * nv);
  R->mat_a.assign(d->mat_a, d->mat_a + E);
  R->mat_b.assign(d->mat_b, d->mat_b + E);
  if (d->dirichlet_mask) R->mask.assign(d->dirichlet_mask, d->dirichlet_mask + N * dim);
  if (d->dirichlet_values) R->values.assign(d->dirichlet_values, d->dirichlet_values + N * dim);
  if (F > 0) {
    R->facets.assign(d->facets, d->facets + F * dim);
    R->traction.assign(d->traction, d->traction + F * dim);
  }
  if (d->f_ext_extra) R->f_extra.assign(d->f_ext_extra, d->f_ext_extra + N * dim);
  if (u0_host) R->u0.assign(u0_host, u0_host + N * dim);
  R->desc = *d;
  R->desc.coords = R->coords.data();
  R->desc.conn = R->conn.empty() ? nullptr : R->conn.data();
  R->desc.mat_a = R->mat_a.empty() ? nullptr : R->mat_a.data();
  R->desc.mat_b = R->mat_b.empty() ? nullptr : R->mat_b.data();
  R->desc.dirichlet_mask = R->mask.empty() ? nullptr : R->mask.data();
  R->desc.dirichlet_values = R->values.empty() ? nullptr : R->values.data();
  R->desc.facets = R->facets.empty() ? nullptr : R->facets.data();
  R->desc.traction = R->traction.empty() ? nullptr : R->traction.data();
  R->desc.f_ext_extra = R->f_extra.empty() ? nullptr : R->f_extra.data();
  R->solve_kind = kind;
  R->tol = tol;
  R->n_load_steps = n_load_steps;
  R->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    R->ticket = S->next_ticket++;
    S->tickets[R->ticket] = R;
    S->queue.push_back(R);
    S->to_plan.push_back(R);
    S->pending++;
    *ticket = R->ticket;
  }
  S->cv_plan.notify_one();
  S->cv_work.notify_all();
  return PFEM_OK;
}

pfem_status pfem_serve_poll(pfem_server_t S, uint64_t ticket, double* u_out_host, pfem_solve_info* info) {
  if (!S) {
    set_error("null server");
    return PFEM_ERR_INVALID_ARG;
  }
  Request* R = nullptr;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) {
      set_error("unknown ticket %llu", (unsigned long long)ticket);
      return PFEM_ERR_INVALID_ARG;
    }
    R = it->second;
    if (!R->done) return PFEM_PENDING;
    S->tickets.erase(it);
  }
  if (u_out_host && !R->result.empty()) std::memcpy(u_out_host, R->result.data(), R->result.size() * 8);
  if (info) {
    *info = R->info;
    info->queue_s = R->t_admit > 0 ? R->t_admit - R->t_submit : R->t_done - R->t_submit;
    info->total_s = R->t_done - R->t_submit;
  }
  const pfem_status st = R->status;
  if (st != PFEM_OK) set_error("request %llu finished with status %d", (unsigned long long)ticket, (int)st);
  delete R;
  return st;
}

pfem_status pfem_serve_stats(pfem_server_t S, double* out) {
  if (!S || !out) {
    set_error("pfem_serve_stats: NULL argument");
    return PFEM_ERR_INVALID_ARG;
  }
  out[0] = S->t_wait;
  out[1] = S->t_admit;
  out[2] = S->t_tables;
  out[3] = S->t_advance;
  out[4] = (double)S->n_chunks;
  out[5] = (double)S->n_rebuilds;
  out[6] = (double)S->n_admitted;
  out[7] = 0.0;
  return PFEM_OK;
}

pfem_status pfem_serve_drain(pfem_server_t S, double timeout_s) {
  if (!S) {
    set_error("null server");
    return PFEM_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lock(S->mu);
  const bool ok = S->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] { return S->pending == 0; });
  if (!ok) {
    set_error("%d request(s) still pending after %.1f s", S->pending, timeout_s);
    return PFEM_ERR_TIMEOUT;
  }
  return PFEM_OK;
}

void pfem_serve_destroy(pfem_server_t S) {
  if (!S) return;
  S->stop.store(true);
  S->cv_plan.notify_all();
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& t : S->planners)
    if (t.joinable()) t.join();
  // requests that were never admitted or polled
  for (auto& kv : S->tickets) {
    Request* R = kv.second;
    if (R->block) cudaFreeAsync(R->block, S->stream);
    if (R->mesh) pfem_mesh_destroy(R->mesh);
    delete R;
  }
  cudaStreamSynchronize(S->stream);  // pooled memory returned before the pool goes
  if (S->chunk_exec) cudaGraphExecDestroy(S->chunk_exec);
  cudaFree(S->d_reqs);
  cudaFree(S->d_btile);
  cudaFree(S->d_ublk);
  cudaFree(S->d_stp);
  cudaFree(S->d_auxp);
  cudaFree(S->d_invp);
  cudaFree(S->d_slots);
  if (S->h_slots) cudaFreeHost(S->h_slots);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
