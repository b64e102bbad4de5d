// Internal declarations shared by the translation units of libpfem.
//
// Data layout (device, per mesh)
//   Elements are reordered along a Morton curve of their centroids and cut into tiles of at
//   most kTileElems elements touching at most kTileNodes distinct nodes. A tile is the unit
//   of work of one CTA: its nodes are staged in shared memory and its elements are grouped
//   into fans, one fan per thread. A fan is a chain of k <= kMaxFan simplices around a common
//   hinge (an edge in 3-D, a vertex in 2-D) with ring nodes r_0..r_k; simplex i has the
//   corners (hinge, r_i, r_{i+1}) and consecutive simplices share the face (hinge, r_{i+1}).
//   The thread walks the ring once: every ring node is read once, its contributions from the
//   two simplices that touch it are summed in registers, and it is written once to its own
//   shared-memory slot; the hinge nodes accumulate over the whole fan. Each tile node then
//   sums its slots in a fixed order (rank order), so the result is bitwise reproducible
//   without float atomics.
//   A node whose incident elements all lie in one tile ("complete") is written directly by
//   that tile. A node shared by several tiles ("halo") gets one partial per tile, written to
//   a scratch buffer, and the last tile to publish one sums them in ascending tile order.
//
//   tile_a[t]   = {fan_begin, n_fans, lnode_begin, n_local}
//   tile_b[t]   = {n_complete, partial_begin, step_begin, n_steps (= elements)}
//   tile_cnt[t] = kMaxFan x uint16: cnt_i = fans of the tile with more than i simplices
//                 (fans are sorted by length, longest first, so these are fans 0..cnt_i-1)
//   lnode_f[l]  = {x - x_anchor, y - y_anchor, z - z_anchor, info}  (float4; info bits below)
//   lnode_d[l]  = same coordinates in double (for the FP64 instantiation)
//   slot_off[l] = first slot of the tile node (uint16; a node's slot count is
//                 slot_off[l+1]-slot_off[l], the last node's end is the tile's slot count)
//   fan_head[f] = {h_0, h_1 (3-D), r_0, k} codes: local node index (bits 0-9) | rank
//                 (bits 10-15), rank = position of the incidence among the node's slots
//   step_code[s], step_mat_f/d[s]: code of r_{i+1} and (mu, lambda) of simplex i of fan f,
//                 stored step-major inside the tile: s = step_begin + sum_{j<i} cnt_j + f,
//                 so a warp's fans read consecutive records at every step
//   info        = node id (bits 0-27) | Dirichlet mask of DOF i at bit 28+i
//   halo_rec[i]  = {slot, first, count, info} of the i-th (tile, halo node) pair in tile order:
//                 the node's partials occupy [first, first + count) in ascending tile order, this
//                 tile's at `slot`; the last tile to publish sums that range (ticket at `first`)
//   halo_info[h], halo_ptr[h..h+1], halo_src[k] (host): halo nodes (sorted by id) and the indices
//                of their partials in ascending tile order
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pfem.h"

namespace pfem {

struct __align__(32) PfemDouble4 {
  double x, y, z, w;
};

constexpr int kTileElems = 2048;   // max elements per tile
constexpr int kMaxFan = 8;         // max simplices per fan
constexpr int kTileNodes = 1024;   // max distinct nodes per tile (10-bit local index)
constexpr int kMaxRank = 63;       // max incidences of one node inside one tile (6 bits)
constexpr int kInfoIdBits = 28;
constexpr uint32_t kInfoIdMask = (1u << kInfoIdBits) - 1u;
constexpr int kThreads = 256;      // threads per CTA of the persistent PCG kernel
constexpr int kTileThreads = 256;  // threads per element-tile CTA (tile, batch and serving kernels)
constexpr int kMaxRegions = 3;     // output ops one tile launch can produce (partials/tickets each)
constexpr int kReduceBlocks = 296; // fixed grid of the deterministic FP64 reductions (2 x 148)

// Kernels enqueued by this thread (launches recorded into a graph are counted by the caller
// per replay instead, see solve.cu).
extern thread_local int64_t g_kernel_launches;
#define PFEM_COUNT_LAUNCH() (++::pfem::g_kernel_launches)

void set_error(const char* fmt, ...);

// Bounds-checked build: each translation unit with checked kernels registers a host function
// that reads and clears its device word of bad-index flags (see checked.cuh).
bool register_check_word(unsigned (*read_and_clear)());
pfem_status cuda_fail(cudaError_t e, const char* what);

#define PFEM_CUDA(call)                                         \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return ::pfem::cuda_fail(_e, #call); \
  } while (0)

// Host-side tile plan (built by plan.cpp).
struct HostPlan {
  int dim = 3, nv = 4;
  int64_t n_nodes = 0, n_elems = 0;
  int max_local = 0, max_elems = 0;
  std::vector<int32_t> tile_a;    // 4 per tile
  std::vector<int32_t> tile_b;    // 4 per tile
  std::vector<float> lnode_f;     // 4 per local node
  std::vector<double> lnode_d;    // 4 per local node
  std::vector<uint16_t> slot_off; // 1 per local node
  std::vector<uint16_t> tile_cnt; // kMaxFan per tile
  std::vector<uint16_t> fan_head; // 4 per fan
  std::vector<uint16_t> step_code;// 1 per step (element)
  std::vector<float> step_mat_f;  // 2 per step
  std::vector<double> step_mat_d; // 2 per step
  int max_slots = 0;              // largest tile slot count
  int64_t n_fans = 0;
  std::vector<int32_t> halo_info; // 1 per halo node
  std::vector<int32_t> halo_ptr;  // n_halo + 1
  std::vector<int32_t> halo_src;  // n_partials
  int64_t n_partials = 0;
  std::vector<int32_t> elem_perm; // original element id of each step
  std::vector<int32_t> partial_halo; // halo node index of each partial
  std::vector<int32_t> halo_rec;     // 4 per partial (see halo_rec above)
  std::vector<int32_t> halo_node;    // 4 per halo node: {first, count, info, 0}
  std::vector<int32_t> halo_seq;     // per CSR position: tile-order index of the partial
  int64_t n_tiles() const { return (int64_t)tile_a.size() / 4; }
  int64_t n_local() const { return (int64_t)slot_off.size(); }
  int64_t n_halo() const { return (int64_t)halo_info.size(); }
};

// Validates desc and builds the plan plus the FP64 external force. Returns status.
// tile_elems <= 0 or > kTileElems selects default_tile_elems(n_elems).
pfem_status build_plan(const pfem_mesh_desc* d, HostPlan* plan, std::vector<double>* f_ext, int tile_elems = 0);

// Device bytes of a mesh built from hp, and the upload that builds it (capi.cu).
size_t mesh_arena_bytes(const HostPlan& hp);
// pool != nullptr (serving): the arena comes from that stream-ordered memory pool on `stream`
// and is returned to it without a device synchronisation; no pinned host scratch.
pfem_status mesh_upload(const HostPlan& hp, const std::vector<double>& fext, const pfem_mesh_desc* desc,
                        cudaStream_t stream, pfem_mesh_t* out, cudaMemPool_t pool = nullptr);

// Default elements per tile for a mesh of n_elems elements.
int default_tile_elems(int64_t n_elems);

// Structural self-check of a plan against its description (host only).
pfem_status verify_plan(const pfem_mesh_desc* d, const HostPlan& plan);

// Device view of one mesh's plan (kernel argument, passed by value).
struct DevPlan {
  int dim;
  int kind;              // pfem_material_kind
  int n_tiles;
  int n_halo;
  int max_local;         // largest tile node count (shared-memory sizing)
  int slot_cap;          // largest tile slot count
  int step_cap;          // largest tile element (step) count
  int64_t n_nodes;
  int64_t n_partials;
  const int4* tile_a;
  const int4* tile_b;
  const float4* lnode_f;
  const PfemDouble4* lnode_d;
  const uint16_t* slot_off;
  const uint4* tile_cnt;   // kMaxFan uint16 per tile
  const ushort4* fan_head;
  const uint16_t* step_code;
  const float2* step_mat_f;
  const double2* step_mat_d;
  const int4* halo_rec;  // per (tile, halo node) pair in tile order
  const int4* halo_node; // per halo node {first CSR position, count, info, 0}
  const int32_t* halo_seq;  // per CSR position: tile-order index of its partial (deferred mode)
  const int2* node_part;    // per node: {first, count} of its contiguous halo partials (count 0:
                            // complete node, written by the tile holding all its elements)
  int32_t* halo_count;   // per region x partial slot (used at each halo node's first slot):
                         // partials published so far (reset by the last)
  void* partial;         // scratch: per region n_partials slots of 4 compute-type values
  double* tile_energy;   // per-tile strain-energy partials
  int32_t* inverted;     // count of J <= 0 elements (device int)
  const double* f_ext;   // n_dofs, FP64, at full load
  const float* f_ext_f;  // n_dofs, the same rounded to FP32
  const double* dvalues; // n_dofs prescribed values at full load
  const uint8_t* dmask;  // n_dofs
  // quadrilaterals (quad.cu): elem_npe = 4 (Q4) or 8 (Q8), 0 for simplex meshes. Element-major
  // path: one thread per element over its Gauss points writes one record per (element, local
  // node) to qbuf; each node sums its records in ascending (element, local) order (CSR).
  // n_tiles counts blocks of kQuadBlock elements (energy and p.Ap partials per block).
  int elem_npe;
  int64_t n_elems;
  const int32_t* qconn;  // n_elems x npe
  const double2* qxd;    // node coordinates
  const float2* qxf;
  const double2* qmatd;  // per element (mu, lambda)
  const float2* qmatf;
  const int32_t* qptr;   // n_nodes + 1
  const int32_t* qidx;   // element * npe + local, ascending per node
  void* qbuf;            // kMaxRegions x n_elems x npe x 2 values (double capacity)
};

constexpr int kQuadBlock = 128;  // elements per block of the quadrilateral element kernel

// Operation bits of the element-tile kernel.
enum : int {
  OP_TANGENT = 1,   // y = A(u) v
  OP_RESIDUAL = 2,  // r = P (f_int(u) - s f_ext)
  OP_ENERGY = 4,    // per-tile sum of V Psi
  OP_DIAG = 8,      // d = diag A(u)
  OP_PCG = 16,      // with OP_TANGENT: PCG-fused apply (direction update + p.Ap + alpha)
  OP_PERSIST = 32,  // with OP_PCG: inside the persistent PCG kernel (beta and parity passed in,
                    // alpha formed by the caller after a grid barrier)
};

enum : int {
  PCG_RUNNING = 0,
  PCG_CONVERGED = 1,
  PCG_MAXITER = 2,
  PCG_NONFINITE = 3,
  PCG_BREAKDOWN = 4,
  PCG_BARRIER_TIMEOUT = 6,  // a grid barrier of the persistent kernel gave up waiting
  PCG_STAGNATED = 7,        // the FP64 true residual stopped decreasing between replacements
  PCG_NEGCURV = 8,          // p.Ap < 0 with truncate set: the iterate so far is the result
};
// Newton inner solves stop after this many PCG iterations at most (a tangent that is not
// positive definite can keep plain CG from converging at all).
constexpr int kInnerMaxIter = 20000;

// Device-resident scalars of one Jacobi-PCG solve (FP64).
struct PcgState {
  double rho;             // r . z of the current residual
  double alpha, beta;
  double rel;             // latest relative residual (recursive, or true right after a replacement)
  double rel_true;        // latest FP64 true relative residual
  double ref;             // reference norm of the stopping rule
  double tol;
  double repl_threshold;  // a recursive residual below this triggers an FP64 replacement
  double repl_factor;     // next threshold = factor * true residual at the last replacement
  int iter;               // completed iterations; direction buffers alternate with its parity
  int max_iter;
  int done;               // PCG_* code, 0 while running
  int repl;               // 1 = stop the device loop for an FP64 residual replacement
  int replacements;
  int truncate;           // 1: stop at negative curvature after the first iteration (Newton inner solves)
  int bodies;             // replays of the graph loop body (counted by its last kernel)
};

// Extra inputs of the PCG-fused tangent apply (OP_PCG): the search direction is formed on
// the fly, p = dinv r + beta p_old, written to p[(iter + 1) & 1], and A p goes to y; each tile
// also sums p_e . (A_e p_e) over its elements; alpha = rho / (p . A p) is formed from the
// tile sums either by the last tile (ticket) or, with alpha_by_update, by the update kernel.
struct PcgArgs {
  const double* r;
  const double* dinv;
  double* p[2];           // direction buffers (p_old = p[iter & 1])
  PcgState* st;
  double* tile_part;      // n_tiles doubles
  unsigned int* ticket;   // zero-initialised; reset by the last tile (unused with alpha_by_update)
  double beta;            // OP_PERSIST: beta of this iteration
  int odd;                // OP_PERSIST: parity of the completed iteration count
  int alpha_by_update;    // 1: tiles only store their sums; the update kernel forms alpha
};

// Grid barrier of the persistent PCG kernels (zeroed before every launch). The arrival
// counter and the words the waiting CTAs poll sit on different 128-byte lines, so that the
// polls do not slow the arrivals.
struct GridBar {
  unsigned int count;  // arrivals at the current barrier
  unsigned int pad0[31];
  unsigned int gen;    // completed barriers
  int err;             // 1 = some CTA gave up waiting
  // scalars the last CTA to arrive computes and publishes with the release (same line as gen)
  int b_stop, b_iter;
  double b_alpha, b_beta, b_rho;
  unsigned int pad1[20];
};

// Buffers of the persistent PCG kernel: one launch runs whole iterations (fused direction /
// apply / p.Ap, grid barrier, alpha and update, grid barrier, beta) until the state asks for
// an FP64 replacement or terminates.
struct PersistArgs {
  const double* u;      // linearisation point of a Newton inner solve (null for linear)
  double* x;
  double* r;
  const double* dinv;
  double* p[2];
  double* q;
  PcgState* st;
  double* tile_part;    // n_tiles doubles
  unsigned int* ticket; // last-tile ticket of the apply (zero; reset by its user)
  double* red_part;     // kReduceBlocks * 2 doubles
  unsigned int* red_counter;  // last-block ticket of the update (zero; reset by its user)
  GridBar* bar;
  int64_t n;            // DOFs
  long long spin_limit; // polls of a grid-barrier wait before it gives up (each >= 32 ns)
  int absent_cta;       // failure-detection test: this CTA leaves at its first grid barrier
                        // without arriving (-1 = none), so the others' waits run out
};

// Default and test settings of the persistent kernel's barrier waits (solve.cu).
constexpr long long kBarrierSpinLimit = 1ll << 25;  // x >= 32 ns sleep: more than a second

struct OpArgs {
  const void* u;    // VT*, may be null for linear tangent/diag
  const void* v;    // VT*
  void* y;          // VT* tangent output
  void* r;          // VT* residual output
  void* d;          // VT* diagonal output
  double load_scale;
  PcgArgs pcg;      // OP_PCG only
  const void* out_scale;   // device scalar of the vector type multiplying residual / tangent
                           // outputs (null = 1)
  int hess;                // tangent on prescribed DOFs: 0 = identity block (y = v), 1 = zero
  int defer_halo;          // 1: tiles publish halo partials in tile order (no loads, no tickets);
                           // halo_finish_kernel completes them
};

// A ragged batch of meshes evaluated in one launch (batch.cu builds it).
struct BatchDev {
  const DevPlan* plans;    // n_meshes device copies (inverted -> the batch's counter)
  const int2* btile;       // per launch block: (mesh, tile of that mesh)
  const int64_t* dof_off;  // n_meshes + 1 DOF offsets into the concatenated vectors
  const float* mesh_scale; // n_meshes upstream factors for grad / hvp (null = 1)
  int max_local;           // largest tile node count over the batch
  int slot_cap;            // largest tile slot count over the batch
  int step_cap;            // largest tile element count over the batch
};

pfem_status launch_batch(const BatchDev& B, int n_blocks, int n_meshes, const float* u, const float* v, float* grad,
                         float* hvp, double* energy, cudaStream_t s);

// One resident solve of the server (device view). Every active solve takes part in the
// shared PCG step launches; the reduction of each solve uses its own fixed block count so
// its rounding does not depend on which other solves share the launch.
struct ReqDev {
  DevPlan plan;
  PcgArgs pcg;             // r, dinv, p[2], st, tile_part, ticket
  double* q;               // A p
  double* x;               // iterate (or Newton correction)
  const double* u;         // Neo-Hookean: linearisation point (null for linear)
  int64_t n;               // DOFs
  int ublk0, nublk;        // blocks of the update launch owned by this solve
  double* upart;           // nublk * 2 partial sums
  unsigned int* ucount;    // last-block ticket of the update
};

// Apply blocks of one material kind in a shared serving step, and the largest tile shape
// among their solves (sizes the shared memory of that kind's launch).
struct ServeTiles {
  int n_blocks = 0, max_local = 1, slot_cap = 4, step_cap = 1;
};

// Shared PCG step over many solves: fused apply (one CTA per (solve, tile); a launch for the
// linear solves' tiles, then one for the Neo-Hookean solves') and update (one CTA range per
// solve). btile: (solve, tile) per apply block, linear blocks first; ublk: solve per update
// block.
pfem_status launch_serve_step(const ReqDev* reqs, const int2* btile, const ServeTiles (&tiles)[2], const int* ublk,
                              int n_update_blocks, cudaStream_t s);

// Blocks the update launch gives a solve of n DOFs (depends on n only).
inline int serve_update_blocks(int64_t n) {
  int64_t b = (n + 256 * 8 - 1) / (256 * 8);
  return (int)(b < 1 ? 1 : (b > 296 ? 296 : b));
}

// Launches the tile kernel and the halo pass for one mesh (kernels_tile.cu); quadrilateral
// meshes go to launch_quad_op.
pfem_status launch_element_op(const DevPlan& P, int ops, pfem_dtype vt, pfem_dtype ct,
                              const OpArgs& a, cudaStream_t s);
// Element operators of quadrilateral meshes (quad.cu); same contract as launch_element_op.
pfem_status launch_quad_op(const DevPlan& P, int ops, pfem_dtype vt, pfem_dtype ct, const OpArgs& a, cudaStream_t s);

// Launches the persistent PCG kernel (FP32 element arithmetic only); PFEM_ERR_UNSUPPORTED
// when it cannot run here (other arithmetic, no co-resident grid), without side effects.
// Load levels of Newton's load stepping (App. B: equal steps of 1/n). A level whose Newton
// iteration fails (every step halving inverts an element, no convergence, or a non-finite
// residual) is retried from the last converged state with half the load increment, at most
// kMaxLoadCuts times per solve; each converged level doubles the increment back (up to 1/n).
// Levels are integers over n * 2^kCutBits, so without cuts the load fractions are exactly
// step / n.
constexpr int kMaxLoadCuts = 8;
struct LoadSchedule {
  static constexpr int kCutBits = 6;
  int64_t den = 1, prev = 0, inc = 1, cur = 1;
  int cuts = 0;
  void start(int n_steps) {
    den = (int64_t)n_steps << kCutBits;
    inc = int64_t(1) << kCutBits;
    prev = 0;
    cur = inc;
    cuts = 0;
  }
  double fraction() const { return (double)cur / (double)den; }
  bool last() const { return cur == den; }
  void converged() {  // the current level converged and is not the last
    prev = cur;
    inc = std::min<int64_t>(inc * 2, int64_t(1) << kCutBits);
    cur = std::min(den, prev + inc);
  }
  bool cut() {  // retry the current level with half the increment; false when out of cuts
    if (inc <= 1 || cuts >= kMaxLoadCuts) return false;
    ++cuts;
    inc /= 2;
    cur = prev + inc;
    return true;
  }
};

pfem_status launch_pcg_persistent(const DevPlan& P, pfem_dtype ct, const PersistArgs& a, cudaStream_t s);

// Halo partials from which launch_element_op completes halo nodes in a separate pass instead
// of inside the tiles (removes the per-tile fence / ticket / reload chain; costs a launch).
constexpr int64_t kDeferHaloPartials = 1 << 18;

// Device address of the allocation-free apply's fixed scratch array on the current device
// (noalloc.cu); the first call per device loads the array's module. pfem_mesh_create calls it.
pfem_status noalloc_scratch(void** out);

// Multi-right-hand-side linear tangent action y_j = A v_j (kernels_multi.cu); vt = PFEM_F32
// (float vectors) or PFEM_F64 (double vectors), FP32 element arithmetic.
pfem_status launch_multi_apply(const DevPlan& P, pfem_dtype vt, int k, const void* v, void* y, cudaStream_t s);

// Penalty springs of a mesh (springs.cu): y_j += S v_j on free DOFs (v read as 0 on prescribed
// DOFs) for k vectors of the vector type vt; d += diag S on free DOFs. No-ops without springs.
pfem_status springs_apply(pfem_mesh_t m, pfem_dtype vt, int k, const void* v, void* y, cudaStream_t s);
pfem_status springs_diag(pfem_mesh_t m, pfem_dtype vt, void* d, cudaStream_t s);
void springs_release(pfem_mesh_t m);

// Dynamic shared memory one tile CTA of launch_element_op needs.
size_t element_op_smem(const DevPlan& P, int ops, pfem_dtype ct);

// Deterministic FP64 reductions (kernels_vec.cu). partials: kReduceBlocks doubles,
// counter: one zero-initialised unsigned int (reset by the last block).
// out[0] = sum over tiles of tile_energy; out[1] = out[0] - s * f_ext . u
pfem_status launch_energy_finalize(const DevPlan& P, pfem_dtype vt, const void* u, double s,
                                   double* partials, unsigned int* counter, double* out,
                                   cudaStream_t st);

}  // namespace pfem

struct pfem_mesh_s {
  pfem::DevPlan plan;
  pfem_mesh_stats stats;
  cudaStream_t stream = nullptr;
  int device = 0;
  double load_scale = 1.0;
  void* arena = nullptr;     // single device allocation holding every plan array
  bool pooled = false;       // arena from a stream-ordered pool (serving): freed on `stream`
  size_t arena_bytes = 0;
  // small device scratch for reductions
  double* red_partials = nullptr;   // kReduceBlocks * 4 doubles
  unsigned int* red_counter = nullptr;
  double* red_out = nullptr;        // 8 doubles
  double* host_out = nullptr;       // pinned, 8 doubles
  int32_t* host_int = nullptr;      // pinned, 4 ints
  int64_t n_dofs = 0, n_free = 0;
  void* solver = nullptr;          // solver workspace (solve.cu), created on first solve
  // penalty springs ("virtual elements" between node pairs, springs.cu): per node with
  // springs its partners in ascending id order (CSR), one stiffness for all
  int32_t n_spring_nodes = 0;
  int32_t* spring_node = nullptr;    // device, n_spring_nodes ids (ascending)
  int32_t* spring_ptr = nullptr;     // device, n_spring_nodes + 1
  int32_t* spring_partner = nullptr; // device
  void* spring_block = nullptr;      // one allocation holding the three arrays
  double spring_k = 0.0;
};
