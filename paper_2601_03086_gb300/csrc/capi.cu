// C ABI: mesh lifetime and the element-operator entry points (see include/pfem.h).

#include <cstring>
#include <cstdlib>
#include <new>

#include "kernels_vec.cuh"
#include "pfem_internal.h"
#include "solver.h"

namespace pfem {
const char* last_error_cstr();

namespace {

struct ArenaBuilder {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  }
};

template <typename T>
pfem_status upload(void* base, size_t off, const std::vector<T>& v, cudaStream_t s) {
  if (v.empty()) return PFEM_OK;
  PFEM_CUDA(cudaMemcpyAsync(static_cast<char*>(base) + off, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return PFEM_OK;
}

}  // namespace

// Readers of the bad-index words of the checked kernels' modules (bounds-checked build only;
// registered at load time, before any other thread runs).
static std::vector<unsigned (*)()>& check_words() {
  static std::vector<unsigned (*)()> v;
  return v;
}

bool register_check_word(unsigned (*read_and_clear)()) {
  check_words().push_back(read_and_clear);
  return true;
}

pfem_status check_mesh(pfem_mesh_t m) {
  if (!m) {
    set_error("null mesh");
    return PFEM_ERR_INVALID_ARG;
  }
  return PFEM_OK;
}

}  // namespace pfem

using namespace pfem;

extern "C" {

const char* pfem_last_error(void) { return last_error_cstr(); }
#ifdef PFEM_CHECKED
const char* pfem_version(void) { return "pfem-gb300 0.1 (sm_103a, bounds-checked)"; }
#else
const char* pfem_version(void) { return "pfem-gb300 0.1 (sm_103a)"; }
#endif

pfem_status pfem_check_status(uint32_t* word) {
  if (!word) {
    set_error("pfem_check_status: word is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  *word = 0;
#ifdef PFEM_CHECKED
  PFEM_CUDA(cudaDeviceSynchronize());
  for (auto f : check_words()) *word |= f();
  return PFEM_OK;
#else
  set_error("not a bounds-checked build (libpfem_checked.so has the checks)");
  return PFEM_ERR_UNSUPPORTED;
#endif
}

pfem_status pfem_debug_set_node_id(pfem_mesh_t m, int64_t local_node, int64_t node_id) {
#ifdef PFEM_CHECKED
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (local_node < 0 || local_node >= m->stats.n_local_nodes || node_id < 0 || node_id > (int64_t)kInfoIdMask) {
    set_error("pfem_debug_set_node_id: index out of range");
    return PFEM_ERR_INVALID_ARG;
  }
  float4* rec = const_cast<float4*>(m->plan.lnode_f) + local_node;
  float4 r;
  PFEM_CUDA(cudaStreamSynchronize(m->stream));
  PFEM_CUDA(cudaMemcpy(&r, rec, sizeof(r), cudaMemcpyDeviceToHost));
  unsigned info;
  std::memcpy(&info, &r.w, sizeof(info));
  info = (info & ~kInfoIdMask) | ((unsigned)node_id & kInfoIdMask);
  std::memcpy(&r.w, &info, sizeof(info));
  PFEM_CUDA(cudaMemcpy(rec, &r, sizeof(r), cudaMemcpyHostToDevice));
  return PFEM_OK;
#else
  (void)m;
  (void)local_node;
  (void)node_id;
  set_error("pfem_debug_set_node_id exists only in the bounds-checked build");
  return PFEM_ERR_UNSUPPORTED;
#endif
}

pfem_status pfem_mesh_create(const pfem_mesh_desc* desc, void* cuda_stream, pfem_mesh_t* out) {
  if (!out) {
    set_error("out is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  HostPlan hp;
  std::vector<double> fext;
  int tile_elems = 0;  // 0: size-dependent default; PFEM_TILE_ELEMS overrides (experiments)
  if (const char* env = std::getenv("PFEM_TILE_ELEMS")) tile_elems = std::atoi(env);
  pfem_status st = build_plan(desc, &hp, &fext, tile_elems);
  if (st != PFEM_OK) return st;
  if ((st = mesh_upload(hp, fext, desc, static_cast<cudaStream_t>(cuda_stream), out))) return st;
  // the allocation-free apply's scratch array is created here, on the mesh's device, so that
  // pfem_tangent_apply_noalloc never triggers the (lazy) load of its module itself
  void* scratch = nullptr;
  if ((st = noalloc_scratch(&scratch))) {
    pfem_mesh_destroy(*out);
    *out = nullptr;
  }
  return st;
}

}  // extern "C"

namespace pfem {

size_t mesh_arena_bytes(const HostPlan& hp) {
  size_t o = 0;
  auto take = [&](size_t b) { o = (o + b + 255) & ~size_t(255); };
  const int64_t nd = hp.n_nodes * hp.dim;
  take(hp.tile_a.size() * 4);
  take(hp.tile_b.size() * 4);
  take(hp.lnode_f.size() * 4);
  take(hp.lnode_d.size() * 8);
  take(hp.slot_off.size() * 2 + 2);
  take(hp.tile_cnt.size() * 2);
  take(hp.fan_head.size() * 2);
  take(hp.step_code.size() * 2);
  take(hp.step_mat_f.size() * 4);
  take(hp.step_mat_d.size() * 8);
  take(hp.halo_rec.size() * 4);
  take(hp.halo_node.size() * 4);
  take(hp.halo_seq.size() * 4);
  take((size_t)hp.n_nodes * 8);
  take((size_t)std::max<int64_t>(hp.n_partials, 1) * kMaxRegions * sizeof(int32_t));
  take((size_t)std::max<int64_t>(hp.n_partials, 1) * 4 * sizeof(double) * kMaxRegions);
  take((size_t)std::max<int64_t>(hp.n_tiles(), 1) * sizeof(double));
  take(16);
  take((size_t)nd * 8);
  take((size_t)nd * 4);
  take((size_t)nd * 8);
  take((size_t)nd);
  take((size_t)kReduceBlocks * 4 * sizeof(double));
  take(64);
  take(8 * sizeof(double));
  return o;
}

pfem_status mesh_upload(const HostPlan& hp, const std::vector<double>& fext, const pfem_mesh_desc* desc,
                        cudaStream_t stream, pfem_mesh_t* out, cudaMemPool_t pool) {
  pfem_status st = PFEM_OK;
  void* cuda_stream = stream;
  const int dim = hp.dim;
  const int64_t nd = hp.n_nodes * dim;
  // per node {first, count} of its contiguous halo partials (count 0 for complete nodes)
  std::vector<int32_t> node_part((size_t)hp.n_nodes * 2, 0);
  for (int64_t h = 0; h < hp.n_halo(); ++h) {
    const int64_t gid = (int64_t)((uint32_t)hp.halo_info[(size_t)h] & kInfoIdMask);
    node_part[(size_t)gid * 2] = hp.halo_ptr[(size_t)h];
    node_part[(size_t)gid * 2 + 1] = hp.halo_ptr[(size_t)h + 1] - hp.halo_ptr[(size_t)h];
  }
  std::vector<float> fext_f(fext.size());
  for (size_t i = 0; i < fext.size(); ++i) fext_f[i] = (float)fext[i];
  std::vector<double> vals((size_t)nd, 0.0);
  std::vector<uint8_t> mask((size_t)nd, 0);
  int64_t n_free = nd;
  for (int64_t i = 0; i < nd; ++i) {
    if (desc->dirichlet_mask && desc->dirichlet_mask[i]) {
      mask[(size_t)i] = 1;
      --n_free;
      if (desc->dirichlet_values) vals[(size_t)i] = desc->dirichlet_values[i];
    }
  }

  ArenaBuilder ab;
  const int64_t nt = hp.n_tiles();
  const size_t o_ta = ab.take(hp.tile_a.size() * 4);
  const size_t o_tb = ab.take(hp.tile_b.size() * 4);
  const size_t o_lf = ab.take(hp.lnode_f.size() * 4);
  const size_t o_ld = ab.take(hp.lnode_d.size() * 8);
  const size_t o_so = ab.take(hp.slot_off.size() * 2 + 2);
  const size_t o_tc = ab.take(hp.tile_cnt.size() * 2);
  const size_t o_fh = ab.take(hp.fan_head.size() * 2);
  const size_t o_sc = ab.take(hp.step_code.size() * 2);
  const size_t o_mf = ab.take(hp.step_mat_f.size() * 4);
  const size_t o_md = ab.take(hp.step_mat_d.size() * 8);
  const size_t o_hr = ab.take(hp.halo_rec.size() * 4);
  const size_t o_hn = ab.take(hp.halo_node.size() * 4);
  const size_t o_hq = ab.take(hp.halo_seq.size() * 4);
  const size_t o_np = ab.take((size_t)hp.n_nodes * 8);
  const size_t o_hc = ab.take((size_t)std::max<int64_t>(hp.n_partials, 1) * kMaxRegions * sizeof(int32_t));
  const size_t o_pa = ab.take((size_t)std::max<int64_t>(hp.n_partials, 1) * 4 * sizeof(double) * kMaxRegions);
  const size_t o_te = ab.take((size_t)std::max<int64_t>(nt, 1) * sizeof(double));
  const size_t o_inv = ab.take(16);
  const size_t o_fe = ab.take((size_t)nd * 8);
  const size_t o_ff = ab.take((size_t)nd * 4);
  const size_t o_dv = ab.take((size_t)nd * 8);
  const size_t o_dm = ab.take((size_t)nd);
  const size_t o_rp = ab.take((size_t)kReduceBlocks * 4 * sizeof(double));
  const size_t o_rc = ab.take(64);
  const size_t o_ro = ab.take(8 * sizeof(double));

  pfem_mesh_s* m = new (std::nothrow) pfem_mesh_s();
  if (!m) {
    set_error("host allocation failed");
    return PFEM_ERR_OUT_OF_MEMORY;
  }
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&m->device);
  m->pooled = pool != nullptr;
  cudaError_t ce = m->pooled ? cudaMallocFromPoolAsync(&m->arena, ab.off, pool, m->stream) : cudaMalloc(&m->arena, ab.off);
  if (ce != cudaSuccess) {
    delete m;
    return cuda_fail(ce, "device allocation (mesh arena)");
  }
  m->arena_bytes = ab.off;
  auto release = [m]() {
    if (m->pooled) {
      cudaFreeAsync(m->arena, m->stream);
    } else {
      cudaFree(m->arena);
    }
    if (m->host_out) cudaFreeHost(m->host_out);
  };
  if (!m->pooled) {  // pinned scratch of the synchronous host-result calls
    ce = cudaMallocHost(&m->host_out, 8 * sizeof(double) + 4 * sizeof(int32_t));
    if (ce != cudaSuccess) {
      cudaFree(m->arena);
      delete m;
      return cuda_fail(ce, "cudaMallocHost");
    }
    m->host_int = reinterpret_cast<int32_t*>(m->host_out + 8);
  }
  char* base = static_cast<char*>(m->arena);
  cudaStream_t s = m->stream;
  auto fail = [&](pfem_status e) {
    cudaStreamSynchronize(s);
    release();
    delete m;
    return e;
  };
  if ((st = upload(base, o_ta, hp.tile_a, s)) || (st = upload(base, o_tb, hp.tile_b, s)) ||
      (st = upload(base, o_lf, hp.lnode_f, s)) || (st = upload(base, o_ld, hp.lnode_d, s)) ||
      (st = upload(base, o_so, hp.slot_off, s)) || (st = upload(base, o_tc, hp.tile_cnt, s)) ||
      (st = upload(base, o_fh, hp.fan_head, s)) || (st = upload(base, o_sc, hp.step_code, s)) ||
      (st = upload(base, o_mf, hp.step_mat_f, s)) || (st = upload(base, o_md, hp.step_mat_d, s)) ||
      (st = upload(base, o_hr, hp.halo_rec, s)) || (st = upload(base, o_hn, hp.halo_node, s)) ||
      (st = upload(base, o_hq, hp.halo_seq, s)) || (st = upload(base, o_np, node_part, s)) ||
      (st = upload(base, o_fe, fext, s)) ||
      (st = upload(base, o_ff, fext_f, s)) || (st = upload(base, o_dv, vals, s)) || (st = upload(base, o_dm, mask, s)))
    return fail(st);
  ce = cudaMemsetAsync(base + o_inv, 0, 16, s);
  if (ce == cudaSuccess)
    ce = cudaMemsetAsync(base + o_hc, 0, (size_t)std::max<int64_t>(hp.n_partials, 1) * kMaxRegions * sizeof(int32_t), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + o_rc, 0, 64, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);  // host vectors die at return
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "mesh upload"));

  DevPlan& P = m->plan;
  P.dim = dim;
  P.kind = desc->kind;
  P.n_tiles = (int)nt;
  P.n_halo = (int)hp.n_halo();
  P.max_local = hp.max_local;
  P.slot_cap = std::max(hp.max_slots, 1);
  P.step_cap = std::max(hp.max_elems, 1);
  P.n_nodes = hp.n_nodes;
  P.n_partials = hp.n_partials;
  P.tile_a = reinterpret_cast<const int4*>(base + o_ta);
  P.tile_b = reinterpret_cast<const int4*>(base + o_tb);
  P.lnode_f = reinterpret_cast<const float4*>(base + o_lf);
  P.lnode_d = reinterpret_cast<const PfemDouble4*>(base + o_ld);
  P.slot_off = reinterpret_cast<const uint16_t*>(base + o_so);
  P.tile_cnt = reinterpret_cast<const uint4*>(base + o_tc);
  P.fan_head = reinterpret_cast<const ushort4*>(base + o_fh);
  P.step_code = reinterpret_cast<const uint16_t*>(base + o_sc);
  P.step_mat_f = reinterpret_cast<const float2*>(base + o_mf);
  P.step_mat_d = reinterpret_cast<const double2*>(base + o_md);
  P.halo_rec = reinterpret_cast<const int4*>(base + o_hr);
  P.halo_node = reinterpret_cast<const int4*>(base + o_hn);
  P.halo_seq = reinterpret_cast<const int32_t*>(base + o_hq);
  P.node_part = reinterpret_cast<const int2*>(base + o_np);
  P.halo_count = reinterpret_cast<int32_t*>(base + o_hc);
  P.partial = base + o_pa;
  P.tile_energy = reinterpret_cast<double*>(base + o_te);
  P.inverted = reinterpret_cast<int32_t*>(base + o_inv);
  P.f_ext = reinterpret_cast<const double*>(base + o_fe);
  P.f_ext_f = reinterpret_cast<const float*>(base + o_ff);
  P.dvalues = reinterpret_cast<const double*>(base + o_dv);
  P.dmask = reinterpret_cast<const uint8_t*>(base + o_dm);
  m->red_partials = reinterpret_cast<double*>(base + o_rp);
  m->red_counter = reinterpret_cast<unsigned int*>(base + o_rc);
  m->red_out = reinterpret_cast<double*>(base + o_ro);
  m->n_dofs = nd;
  m->n_free = n_free;

  pfem_mesh_stats& S = m->stats;
  S.n_nodes = hp.n_nodes;
  S.n_elems = hp.n_elems;
  S.n_dofs = nd;
  S.n_free_dofs = n_free;
  S.n_tiles = nt;
  S.n_local_nodes = hp.n_local();
  S.n_halo_nodes = hp.n_halo();
  S.n_partials = hp.n_partials;
  S.device_bytes = (int64_t)ab.off;
  S.max_tile_elems = hp.max_elems;
  S.max_tile_nodes = hp.max_local;
  S.n_fans = hp.n_fans;
  S.max_tile_slots = hp.max_slots;
  *out = m;
  return PFEM_OK;
}

}  // namespace pfem

extern "C" {

pfem_status pfem_plan_check(const pfem_mesh_desc* desc, pfem_mesh_stats* out) {
  HostPlan hp;
  std::vector<double> fext;
  int tile_elems = 0;
  if (const char* env = std::getenv("PFEM_TILE_ELEMS")) tile_elems = std::atoi(env);
  pfem_status st = build_plan(desc, &hp, &fext, tile_elems);
  if (st != PFEM_OK) return st;
  if ((st = verify_plan(desc, hp)) != PFEM_OK) return st;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->n_nodes = hp.n_nodes;
    out->n_elems = hp.n_elems;
    out->n_dofs = hp.n_nodes * hp.dim;
    int64_t nf = out->n_dofs;
    if (desc->dirichlet_mask)
      for (int64_t i = 0; i < out->n_dofs; ++i) nf -= desc->dirichlet_mask[i] ? 1 : 0;
    out->n_free_dofs = nf;
    out->n_tiles = hp.n_tiles();
    out->n_local_nodes = hp.n_local();
    out->n_halo_nodes = hp.n_halo();
    out->n_partials = hp.n_partials;
    out->max_tile_elems = hp.max_elems;
    out->max_tile_nodes = hp.max_local;
    out->n_fans = hp.n_fans;
    out->max_tile_slots = hp.max_slots;
  }
  return PFEM_OK;
}

void pfem_mesh_destroy(pfem_mesh_t m) {
  if (!m) return;
  if (m->pooled) {  // serving: returned to the pool in stream order, no device synchronisation
    cudaFreeAsync(m->arena, m->stream);
    delete m;
    return;
  }
  cudaStreamSynchronize(m->stream);
  solver_release(m);
  springs_release(m);
  cudaFree(m->arena);
  cudaFreeHost(m->host_out);
  delete m;
}

pfem_status pfem_mesh_stats_get(pfem_mesh_t m, pfem_mesh_stats* out) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (!out) {
    set_error("out is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  *out = m->stats;
  out->device_bytes += (int64_t)solver_bytes(m);
  return PFEM_OK;
}

pfem_status pfem_mesh_set_load_scale(pfem_mesh_t m, double s) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (!std::isfinite(s)) {
    set_error("non-finite load scale");
    return PFEM_ERR_INVALID_ARG;
  }
  m->load_scale = s;
  return PFEM_OK;
}

static pfem_status no_springs(pfem_mesh_t m, const char* what) {
  if (m->n_spring_nodes) {
    set_error("%s does not include penalty springs; remove them with pfem_mesh_set_springs(mesh, 0, NULL, 0)", what);
    return PFEM_ERR_UNSUPPORTED;
  }
  return PFEM_OK;
}

static pfem_status op_common(pfem_mesh_t m, pfem_dtype dt) {
  pfem_status st = check_mesh(m);
  if (st) return st;
  if (dt != PFEM_F32 && dt != PFEM_F64 && dt != PFEM_F64_F32) {
    set_error("unknown dtype %d", (int)dt);
    return PFEM_ERR_INVALID_ARG;
  }
  return PFEM_OK;
}

// vector type / element arithmetic of a dtype
static pfem_dtype vt_of(pfem_dtype d) { return d == PFEM_F32 ? PFEM_F32 : PFEM_F64; }
static pfem_dtype ct_of(pfem_dtype d) { return d == PFEM_F64 ? PFEM_F64 : PFEM_F32; }

pfem_status pfem_energy(pfem_mesh_t m, pfem_dtype dt, const void* u, double* energy, double* strain_energy) {
  pfem_status st = op_common(m, dt);
  if (st || (st = no_springs(m, "pfem_energy"))) return st;
  if (!u) {
    set_error("u is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  OpArgs a{u, nullptr, nullptr, nullptr, nullptr, m->load_scale};
  PFEM_CUDA(cudaMemsetAsync(m->plan.inverted, 0, sizeof(int32_t), m->stream));
  if ((st = launch_element_op(m->plan, OP_ENERGY, vt_of(dt), ct_of(dt), a, m->stream))) return st;
  if ((st = launch_energy_finalize(m->plan, vt_of(dt), u, m->load_scale, m->red_partials, m->red_counter, m->red_out,
                                   m->stream)))
    return st;
  PFEM_CUDA(cudaMemcpyAsync(m->host_out, m->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PFEM_CUDA(cudaMemcpyAsync(m->host_int, m->plan.inverted, sizeof(int32_t), cudaMemcpyDeviceToHost, m->stream));
  PFEM_CUDA(cudaStreamSynchronize(m->stream));
  if (energy) *energy = m->host_out[0];
  if (strain_energy) *strain_energy = m->host_out[1];
  if (m->host_int[0] > 0) {
    set_error("%d element(s) with J <= 0", m->host_int[0]);
    return PFEM_ERR_INVERTED;
  }
  return PFEM_OK;
}

pfem_status pfem_residual(pfem_mesh_t m, pfem_dtype dt, const void* u, void* r) {
  pfem_status st = op_common(m, dt);
  if (st) return st;
  if (!u || !r) {
    set_error("u/r is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  OpArgs a{u, nullptr, nullptr, r, nullptr, m->load_scale};
  if ((st = launch_element_op(m->plan, OP_RESIDUAL, vt_of(dt), ct_of(dt), a, m->stream))) return st;
  return springs_apply(m, vt_of(dt), 1, u, r, m->stream);
}

pfem_status pfem_tangent_apply(pfem_mesh_t m, pfem_dtype dt, const void* u, const void* v, void* y) {
  pfem_status st = op_common(m, dt);
  if (st) return st;
  if (!v || !y || (m->plan.kind == PFEM_NEOHOOKEAN && !u)) {
    set_error("u/v/y is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  OpArgs a{u, v, y, nullptr, nullptr, m->load_scale};
  if ((st = launch_element_op(m->plan, OP_TANGENT, vt_of(dt), ct_of(dt), a, m->stream))) return st;
  return springs_apply(m, vt_of(dt), 1, v, y, m->stream);
}

pfem_status pfem_energy_gradient(pfem_mesh_t m, pfem_dtype dt, const void* u, const void* scale, void* g) {
  pfem_status st = op_common(m, dt);
  if (st || (st = no_springs(m, "pfem_energy_gradient"))) return st;
  if (!u || !g) {
    set_error("u/g is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  OpArgs a{u, nullptr, nullptr, g, nullptr, m->load_scale};
  a.out_scale = scale;
  return launch_element_op(m->plan, OP_RESIDUAL, vt_of(dt), ct_of(dt), a, m->stream);
}

pfem_status pfem_energy_hvp(pfem_mesh_t m, pfem_dtype dt, const void* u, const void* v, const void* scale,
                            void* y) {
  pfem_status st = op_common(m, dt);
  if (st || (st = no_springs(m, "pfem_energy_hvp"))) return st;
  if (!v || !y || (m->plan.kind == PFEM_NEOHOOKEAN && !u)) {
    set_error("u/v/y is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  OpArgs a{u, v, y, nullptr, nullptr, m->load_scale};
  a.out_scale = scale;
  a.hess = 1;  // rows and columns of prescribed DOFs are zero
  return launch_element_op(m->plan, OP_TANGENT, vt_of(dt), ct_of(dt), a, m->stream);
}

pfem_status pfem_dot(pfem_mesh_t m, pfem_dtype dt, const void* a, const void* b, void* out) {
  pfem_status st = op_common(m, dt);
  if (st) return st;
  if (!a || !b || !out) {
    set_error("a/b/out is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  return vk_dot(m->n_dofs, vt_of(dt), a, b, out, m->red_partials, m->red_counter, m->stream);
}

pfem_status pfem_jacobi_diag(pfem_mesh_t m, pfem_dtype dt, const void* u, void* d) {
  pfem_status st = op_common(m, dt);
  if (st) return st;
  if (!d || (m->plan.kind == PFEM_NEOHOOKEAN && !u)) {
    set_error("u/d is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  OpArgs a{u, nullptr, nullptr, nullptr, d, m->load_scale};
  if ((st = launch_element_op(m->plan, OP_DIAG, vt_of(dt), ct_of(dt), a, m->stream))) return st;
  return springs_diag(m, vt_of(dt), d, m->stream);
}

}  // extern "C"
