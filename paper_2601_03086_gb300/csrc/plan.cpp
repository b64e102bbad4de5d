// Host-side mesh validation and tile planning.
//
// The plan turns an unstructured P1 mesh into shared-memory work units (tiles) for the
// element kernels: elements are sorted along a Morton curve of their centroids and cut
// greedily into tiles; each tile lists the nodes it touches (complete nodes first, then
// halo nodes, each group by ascending node id) and gives every element corner the slot it
// writes its contribution to. See pfem_internal.h for the layout.
//
// External force (App. B, f_ext = int N_I f + int_Gamma_t N_I t): a P1 facet of measure |F|
// with constant traction t adds t |F| / dim to each of its dim nodes.

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "pfem_internal.h"

namespace pfem {

static thread_local std::string g_last_error;
thread_local int64_t g_kernel_launches = 0;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char* last_error_cstr() { return g_last_error.c_str(); }

pfem_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? PFEM_ERR_OUT_OF_MEMORY : PFEM_ERR_CUDA;
}

static inline uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

static inline uint64_t spread2(uint64_t x) {  // 31 bits -> every second bit
  x &= 0x7fffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

static bool finite_all(const double* p, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Tile size: 512 elements once the mesh fills the GPU several times over (fewer halo
// partials per element); smaller tiles for small meshes so that at least ~8 tiles land on
// each of the 152 SMs (latency hiding beats halo overhead there).
int default_tile_elems(int64_t n_elems) {
  const int64_t per = (n_elems + 152 * 8 - 1) / (152 * 8);
  int64_t t = (per + 63) / 64 * 64;
  if (t < 128) t = 128;
  if (t > 512) t = 512;
  return (int)t;
}

pfem_status build_plan(const pfem_mesh_desc* d, HostPlan* P, std::vector<double>* f_ext, int tile_elems) {
  if (!d || !P || !f_ext) {
    set_error("null argument");
    return PFEM_ERR_INVALID_ARG;
  }
  const int dim = d->dim;
  if (dim != 2 && dim != 3) {
    set_error("dim must be 2 or 3 (got %d)", dim);
    return PFEM_ERR_INVALID_ARG;
  }
  const int nv = dim + 1;
  const int64_t N = d->n_nodes, E = d->n_elems;
  if (N < 1 || N > (int64_t)kInfoIdMask + 1) {
    set_error("n_nodes must be in [1, 2^28] (got %lld)", (long long)N);
    return PFEM_ERR_INVALID_ARG;
  }
  if (E < 0 || E > ((int64_t)1 << 31) - 1 - kTileElems) {
    set_error("n_elems out of range (got %lld)", (long long)E);
    return PFEM_ERR_INVALID_ARG;
  }
  if (!d->coords || (E > 0 && (!d->conn || !d->mat_a || !d->mat_b))) {
    set_error("coords/conn/mat_a/mat_b must not be NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  if (d->kind != PFEM_LINEAR && d->kind != PFEM_NEOHOOKEAN) {
    set_error("unknown material kind %d", d->kind);
    return PFEM_ERR_INVALID_ARG;
  }
  if (tile_elems < 1 || tile_elems > kTileElems) tile_elems = default_tile_elems(E);
  const double* X = d->coords;
  if (!finite_all(X, N * dim)) {
    set_error("non-finite coordinate");
    return PFEM_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < E * nv; ++i) {
    if (d->conn[i] < 0 || d->conn[i] >= N) {
      set_error("conn[%lld] = %d out of range [0, %lld)", (long long)i, d->conn[i], (long long)N);
      return PFEM_ERR_INVALID_ARG;
    }
  }
  for (int64_t e = 0; e < E; ++e) {
    const double a = d->mat_a[e], b = d->mat_b[e];
    bool ok = std::isfinite(a) && std::isfinite(b) && a > 0.0;
    if (d->kind == PFEM_LINEAR) ok = ok && b > -1.0 && b < 0.5;
    else ok = ok && b >= 0.0;
    if (!ok) {
      set_error("invalid material of element %lld: (%g, %g)", (long long)e, a, b);
      return PFEM_ERR_INVALID_ARG;
    }
  }
  if (d->n_facets < 0 || (d->n_facets > 0 && (!d->facets || !d->traction))) {
    set_error("facets/traction missing");
    return PFEM_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < d->n_facets * dim; ++i) {
    if (d->facets[i] < 0 || d->facets[i] >= N) {
      set_error("facet node id out of range");
      return PFEM_ERR_INVALID_ARG;
    }
  }
  if (d->n_facets > 0 && !finite_all(d->traction, d->n_facets * dim)) {
    set_error("non-finite traction");
    return PFEM_ERR_INVALID_ARG;
  }
  if (d->dirichlet_values && !finite_all(d->dirichlet_values, N * dim)) {
    set_error("non-finite Dirichlet value");
    return PFEM_ERR_INVALID_ARG;
  }
  if (d->f_ext_extra && !finite_all(d->f_ext_extra, N * dim)) {
    set_error("non-finite f_ext_extra");
    return PFEM_ERR_INVALID_ARG;
  }

  // ---- geometry check and Morton keys --------------------------------------------------
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int i = 0; i < dim; ++i) lo[i] = hi[i] = X[i];
  for (int64_t n = 0; n < N; ++n)
    for (int i = 0; i < dim; ++i) {
      lo[i] = std::min(lo[i], X[n * dim + i]);
      hi[i] = std::max(hi[i], X[n * dim + i]);
    }
  const int bits = dim == 3 ? 21 : 31;
  const double cells = (double)((1ull << bits) - 1);
  double sc[3];
  for (int i = 0; i < dim; ++i) sc[i] = cells / std::max(hi[i] - lo[i], 1e-300);
  std::vector<std::pair<uint64_t, int32_t>> keyed((size_t)E);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* c = d->conn + e * nv;
    double xc[3] = {0, 0, 0}, D[3][3] = {{0}}, maxe2 = 0.0;
    for (int a = 0; a < nv; ++a)
      for (int i = 0; i < dim; ++i) xc[i] += X[(int64_t)c[a] * dim + i] / nv;
    for (int a = 1; a < nv; ++a)
      for (int i = 0; i < dim; ++i) D[i][a - 1] = X[(int64_t)c[a] * dim + i] - X[(int64_t)c[0] * dim + i];
    for (int a = 0; a < nv; ++a)
      for (int b = a + 1; b < nv; ++b) {
        double l2 = 0;
        for (int i = 0; i < dim; ++i) {
          double t = X[(int64_t)c[a] * dim + i] - X[(int64_t)c[b] * dim + i];
          l2 += t * t;
        }
        maxe2 = std::max(maxe2, l2);
      }
    double det = dim == 2 ? D[0][0] * D[1][1] - D[0][1] * D[1][0]
                          : D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                                D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                                D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
    const double hd = std::pow(std::sqrt(maxe2), dim);
    if (!(std::fabs(det) > 1e-12 * hd)) {
      set_error("degenerate element %lld (|det D| = %g, max edge^d = %g)", (long long)e, std::fabs(det), hd);
      return PFEM_ERR_DEGENERATE_ELEMENT;
    }
    uint64_t q[3];
    for (int i = 0; i < dim; ++i) q[i] = (uint64_t)std::llround((xc[i] - lo[i]) * sc[i]);
    uint64_t key = dim == 3 ? (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2))
                            : (spread2(q[0]) | (spread2(q[1]) << 1));
    keyed[(size_t)e] = {key, (int32_t)e};
  }
  std::sort(keyed.begin(), keyed.end());

  // ---- global node degree ----------------------------------------------------------------
  std::vector<int32_t> gdeg((size_t)N, 0);
  for (int64_t i = 0; i < E * nv; ++i) gdeg[(size_t)d->conn[i]]++;

  auto info_of = [&](int64_t n) -> int32_t {
    uint32_t m = 0;
    if (d->dirichlet_mask)
      for (int i = 0; i < dim; ++i)
        if (d->dirichlet_mask[n * dim + i]) m |= 1u << i;
    return (int32_t)((uint32_t)n | (m << kInfoIdBits));
  };

  // ---- greedy tiling ----------------------------------------------------------------------
  P->dim = dim;
  P->nv = nv;
  P->n_nodes = N;
  P->n_elems = E;
  P->tile_a.clear();
  P->tile_b.clear();
  P->lnode_f.clear();
  P->lnode_d.clear();
  P->slot_off.clear();
  P->ecode.assign((size_t)E * 4, 0);
  P->emat_f.assign((size_t)E * 2, 0.f);
  P->emat_d.assign((size_t)E * 2, 0.0);
  P->max_local = 0;
  P->max_elems = 0;
  std::vector<int32_t> stamp((size_t)N, -1), tdeg((size_t)N, 0), lmap((size_t)N, 0), rk;
  std::vector<int32_t> cur_nodes, comp, halo;
  std::vector<std::pair<int32_t, int32_t>> halo_pairs;  // (node, partial index), tile order
  halo_pairs.reserve((size_t)(E / 2 + 16));
  int64_t n_partials = 0;
  int32_t tile = 0;
  int64_t tbegin = 0;

  auto close_tile = [&](int64_t tend) {
    comp.clear();
    halo.clear();
    for (int32_t n : cur_nodes) (tdeg[n] == gdeg[n] ? comp : halo).push_back(n);
    std::sort(comp.begin(), comp.end());
    std::sort(halo.begin(), halo.end());
    const int n_local = (int)(comp.size() + halo.size());
    const int64_t lbeg = P->n_local();
    int li = 0;
    int off = 0;
    const int32_t anchor = comp.empty() ? halo[0] : comp[0];
    auto push = [&](int32_t n) {
      lmap[n] = li++;
      float f4[4];
      double d4[4] = {0, 0, 0, 0};
      for (int i = 0; i < dim; ++i) {
        d4[i] = X[(int64_t)n * dim + i] - X[(int64_t)anchor * dim + i];
        f4[i] = (float)d4[i];
      }
      for (int i = dim; i < 3; ++i) f4[i] = 0.f;
      int32_t inf = info_of(n);
      std::memcpy(&f4[3], &inf, 4);
      std::memcpy(&d4[3], &inf, 4);
      P->lnode_f.insert(P->lnode_f.end(), f4, f4 + 4);
      P->lnode_d.insert(P->lnode_d.end(), d4, d4 + 4);
      P->slot_off.push_back((uint16_t)off);
      off += tdeg[n];
    };
    for (int32_t n : comp) push(n);
    for (int32_t n : halo) push(n);
    rk.assign((size_t)n_local, 0);
    for (int64_t p = tbegin; p < tend; ++p) {
      const int32_t e = keyed[(size_t)p].second;
      const int32_t* c = d->conn + (int64_t)e * nv;
      for (int a = 0; a < nv; ++a) {
        const int l = lmap[c[a]];
        const int r = rk[l]++;
        P->ecode[(size_t)p * 4 + a] = (uint16_t)(l | (r << 10));
      }
      double a_ = d->mat_a[e], b_ = d->mat_b[e], mu, lam;
      if (d->kind == PFEM_LINEAR) {
        mu = a_ / (2.0 * (1.0 + b_));
        lam = a_ * b_ / ((1.0 + b_) * (1.0 - 2.0 * b_));
      } else {
        mu = a_;
        lam = b_;
      }
      P->emat_d[(size_t)p * 2] = mu;
      P->emat_d[(size_t)p * 2 + 1] = lam;
      P->emat_f[(size_t)p * 2] = (float)mu;
      P->emat_f[(size_t)p * 2 + 1] = (float)lam;
    }
    for (size_t j = 0; j < halo.size(); ++j) halo_pairs.push_back({halo[j], (int32_t)(n_partials + (int64_t)j)});
    const int32_t ta[4] = {(int32_t)tbegin, (int32_t)(tend - tbegin), (int32_t)lbeg, n_local};
    const int32_t tb[4] = {(int32_t)comp.size(), (int32_t)n_partials, 0, 0};
    P->tile_a.insert(P->tile_a.end(), ta, ta + 4);
    P->tile_b.insert(P->tile_b.end(), tb, tb + 4);
    n_partials += (int64_t)halo.size();
    P->max_local = std::max(P->max_local, n_local);
    P->max_elems = std::max(P->max_elems, (int)(tend - tbegin));
    cur_nodes.clear();
    ++tile;
    tbegin = tend;
  };

  for (int64_t p = 0; p < E; ++p) {
    const int32_t e = keyed[(size_t)p].second;
    const int32_t* c = d->conn + (int64_t)e * nv;
    int newn = 0;
    bool over = false;
    for (int a = 0; a < nv; ++a) {
      const int32_t n = c[a];
      if (stamp[n] != tile) ++newn;
      else if (tdeg[n] + 1 > kMaxRank + 1) over = true;
    }
    const int64_t cur_e = p - tbegin;
    if (cur_e > 0 && (cur_e + 1 > tile_elems || (int64_t)cur_nodes.size() + newn > kTileNodes || over))
      close_tile(p);
    for (int a = 0; a < nv; ++a) {
      const int32_t n = c[a];
      if (stamp[n] != tile) {
        stamp[n] = tile;
        tdeg[n] = 0;
        cur_nodes.push_back(n);
      }
      tdeg[n]++;
    }
  }
  if (E > 0) close_tile(E);
  // Orphan nodes (no element) go to element-free tiles as complete nodes of degree zero, so
  // the tile kernel writes their outputs too.
  for (int64_t n = 0; n < N; ++n) {
    if (gdeg[(size_t)n] != 0) continue;
    cur_nodes.push_back((int32_t)n);
    if ((int)cur_nodes.size() == kTileNodes) close_tile(E);
  }
  if (!cur_nodes.empty()) close_tile(E);

  // ---- halo CSR: nodes shared by several tiles, by ascending id ---------------------------
  std::vector<int32_t> cnt((size_t)N, 0);
  for (auto& pr : halo_pairs) cnt[pr.first]++;
  P->halo_info.clear();
  P->halo_ptr.assign(1, 0);
  std::vector<int32_t> start((size_t)N, -1);
  int64_t acc = 0;
  for (int64_t n = 0; n < N; ++n) {
    if (cnt[n] > 0) {
      P->halo_info.push_back(info_of(n));
      start[n] = (int32_t)acc;
      acc += cnt[n];
      P->halo_ptr.push_back((int32_t)acc);
    }
  }
  P->halo_src.assign((size_t)acc, 0);
  std::vector<int32_t> fill((size_t)N, 0);
  for (auto& pr : halo_pairs) P->halo_src[(size_t)(start[pr.first] + fill[pr.first]++)] = pr.second;
  P->n_partials = n_partials;
  P->partial_halo.assign((size_t)n_partials, 0);
  for (int64_t h = 0; h < P->n_halo(); ++h)
    for (int32_t k = P->halo_ptr[(size_t)h]; k < P->halo_ptr[(size_t)h + 1]; ++k)
      P->partial_halo[(size_t)P->halo_src[(size_t)k]] = (int32_t)h;

  // ---- external force ---------------------------------------------------------------------
  f_ext->assign((size_t)(N * dim), 0.0);
  for (int64_t f = 0; f < d->n_facets; ++f) {
    const int32_t* c = d->facets + f * dim;
    double meas;
    if (dim == 2) {
      const double dx = X[(int64_t)c[1] * 2] - X[(int64_t)c[0] * 2];
      const double dy = X[(int64_t)c[1] * 2 + 1] - X[(int64_t)c[0] * 2 + 1];
      meas = std::sqrt(dx * dx + dy * dy);
    } else {
      double a[3], b[3];
      for (int i = 0; i < 3; ++i) {
        a[i] = X[(int64_t)c[1] * 3 + i] - X[(int64_t)c[0] * 3 + i];
        b[i] = X[(int64_t)c[2] * 3 + i] - X[(int64_t)c[0] * 3 + i];
      }
      const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
      meas = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    for (int k = 0; k < dim; ++k)
      for (int i = 0; i < dim; ++i) (*f_ext)[(size_t)c[k] * dim + i] += d->traction[f * dim + i] * meas / dim;
  }
  if (d->f_ext_extra)
    for (int64_t i = 0; i < N * dim; ++i) (*f_ext)[(size_t)i] += d->f_ext_extra[i];
  P->elem_perm.resize((size_t)E);
  for (int64_t p = 0; p < E; ++p) P->elem_perm[(size_t)p] = keyed[(size_t)p].second;
  return PFEM_OK;
}

// Structural invariants of a plan (host only): every element in exactly one tile, corner
// codes pointing at the right nodes, slots forming a permutation of each tile's incidences
// with ranks in element order, complete nodes holding all their incidences, and every other
// node (halo or orphan) listed once with one partial per tile that touches it.
pfem_status verify_plan(const pfem_mesh_desc* d, const HostPlan& P) {
  const int nv = P.nv, dim = P.dim;
  const int64_t N = P.n_nodes, E = P.n_elems, T = P.n_tiles();
  auto bad = [](const char* what, long long a, long long b) {
    set_error("plan check failed: %s (%lld, %lld)", what, a, b);
    return PFEM_ERR_INVALID_ARG;
  };
  std::vector<int32_t> gdeg((size_t)N, 0);
  for (int64_t i = 0; i < E * nv; ++i) gdeg[(size_t)d->conn[i]]++;
  std::vector<int32_t> owner((size_t)N, -1), partial_tiles((size_t)N, 0), partial_deg((size_t)N, 0);
  std::vector<int64_t> partial_node((size_t)std::max<int64_t>(P.n_partials, 1), -1), partial_deg_of;
  partial_deg_of.assign((size_t)std::max<int64_t>(P.n_partials, 1), 0);
  int64_t next_e = 0;
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* ta = &P.tile_a[(size_t)t * 4];
    const int32_t* tb = &P.tile_b[(size_t)t * 4];
    const int eb = ta[0], ne = ta[1], lb = ta[2], nl = ta[3], nc = tb[0], pb = tb[1];
    if (eb != next_e || ne < 0 || (ne == 0 && eb != E)) return bad("tiles must cover elements contiguously", t, eb);
    next_e = eb + ne;
    if (nl < 1 || nl > kTileNodes || nc > nl) return bad("tile node count", t, nl);
    std::vector<int> seen((size_t)ne * nv, 0), next_rank((size_t)nl, 0);
    for (int l = 0; l < nl; ++l) {
      const int off = P.slot_off[(size_t)(lb + l)];
      const int end = l + 1 < nl ? P.slot_off[(size_t)(lb + l + 1)] : ne * nv;
      if (end < off) return bad("slot offsets not monotone", t, l);
    }
    for (int e = 0; e < ne; ++e) {
      const int32_t orig = P.elem_perm[(size_t)(eb + e)];
      for (int a = 0; a < nv; ++a) {
        const uint16_t code = P.ecode[(size_t)(eb + e) * 4 + a];
        const int l = code & 1023, r = code >> 10;
        if (l >= nl) return bad("local index out of range", t, l);
        int32_t info;
        std::memcpy(&info, &P.lnode_f[(size_t)(lb + l) * 4 + 3], 4);
        const int64_t gid = (int64_t)((uint32_t)info & kInfoIdMask);
        if (gid != d->conn[(int64_t)orig * nv + a]) return bad("corner code points at the wrong node", orig, a);
        if (r != next_rank[l]++) return bad("ranks not in element order", t, l);
        const int off = P.slot_off[(size_t)(lb + l)];
        const int end = l + 1 < nl ? P.slot_off[(size_t)(lb + l + 1)] : ne * nv;
        if (off + r >= end) return bad("rank beyond the node's slot range", t, l);
        if (seen[(size_t)(off + r)]++) return bad("slot used twice", t, off + r);
      }
    }
    for (int l = 0; l < nl; ++l) {
      int32_t info;
      std::memcpy(&info, &P.lnode_f[(size_t)(lb + l) * 4 + 3], 4);
      const int64_t gid = (int64_t)((uint32_t)info & kInfoIdMask);
      if (l < nc) {
        if (next_rank[l] != gdeg[(size_t)gid]) return bad("complete node misses incidences", gid, next_rank[l]);
        if (owner[(size_t)gid] != -1) return bad("node complete in two tiles", gid, t);
        owner[(size_t)gid] = (int32_t)t;
      } else {
        const int64_t pi = pb + (l - nc);
        if (pi >= P.n_partials) return bad("partial index out of range", t, pi);
        partial_node[(size_t)pi] = gid;
        partial_deg_of[(size_t)pi] = next_rank[l];
        partial_tiles[(size_t)gid]++;
        partial_deg[(size_t)gid] += next_rank[l];
      }
    }
  }
  if (next_e != E) return bad("tiles do not cover all elements", next_e, E);
  std::vector<int> listed((size_t)N, 0);
  for (int64_t h = 0; h < P.n_halo(); ++h) {
    const int64_t gid = (int64_t)((uint32_t)P.halo_info[(size_t)h] & kInfoIdMask);
    if (listed[(size_t)gid]++) return bad("halo node listed twice", gid, h);
    if (owner[(size_t)gid] != -1) return bad("halo node also complete", gid, owner[(size_t)gid]);
    const int b = P.halo_ptr[(size_t)h], e = P.halo_ptr[(size_t)h + 1];
    if (e - b != partial_tiles[(size_t)gid]) return bad("halo partial count", gid, e - b);
    int deg = 0;
    for (int k = b; k < e; ++k) {
      const int32_t pi = P.halo_src[(size_t)k];
      if (partial_node[(size_t)pi] != gid) return bad("halo partial of another node", gid, pi);
      if (k > b && pi <= P.halo_src[(size_t)k - 1]) return bad("halo partials not in tile order", gid, k);
      deg += (int)partial_deg_of[(size_t)pi];
    }
    if (deg != gdeg[(size_t)gid]) return bad("halo node incidences", gid, deg);
    for (int k = b; k < e; ++k)
      if (P.partial_halo[(size_t)P.halo_src[(size_t)k]] != (int32_t)h) return bad("partial -> halo map", gid, k);
    if (gdeg[(size_t)gid] == 0) return bad("orphan node in the halo list", gid, h);
  }
  for (int64_t n = 0; n < N; ++n)
    if (owner[(size_t)n] == -1 && !listed[(size_t)n]) return bad("node neither complete nor listed", n, 0);
  (void)dim;
  return PFEM_OK;
}

}  // namespace pfem
