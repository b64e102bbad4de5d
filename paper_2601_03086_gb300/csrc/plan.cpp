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

// Tile size: 768 elements once the mesh fills the GPU several times over (longer fans and
// fewer halo partials per element, while four tiles still fit on an SM); smaller tiles for
// small meshes so that at least ~4 tiles land on each of the 152 SMs.
int default_tile_elems(int64_t n_elems) {
  const int64_t per = (n_elems + 152 * 4 - 1) / (152 * 4);
  int64_t t = (per + 63) / 64 * 64;
  if (t < 256) t = 256;
  if (t > 768) t = 768;
  return (int)t;
}

// One fan (see pfem_internal.h): hinge and ring as tile-local node indices, and the keyed
// positions of its simplices (simplex i spans hinge, ring[i], ring[i+1]).
struct Fan {
  int h[2] = {0, 0};
  int ring[kMaxFan + 1];
  int64_t pos[kMaxFan];
  int k = 0;
};

constexpr int kFanCap = kMaxFan;  // longest fan the planner builds

// Greedy fans over the elements at keyed positions [b, e) (one tile). Elements are taken in
// order; each unassigned element tries every hinge (edge in 3-D, vertex in 2-D), walks both
// ways around it through face-adjacent unassigned elements of the tile, and keeps the
// longest chain (first hinge on ties, at most kFanCap simplices).
static void build_fans(const pfem_mesh_desc* d, int nv, const std::vector<std::pair<uint64_t, int32_t>>& keyed,
                       int64_t b, int64_t e, const std::vector<int32_t>& lmap, std::vector<Fan>& fans) {
  const int ne = (int)(e - b);
  const int hs = nv - 2;  // hinge size
  std::vector<int> L((size_t)ne * 4, 0);
  for (int j = 0; j < ne; ++j) {
    const int32_t* c = d->conn + (int64_t)keyed[(size_t)(b + j)].second * nv;
    for (int a = 0; a < nv; ++a) L[(size_t)j * 4 + a] = lmap[c[a]];
  }
  // face adjacency inside the tile: nb[j*4+o] = element across the face opposite corner o
  std::vector<std::pair<uint32_t, int32_t>> faces;
  faces.reserve((size_t)ne * nv);
  for (int j = 0; j < ne; ++j)
    for (int o = 0; o < nv; ++o) {
      int f[3], m = 0;
      for (int a = 0; a < nv; ++a)
        if (a != o) f[m++] = L[(size_t)j * 4 + a];
      std::sort(f, f + m);
      uint32_t key = 0;
      for (int i = 0; i < m; ++i) key |= (uint32_t)f[i] << (10 * i);
      faces.push_back({key, j * 4 + o});
    }
  std::sort(faces.begin(), faces.end());
  std::vector<int> nb((size_t)ne * 4, -1);
  for (size_t i = 0; i + 1 < faces.size(); ++i)
    if (faces[i].first == faces[i + 1].first) {
      nb[(size_t)faces[i].second] = faces[i + 1].second >> 2;
      nb[(size_t)faces[i + 1].second] = faces[i].second >> 2;
      ++i;
    }
  std::vector<char> used((size_t)ne, 0);
  auto corner_of = [&](int j, int node) {
    for (int a = 0; a < nv; ++a)
      if (L[(size_t)j * 4 + a] == node) return a;
    return -1;
  };
  // walks from element j, leaving ring node `from` behind and entering `to`, up to `room`
  // simplices; appends (element, apex) pairs
  auto walk = [&](int j, const int* hinge, int from, int to, int room, const int* chain, int n_chain,
                  int* els, int* apex) {
    int n = 0;
    while (n < room) {
      const int o = corner_of(j, from);
      const int nj = o < 0 ? -1 : nb[(size_t)j * 4 + o];
      if (nj < 0 || used[(size_t)nj]) break;
      bool dup = false;
      for (int i = 0; i < n_chain && !dup; ++i) dup = chain[i] == nj;
      for (int i = 0; i < n && !dup; ++i) dup = els[i] == nj;
      if (dup) break;
      int ap = -1;
      for (int a = 0; a < nv; ++a) {
        const int x = L[(size_t)nj * 4 + a];
        bool in = x == to;
        for (int h = 0; h < hs; ++h) in = in || x == hinge[h];
        if (!in) ap = x;
      }
      if (ap < 0) break;
      els[n] = nj;
      apex[n] = ap;
      ++n;
      from = to;
      to = ap;
      j = nj;
    }
    return n;
  };
  for (int j = 0; j < ne; ++j) {
    if (used[(size_t)j]) continue;
    int best = -1, best_nf = 0, best_nb = 0, bf_el[kMaxFan], bf_ap[kMaxFan], bb_el[kMaxFan], bb_ap[kMaxFan];
    int best_h[2] = {0, 0}, best_c = 0, best_d = 0;
    const int* Lj = &L[(size_t)j * 4];
    const int n_hinges = nv == 4 ? 6 : 3;
    static const int kPairs[6][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}, {1, 2, 0, 3}, {1, 3, 0, 2}, {2, 3, 0, 1}};
    static const int kVerts[3][3] = {{0, 1, 2}, {1, 0, 2}, {2, 0, 1}};
    for (int hc = 0; hc < n_hinges; ++hc) {
      int hinge[2], c, dd;
      if (nv == 4) {
        hinge[0] = Lj[kPairs[hc][0]];
        hinge[1] = Lj[kPairs[hc][1]];
        c = Lj[kPairs[hc][2]];
        dd = Lj[kPairs[hc][3]];
      } else {
        hinge[0] = Lj[kVerts[hc][0]];
        hinge[1] = -1;
        c = Lj[kVerts[hc][1]];
        dd = Lj[kVerts[hc][2]];
      }
      int f_el[kMaxFan], f_ap[kMaxFan], b_el[kMaxFan], b_ap[kMaxFan];
      const int nf = walk(j, hinge, c, dd, kFanCap - 1, &j, 1, f_el, f_ap);
      int chain[kMaxFan + 1];
      chain[0] = j;
      for (int i = 0; i < nf; ++i) chain[i + 1] = f_el[i];
      const int nbk = walk(j, hinge, dd, c, kFanCap - 1 - nf, chain, nf + 1, b_el, b_ap);
      if (1 + nf + nbk > best) {
        best = 1 + nf + nbk;
        best_nf = nf;
        best_nb = nbk;
        std::copy(f_el, f_el + nf, bf_el);
        std::copy(f_ap, f_ap + nf, bf_ap);
        std::copy(b_el, b_el + nbk, bb_el);
        std::copy(b_ap, b_ap + nbk, bb_ap);
        best_h[0] = hinge[0];
        best_h[1] = hinge[1];
        best_c = c;
        best_d = dd;
      }
    }
    Fan F;
    F.h[0] = best_h[0];
    F.h[1] = best_h[1] < 0 ? 0 : best_h[1];
    int r = 0, k = 0;
    for (int i = best_nb - 1; i >= 0; --i) {  // backward chain, outermost first
      F.ring[r++] = bb_ap[i];
      F.pos[k++] = b + bb_el[i];
      used[(size_t)bb_el[i]] = 1;
    }
    F.ring[r++] = best_c;
    F.ring[r++] = best_d;
    F.pos[k++] = b + j;
    used[(size_t)j] = 1;
    for (int i = 0; i < best_nf; ++i) {
      F.ring[r++] = bf_ap[i];
      F.pos[k++] = b + bf_el[i];
      used[(size_t)bf_el[i]] = 1;
    }
    F.k = k;
    fans.push_back(F);
  }
  // longest first (stable: equal lengths keep the element order)
  std::stable_sort(fans.begin(), fans.end(), [](const Fan& x, const Fan& y) { return x.k > y.k; });
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
  P->tile_cnt.clear();
  P->fan_head.clear();
  P->step_code.assign((size_t)E, 0);
  P->step_mat_f.assign((size_t)E * 2, 0.f);
  P->step_mat_d.assign((size_t)E * 2, 0.0);
  P->elem_perm.assign((size_t)E, 0);
  P->n_fans = 0;
  P->max_slots = 0;
  P->max_local = 0;
  P->max_elems = 0;
  std::vector<int32_t> stamp((size_t)N, -1), tdeg((size_t)N, 0), lmap((size_t)N, 0), rk;
  std::vector<int32_t> cur_nodes, comp, halo;
  std::vector<std::pair<int32_t, int32_t>> halo_pairs;  // (node, partial index), tile order
  halo_pairs.reserve((size_t)(E / 2 + 16));
  int64_t n_partials = 0;
  int32_t tile = 0;
  int64_t tbegin = 0;

  std::vector<Fan> fans;
  std::vector<int32_t> fdeg;

  auto close_tile = [&](int64_t tend) {
    comp.clear();
    halo.clear();
    for (int32_t n : cur_nodes) (tdeg[n] == gdeg[n] ? comp : halo).push_back(n);
    std::sort(comp.begin(), comp.end());
    std::sort(halo.begin(), halo.end());
    const int n_local = (int)(comp.size() + halo.size());
    const int64_t lbeg = P->n_local();
    int li = 0;
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
    };
    for (int32_t n : comp) push(n);
    for (int32_t n : halo) push(n);

    // fans, slots per node (one per fan the node belongs to, per ring position), ranks
    fans.clear();
    if (tend > tbegin) build_fans(d, nv, keyed, tbegin, tend, lmap, fans);
    const int hs = nv - 2;
    fdeg.assign((size_t)n_local, 0);
    for (const Fan& F : fans) {
      for (int h = 0; h < hs; ++h) fdeg[(size_t)F.h[h]]++;
      for (int i = 0; i <= F.k; ++i) fdeg[(size_t)F.ring[i]]++;
    }
    int off = 0;
    for (int l = 0; l < n_local; ++l) {
      P->slot_off.push_back((uint16_t)off);
      off += fdeg[(size_t)l];
    }
    P->max_slots = std::max(P->max_slots, off);
    rk.assign((size_t)n_local, 0);
    auto code = [&](int l) { return (uint16_t)(l | (rk[(size_t)l]++ << 10)); };
    int cnt[kMaxFan] = {0};
    for (const Fan& F : fans)
      for (int i = 0; i < F.k; ++i) cnt[i]++;
    int base[kMaxFan] = {0};
    for (int i = 1; i < kMaxFan; ++i) base[i] = base[i - 1] + cnt[i - 1];
    for (int i = 0; i < kMaxFan; ++i) P->tile_cnt.push_back((uint16_t)cnt[i]);
    const int64_t fan_beg = P->n_fans;
    for (size_t f = 0; f < fans.size(); ++f) {
      const Fan& F = fans[f];
      const uint16_t h0 = code(F.h[0]);
      const uint16_t h1 = hs == 2 ? code(F.h[1]) : (uint16_t)0;
      const uint16_t r0 = code(F.ring[0]);
      const uint16_t head[4] = {h0, h1, r0, (uint16_t)F.k};
      P->fan_head.insert(P->fan_head.end(), head, head + 4);
      for (int i = 0; i < F.k; ++i) {
        const size_t st = (size_t)(tbegin + base[i] + (int64_t)f);
        P->step_code[st] = code(F.ring[i + 1]);
        const int32_t e = keyed[(size_t)F.pos[i]].second;
        P->elem_perm[st] = e;
        double a_ = d->mat_a[e], b_ = d->mat_b[e], mu, lam;
        if (d->kind == PFEM_LINEAR) {
          mu = a_ / (2.0 * (1.0 + b_));
          lam = a_ * b_ / ((1.0 + b_) * (1.0 - 2.0 * b_));
        } else {
          mu = a_;
          lam = b_;
        }
        P->step_mat_d[st * 2] = mu;
        P->step_mat_d[st * 2 + 1] = lam;
        P->step_mat_f[st * 2] = (float)mu;
        P->step_mat_f[st * 2 + 1] = (float)lam;
      }
    }
    P->n_fans += (int64_t)fans.size();
    for (size_t j = 0; j < halo.size(); ++j) halo_pairs.push_back({halo[j], (int32_t)(n_partials + (int64_t)j)});
    const int32_t ta[4] = {(int32_t)fan_beg, (int32_t)fans.size(), (int32_t)lbeg, n_local};
    const int32_t tb[4] = {(int32_t)comp.size(), (int32_t)n_partials, (int32_t)tbegin, (int32_t)(tend - tbegin)};
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
  P->halo_rec.assign((size_t)n_partials * 4, 0);
  P->halo_seq = P->halo_src;
  P->halo_node.assign((size_t)P->n_halo() * 4, 0);
  for (int64_t h = 0; h < P->n_halo(); ++h) {
    P->halo_node[(size_t)h * 4] = P->halo_ptr[(size_t)h];
    P->halo_node[(size_t)h * 4 + 1] = P->halo_ptr[(size_t)h + 1] - P->halo_ptr[(size_t)h];
    P->halo_node[(size_t)h * 4 + 2] = P->halo_info[(size_t)h];
  }
  for (int64_t h = 0; h < P->n_halo(); ++h)
    for (int32_t k = P->halo_ptr[(size_t)h]; k < P->halo_ptr[(size_t)h + 1]; ++k) {
      const int32_t pi = P->halo_src[(size_t)k];
      P->partial_halo[(size_t)pi] = (int32_t)h;
      int32_t* rec = &P->halo_rec[(size_t)pi * 4];
      rec[0] = k;
      rec[1] = P->halo_ptr[(size_t)h];
      rec[2] = P->halo_ptr[(size_t)h + 1] - P->halo_ptr[(size_t)h];
      rec[3] = P->halo_info[(size_t)h];
    }

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
  int64_t next_e = 0, next_f = 0;
  std::vector<char> elem_seen((size_t)std::max<int64_t>(E, 1), 0);
  const int hs = nv - 2;
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* ta = &P.tile_a[(size_t)t * 4];
    const int32_t* tb = &P.tile_b[(size_t)t * 4];
    const int fb = ta[0], nf = ta[1], lb = ta[2], nl = ta[3], nc = tb[0], pb = tb[1], sb = tb[2], ns = tb[3];
    if (sb != next_e || ns < 0) return bad("tiles must cover elements contiguously", t, sb);
    if (fb != next_f || nf < 0) return bad("tiles must cover fans contiguously", t, fb);
    next_e = sb + ns;
    next_f = fb + nf;
    if (nl < 1 || nl > kTileNodes || nc > nl) return bad("tile node count", t, nl);
    const uint16_t* cnt = &P.tile_cnt[(size_t)t * kMaxFan];
    int base[kMaxFan + 1] = {0};
    for (int i = 0; i < kMaxFan; ++i) {
      if (i > 0 && cnt[i] > cnt[i - 1]) return bad("fan counts not non-increasing", t, i);
      base[i + 1] = base[i] + cnt[i];
    }
    if (base[kMaxFan] != ns || (nf > 0 && cnt[0] != nf) || (nf == 0 && ns != 0)) return bad("fan counts", t, ns);
    int total_slots = 0;
    std::vector<int> node_slots((size_t)nl, 0), next_rank((size_t)nl, 0), inc((size_t)nl, 0);
    for (int f = 0; f < nf; ++f) {
      const uint16_t* hd = &P.fan_head[(size_t)(fb + f) * 4];
      total_slots += hs + hd[3] + 1;
    }
    for (int l = 0; l < nl; ++l) {
      const int off = P.slot_off[(size_t)(lb + l)];
      const int end = l + 1 < nl ? P.slot_off[(size_t)(lb + l + 1)] : total_slots;
      if (end < off) return bad("slot offsets not monotone", t, l);
      node_slots[(size_t)l] = end - off;
    }
    std::vector<int> seen((size_t)std::max(total_slots, 1), 0);
    auto gid_of = [&](int l) {
      int32_t info;
      std::memcpy(&info, &P.lnode_f[(size_t)(lb + l) * 4 + 3], 4);
      return (int64_t)((uint32_t)info & kInfoIdMask);
    };
    auto take = [&](uint16_t code, int* l_out) -> bool {
      const int l = code & 1023, r = code >> 10;
      if (l >= nl) return false;
      if (r != next_rank[(size_t)l]++) return false;
      const int off = P.slot_off[(size_t)(lb + l)];
      if (r >= node_slots[(size_t)l]) return false;
      if (seen[(size_t)(off + r)]++) return false;
      *l_out = l;
      return true;
    };
    for (int f = 0; f < nf; ++f) {
      const uint16_t* hd = &P.fan_head[(size_t)(fb + f) * 4];
      const int k = hd[3];
      if (k < 1 || k > kMaxFan) return bad("fan length", t, k);
      if (f > 0 && k > P.fan_head[(size_t)(fb + f - 1) * 4 + 3]) return bad("fans not sorted by length", t, f);
      int hl[2] = {0, 0}, rprev = 0;
      if (!take(hd[0], &hl[0])) return bad("hinge code", t, f);
      if (hs == 2 && !take(hd[1], &hl[1])) return bad("hinge code", t, f);
      if (!take(hd[2], &rprev)) return bad("ring code", t, f);
      for (int i = 0; i < k; ++i) {
        const int64_t st = sb + base[i] + f;
        if (f >= cnt[i]) return bad("fan step outside its count", t, f);
        int rnext = 0;
        if (!take(P.step_code[(size_t)st], &rnext)) return bad("ring code", t, f);
        const int32_t orig = P.elem_perm[(size_t)st];
        if (orig < 0 || orig >= E || elem_seen[(size_t)orig]++) return bad("element missing or repeated", orig, st);
        int64_t want[4];
        int m = 0;
        for (int h = 0; h < hs; ++h) want[m++] = gid_of(hl[h]);
        want[m++] = gid_of(rprev);
        want[m++] = gid_of(rnext);
        int64_t have[4];
        for (int a = 0; a < nv; ++a) have[a] = d->conn[(int64_t)orig * nv + a];
        std::sort(want, want + nv);
        std::sort(have, have + nv);
        for (int a = 0; a < nv; ++a)
          if (want[a] != have[a]) return bad("simplex corners do not match the element", orig, a);
        for (int h = 0; h < hs; ++h) inc[(size_t)hl[h]]++;
        inc[(size_t)rprev]++;
        inc[(size_t)rnext]++;
        rprev = rnext;
      }
    }
    for (int l = 0; l < nl; ++l)
      if (next_rank[(size_t)l] != node_slots[(size_t)l]) return bad("node slots not all used", t, l);
    for (int l = 0; l < nl; ++l) {
      const int64_t gid = gid_of(l);
      if (l < nc) {
        if (inc[(size_t)l] != gdeg[(size_t)gid]) return bad("complete node misses incidences", gid, inc[(size_t)l]);
        if (owner[(size_t)gid] != -1) return bad("node complete in two tiles", gid, t);
        owner[(size_t)gid] = (int32_t)t;
      } else {
        const int64_t pi = pb + (l - nc);
        if (pi >= P.n_partials) return bad("partial index out of range", t, pi);
        partial_node[(size_t)pi] = gid;
        partial_deg_of[(size_t)pi] = inc[(size_t)l];
        partial_tiles[(size_t)gid]++;
        partial_deg[(size_t)gid] += inc[(size_t)l];
      }
    }
  }
  if (next_e != E) return bad("tiles do not cover all elements", next_e, E);
  if (next_f != P.n_fans) return bad("tiles do not cover all fans", next_f, P.n_fans);
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
    for (int k = b; k < e; ++k) {
      const int32_t pi = P.halo_src[(size_t)k];
      if (P.partial_halo[(size_t)pi] != (int32_t)h) return bad("partial -> halo map", gid, k);
      const int32_t* rec = &P.halo_rec[(size_t)pi * 4];
      if (rec[0] != k || rec[1] != b || rec[2] != e - b || rec[3] != P.halo_info[(size_t)h])
        return bad("halo record", gid, k);
    }
    if (gdeg[(size_t)gid] == 0) return bad("orphan node in the halo list", gid, h);
  }
  for (int64_t n = 0; n < N; ++n)
    if (owner[(size_t)n] == -1 && !listed[(size_t)n]) return bad("node neither complete nor listed", n, 0);
  (void)dim;
  return PFEM_OK;
}

}  // namespace pfem
