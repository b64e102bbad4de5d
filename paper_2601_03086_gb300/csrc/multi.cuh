// Multi-right-hand-side tangent action of the linear element operator: y_j = A v_j for k
// vectors per pass over the element data (several load cases on one mesh, e.g. the six unit
// strains of a homogenisation or k independent solves sharing each operator application).
//
// A tile is staged once (step records, fan heads, coordinates, ids, slot offsets), then the
// right-hand sides are processed two at a time. The element geometry (edge vectors, adjugate
// rows, 1/det, the material scale) depends on the mesh only and is formed once per simplex
// as FP32 scalars; everything that depends on a field (corner differences, G', the stress,
// its contraction with the adjugate rows, the ring-node sums) is carried for both vectors of
// a pair in the two lanes of packed FP32x2 arithmetic (sm_100+ FFMA2/FADD2/FMUL2), so one
// instruction stream serves two right-hand sides. Per-lane rounding is IEEE FP32 (round to
// nearest even, fused multiply-add where the code says fma).
//
// Shared-memory records of a pair are 32 bytes: (d0 of both vectors, d1, d2, pad) as float2.
#pragma once

#include <cuda_runtime.h>

#include "pfem_internal.h"
#include "tile.cuh"

namespace pfem {

struct __align__(8) F2 {
  float x, y;
};

__device__ __forceinline__ float2 to2(F2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ F2 of2(float2 a) { return F2{a.x, a.y}; }
__device__ __forceinline__ F2 bc(float s) { return F2{s, s}; }  // one scalar in both lanes
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return of2(__fadd2_rn(to2(a), to2(b))); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return of2(__fadd2_rn(to2(a), make_float2(-b.x, -b.y))); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return of2(__fmul2_rn(to2(a), to2(b))); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return of2(__ffma2_rn(to2(a), to2(b), to2(c))); }
__device__ __forceinline__ F2 neg2(F2 a) { return F2{-a.x, -a.y}; }

// Shared-memory layout of the multi-RHS kernel.
struct MultiLayout {
  size_t slot, x, v, off, info, fb, head, smat, scode, total;
};

__host__ __device__ inline MultiLayout multi_layout(int max_local, int slot_cap, int step_cap) {
  MultiLayout L;
  size_t o = 0;
  auto al = [](size_t x) { return (x + 31) & ~size_t(31); };
  L.head = o;
  o = al(o + (size_t)step_cap * sizeof(ushort4));
  L.smat = o;
  o = al(o + (size_t)step_cap * sizeof(float2));
  L.scode = o;
  o = al(o + (size_t)step_cap * sizeof(uint16_t));
  L.slot = o;
  o = al(o + (size_t)slot_cap * 32);
  L.x = o;
  o = al(o + (size_t)max_local * 16);
  L.v = o;
  o = al(o + (size_t)max_local * 32);
  L.off = o;
  o = al(o + (size_t)(max_local + 1) * sizeof(int));
  L.info = o;
  o = al(o + (size_t)max_local * sizeof(int));
  L.fb = o;
  o = al(o + kMaxFan * sizeof(int));
  L.total = o;
  return L;
}

// a pair record: components 0..2 of both vectors
__device__ __forceinline__ void ld_pair(const unsigned char* base, int i, F2 (&d)[3]) {
  const float4 a = *reinterpret_cast<const float4*>(base + 32 * (size_t)i);
  const float2 b = *reinterpret_cast<const float2*>(base + 32 * (size_t)i + 16);
  d[0] = F2{a.x, a.y};
  d[1] = F2{a.z, a.w};
  d[2] = F2{b.x, b.y};
}
__device__ __forceinline__ void st_pair(unsigned char* base, int i, const F2* d, int dim) {
  const F2 z{0.f, 0.f};
  const F2 d2 = dim == 3 ? d[2] : z;
  *reinterpret_cast<float4*>(base + 32 * (size_t)i) = make_float4(d[0].x, d[0].y, d[1].x, d[1].y);
  *reinterpret_cast<float2*>(base + 32 * (size_t)i + 16) = make_float2(d2.x, d2.y);
}

}  // namespace pfem

namespace pfem {

// One fan pass of a pair of right-hand sides (linear tangent action), the same ring walk and
// slot order as fan_pass<DIM, K_LIN, OUT_TAN>: geometry in FP32 scalars, fields in FP32x2.
template <int DIM>
__device__ __forceinline__ void fan_pass_pair(unsigned char* smem, const MultiLayout& L, int nf) {
  constexpr int HS = DIM - 1;  // hinge nodes
  const float* sx = reinterpret_cast<const float*>(smem + L.x);
  const unsigned char* sv = smem + L.v;
  const int* soff = reinterpret_cast<const int*>(smem + L.off);
  const int* scnt = reinterpret_cast<const int*>(smem + L.fb);
  const ushort4* shead = reinterpret_cast<const ushort4*>(smem + L.head);
  const float2* smat = reinterpret_cast<const float2*>(smem + L.smat);
  const uint16_t* scode = reinterpret_cast<const uint16_t*>(smem + L.scode);
  unsigned char* slot = smem + L.slot;
  auto put = [&](unsigned code, const F2 (&acc)[DIM]) {
    st_pair(slot, soff[code & 1023u] + (int)(code >> 10), acc, DIM);
  };
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    const ushort4 hd = shead[f];
    const int k = hd.w;
    float x0[4];
    ld4(sx + 4 * (hd.x & 1023), x0);
    F2 v0[3];
    ld_pair(sv, hd.x & 1023, v0);
    float H[3] = {0.f, 0.f, 0.f};
    F2 dvH[3] = {};
    if constexpr (DIM == 3) {
      float t[4];
      ld4(sx + 4 * (hd.y & 1023), t);
      F2 w[3];
      ld_pair(sv, hd.y & 1023, w);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        H[i] = t[i] - x0[i];
        dvH[i] = sub2(w[i], v0[i]);
      }
    }
    struct Ring {
      float x[4];
      F2 v[3];
    };
    auto fetch = [&](unsigned code, Ring& g) {
      const int l = (int)(code & 1023u);
      ld4(sx + 4 * l, g.x);
      ld_pair(sv, l, g.v);
    };
    auto derive = [&](const Ring& g, float (&E)[3], float (&Q)[3], F2 (&dv)[3]) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        E[i] = g.x[i] - x0[i];
        dv[i] = sub2(g.v[i], v0[i]);
      }
      if constexpr (DIM == 3) {
        Q[0] = H[1] * E[2] - H[2] * E[1];
        Q[1] = H[2] * E[0] - H[0] * E[2];
        Q[2] = H[0] * E[1] - H[1] * E[0];
      }
    };
    F2 acc0[DIM], acc1[DIM], accc[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc0[i] = acc1[i] = accc[i] = F2{0.f, 0.f};
    unsigned cc = hd.z;
    float Ec[3], Qc[3] = {0.f, 0.f, 0.f};
    F2 dvc[3];
    Ring gn;
    fetch(cc, gn);
    derive(gn, Ec, Qc, dvc);
    int s = f;  // step-major records: step i of fan f at sum_{j<i} cnt_j + f
    unsigned cnext = 0;
    float2 mnext = make_float2(0.f, 0.f);
    if (k > 0) {
      cnext = scode[s];
      mnext = smat[s];
      fetch(cnext, gn);
    }
    for (int i = 0; i < k; ++i) {
      const unsigned cn = cnext;
      const float mu = mnext.x, lam = mnext.y;
      float En[3], Qn[3] = {0.f, 0.f, 0.f};
      F2 dvn[3];
      derive(gn, En, Qn, dvn);
      s += scnt[i];
      if (i + 1 < k) {  // the next step's record and ring node, in flight during this simplex
        cnext = scode[s];
        mnext = smat[s];
        fetch(cnext, gn);
      }
      ElemGeo<DIM, float> G;
      fan_geometry<DIM, float>(H, Ec, En, Qc, Qn, G);
      F2 dw[DIM][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if constexpr (DIM == 3) {
          dw[0][j] = dvH[j];
          dw[1][j] = dvc[j];
          dw[2][j] = dvn[j];
        } else {
          dw[0][j] = dvc[j];
          dw[1][j] = dvn[j];
        }
      }
      F2 Gp[DIM][DIM];  // G' = sum_a dw_a (x) c_a (grad v times det)
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
          F2 t = mul2(dw[0][a], bc(G.c[0][b]));
#pragma unroll
          for (int c = 1; c < DIM; ++c) t = fma2(dw[c][a], bc(G.c[c][b]), t);
          Gp[a][b] = t;
        }
      const float mus = mu * G.s, lams = lam * G.s;
      F2 tr = Gp[0][0];
#pragma unroll
      for (int a = 1; a < DIM; ++a) tr = add2(tr, Gp[a][a]);
      const F2 lt = mul2(bc(lams), tr);
      F2 S[DIM][DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        S[a][a] = fma2(bc(2.f * mus), Gp[a][a], lt);
#pragma unroll
        for (int b = a + 1; b < DIM; ++b) {
          S[a][b] = mul2(bc(mus), add2(Gp[a][b], Gp[b][a]));
          S[b][a] = S[a][b];
        }
      }
      F2 out[DIM + 1][DIM];  // out_{a+1} = S c_a, out_0 = -sum
#pragma unroll
      for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int r = 0; r < DIM; ++r) {
          F2 t = mul2(S[r][0], bc(G.c[a][0]));
#pragma unroll
          for (int c = 1; c < DIM; ++c) t = fma2(S[r][c], bc(G.c[a][c]), t);
          out[a + 1][r] = t;
        }
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        F2 t = out[1][r];
#pragma unroll
        for (int a = 2; a <= DIM; ++a) t = add2(t, out[a][r]);
        out[0][r] = neg2(t);
      }
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        acc0[j] = add2(acc0[j], out[0][j]);
        if constexpr (DIM == 3) acc1[j] = add2(acc1[j], out[1][j]);
        accc[j] = add2(accc[j], out[HS][j]);
      }
      put(cc, accc);  // ring node i is complete: it touches simplices i - 1 and i only
#pragma unroll
      for (int j = 0; j < DIM; ++j) accc[j] = out[HS + 1][j];
      cc = cn;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Ec[j] = En[j];
        Qc[j] = Qn[j];
        dvc[j] = dvn[j];
      }
    }
    put(cc, accc);
    put(hd.x, acc0);
    if constexpr (DIM == 3) put(hd.y, acc1);
  }
}

}  // namespace pfem
