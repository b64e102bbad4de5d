// Physics attention of the Transolver backbone (Method, subsection "Transolver") on the
// sm_103a tensor cores.  Forward pass for N points with C = 128 channels and S tokens:
//
//   slice   (tcgen05):  [U' | logits] = X [W_U | W_M] + [0 | b_M]     one 128 x (C+S) MMA/tile
//                       M = softmax_S(logits)                            epilogue, FP32
//                       [Z_num | w] += M^T [U' | 1]                      one 128 x 144 MMA/tile
//                       M stored (bf16, TMA) for the deslice
//   reduce              per-CTA partial token sums added in a fixed order
//   tokens  (FP32)      Z = Z_num / w + b_U (the weights sum to w, so the bias of U moves
//                       out of the per-point work); Q, K, V = Z W + b; per head
//                       softmax(scale Q K^T) V
//                       (two kernels: the projections, then the heads)
//   deslice (tcgen05):  X^t = M Z^t                                      one 128 x C MMA/tile
//
// Data layout: X, X^t row-major [N][C] bf16; M row-major [N][S_pad] bf16 (S_pad = 64 or 128,
// columns S..S_pad-1 zero).  Each 128-point tile moves through shared memory in 64-column
// regions with the 128-byte swizzle, the layout TMA writes and the MMA descriptors read.
// Operands the epilogue produces (M and [U | 1] of the slice MMA) are written row by row,
// four threads per point (a quarter of the columns each), as MN-major operands, so no
// transpose is needed.
//
// Precision: bf16 operands, FP32 accumulation; X W_U, M, Z^t and X^t are stored in bf16, the
// tokens, Q/K/V and the attention in FP32.  Deterministic: fixed tile-to-CTA assignment and
// fixed-order reductions, no atomics.
//
// Every wait is bounded (wall-clock limit); a wait that expires raises the handle's error
// word, the other roles see it and stop, in-flight copies are waited for (bounded) and the
// tensor memory is released before the kernel returns.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "pfem_internal.h"
#include "sm100.cuh"

namespace pfem {
namespace attn {

using namespace sm100;

constexpr int kC = 128;            // channels (the kernels are built for this width)
constexpr int kTile = 128;         // points per tile = MMA M = TMEM lanes
constexpr int kRegion = kTile * 128;  // one 64-column bf16 region of a 128-row tile (16 KB)
constexpr int kZCols = 144;        // slice MMA N: C channels, the weight-sum column, zero pad
constexpr int kPartPitch = 132;    // floats per token row of a CTA partial (C sums, w, pad)
constexpr int kThreads = 192;      // deslice: warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kEpi = 128;
// slice: warp 0 TMA, warp 1 MMA, 16 epilogue warps: four per TMEM lane quarter, each taking
// a quarter of the columns (32 channels of U and S_pad / 4 slice logits of its 32 points)
constexpr int kSliceEpi = 512;
constexpr int kSliceThreads = 64 + kSliceEpi;
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ bool vote_any(bool pred, uint32_t id, uint32_t count) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(pred ? 1u : 0u), "r"(id), "r"(count)
      : "memory");
  return out != 0;
}

constexpr float kLog2e = 1.4426950408889634f;

// 2^x by the hardware approximation (relative error far below the bf16 rounding the slice
// weights get next); 2^-inf = 0
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 8 consecutive values of one point row into a swizzled 128-byte row: region base `reg`,
// row `row`, logical 16-byte chunk `c8`.
__device__ __forceinline__ void st_chunk(uint8_t* reg, int row, int c8, const float* v) {
  uint4 w;
  w.x = pack_bf16(v[0], v[1]);
  w.y = pack_bf16(v[2], v[3]);
  w.z = pack_bf16(v[4], v[5]);
  w.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(reg + row * 128 + ((c8 ^ (row & 7)) << 4)) = w;
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = smem_addr(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

struct SliceArgs {
  int64_t n_points;
  int32_t n_tiles, S;
  const float* bias;  // [C + S_pad]: b_U, then b_M with -inf for the padded tokens
  float* partial;     // [gridDim.x][S][kPartPitch]
  int* err;
};

enum { B_FULL0, B_FULL1, B_EMPTY0, B_EMPTY1, B_WFULL, B_MMA, B_TFREE, B_EPI, B_SLICE, B_FINAL, B_COUNT };

template <int SP>
constexpr size_t slice_smem_bytes() {
  return 1024 + 2 * (kC + SP) * 128 + 2 * 2 * kRegion + 2 * kRegion + 3 * kRegion + 256 * 4 + 2 * 4 * kTile * 4 +
         16 * 8 + 16;
}

// One persistent CTA per SM; CTA b takes tiles b, b + grid, ...
template <int SP>
__global__ void __launch_bounds__(kSliceThreads, 1)
    attn_slice_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                      const __grid_constant__ CUtensorMap map_m, SliceArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  // token columns S .. SP - 1 of W_M are zero and their logit biases -inf, so the padded
  // slice weights come out exactly 0 without a test on S
  constexpr int CS = kC + SP;
  const int S = a.S;
  uint8_t* sw = base;                           // [W_U^T ; W_M^T]: 2 K-regions of CS rows
  uint8_t* sx = sw + 2 * (kC + SP) * 128;       // X: 2 stages x 2 K-regions
  uint8_t* sa = sx + 4 * kRegion;               // M (MN-major A of the slice MMA): 2 regions
  uint8_t* sb = sa + 2 * kRegion;               // [U | 1] (MN-major B): 3 regions
  float* sbias = reinterpret_cast<float*>(sb + 3 * kRegion);
  float* xmax = sbias + 256;        // [4][kTile]: per column quarter, partial row maxima
  float* xsum = xmax + 4 * kTile;   // [4][kTile]: partial row sums
  uint64_t* bar = reinterpret_cast<uint64_t*>(xsum + 4 * kTile);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 16);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = a.n_tiles;
  const int T = (n_tiles - static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) - 1) / static_cast<int>(gridDim.x);

  // constant operand parts: token rows past SP (and all of region 1 when SP = 64) are zero;
  // region 2 of [U | 1] holds the ones column (n = 128) and zeros
  for (int i = threadIdx.x; i < (2 * kRegion) / 16; i += kSliceThreads) {
    const int r = (i * 16) / kRegion;
    if (r >= SP / 64) reinterpret_cast<uint4*>(sa)[i] = make_uint4(0, 0, 0, 0);
  }
  for (int i = threadIdx.x; i < kRegion / 16; i += kSliceThreads)
    reinterpret_cast<uint4*>(sb + 2 * kRegion)[i] = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < CS; i += kSliceThreads) sbias[i] = a.bias[i];
  __syncthreads();
  if (threadIdx.x < kTile) {
    const int row = threadIdx.x;  // n = 128 sits in logical chunk 0, element 0 of the row
    *reinterpret_cast<uint16_t*>(sb + 2 * kRegion + row * 128 + ((0 ^ (row & 7)) << 4)) = 0x3F80;  // bf16 1.0
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[B_FULL0], 1);
    mbar_init(&bar[B_FULL1], 1);
    mbar_init(&bar[B_EMPTY0], 1);
    mbar_init(&bar[B_EMPTY1], 1);
    mbar_init(&bar[B_WFULL], 1);
    mbar_init(&bar[B_MMA], 1);
    mbar_init(&bar[B_TFREE], kSliceEpi / 32);  // one arrival per epilogue warp
    mbar_init(&bar[B_EPI], kSliceEpi / 32);
    mbar_init(&bar[B_SLICE], 1);
    mbar_init(&bar[B_FINAL], 1);
    fence_barrier_init();
    prefetch_map(&map_x);
    prefetch_map(&map_w);
    prefetch_map(&map_m);
  }
  fence_async_smem();
  if (warp == 1) tmem_alloc(tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    mbar_arrive_expect_tx(&bar[B_WFULL], 2 * CS * 128);
    tma_load_2d(sw, &map_w, &bar[B_WFULL], 0, 0);
    tma_load_2d(sw + CS * 128, &map_w, &bar[B_WFULL], 64, 0);
    int issued = 0;
    for (int i = 0; i < T; ++i) {
      const int s = i & 1, k = i >> 1;
      if (!mbar_wait(&bar[B_EMPTY0 + s], (k & 1) ^ 1, a.err, kWaitNs)) break;
      const int y = (static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x)) * kTile;
      mbar_arrive_expect_tx(&bar[B_FULL0 + s], 2 * kRegion);
      tma_load_2d(sx + s * 2 * kRegion, &map_x, &bar[B_FULL0 + s], 0, y);
      tma_load_2d(sx + s * 2 * kRegion + kRegion, &map_x, &bar[B_FULL0 + s], 64, y);
      issued = i + 1;
    }
    // every copy issued must have landed before the CTA exits (bounded)
    mbar_wait(&bar[B_WFULL], 0, a.err, kWaitNs);
    for (int s = 0; s < 2; ++s) {
      const int fills = (issued + 1 - s) / 2;
      if (fills > 0) mbar_wait(&bar[B_FULL0 + s], (fills - 1) & 1, a.err, kWaitNs);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // The projection MMA of tile i + 1 is issued as soon as the epilogue has read tile i's
    // accumulators (B_TFREE), before the slice MMA of tile i waits for the epilogue's
    // operands (B_EPI), so the epilogues run back to back.
    const uint32_t id1 = idesc_bf16(kTile, CS, false, false);
    const uint32_t id3 = idesc_bf16(kTile, kZCols, true, true);
    const uint32_t ax = smem_addr(sx), aw = smem_addr(sw), aa = smem_addr(sa), ab = smem_addr(sb);
    auto project = [&](int i) -> bool {
      const int s = i & 1, k = i >> 1;
      if (!mbar_wait(&bar[B_FULL0 + s], k & 1, a.err, kWaitNs)) return false;
      if (!mbar_wait(&bar[B_TFREE], (i & 1) ^ 1, a.err, kWaitNs)) return false;
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kC / 16; ++kk) {
        const uint32_t off = (kk & 3) * 32;  // 16 bf16 of K inside the swizzled 128-byte row
        const uint64_t da = sdesc_sw128(ax + s * 2 * kRegion + (kk >> 2) * kRegion + off, 16, 1024);
        const uint64_t db = sdesc_sw128(aw + (kk >> 2) * CS * 128 + off, 16, 1024);
        mma_bf16(tmem, da, db, id1, kk > 0 ? 1u : 0u);
      }
      mma_commit(&bar[B_EMPTY0 + s]);
      mma_commit(&bar[B_MMA]);
      return true;
    };
    bool ok = mbar_wait(&bar[B_WFULL], 0, a.err, kWaitNs) && project(0);
    for (int i = 0; ok && i < T; ++i) {
      if (i + 1 < T && !project(i + 1)) break;
      if (!mbar_wait(&bar[B_EPI], i & 1, a.err, kWaitNs)) break;
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kTile / 16; ++kk) {
        const uint64_t da = sdesc_sw128(aa + kk * 2048, kRegion, 1024);
        const uint64_t db = sdesc_sw128(ab + kk * 2048, kRegion, 1024);
        mma_bf16(tmem + 256, da, db, id3, (i > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bar[B_SLICE]);
    }
    mma_commit(&bar[B_FINAL]);  // all MMAs done before the tensor memory is released
    mbar_wait(&bar[B_FINAL], 0, a.err, kWaitNs);
  } else if (warp >= 2) {
    // ---------------- epilogue: one thread per (point, column quarter) ----------------
    // Barriers: 1 + q among the four warps of lane quarter q (softmax exchange), 5 and 6
    // among all epilogue threads (vote on the waits, operands complete before the M store).
    constexpr int LQ = SP / 4;  // slice logits per thread
    const int q = warp & 3, part = (warp - 2) >> 2;
    const int row = 32 * q + lane;
    const uint32_t tl = tmem + (static_cast<uint32_t>(32 * q) << 16);
    const bool leader = (warp == 2 && lane == 0);
    bool failed = false;
    for (int i = 0; i < T; ++i) {
      const int tile = static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x);
      // one thread waits (the others sleep in the vote barrier, which orders them after it):
      // the tile's accumulators are ready
      bool ok = true;
      if (leader) ok = mbar_wait(&bar[B_MMA], i & 1, a.err, kWaitNs);
      if (vote_any(!ok, 5, kSliceEpi)) {
        failed = true;
        break;
      }
      tc_fence_after();
      float u[32], lg[LQ];
      tmem_ld32(tl + 32 * part, u);
      if constexpr (LQ == 32) {
        tmem_ld32(tl + kC + 32 * part, lg);
      } else {
        tmem_ld16(tl + kC + 16 * part, lg);
      }
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar[B_TFREE]);
      // M = softmax over the S tokens, the row spread over four threads (zero rows for points
      // past the end); partial maxima and sums combined in quarter order
      const int j0 = LQ * part;
      float pm = -INFINITY;
#pragma unroll
      for (int j = 0; j < LQ; j += 4) {
        const float4 b4 = *reinterpret_cast<const float4*>(sbias + kC + j0 + j);
        lg[j] += b4.x;
        lg[j + 1] += b4.y;
        lg[j + 2] += b4.z;
        lg[j + 3] += b4.w;
        pm = fmaxf(pm, fmaxf(fmaxf(lg[j], lg[j + 1]), fmaxf(lg[j + 2], lg[j + 3])));
      }
      xmax[part * kTile + row] = pm;
      named_sync(1 + q, 128);
      const float mx = fmaxf(fmaxf(xmax[row], xmax[kTile + row]), fmaxf(xmax[2 * kTile + row], xmax[3 * kTile + row]));
      const float mxl = mx * kLog2e;
      float ps = 0.0f;
#pragma unroll
      for (int j = 0; j < LQ; ++j) {
        lg[j] = fast_exp2(fmaf(lg[j], kLog2e, -mxl));
        ps += lg[j];
      }
      xsum[part * kTile + row] = ps;
      named_sync(1 + q, 128);
      const float sum = ((xsum[row] + xsum[kTile + row]) + xsum[2 * kTile + row]) + xsum[3 * kTile + row];
      const bool valid = static_cast<int64_t>(tile) * kTile + row < a.n_points;
      const float inv = valid ? 1.0f / sum : 0.0f;
#pragma unroll
      for (int j = 0; j < LQ; ++j) lg[j] *= inv;
      // the operand buffers are free once the previous tile's slice MMA has read them and its
      // M store has read sa (the softmax above overlapped that MMA)
      ok = true;
      if (leader) {
        ok = mbar_wait(&bar[B_SLICE], (i & 1) ^ 1, a.err, kWaitNs);
        bulk_wait_read_all();
      }
      if (vote_any(!ok, 5, kSliceEpi)) {
        failed = true;
        break;
      }
      // X W_U -> bf16, channels 32 part .. 32 part + 31 of the row of [U | 1]; b_U is added to
      // the tokens instead (sum_I M_IJ (X_I W_U + b_U) / sum_I M_IJ = Z'_J + b_U)
#pragma unroll
      for (int m = 0; m < 4; ++m) st_chunk(sb + (part >> 1) * kRegion, row, (part & 1) * 4 + m, u + 8 * m);
      if constexpr (LQ == 32) {
#pragma unroll
        for (int m = 0; m < 4; ++m) st_chunk(sa + (part >> 1) * kRegion, row, (part & 1) * 4 + m, lg + 8 * m);
      } else {
#pragma unroll
        for (int m = 0; m < 2; ++m) st_chunk(sa, row, 2 * part + m, lg + 8 * m);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar[B_EPI]);
      named_sync(6, kSliceEpi);
      if (leader) {
#pragma unroll
        for (int r = 0; r < SP / 64; ++r) tma_store_2d(&map_m, sa + r * kRegion, 64 * r, tile * kTile);
        bulk_commit();
      }
    }
    // this CTA's token sums: lane j of the slice accumulator = token j; quarter `part` of
    // the columns per thread, the weight sums (column 128) by the first quarter
    bool ok = !failed;
    if (leader && ok) ok = mbar_wait(&bar[B_SLICE], (T - 1) & 1, a.err, kWaitNs);
    if (!vote_any(!ok, 5, kSliceEpi)) {
      tc_fence_after();
      float* dst = a.partial + (static_cast<int64_t>(blockIdx.x) * S + row) * kPartPitch;
      float v[32];
      tmem_ld32(tl + 256 + 32 * part, v);
      tmem_ld_wait();
      if (row < S) {
#pragma unroll
        for (int e = 0; e < 32; e += 4)
          *reinterpret_cast<float4*>(dst + 32 * part + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      }
      if (part == 0) {
        tmem_ld32(tl + 256 + kC, v);
        tmem_ld_wait();
        if (row < S) *reinterpret_cast<float4*>(dst + kC) = make_float4(v[0], 0.0f, 0.0f, 0.0f);
      }
    }
    if (leader) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- deslice: X^t = M Z^t ---------------------------------------------------------------

struct DesliceArgs {
  int32_t n_tiles;
  int* err;
};

enum { D_FULL0, D_EMPTY0 = 3, D_ZFULL = 6, D_MMA0, D_MMA1, D_TFREE0, D_TFREE1, D_FINAL, D_COUNT };
constexpr int kDStages = 3;

template <int SP>
constexpr size_t deslice_smem_bytes() {
  return 1024 + (SP / 64) * kC * 128 + kDStages * (SP / 64) * kRegion + 2 * 2 * kRegion + 16 * 8 + 16;
}

template <int SP>
__global__ void __launch_bounds__(kThreads, 1)
    attn_deslice_kernel(const __grid_constant__ CUtensorMap map_m, const __grid_constant__ CUtensorMap map_zt,
                        const __grid_constant__ CUtensorMap map_xt, DesliceArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = align1024(smem_raw);
  constexpr int KR = SP / 64;            // K regions (64 tokens each)
  constexpr int kStage = KR * kRegion;   // one M tile
  uint8_t* sz = base;                    // (Z^t)^T: KR regions of C rows
  uint8_t* sm = sz + KR * kC * 128;      // M tiles
  uint8_t* so = sm + kDStages * kStage;  // X^t staging: 2 buffers x 2 regions
  uint64_t* bar = reinterpret_cast<uint64_t*>(so + 4 * kRegion);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 16);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = (a.n_tiles - static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) - 1) / static_cast<int>(gridDim.x);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDStages; ++s) {
      mbar_init(&bar[D_FULL0 + s], 1);
      mbar_init(&bar[D_EMPTY0 + s], 1);
    }
    mbar_init(&bar[D_ZFULL], 1);
    mbar_init(&bar[D_MMA0], 1);
    mbar_init(&bar[D_MMA1], 1);
    mbar_init(&bar[D_TFREE0], kEpi);
    mbar_init(&bar[D_TFREE1], kEpi);
    mbar_init(&bar[D_FINAL], 1);
    fence_barrier_init();
    prefetch_map(&map_m);
    prefetch_map(&map_zt);
    prefetch_map(&map_xt);
  }
  if (warp == 1) tmem_alloc(tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    mbar_arrive_expect_tx(&bar[D_ZFULL], KR * kC * 128);
    for (int r = 0; r < KR; ++r) tma_load_2d(sz + r * kC * 128, &map_zt, &bar[D_ZFULL], 64 * r, 0);
    int issued = 0;
    for (int i = 0; i < T; ++i) {
      const int s = i % kDStages, k = i / kDStages;
      if (!mbar_wait(&bar[D_EMPTY0 + s], (k & 1) ^ 1, a.err, kWaitNs)) break;
      const int y = (static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x)) * kTile;
      mbar_arrive_expect_tx(&bar[D_FULL0 + s], kStage);
      for (int r = 0; r < KR; ++r) tma_load_2d(sm + s * kStage + r * kRegion, &map_m, &bar[D_FULL0 + s], 64 * r, y);
      issued = i + 1;
    }
    mbar_wait(&bar[D_ZFULL], 0, a.err, kWaitNs);
    for (int s = 0; s < kDStages; ++s) {
      const int fills = (issued - s + kDStages - 1) / kDStages;
      if (fills > 0) mbar_wait(&bar[D_FULL0 + s], (fills - 1) & 1, a.err, kWaitNs);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t id = idesc_bf16(kTile, kC, false, false);
    const uint32_t am = smem_addr(sm), az = smem_addr(sz);
    bool ok = mbar_wait(&bar[D_ZFULL], 0, a.err, kWaitNs);
    for (int i = 0; ok && i < T; ++i) {
      const int s = i % kDStages, k = i / kDStages, b = i & 1, use = i >> 1;
      if (!mbar_wait(&bar[D_FULL0 + s], k & 1, a.err, kWaitNs)) break;
      if (!mbar_wait(&bar[D_TFREE0 + b], (use & 1) ^ 1, a.err, kWaitNs)) break;
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < SP / 16; ++kk) {
        const uint32_t off = (kk & 3) * 32;
        const uint64_t da = sdesc_sw128(am + s * kStage + (kk >> 2) * kRegion + off, 16, 1024);
        const uint64_t db = sdesc_sw128(az + (kk >> 2) * kC * 128 + off, 16, 1024);
        mma_bf16(tmem + b * kC, da, db, id, kk > 0 ? 1u : 0u);
      }
      mma_commit(&bar[D_EMPTY0 + s]);
      mma_commit(&bar[D_MMA0 + b]);
    }
    mma_commit(&bar[D_FINAL]);
    mbar_wait(&bar[D_FINAL], 0, a.err, kWaitNs);
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const bool leader = (warp == 2 && lane == 0);
    for (int i = 0; i < T; ++i) {
      const int tile = static_cast<int>(blockIdx.x) + i * static_cast<int>(gridDim.x);
      const int b = i & 1, use = i >> 1;
      bool ok = mbar_wait(&bar[D_MMA0 + b], use & 1, a.err, kWaitNs);
      if (leader) bulk_wait_read_1();  // the store from this staging buffer two tiles ago has read it
      if (vote_any(!ok, 1, kEpi)) break;
      tc_fence_after();
      const uint32_t tl = tmem + b * kC + (static_cast<uint32_t>(32 * q) << 16);
      uint8_t* out = so + b * 2 * kRegion;
#pragma unroll
      for (int c = 0; c < kC / 32; ++c) {
        float v[32];
        tmem_ld32(tl + 32 * c, v);
        tmem_ld_wait();
#pragma unroll
        for (int m = 0; m < 4; ++m) st_chunk(out + (c >> 1) * kRegion, row, (c & 1) * 4 + m, v + 8 * m);
      }
      tc_fence_before();
      mbar_arrive(&bar[D_TFREE0 + b]);
      fence_async_smem();
      named_sync(1, kEpi);
      if (leader) {
        tma_store_2d(&map_xt, out, 0, tile * kTile);
        tma_store_2d(&map_xt, out + kRegion, 64, tile * kTile);
        bulk_commit();
      }
    }
    if (leader) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// ---- token sums: fixed-order sum of the CTA partials ------------------------------------

// grid (S, 5): block (j, cb) sums columns 32 cb .. 32 cb + 31 (<= 128) of token j over the
// G partials; 8 lanes of g per column, combined in lane order.
__global__ void __launch_bounds__(256) attn_reduce_kernel(const float* partial, int G, int S, float* zsum) {
  __shared__ float red[8][33];
  const int j = blockIdx.x, cb = blockIdx.y;
  const int cl = threadIdx.x & 31, g0 = threadIdx.x >> 5;
  const int c = 32 * cb + cl;
  // partials g0, g0 + 8, ... in that order; loads issued kBatch at a time before their sums
  constexpr int kBatch = 10;
  float acc = 0.0f;
  if (c <= kC)
    for (int g1 = g0; g1 < G; g1 += 8 * kBatch) {
      float v[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) {
        const int g = g1 + 8 * k;
        v[k] = g < G ? partial[(static_cast<int64_t>(g) * S + j) * kPartPitch + c] : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < kBatch; ++k) acc += v[k];
    }
  red[g0][cl] = acc;
  __syncthreads();
  if (g0 == 0 && c <= kC) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k][cl];
    zsum[j * kPartPitch + c] = s;
  }
}

// ---- token attention (FP32 CUDA cores; S x C is tiny) -------------------------------------

// Q, K, V = Z W + b for all heads, Z = token sums / weight sums + b_U: CTA (x, y) forms the 32 x 32
// block of token rows 32 y .. and columns 32 (x % 4) .. of matrix x / 4 (Q, K, V) from the
// staged token rows and weight columns; CTA (0, y) also writes those rows of Z.
__global__ void __launch_bounds__(256) attn_qkv_kernel(const float* zsum, const float* bias_u, const float* wqkv,
                                                       const float* bqkv, int S, float* z, float* qkv) {
  __shared__ float sz[32][kC + 1];
  __shared__ float sw[kC][33];
  __shared__ float sden[32];
  const int m = blockIdx.x >> 2, c0 = (blockIdx.x & 3) * 32, r0 = blockIdx.y * 32;
  if (threadIdx.x < 32) sden[threadIdx.x] = r0 + threadIdx.x < S ? zsum[(r0 + threadIdx.x) * kPartPitch + kC] : 0.0f;
  // every load of the staging issued before the first use (fixed trip counts, 256 threads)
  constexpr int kIt = 32 * kC / 256;
  float zv[kIt], wv[kIt];
#pragma unroll
  for (int k = 0; k < kIt; ++k) {
    const int e = threadIdx.x + 256 * k;
    const int j = e / kC, c = e % kC;
    zv[k] = r0 + j < S ? zsum[(r0 + j) * kPartPitch + c] : 0.0f;
    wv[k] = wqkv[static_cast<int64_t>(m) * kC * kC + (e >> 5) * kC + c0 + (e & 31)];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kIt; ++k) {
    const int e = threadIdx.x + 256 * k;
    const int j = e / kC, c = e % kC, row = r0 + j;
    const float w = sden[j];
    const float v = w > 0.0f ? zv[k] / w + bias_u[c] : 0.0f;
    if (blockIdx.x == 0 && row < S) z[row * kC + c] = v;
    sz[j][c] = v;
    sw[e >> 5][e & 31] = wv[k];
  }
  __syncthreads();
  const int t = threadIdx.x & 31, jb = threadIdx.x >> 5;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
  for (int c = 0; c < kC; ++c) {
    const float w = sw[c][t];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = fmaf(sz[jb + 8 * k][c], w, acc[k]);
  }
  const float b = bqkv[m * kC + c0 + t];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int row = r0 + jb + 8 * k;
    if (row < S) qkv[(static_cast<int64_t>(m) * S + row) * kC + c0 + t] = acc[k] + b;
  }
}

// Per head h (D = C / H channels): CTA (h, y) takes the query tokens 32 y .. 32 y + 31, four
// threads per query, each running an online softmax over the keys b = part, part + 4, ...;
// the four partial (max, sum, output) triples are merged by shuffles in a fixed order.
// Writes Z^t (FP32, [S][C]) and (Z^t)^T in bf16 ([C][S_pad], the deslice's B operand).
template <int D>
__global__ void __launch_bounds__(128) attn_heads_kernel(const float* qkv, int S, int SP, float scale, float* zt,
                                                         __nv_bfloat16* ztT) {
  extern __shared__ float sh[];
  float* sk = sh;          // [S][D]
  float* sv = sh + S * D;  // [S][D]
  const int h = blockIdx.x, a = blockIdx.y * 32 + (threadIdx.x >> 2), part = threadIdx.x & 3;
  // staging with every load issued first: S * D <= 128 D elements over 128 threads
  float kv[D], vv[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int e = threadIdx.x + 128 * k, b = e / D, t = e % D;
    kv[k] = e < S * D ? qkv[(static_cast<int64_t>(S) + b) * kC + h * D + t] : 0.0f;
    vv[k] = e < S * D ? qkv[(2 * static_cast<int64_t>(S) + b) * kC + h * D + t] : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int e = threadIdx.x + 128 * k;
    if (e < S * D) {
      sk[e] = kv[k];
      sv[e] = vv[k];
    }
  }
  __syncthreads();
  float qa[D], o[D];
#pragma unroll
  for (int t = 0; t < D; ++t) {
    qa[t] = a < S ? qkv[static_cast<int64_t>(a) * kC + h * D + t] * scale : 0.0f;
    o[t] = 0.0f;
  }
  float mx = -INFINITY, l = 0.0f;
  for (int b = part; b < S; b += 4) {
    float s = 0.0f;
#pragma unroll
    for (int t = 0; t < D; ++t) s = fmaf(qa[t], sk[b * D + t], s);
    if (s > mx) {
      const float f = expf(mx - s);
      l *= f;
#pragma unroll
      for (int t = 0; t < D; ++t) o[t] *= f;
      mx = s;
    }
    const float w = expf(s - mx);
    l += w;
#pragma unroll
    for (int t = 0; t < D; ++t) o[t] = fmaf(w, sv[b * D + t], o[t]);
  }
#pragma unroll
  for (int off = 1; off <= 2; off <<= 1) {
    const float m2 = __shfl_xor_sync(0xffffffffu, mx, off);
    const float l2 = __shfl_xor_sync(0xffffffffu, l, off);
    const float mn = fmaxf(mx, m2);
    const float f1 = mx == -INFINITY ? 0.0f : expf(mx - mn);
    const float f2 = m2 == -INFINITY ? 0.0f : expf(m2 - mn);
    l = __fadd_rn(__fmul_rn(l, f1), __fmul_rn(l2, f2));
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const float o2 = __shfl_xor_sync(0xffffffffu, o[t], off);
      o[t] = __fadd_rn(__fmul_rn(o[t], f1), __fmul_rn(o2, f2));
    }
    mx = mn;
  }
  if (part == 0 && a < S) {
    const float il = 1.0f / l;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      const float v = o[t] * il;
      zt[a * kC + h * D + t] = v;
      ztT[(h * D + t) * SP + a] = __float2bfloat16_rn(v);
    }
  }
}

}  // namespace attn
}  // namespace pfem

// ---- host side ---------------------------------------------------------------------------

using namespace pfem;
using namespace pfem::attn;

struct pfem_attn_s {
  int S = 0, SP = 0, H = 0;
  float scale = 1.0f;
  cudaStream_t stream = nullptr;
  int n_sm = 0;
  __nv_bfloat16* wcat = nullptr;  // [C + S_pad][C]: rows = output channels of W_U, W_M, zero pad (K-major)
  float* bias = nullptr;          // [C + S_pad]: b_U, b_M, -inf pad
  float* wqkv = nullptr;          // [3][C][C] (in, out)
  float* bqkv = nullptr;          // [3][C]
  float* partial = nullptr;       // [n_sm][S][kPartPitch]
  float* zsum = nullptr;          // [S][kPartPitch]
  float* z = nullptr;             // [S][C]
  float* zt = nullptr;            // [S][C]
  float* qkv = nullptr;            // [3][S][C]: Q, K, V
  __nv_bfloat16* ztT = nullptr;   // [C][SP]
  __nv_bfloat16* mbuf = nullptr;  // [mbuf_rows][SP] workspace for M when the caller gives none
  int64_t mbuf_rows = 0;
  int* err = nullptr;
  CUtensorMap map_w{}, map_zt{};
  bool timing = false;
  cudaEvent_t ev[5] = {};  // around the slice, reduce, tokens and deslice kernels
};

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

// 2-D bf16 row-major [rows][cols] map with a {64, box_rows} box and the 128-byte swizzle
pfem_status make_map(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return PFEM_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols) * 2};
  const cuuint32_t box[2] = {64, static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor map encoding failed (%d)", static_cast<int>(r));
    return PFEM_ERR_CUDA;
  }
  return PFEM_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int SP>
pfem_status set_smem_attrs() {
  static cudaError_t e = [] {
    cudaError_t r = cudaFuncSetAttribute(attn_slice_kernel<SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(slice_smem_bytes<SP>()));
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(attn_deslice_kernel<SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(deslice_smem_bytes<SP>()));
    if (r == cudaSuccess)  // K and V of one head, S x 64 each at most
      r = cudaFuncSetAttribute(attn_heads_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(2 * 128 * 64 * sizeof(float)));
    return r;
  }();
  PFEM_CUDA(e);
  return PFEM_OK;
}

template <int SP>
pfem_status launch_forward(pfem_attn_t a, int64_t n, const void* x, void* xt, __nv_bfloat16* m) {
  pfem_status st = set_smem_attrs<SP>();
  if (st) return st;
  CUtensorMap mx, mm, mxt;
  if ((st = make_map(&mx, x, n, kC, kTile)) || (st = make_map(&mm, m, n, SP, kTile)) ||
      (st = make_map(&mxt, xt, n, kC, kTile)))
    return st;
  const int n_tiles = static_cast<int>((n + kTile - 1) / kTile);
  const int grid = std::min(a->n_sm, n_tiles);
  SliceArgs sa{n, n_tiles, a->S, a->bias, a->partial, a->err};
  if (a->timing) PFEM_CUDA(cudaEventRecord(a->ev[0], a->stream));
  attn_slice_kernel<SP><<<grid, kSliceThreads, slice_smem_bytes<SP>(), a->stream>>>(mx, a->map_w, mm, sa);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  if (a->timing) PFEM_CUDA(cudaEventRecord(a->ev[1], a->stream));
  attn_reduce_kernel<<<dim3(a->S, 5), 256, 0, a->stream>>>(a->partial, grid, a->S, a->zsum);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  if (a->timing) PFEM_CUDA(cudaEventRecord(a->ev[2], a->stream));
  attn_qkv_kernel<<<dim3(12, (a->S + 31) / 32), 256, 0, a->stream>>>(a->zsum, a->bias, a->wqkv, a->bqkv, a->S, a->z,
                                                                      a->qkv);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  const dim3 hg(a->H, (a->S + 31) / 32);
  const size_t hsm = 2 * static_cast<size_t>(a->S) * (kC / a->H) * sizeof(float);
  switch (a->H) {
    case 2: attn_heads_kernel<64><<<hg, 128, hsm, a->stream>>>(a->qkv, a->S, SP, a->scale, a->zt, a->ztT); break;
    case 4: attn_heads_kernel<32><<<hg, 128, hsm, a->stream>>>(a->qkv, a->S, SP, a->scale, a->zt, a->ztT); break;
    case 8: attn_heads_kernel<16><<<hg, 128, hsm, a->stream>>>(a->qkv, a->S, SP, a->scale, a->zt, a->ztT); break;
    default: attn_heads_kernel<8><<<hg, 128, hsm, a->stream>>>(a->qkv, a->S, SP, a->scale, a->zt, a->ztT); break;
  }
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  DesliceArgs da{n_tiles, a->err};
  if (a->timing) PFEM_CUDA(cudaEventRecord(a->ev[3], a->stream));
  attn_deslice_kernel<SP><<<grid, attn::kThreads, deslice_smem_bytes<SP>(), a->stream>>>(mm, a->map_zt, mxt, da);
  PFEM_COUNT_LAUNCH();
  PFEM_CUDA(cudaGetLastError());
  if (a->timing) PFEM_CUDA(cudaEventRecord(a->ev[4], a->stream));
  return PFEM_OK;
}

void release(pfem_attn_t a) {
  if (!a) return;
  cudaFree(a->wcat);
  cudaFree(a->bias);
  cudaFree(a->wqkv);
  cudaFree(a->bqkv);
  cudaFree(a->partial);
  cudaFree(a->zsum);
  cudaFree(a->z);
  cudaFree(a->zt);
  cudaFree(a->qkv);
  cudaFree(a->ztT);
  cudaFree(a->mbuf);
  cudaFree(a->err);
  for (cudaEvent_t e : a->ev)
    if (e) cudaEventDestroy(e);
  delete a;
}

}  // namespace

extern "C" pfem_status pfem_attn_create(int32_t n_channels, int32_t n_tokens, int32_t n_heads, double scale,
                                        const pfem_attn_weights* w, void* cuda_stream, pfem_attn_t* out) {
  if (!out) {
    set_error("pfem_attn_create: out is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!w || !w->wu || !w->bu || !w->wm || !w->bm || !w->wq || !w->bq || !w->wk || !w->bk || !w->wv || !w->bv) {
    set_error("pfem_attn_create: a weight pointer is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  if (n_channels != kC) {
    set_error("pfem_attn_create: the kernels are built for %d channels (got %d)", kC, n_channels);
    return PFEM_ERR_UNSUPPORTED;
  }
  if (n_tokens < 16 || n_tokens > 128 || n_tokens % 16) {
    set_error("pfem_attn_create: tokens must be a multiple of 16 in [16, 128] (got %d)", n_tokens);
    return PFEM_ERR_UNSUPPORTED;
  }
  if (n_heads != 2 && n_heads != 4 && n_heads != 8 && n_heads != 16) {
    set_error("pfem_attn_create: heads must be 2, 4, 8 or 16 (got %d)", n_heads);
    return PFEM_ERR_UNSUPPORTED;
  }
  if (!std::isfinite(scale)) {
    set_error("pfem_attn_create: scale is not finite");
    return PFEM_ERR_INVALID_ARG;
  }
  const int S = n_tokens, SP = S <= 64 ? 64 : 128, CS = kC + SP;  // W_M padded to SP tokens
  auto* a = new pfem_attn_s();
  a->S = S;
  a->SP = SP;
  a->H = n_heads;
  a->scale = static_cast<float>(scale);
  a->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&a->n_sm, cudaDevAttrMultiProcessorCount, dev);
  std::vector<__nv_bfloat16> wcat(static_cast<size_t>(CS) * kC);
  std::vector<float> bias(CS), wqkv(3 * static_cast<size_t>(kC) * kC), bqkv(3 * kC);
  for (int o = 0; o < kC; ++o)
    for (int i = 0; i < kC; ++i) wcat[static_cast<size_t>(o) * kC + i] = __float2bfloat16_rn(w->wu[i * kC + o]);
  for (int o = 0; o < S; ++o)
    for (int i = 0; i < kC; ++i) wcat[static_cast<size_t>(kC + o) * kC + i] = __float2bfloat16_rn(w->wm[i * S + o]);
  for (int o = 0; o < kC; ++o) bias[o] = w->bu[o];
  for (int o = 0; o < SP; ++o) bias[kC + o] = o < S ? w->bm[o] : -INFINITY;
  const float* ws[3] = {w->wq, w->wk, w->wv};
  const float* bs[3] = {w->bq, w->bk, w->bv};
  for (int m = 0; m < 3; ++m) {
    std::memcpy(wqkv.data() + static_cast<size_t>(m) * kC * kC, ws[m], sizeof(float) * kC * kC);
    std::memcpy(bqkv.data() + m * kC, bs[m], sizeof(float) * kC);
  }
  for (float v : wqkv)
    if (!std::isfinite(v)) e = cudaErrorInvalidValue;
  auto alloc = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  };
  alloc(&a->wcat, wcat.size() * 2);
  alloc(&a->bias, CS * sizeof(float));
  alloc(&a->wqkv, wqkv.size() * sizeof(float));
  alloc(&a->bqkv, bqkv.size() * sizeof(float));
  alloc(&a->partial, static_cast<size_t>(std::max(a->n_sm, 1)) * S * kPartPitch * sizeof(float));
  alloc(&a->zsum, static_cast<size_t>(S) * kPartPitch * sizeof(float));
  alloc(&a->z, static_cast<size_t>(S) * kC * sizeof(float));
  alloc(&a->zt, static_cast<size_t>(S) * kC * sizeof(float));
  alloc(&a->qkv, 3 * static_cast<size_t>(S) * kC * sizeof(float));
  alloc(&a->ztT, static_cast<size_t>(kC) * SP * 2);
  alloc(&a->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(a->wcat, wcat.data(), wcat.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(a->bias, bias.data(), CS * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(a->wqkv, wqkv.data(), wqkv.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(a->bqkv, bqkv.data(), bqkv.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(a->ztT, 0, static_cast<size_t>(kC) * SP * 2);
  if (e == cudaSuccess) e = cudaMemset(a->err, 0, sizeof(int));
  for (cudaEvent_t& ev : a->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e != cudaSuccess) {
    release(a);
    if (e == cudaErrorInvalidValue) {
      set_error("pfem_attn_create: non-finite weight");
      return PFEM_ERR_INVALID_ARG;
    }
    return cuda_fail(e, "pfem_attn_create");
  }
  pfem_status st = make_map(&a->map_w, a->wcat, CS, kC, CS);
  if (!st) st = make_map(&a->map_zt, a->ztT, kC, SP, kC);
  if (st) {
    release(a);
    return st;
  }
  *out = a;
  return PFEM_OK;
}

extern "C" void pfem_attn_destroy(pfem_attn_t a) {
  if (a) cudaStreamSynchronize(a->stream);
  release(a);
}

extern "C" pfem_status pfem_attn_forward(pfem_attn_t a, int64_t n_points, const void* x, void* xt, void* m,
                                         float* z, float* zt) {
  if (!a) {
    set_error("pfem_attn_forward: handle is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  if (n_points < 0 || n_points > (int64_t(1) << 31) - kTile) {
    set_error("pfem_attn_forward: point count out of range");
    return PFEM_ERR_INVALID_ARG;
  }
  if (n_points == 0) return PFEM_OK;
  if (!x || !xt || !aligned16(x) || !aligned16(xt) || (m && !aligned16(m))) {
    set_error("pfem_attn_forward: x and xt (and m) must be non-NULL, 16-byte aligned device pointers");
    return PFEM_ERR_INVALID_ARG;
  }
  __nv_bfloat16* mb = static_cast<__nv_bfloat16*>(m);
  if (!mb) {
    if (a->mbuf_rows < n_points) {
      PFEM_CUDA(cudaStreamSynchronize(a->stream));
      cudaFree(a->mbuf);
      a->mbuf = nullptr;
      a->mbuf_rows = 0;
      PFEM_CUDA(cudaMalloc(reinterpret_cast<void**>(&a->mbuf), static_cast<size_t>(n_points) * a->SP * 2));
      a->mbuf_rows = n_points;
    }
    mb = a->mbuf;
  }
  pfem_status st = a->SP == 64 ? launch_forward<64>(a, n_points, x, xt, mb) : launch_forward<128>(a, n_points, x, xt, mb);
  if (st) return st;
  if (z) PFEM_CUDA(cudaMemcpyAsync(z, a->z, static_cast<size_t>(a->S) * kC * sizeof(float), cudaMemcpyDeviceToDevice, a->stream));
  if (zt)
    PFEM_CUDA(cudaMemcpyAsync(zt, a->zt, static_cast<size_t>(a->S) * kC * sizeof(float), cudaMemcpyDeviceToDevice, a->stream));
  return PFEM_OK;
}

extern "C" pfem_status pfem_attn_sync(pfem_attn_t a) {
  if (!a) {
    set_error("pfem_attn_sync: handle is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  int flag = 0;
  PFEM_CUDA(cudaMemcpyAsync(&flag, a->err, sizeof(int), cudaMemcpyDeviceToHost, a->stream));
  PFEM_CUDA(cudaStreamSynchronize(a->stream));
  if (flag) {
    PFEM_CUDA(cudaMemsetAsync(a->err, 0, sizeof(int), a->stream));
    PFEM_CUDA(cudaStreamSynchronize(a->stream));
    set_error("physics attention: a bounded wait expired; outputs are incomplete");
    return PFEM_ERR_TIMEOUT;
  }
  return PFEM_OK;
}

extern "C" pfem_status pfem_attn_set_timing(pfem_attn_t a, int32_t on) {
  if (!a) {
    set_error("pfem_attn_set_timing: handle is NULL");
    return PFEM_ERR_INVALID_ARG;
  }
  a->timing = on != 0;
  return PFEM_OK;
}

extern "C" pfem_status pfem_attn_kernel_ms(pfem_attn_t a, double* ms) {
  if (!a || !ms || !a->timing) {
    set_error("pfem_attn_kernel_ms: NULL argument or timing off");
    return PFEM_ERR_INVALID_ARG;
  }
  PFEM_CUDA(cudaEventSynchronize(a->ev[4]));
  for (int k = 0; k < 4; ++k) {
    float t = 0.0f;
    PFEM_CUDA(cudaEventElapsedTime(&t, a->ev[k], a->ev[k + 1]));
    ms[k] = t;
  }
  return PFEM_OK;
}
