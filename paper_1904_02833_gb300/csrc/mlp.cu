// Warm-start network on the 5th-generation tensor cores: 24 features -> 128 -> 128 -> 1
// with SiLU, BF16 operands, FP32 accumulation in tensor memory.
//
// Inference (mlp_infer_kernel) and training (mlp_train_kernel: forward, MSE loss,
// backward, weight-gradient accumulation across tiles in tensor memory) process tiles
// of 128 constraint rows.  Every GEMM is one or more tcgen05.mma of M = 128 issued by one
// thread; operands are staged in shared memory in the canonical no-swizzle K-major
// layout (tc.cuh); transposed operands of the weight gradients are written transposed
// by the epilogue threads, so every MMA reads K-major tiles.  Adam runs on FP32 master
// weights (mlp_adam_kernel) and refreshes the BF16 copies the GEMMs read.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "snakesim.h"
#include "tc.cuh"

using namespace snakesim;

namespace {

constexpr int kIn = 24;      // features
constexpr int kInPad = 32;   // K of the first GEMM (two K = 16 steps)
constexpr int kHid = 128;
constexpr int kTile = 128;   // rows per tile (M of every MMA)
constexpr uint32_t kWaitLimit = 1u << 26;

// parameter vector (FP32): W1 [128][24], b1 [128], W2 [128][128], b2 [128], w3 [128], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
constexpr int kNumParams = kOffB3 + 1;  // 19841
static_assert(kNumParams == MLP_NUM_PARAMS, "parameter count");

// After a timed-out wait on an MMA: thread 0, the only thread that issues MMAs, commits
// once more to a barrier of its own, which arrives only when every MMA the thread issued
// before has completed (tcgen05.commit tracks all of the issuing thread's earlier
// tensor-core operations, not one group), and the block waits for that arrival before
// its TMEM columns are freed.  Like every wait it is bounded: an MMA completes in
// microseconds, so a drain that runs out means no completion will ever arrive (the
// columns are not being written) and the block still frees them, which it must do
// before it exits.
__device__ __forceinline__ void drain_mma(uint64_t* drain, int t) {
  if (t == 0) tc::mma_commit(drain);
  tc::mbar_wait(drain, 0, kWaitLimit);
}

struct MlpDev {
  const __nv_bfloat16* w1;  // [128][32] row-major (out x in, zero-padded in 24..31)
  const __nv_bfloat16* w2;  // [128][128] (out x in)
  const float* b1;
  const float* b2;
  const float* w3;
  const float* b3;
};

__device__ __forceinline__ float silu(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  return z * fmaf(0.5f, t, 0.5f);
}
__device__ __forceinline__ float silu_grad(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  const float s = fmaf(0.5f, t, 0.5f);
  return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
// silu of two values, evaluated in bfloat16 pairs (the result feeds a bfloat16 operand
// anyway): silu(z) = hz + hz tanh(hz) with hz = z / 2, one packed tanh for two values.
__device__ __forceinline__ uint32_t silu_bf16x2(float z0, float z1) {
  const uint32_t hz = pack_bf16x2(0.5f * z0, 0.5f * z1);
  uint32_t th, r;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(th) : "r"(hz));
  asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(hz), "r"(th));
  return r;
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}
__device__ __forceinline__ void st_shared_u16(uint32_t addr, uint16_t v) {
  asm volatile("st.shared.u16 [%0], %1;\n" ::"r"(addr), "h"(v) : "memory");
}

// Copies a row-major bf16 matrix [rows][K] into the canonical K-major smem layout.
__device__ void stage_kmajor(uint8_t* dst, const __nv_bfloat16* src, int rows, int K) {
  const int chunks = rows * (K / 8);
  const uint32_t base = tc::smem_u32(dst);
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int m = c / (K / 8), kc = (c % (K / 8)) * 8;
    const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)m * K + kc);
    st_shared_v4(base + tc::kmajor_off(m, kc, K), v.x, v.y, v.z, v.w);
  }
}
// Same, transposed: dst holds src^T ([K][rows] K-major over `rows`).
__device__ void stage_kmajor_t(uint8_t* dst, const __nv_bfloat16* src, int rows, int K) {
  const uint32_t base = tc::smem_u32(dst);
  for (int e = threadIdx.x; e < rows * K; e += blockDim.x) {
    const int m = e / K, k = e % K;
    const __nv_bfloat16 v = src[(size_t)m * K + k];
    st_shared_u16(base + tc::kmajor_off(k, m, rows), *reinterpret_cast<const uint16_t*>(&v));
  }
}

struct InferSmem {
  uint8_t w1[kHid * kInPad * 2];
  uint8_t w2[kHid * kHid * 2];
  uint8_t x[kTile * kInPad * 2];
  uint8_t h[kTile * kHid * 2];
  float b1[kHid], b2[kHid], w3[kHid];
  float part[kTile];  // second column half's share of y, per row
  uint64_t mbar;
  uint64_t drain;  // drain_mma: arrives once every MMA issued so far has completed
  uint32_t tmem;
};
constexpr int kInferThreads = 256;

}  // namespace

// y[r] = w3 . silu(W2 silu(W1 x_r + b1) + b2) + b3 for feat [rows][32] bf16.
// Eight warps per block, two blocks per SM: warp w reads TMEM lane quarter w % 4 (rows
// 32 (w % 4) .. +31) and takes the column half w / 4 of both epilogues, so each row's
// 256 SiLU evaluations are split between two threads; the next tile's features are
// loaded into registers while the current tile's MMAs run.
// The rows the network runs on, in the solver's six-rows-per-node order: sel = 0 all rows;
// sel = 1 the stretch, yaw and pitch rows (row r is row 6 (r / 3) + r % 3 of feat and out);
// sel = 2 the stretch rows (row r is row 6 r).
__device__ __forceinline__ long long infer_row(long long r, int sel) {
  return sel == 1 ? 6 * (r / 3) + r % 3 : (sel == 2 ? 6 * r : r);
}
__global__ void __launch_bounds__(kInferThreads, 2) mlp_infer_kernel(const __nv_bfloat16* __restrict__ feat,
                                                                    long long rows, MlpDev w,
                                                                    float* __restrict__ out, int* err,
                                                                    int sel) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;  // the TMEM lane (tile row) this thread reads
  if (warp == 0) tc::tmem_alloc(&S.tmem, 256);
  if (t == 0) { tc::mbar_init(&S.mbar, 1); tc::mbar_init(&S.drain, 1); }
  stage_kmajor(S.w1, w.w1, kHid, kInPad);
  stage_kmajor(S.w2, w.w2, kHid, kHid);
  if (t < kHid) { S.b1[t] = w.b1[t]; S.b2[t] = w.b2[t]; S.w3[t] = w.w3[t]; }
  const float b3 = w.b3[0];
  tc::fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
  const uint32_t idesc = tc::make_idesc_bf16(kTile, kHid);
  const uint32_t sx = tc::smem_u32(S.x), sh = tc::smem_u32(S.h);
  const uint32_t sw1 = tc::smem_u32(S.w1), sw2 = tc::smem_u32(S.w2);
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (rows + kTile - 1) / kTile;
  // a tile is 128 rows x 4 chunks of 16 bytes: chunks t and t + 256 of this thread
  auto load_tile = [&](long long tile, uint4 (&v)[2]) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int c = t + u * kInferThreads;
      const long long r = tile * kTile + (c >> 2);
      v[u] = make_uint4(0u, 0u, 0u, 0u);
      if (tile < ntiles && r < rows) v[u] = reinterpret_cast<const uint4*>(feat + infer_row(r, sel) * kInPad)[c & 3];
    }
  };
  uint4 nxt[2];
  load_tile(blockIdx.x, nxt);
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int c = t + u * kInferThreads;
      st_shared_v4(sx + tc::kmajor_off(c >> 2, 8 * (c & 3), kInPad), nxt[u].x, nxt[u].y, nxt[u].z, nxt[u].w);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int kk = 0; kk < kInPad / 16; ++kk)
        tc::mma_bf16(tmem, tc::make_sdesc(sx + kk * 256, 128, kInPad / 8 * 128),
                     tc::make_sdesc(sw1 + kk * 256, 128, kInPad / 8 * 128), idesc, kk > 0);
      tc::mma_commit(&S.mbar);
    }
    load_tile(tile + gridDim.x, nxt);  // in flight while the tensor core works
    if (__syncthreads_or(!tc::mbar_wait(&S.mbar, phase, kWaitLimit))) { ok = false; break; }
    phase ^= 1;
    tc::fence_after_sync();
    // epilogue 1: h = silu(z1 + b1) -> bf16 -> shared (A operand of the second GEMM)
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
      float a[32];
      tc::tmem_ld32(tmem + lane_base + c0, a);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = c0 + 8 * q + 2 * e;
          p[e] = silu_bf16x2(a[8 * q + 2 * e] + S.b1[c], a[8 * q + 2 * e + 1] + S.b1[c + 1]);
        }
        st_shared_v4(sh + tc::kmajor_off(row, c0 + 8 * q, kHid), p[0], p[1], p[2], p[3]);
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc::mma_bf16(tmem + kHid, tc::make_sdesc(sh + kk * 256, 128, kHid / 8 * 128),
                     tc::make_sdesc(sw2 + kk * 256, 128, kHid / 8 * 128), idesc, kk > 0);
      tc::mma_commit(&S.mbar);
    }
    if (__syncthreads_or(!tc::mbar_wait(&S.mbar, phase, kWaitLimit))) { ok = false; break; }
    phase ^= 1;
    tc::fence_after_sync();
    // epilogue 2: y = w3 . silu(z2 + b2) + b3, the two column halves added through shared
    float y = 0.f;
#pragma unroll 1
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
      float a[32];
      tc::tmem_ld32(tmem + lane_base + kHid + c0, a);
#pragma unroll
      for (int i = 0; i < 32; ++i) y = fmaf(S.w3[c0 + i], silu(a[i] + S.b2[c0 + i]), y);
    }
    if (half == 1) S.part[row] = y;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const long long r = tile * kTile + row;
    if (half == 0 && r < rows) out[infer_row(r, sel)] = (y + S.part[row]) + b3;
  }
  if (!ok) {
    if (t == 0) atomicExch(err, 1);
    drain_mma(&S.drain, t);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Self-test of the bounded tensor-core waits: one block allocates tensor memory, waits
// with a bound of `polls` on an mbarrier that nothing arrives on (so the wait runs out, as
// a lost MMA completion would make the network kernels' waits run out), records the
// timeout in *err and frees its tensor memory before returning, as those kernels do.
__global__ void __launch_bounds__(128) mlp_wait_selftest_kernel(uint32_t polls, int* err) {
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_addr;
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&tmem_addr, 32);
  if (t == 0) tc::mbar_init(&mbar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (__syncthreads_or(!tc::mbar_wait(&mbar, 0, polls)) && t == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_addr, 32);
}

namespace {

struct TrainSmem {
  uint8_t w1[kHid * kInPad * 2];   // W1 [h1][in]
  uint8_t w2[kHid * kHid * 2];     // W2 [h2][h1]
  uint8_t w2t[kHid * kHid * 2];    // W2^T [h1][h2]
  uint8_t x[kTile * kInPad * 2];   // X [row][in]
  uint8_t xt[kInPad * kTile * 2];  // X^T [in][row]
  uint8_t h[kTile * kHid * 2];     // H1 [row][h1], later dZ2 [row][h2]
  uint8_t ht[kHid * kTile * 2];    // H1^T [h1][row]
  uint8_t dt[kHid * kTile * 2];    // dZ2^T [h2][row], later dZ1^T [h1][row]
  float b1[kHid], b2[kHid], w3[kHid];
  float gb1[kHid], gb2[kHid], gw3[kHid];
  float gb3, loss;
  uint64_t mbar;
  uint64_t drain;  // drain_mma: arrives once every MMA issued so far has completed
  uint32_t tmem;
};

}  // namespace

// Accumulates the gradient of L = sum_r (y_r - target_r)^2 * scale over `rows` rows into
// grad[kNumParams] (FP32, atomically) and L into *loss.
__global__ void __launch_bounds__(128, 1) mlp_train_kernel(const __nv_bfloat16* __restrict__ feat,
                                                           const float* __restrict__ target,
                                                           long long rows, float scale, MlpDev w,
                                                           float* __restrict__ grad,
                                                           float* __restrict__ loss, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) tc::tmem_alloc(&S.tmem, 512);
  if (t == 0) { tc::mbar_init(&S.mbar, 1); tc::mbar_init(&S.drain, 1); S.gb3 = 0.f; S.loss = 0.f; }
  stage_kmajor(S.w1, w.w1, kHid, kInPad);
  stage_kmajor(S.w2, w.w2, kHid, kHid);
  stage_kmajor_t(S.w2t, w.w2, kHid, kHid);
  S.b1[t] = w.b1[t]; S.b2[t] = w.b2[t]; S.w3[t] = w.w3[t];
  S.gb1[t] = 0.f; S.gb2[t] = 0.f; S.gw3[t] = 0.f;
  const float b3 = w.b3[0];
  tc::fence_proxy_async();
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t T_Z1 = 0, T_Z2 = 128, T_DW1 = 256, T_DW2 = 384;  // TMEM columns
  const uint32_t id_128 = tc::make_idesc_bf16(kTile, kHid);
  const uint32_t id_32 = tc::make_idesc_bf16(kHid, kInPad);
  const uint32_t sx = tc::smem_u32(S.x), sxt = tc::smem_u32(S.xt), sh = tc::smem_u32(S.h);
  const uint32_t sht = tc::smem_u32(S.ht), sdt = tc::smem_u32(S.dt);
  const uint32_t sw1 = tc::smem_u32(S.w1), sw2 = tc::smem_u32(S.w2), sw2t = tc::smem_u32(S.w2t);
  const uint32_t SB32 = kInPad / 8 * 128, SB128 = kHid / 8 * 128;
  uint32_t phase = 0;
  bool ok = true, first = true;
  auto sync_mma = [&]() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  auto wait_mma = [&]() -> bool {
    if (__syncthreads_or(!tc::mbar_wait(&S.mbar, phase, kWaitLimit))) {
      if (t == 0) atomicExch(err, 1);
      return false;
    }
    phase ^= 1;
    tc::fence_after_sync();
    return true;
  };
  const long long ntiles = (rows + kTile - 1) / kTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long r = tile * kTile + t;
    const bool valid = r < rows;
    // X row -> sX (K-major over inputs) and X^T -> sXT (K-major over rows)
    uint4 v[4] = {};
    if (valid) {
      const uint4* src = reinterpret_cast<const uint4*>(feat + r * kInPad);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = src[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      st_shared_v4(sx + tc::kmajor_off(t, 8 * q, kInPad), v[q].x, v[q].y, v[q].z, v[q].w);
      const uint16_t* e = reinterpret_cast<const uint16_t*>(&v[q]);
#pragma unroll
      for (int i = 0; i < 8; ++i) st_shared_u16(sxt + tc::kmajor_off(8 * q + i, t, kTile), e[i]);
    }
    sync_mma();
    if (t == 0) {
      for (int kk = 0; kk < kInPad / 16; ++kk)
        tc::mma_bf16(tmem + T_Z1, tc::make_sdesc(sx + kk * 256, 128, SB32),
                     tc::make_sdesc(sw1 + kk * 256, 128, SB32), id_128, kk > 0);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    // H1 = silu(Z1 + b1) -> sH [row][h1] and sHT [h1][row]
    for (int c0 = 0; c0 < kHid; c0 += 32) {
      float a[32];
      tc::tmem_ld32(tmem + lane_base + T_Z1 + c0, a);
      for (int q = 0; q < 4; ++q) {
        uint32_t p[4];
        for (int e = 0; e < 4; ++e) {
          const int c = c0 + 8 * q + 2 * e;
          p[e] = pack_bf16x2(silu(a[8 * q + 2 * e] + S.b1[c]), silu(a[8 * q + 2 * e + 1] + S.b1[c + 1]));
        }
        st_shared_v4(sh + tc::kmajor_off(t, c0 + 8 * q, kHid), p[0], p[1], p[2], p[3]);
        const uint16_t* e16 = reinterpret_cast<const uint16_t*>(p);
        for (int i = 0; i < 8; ++i) st_shared_u16(sht + tc::kmajor_off(c0 + 8 * q + i, t, kTile), e16[i]);
      }
    }
    sync_mma();
    if (t == 0) {
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc::mma_bf16(tmem + T_Z2, tc::make_sdesc(sh + kk * 256, 128, SB128),
                     tc::make_sdesc(sw2 + kk * 256, 128, SB128), id_128, kk > 0);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    // y, loss, g = dL/dy
    float y = b3;
    for (int c0 = 0; c0 < kHid; c0 += 32) {
      float a[32];
      tc::tmem_ld32(tmem + lane_base + T_Z2 + c0, a);
      for (int i = 0; i < 32; ++i) y = fmaf(S.w3[c0 + i], silu(a[i] + S.b2[c0 + i]), y);
    }
    const float res = valid ? y - target[r] : 0.f;
    const float g = 2.f * res * scale;
    atomicAdd(&S.loss, res * res * scale);
    atomicAdd(&S.gb3, g);
    // dZ2 = g w3 * silu'(Z2) -> sH [row][h2] and sDT [h2][row]; dw3 += g H2; db2 += dZ2
    for (int c0 = 0; c0 < kHid; c0 += 32) {
      float a[32];
      tc::tmem_ld32(tmem + lane_base + T_Z2 + c0, a);
      for (int q = 0; q < 4; ++q) {
        uint32_t p[4];
        for (int e = 0; e < 4; ++e) {
          float d2[2];
          for (int u = 0; u < 2; ++u) {
            const int i = 8 * q + 2 * e + u, c = c0 + i;
            const float z = a[i] + S.b2[c];
            d2[u] = g * S.w3[c] * silu_grad(z);
            if (valid) {
              atomicAdd(&S.gw3[c], g * silu(z));
              atomicAdd(&S.gb2[c], d2[u]);
            }
          }
          p[e] = pack_bf16x2(d2[0], d2[1]);
        }
        st_shared_v4(sh + tc::kmajor_off(t, c0 + 8 * q, kHid), p[0], p[1], p[2], p[3]);
        const uint16_t* e16 = reinterpret_cast<const uint16_t*>(p);
        for (int i = 0; i < 8; ++i) st_shared_u16(sdt + tc::kmajor_off(c0 + 8 * q + i, t, kTile), e16[i]);
      }
    }
    sync_mma();
    if (t == 0) {
      // dH1 = dZ2 W2  (into the Z2 columns, consumed)
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc::mma_bf16(tmem + T_Z2, tc::make_sdesc(sh + kk * 256, 128, SB128),
                     tc::make_sdesc(sw2t + kk * 256, 128, SB128), id_128, kk > 0);
      // dW2 += dZ2^T H1
      for (int kk = 0; kk < kTile / 16; ++kk)
        tc::mma_bf16(tmem + T_DW2, tc::make_sdesc(sdt + kk * 256, 128, SB128),
                     tc::make_sdesc(sht + kk * 256, 128, SB128), id_128, (!first || kk > 0) ? 1u : 0u);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    // dZ1 = dH1 * silu'(Z1) -> sDT [h1][row]; db1 += dZ1
    for (int c0 = 0; c0 < kHid; c0 += 32) {
      float a[32], z1[32];
      tc::tmem_ld32(tmem + lane_base + T_Z2 + c0, a);
      tc::tmem_ld32(tmem + lane_base + T_Z1 + c0, z1);
      for (int i = 0; i < 32; ++i) {
        const int c = c0 + i;
        const float d1 = a[i] * silu_grad(z1[i] + S.b1[c]);
        const __nv_bfloat16 b = __float2bfloat16_rn(d1);
        st_shared_u16(sdt + tc::kmajor_off(c, t, kTile), *reinterpret_cast<const uint16_t*>(&b));
        if (valid) atomicAdd(&S.gb1[c], d1);
      }
    }
    sync_mma();
    if (t == 0) {
      // dW1 += dZ1^T X
      for (int kk = 0; kk < kTile / 16; ++kk)
        tc::mma_bf16(tmem + T_DW1, tc::make_sdesc(sdt + kk * 256, 128, SB128),
                     tc::make_sdesc(sxt + kk * 256, 128, SB128), id_32, (!first || kk > 0) ? 1u : 0u);
      tc::mma_commit(&S.mbar);
    }
    if (!(ok = wait_mma())) break;
    first = false;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (!ok) drain_mma(&S.drain, t);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (ok && !first) {
    // weight gradients out of tensor memory: thread t owns row t of dW2 and dW1
    for (int c0 = 0; c0 < kHid; c0 += 32) {
      float a[32];
      tc::tmem_ld32(tmem + lane_base + T_DW2 + c0, a);
      for (int i = 0; i < 32; ++i) atomicAdd(&grad[kOffW2 + t * kHid + c0 + i], a[i]);
    }
    float a[32];
    tc::tmem_ld32(tmem + lane_base + T_DW1, a);
    for (int i = 0; i < kIn; ++i) atomicAdd(&grad[kOffW1 + t * kIn + i], a[i]);
    atomicAdd(&grad[kOffB1 + t], S.gb1[t]);
    atomicAdd(&grad[kOffB2 + t], S.gb2[t]);
    atomicAdd(&grad[kOffW3 + t], S.gw3[t]);
    if (t == 0) { atomicAdd(&grad[kOffB3], S.gb3); atomicAdd(loss, S.loss); }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Adam on the FP32 master parameters; refreshes the BF16 weight copies.
__global__ void mlp_adam_kernel(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float b1, float b2, float eps,
                                float c1, float c2, __nv_bfloat16* __restrict__ w1b,
                                __nv_bfloat16* __restrict__ w2b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNumParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi; v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  g[i] = 0.f;
  if (i < kOffB1) {
    const int o = i / kIn, k = i % kIn;
    w1b[o * kInPad + k] = __float2bfloat16_rn(pi);
  } else if (i >= kOffW2 && i < kOffB2) {
    w2b[i - kOffW2] = __float2bfloat16_rn(pi);
  }
}

__global__ void mlp_pack_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1b,
                                __nv_bfloat16* __restrict__ w2b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kHid * kInPad) {
    const int o = i / kInPad, k = i % kInPad;
    w1b[i] = __float2bfloat16_rn(k < kIn ? p[kOffW1 + o * kIn + k] : 0.f);
  }
  if (i < kHid * kHid) w2b[i] = __float2bfloat16_rn(p[kOffW2 + i]);
}

// ------------------------------------------------------------------ host
struct MlpHandle;
namespace snakesim {
SimStatus mlp_forward_launch(MlpHandle* h, const void* feat, long long rows, float* out, cudaStream_t st,
                             int sel);
}
struct MlpHandle {
  cudaStream_t stream = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *w1b = nullptr, *w2b = nullptr;
  float* loss = nullptr;
  int* err = nullptr;
  long long adam_t = 0;
  int sms = 0;
};

namespace {
SimStatus mfail(SimStatus s, const std::string& m) { set_last_error(m.c_str()); return s; }
#define MCU(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return mfail(e_ == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,          \
                   std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

MlpDev dev_of(MlpHandle* h) {
  MlpDev d;
  d.w1 = h->w1b; d.w2 = h->w2b; d.b1 = h->p + kOffB1; d.b2 = h->p + kOffB2; d.w3 = h->p + kOffW3;
  d.b3 = h->p + kOffB3;
  return d;
}

SimStatus check_err(MlpHandle* h) {
  int e = 0;
  MCU(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MCU(cudaStreamSynchronize(h->stream));
  if (e) return mfail(SIM_ECUDA, "tensor-core wait timed out");
  return SIM_OK;
}
}  // namespace

SimStatus snakesim::mlp_forward_launch(MlpHandle* h, const void* feat, long long rows, float* out,
                                       cudaStream_t st, int sel) {
  if (rows <= 0) return SIM_OK;
  const long long tiles = (rows + kTile - 1) / kTile;
  const int grid = (int)std::min<long long>(tiles, 2LL * h->sms);
  mlp_infer_kernel<<<grid, kInferThreads, sizeof(InferSmem), st>>>((const __nv_bfloat16*)feat, rows, dev_of(h),
                                                                  out, h->err, sel);
  MCU(cudaGetLastError());
  return SIM_OK;
}

extern "C" {

SimStatus mlp_create(void* stream, MlpHandle** out) {
  if (!out) return mfail(SIM_EINVAL, "null output");
  *out = nullptr;
  MlpHandle* h = new MlpHandle();
  h->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
  alloc((void**)&h->p, kNumParams * sizeof(float));
  alloc((void**)&h->g, kNumParams * sizeof(float));
  alloc((void**)&h->m, kNumParams * sizeof(float));
  alloc((void**)&h->v, kNumParams * sizeof(float));
  alloc((void**)&h->w1b, kHid * kInPad * sizeof(__nv_bfloat16));
  alloc((void**)&h->w2b, kHid * kHid * sizeof(__nv_bfloat16));
  alloc((void**)&h->loss, sizeof(float));
  alloc((void**)&h->err, sizeof(int));
  if (e != cudaSuccess) { mlp_destroy(h); return mfail(SIM_ENOMEM, cudaGetErrorString(e)); }
  cudaMemset(h->p, 0, kNumParams * sizeof(float));
  cudaMemset(h->g, 0, kNumParams * sizeof(float));
  cudaMemset(h->m, 0, kNumParams * sizeof(float));
  cudaMemset(h->v, 0, kNumParams * sizeof(float));
  cudaMemset(h->w1b, 0, kHid * kInPad * sizeof(__nv_bfloat16));
  cudaMemset(h->w2b, 0, kHid * kHid * sizeof(__nv_bfloat16));
  cudaMemset(h->err, 0, sizeof(int));
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(InferSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
  if (e != cudaSuccess) { mlp_destroy(h); return mfail(SIM_ECUDA, cudaGetErrorString(e)); }
  *out = h;
  return SIM_OK;
}

SimStatus mlp_set_params(MlpHandle* h, const float* params, int is_device) {
  if (!h || !params) return mfail(SIM_EINVAL, "null handle or params");
  MCU(cudaMemcpyAsync(h->p, params, kNumParams * sizeof(float),
                      is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  mlp_pack_kernel<<<(kHid * kHid + 255) / 256, 256, 0, h->stream>>>(h->p, h->w1b, h->w2b);
  MCU(cudaGetLastError());
  MCU(cudaMemsetAsync(h->m, 0, kNumParams * sizeof(float), h->stream));
  MCU(cudaMemsetAsync(h->v, 0, kNumParams * sizeof(float), h->stream));
  h->adam_t = 0;
  if (!is_device) MCU(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

SimStatus mlp_get_params(MlpHandle* h, float* params, int is_device) {
  if (!h || !params) return mfail(SIM_EINVAL, "null handle or params");
  MCU(cudaMemcpyAsync(params, h->p, kNumParams * sizeof(float),
                      is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!is_device) MCU(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

SimStatus mlp_forward(MlpHandle* h, const void* feat, int64_t rows, float* out) {
  if (!h || !feat || !out || rows < 0) return mfail(SIM_EINVAL, "bad arguments");
  if (((uintptr_t)feat & 15u) != 0) return mfail(SIM_EINVAL, "feat is not 16-byte aligned");
  SimStatus s = snakesim::mlp_forward_launch(h, feat, rows, out, h->stream, 0);
  if (s != SIM_OK) return s;
  return check_err(h);
}

SimStatus mlp_grad(MlpHandle* h, const void* feat, const float* target, int64_t rows, float scale,
                   float* grad, float* loss) {
  if (!h || !feat || !target || rows < 0) return mfail(SIM_EINVAL, "bad arguments");
  if (((uintptr_t)feat & 15u) != 0) return mfail(SIM_EINVAL, "feat is not 16-byte aligned");
  MCU(cudaMemsetAsync(h->g, 0, kNumParams * sizeof(float), h->stream));
  MCU(cudaMemsetAsync(h->loss, 0, sizeof(float), h->stream));
  if (rows > 0) {
    const long long tiles = (rows + kTile - 1) / kTile;
    const int grid = (int)std::min<long long>(tiles, h->sms);
    mlp_train_kernel<<<grid, 128, sizeof(TrainSmem), h->stream>>>((const __nv_bfloat16*)feat, target, rows,
                                                                   scale, dev_of(h), h->g, h->loss, h->err);
    MCU(cudaGetLastError());
  }
  if (grad) MCU(cudaMemcpyAsync(grad, h->g, kNumParams * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (loss) MCU(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return check_err(h);
}

SimStatus mlp_train_step(MlpHandle* h, const void* feat, const float* target, int64_t rows, float lr,
                         float* loss) {
  if (!h || !feat || !target || rows <= 0 || !(lr > 0.f)) return mfail(SIM_EINVAL, "bad arguments");
  if (((uintptr_t)feat & 15u) != 0) return mfail(SIM_EINVAL, "feat is not 16-byte aligned");
  MCU(cudaMemsetAsync(h->g, 0, kNumParams * sizeof(float), h->stream));
  MCU(cudaMemsetAsync(h->loss, 0, sizeof(float), h->stream));
  const long long tiles = (rows + kTile - 1) / kTile;
  const int grid = (int)std::min<long long>(tiles, h->sms);
  mlp_train_kernel<<<grid, 128, sizeof(TrainSmem), h->stream>>>((const __nv_bfloat16*)feat, target, rows,
                                                                 1.0f / (float)rows, dev_of(h), h->g, h->loss, h->err);
  MCU(cudaGetLastError());
  h->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)h->adam_t), c2 = 1.f - powf(b2, (float)h->adam_t);
  mlp_adam_kernel<<<(kNumParams + 255) / 256, 256, 0, h->stream>>>(h->p, h->g, h->m, h->v, lr, b1, b2, 1e-8f,
                                                                   c1, c2, h->w1b, h->w2b);
  MCU(cudaGetLastError());
  if (loss) MCU(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return SIM_OK;
}

SimStatus mlp_check(MlpHandle* h) {
  if (!h) return mfail(SIM_EINVAL, "null handle");
  return check_err(h);
}

SimStatus mlp_wait_selftest(uint32_t polls, void* stream, int32_t* timed_out) {
  if (polls < 1 || !timed_out) return mfail(SIM_EINVAL, "polls >= 1 and a result pointer");
  cudaStream_t st = (cudaStream_t)stream;
  int* flag = nullptr;
  MCU(cudaMalloc(&flag, sizeof(int)));
  int e = 0;
  cudaError_t c = cudaMemsetAsync(flag, 0, sizeof(int), st);
  if (c == cudaSuccess) {
    mlp_wait_selftest_kernel<<<1, 128, 0, st>>>(polls, flag);
    c = cudaGetLastError();
  }
  if (c == cudaSuccess) c = cudaMemcpyAsync(&e, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (c == cudaSuccess) c = cudaStreamSynchronize(st);
  cudaFree(flag);
  if (c != cudaSuccess) return mfail(SIM_ECUDA, std::string("mlp_wait_selftest: ") + cudaGetErrorString(c));
  *timed_out = e;
  return SIM_OK;
}

SimStatus mlp_destroy(MlpHandle* h) {
  if (!h) return SIM_OK;
  cudaStreamSynchronize(h->stream);
  void* ptrs[] = {h->p, h->g, h->m, h->v, h->w1b, h->w2b, h->loss, h->err};
  for (void* p : ptrs) if (p) cudaFree(p);
  delete h;
  return SIM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free forward
// Some callers cannot allocate device memory: a control loop with a hard real-time
// budget must not stall on the CUDA allocator, and a host application that gives this
// library a fixed device budget owned by its own allocator has no cudaMalloc to offer.
// For them, mlp_forward_noalloc runs the network from a parameter vector they own; the
// only working memory it needs -- the bfloat16 copies of W1 and W2 the tensor cores read,
// and the wait-timeout flag -- lives in the file-scope array below, which every GPU that
// loads the library holds until the process exits.
namespace {
constexpr size_t kNoallocW1 = (size_t)kHid * kInPad * 2;   // 8 KB
constexpr size_t kNoallocW2 = (size_t)kHid * kHid * 2;     // 32 KB
constexpr size_t kNoallocBytes = kNoallocW1 + kNoallocW2 + 256;  // + timeout flag
static_assert(kNoallocBytes == MLP_NOALLOC_SCRATCH_BYTES, "documented size");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {};  // device address of the array, per device
unsigned long long g_noalloc_ctx[kMaxDevices] = {};  // id of the context it belongs to
int g_noalloc_sms[kMaxDevices] = {};

// The id of the calling thread's current CUDA context (0 if none yet), from the driver's
// cuCtxGetCurrent / cuCtxGetId, reached through the runtime's driver entry points (no
// link-time dependency on the driver library).  The driver never reuses an id, so a
// primary context destroyed by cudaDeviceReset and created again has a new one.
SimStatus current_context_id(unsigned long long* id) {
  typedef CUresult (*GetCur)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCur get_cur = nullptr;
  static GetId get_id = nullptr;
  if (!get_cur || !get_id) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void *f1 = nullptr, *f2 = nullptr;
    cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return mfail(SIM_ECUDA, "cuCtxGetCurrent / cuCtxGetId entry points not available");
    get_cur = reinterpret_cast<GetCur>(f1);
    get_id = reinterpret_cast<GetId>(f2);
  }
  CUcontext c = nullptr;
  if (get_cur(&c) != CUDA_SUCCESS) return mfail(SIM_ECUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (c && get_id(c, id) != CUDA_SUCCESS) return mfail(SIM_ECUDA, "cuCtxGetId failed");
  return SIM_OK;
}

// Set-up, once per device and context, with that device current: the array's device
// address (the name g_noalloc_scratch in host code is only a host-side stand-in) and the
// kernel's shared-memory opt-in.  A later context on the device (after cudaDeviceReset)
// is set up again.
SimStatus noalloc_setup(int dev, unsigned char** addr, int* sms) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  unsigned long long ctx = 0;
  SimStatus s = current_context_id(&ctx);
  if (s != SIM_OK) return s;
  if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // creates the context if needed
    if (e != cudaSuccess) return mfail(SIM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(InferSmem));
    if (e != cudaSuccess) return mfail(SIM_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return mfail(SIM_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    if (ctx == 0 && (s = current_context_id(&ctx)) != SIM_OK) return s;
    g_noalloc_sms[dev] = n;
    g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    g_noalloc_ctx[dev] = ctx;
  }
  *addr = g_noalloc_addr[dev];
  *sms = g_noalloc_sms[dev];
  return SIM_OK;
}
}  // namespace

extern "C" SimStatus mlp_forward_noalloc(const float* params, int32_t n_params, const void* feat,
                                         int64_t rows, float* out, void* stream) {
  if (!params || !feat || !out || rows < 0) return mfail(SIM_EINVAL, "null pointer or rows < 0");
  if (((uintptr_t)feat & 15u) != 0) return mfail(SIM_EINVAL, "feat is not 16-byte aligned");
  if (n_params != kNumParams)
    return mfail(SIM_EINVAL, "mlp_forward_noalloc: its static working array holds the bfloat16 weights of "
                             "exactly one 24-128-128-1 network (" + std::to_string(kNumParams) +
                             " parameters, " + std::to_string(kNoallocBytes) + " bytes); got " +
                             std::to_string(n_params) + " parameters");
  int dev = 0;
  MCU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return mfail(SIM_EINVAL, "device index out of range");
  unsigned char* base = nullptr;
  int sms = 0;
  SimStatus s = noalloc_setup(dev, &base, &sms);
  if (s != SIM_OK) return s;
  if (rows == 0) return SIM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16* w1b = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* w2b = reinterpret_cast<__nv_bfloat16*>(base + kNoallocW1);
  int* err = reinterpret_cast<int*>(base + kNoallocW1 + kNoallocW2);
  // the array keeps the previous call's contents: the flag must start at zero
  MCU(cudaMemsetAsync(err, 0, sizeof(int), st));
  mlp_pack_kernel<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(params, w1b, w2b);
  MCU(cudaGetLastError());
  MlpDev d;
  d.w1 = w1b; d.w2 = w2b;
  d.b1 = params + kOffB1; d.b2 = params + kOffB2; d.w3 = params + kOffW3; d.b3 = params + kOffB3;
  const long long tiles = (rows + kTile - 1) / kTile;
  const int grid = (int)std::min<long long>(tiles, 2LL * sms);
  mlp_infer_kernel<<<grid, kInferThreads, sizeof(InferSmem), st>>>((const __nv_bfloat16*)feat, rows, d, out, err, 0);
  MCU(cudaGetLastError());
  int e = 0;
  MCU(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  MCU(cudaStreamSynchronize(st));
  if (e) return mfail(SIM_ECUDA, "tensor-core wait timed out");
  return SIM_OK;
}
