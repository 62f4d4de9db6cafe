// mlp_kernels.cu -- tensor-core kernels of the warm-start network (BF16
// operands, FP32 accumulation in TMEM) and its elementwise pieces.
//
//   dense_kernel   out[t][p] = epi( sum_q A[t][q] * Bt[p][q] )   (M = 128 rows
//                  per tile, N = P <= 256, K = Q in steps of 16): the forward
//                  of a layer (A = activations, Bt = weights [out][in]) and
//                  the gradient of its input (A = dZ, Bt = weights^T); loads,
//                  MMA issue and epilogue run on separate warps, pipelined
//   wgrad_kernel   partial[cta][p][q] = sum_t Dz[t][p] * H[t][q] over the
//                  CTA's row tiles (the gradient of a weight matrix), then
//   wgrad_reduce   dW = sum over CTAs in a fixed order
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "../../include/hcran_mlp.h"
#include "mlp_tc.cuh"

namespace hcran {

enum DenseEpi {
  kEpiBiasRelu = 0,  // relu(acc + b) -> BF16
  kEpiBiasF32 = 1,   // acc + b -> FP32
  kEpiReluMask = 2,  // acc * (H > 0) -> BF16 (gradient through a ReLU)
  kEpiF32 = 3,       // acc -> FP32
};

constexpr int kTcThreads = 128;  // one warpgroup: its 4 warps cover the 128 TMEM lanes
constexpr int kTile = 128;       // rows per tile (MMA M)

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// The dense layer is a pipeline over the CTA's 128-row tiles, one role per
// warp group (256 threads):
//   warps 5-7  stream each tile of A in K-chunks of Kc columns (cp.async, 16
//              bytes a thread, rows past T zero-filled) into a ring of
//              kStages shared-memory slots in the core-matrix layout
//   warp 4     (one thread) issues the tcgen05 MMAs of a chunk once its slot
//              is full, commits the slot back to the producers, and commits
//              the tile's accumulator to the epilogue
//   warps 0-3  (one TMEM lane quadrant each) drain the accumulator through
//              the epilogue into global memory
// Two TMEM accumulators alternate between tiles, so a tile's epilogue runs
// under the next tile's MMAs and loads; the weight matrix stays resident.
// Every wait is bounded: a timeout sets the abort flag and *err, every role
// leaves its loop, and the MMAs and copies in flight are drained before the
// TMEM is freed.
constexpr int kPipeThreads = 256;
constexpr int kStages = 4;         // A-chunk ring slots
constexpr int kProdThreads = 96;   // warps 5-7
constexpr int kLag = 2;            // chunks a producer keeps in flight

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(tc::saddr(bar)) : "memory");
}
// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool pipe_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  for (int i = 0; i < tc::kSpin; i++) {
    if (tc::mbar_try(bar, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  return false;
}

// epilogue of one tile: accumulator columns [0, P) of this thread's TMEM lane
__device__ __forceinline__ void dense_epilogue(uint32_t tacc, int warp, int lane, int64_t row0, int64_t T, int P,
                                               int epi, const float *bias, const __nv_bfloat16 *H, void *out) {
  const int64_t row = row0 + 32 * warp + lane;
  for (int c0 = 0; c0 < P; c0 += 16) {
    float v[16];
    tc::tmem_ld16(tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    if (row >= T) continue;
    if (epi == kEpiBiasRelu || epi == kEpiBiasF32) {
#pragma unroll
      for (int i = 0; i < 16; i++) v[i] += bias ? bias[c0 + i] : 0.f;
    }
    if (epi == kEpiBiasRelu) {
#pragma unroll
      for (int i = 0; i < 16; i++) v[i] = fmaxf(v[i], 0.f);
    } else if (epi == kEpiReluMask) {
      const uint4 *hp = reinterpret_cast<const uint4 *>(H + row * P + c0);
      const uint4 h0 = hp[0], h1 = hp[1];
      const __nv_bfloat16 *hb0 = reinterpret_cast<const __nv_bfloat16 *>(&h0);
      const __nv_bfloat16 *hb1 = reinterpret_cast<const __nv_bfloat16 *>(&h1);
#pragma unroll
      for (int i = 0; i < 8; i++) {
        if (!(__bfloat162float(hb0[i]) > 0.f)) v[i] = 0.f;
        if (!(__bfloat162float(hb1[i]) > 0.f)) v[8 + i] = 0.f;
      }
    }
    if (epi == kEpiBiasF32 || epi == kEpiF32) {
      float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(out) + row * P + c0);
#pragma unroll
      for (int i = 0; i < 4; i++) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
      uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out) + row * P + c0);
      o[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
      o[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                        pack_bf16(v[14], v[15]));
    }
  }
}

// K-chunk width: the largest of 64, 32, 16 that divides Q
__host__ __device__ __forceinline__ int dense_kc(int Q) { return (Q % 64 == 0) ? 64 : ((Q % 32 == 0) ? 32 : 16); }
// TMEM columns of one accumulator (a power of two >= 32)
__host__ __device__ __forceinline__ uint32_t dense_cols(int P) {
  return P <= 32 ? 32u : (P <= 64 ? 64u : (P <= 128 ? 128u : 256u));
}

__global__ void __launch_bounds__(kPipeThreads, 1)
    dense_kernel(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ Bt,
                 const float *__restrict__ bias, const __nv_bfloat16 *__restrict__ H, int64_t T, int Q, int P,
                 int epi, void *__restrict__ out, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[kStages], empty[kStages], accf[2], acce[2], done;
  __shared__ uint32_t tslot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Kc = dense_kc(Q), nchunk = Q / Kc;
  const uint32_t chunk_bytes = (uint32_t)(kTile * Kc * 2);
  unsigned char *sB = smem;                               // [P][Q] core layout, resident
  unsigned char *ring = smem + (size_t)P * Q * 2;         // kStages x [128][Kc] core layout
  const uint32_t ncols = dense_cols(P);
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * ncols);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; i++) {
      tc::mbar_init(&full[i], kProdThreads);
      tc::mbar_init(&empty[i], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 4);
    }
    tc::mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < P * (Q >> 3); i += kPipeThreads) {  // weights into the core layout
    const int r = i / (Q >> 3), j = i - r * (Q >> 3);
    *reinterpret_cast<uint4 *>(sB + tc::core_off(r, 8 * j, Q)) = *reinterpret_cast<const uint4 *>(Bt + (int64_t)r * Q + 8 * j);
  }
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = tslot;
  const int64_t ntiles = (T + kTile - 1) / kTile;
  const int mine = ntiles > blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

  if (warp >= 5) {  // producers
    const int pt = threadIdx.x - 160;
    const int per_row = Kc >> 3;
    int g = 0;
    for (int i = 0; i < mine && !abort_flag; i++) {
      const int64_t row0 = (blockIdx.x + (int64_t)i * gridDim.x) * kTile;
      for (int c = 0; c < nchunk; c++, g++) {
        const int s = g % kStages, u = g / kStages;
        if (u >= 1 && !pipe_wait(&empty[s], (uint32_t)((u - 1) & 1), &abort_flag)) {
          abort_flag = 1;
          break;
        }
        const uint32_t dst0 = tc::saddr(ring + (size_t)s * chunk_bytes);
        for (int q = pt; q < kTile * per_row; q += kProdThreads) {
          const int r = q / per_row, j = q - r * per_row;
          const bool in = row0 + r < T;
          const __nv_bfloat16 *src = A + (in ? (row0 + r) * Q : 0) + c * Kc + 8 * j;
          cp_async16(dst0 + tc::core_off(r, 8 * j, Kc), src, in ? 16u : 0u);
        }
        cp_async_commit();
        if (g >= kLag) {  // chunk g - kLag has landed: publish it to the tensor core
          cp_async_wait<kLag>();
          tc::fence_async_smem();
          mbar_arrive(&full[(g - kLag) % kStages]);
        }
      }
    }
    cp_async_wait<0>();
    tc::fence_async_smem();
    if (!abort_flag)
      for (int k = g - kLag > 0 ? g - kLag : 0; k < g; k++) mbar_arrive(&full[k % kStages]);
  } else if (warp == 4) {  // MMA issue
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16(kTile, P);
      const uint32_t sbo_a = (uint32_t)(Kc >> 3) << 7, sbo_b = (uint32_t)(Q >> 3) << 7;
      int g = 0;
      for (int i = 0; i < mine && !abort_flag; i++) {
        const int b = i & 1;
        if (i >= 2 && !pipe_wait(&acce[b], (uint32_t)(((i >> 1) - 1) & 1), &abort_flag)) {
          abort_flag = 1;
          break;
        }
        tc::tc_fence_after();
        const uint32_t tacc = taddr + (uint32_t)b * ncols;
        for (int c = 0; c < nchunk; c++, g++) {
          const int s = g % kStages, u = g / kStages;
          if (!pipe_wait(&full[s], (uint32_t)(u & 1), &abort_flag)) {
            abort_flag = 1;
            break;
          }
          tc::tc_fence_after();
          const uint32_t a0 = tc::saddr(ring + (size_t)s * chunk_bytes), b0 = tc::saddr(sB);
          for (int k = 0; k < (Kc >> 4); k++) {
            const uint64_t ad = tc::sdesc(a0 + 256u * k, 128u, sbo_a);
            const uint64_t bd = tc::sdesc(b0 + 256u * (c * (Kc >> 4) + k), 128u, sbo_b);
            tc::mma_bf16(tacc, ad, bd, idesc, (c | k) ? 1u : 0u);
          }
          tc::mma_commit(&empty[s]);  // the slot is free once these MMAs complete
        }
        if (abort_flag) break;
        tc::mma_commit(&accf[b]);
      }
      tc::mma_commit(&done);  // every MMA issued has completed when this arrives
      if (!tc::mbar_wait(&done, 0u)) abort_flag = 1;
    }
    __syncwarp();
  } else {  // epilogue (every exit warp-uniform: tcgen05.ld is warp-collective)
    for (int i = 0; i < mine; i++) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      const int b = i & 1;
      const int64_t row0 = (blockIdx.x + (int64_t)i * gridDim.x) * kTile;
      const bool ok = pipe_wait(&accf[b], (uint32_t)((i >> 1) & 1), &abort_flag);
      if (__any_sync(0xffffffffu, !ok)) {  // warp-uniform exit
        abort_flag = 1;
        break;
      }
      tc::tc_fence_after();
      dense_epilogue(taddr + (uint32_t)b * ncols, warp, lane, row0, T, P, epi, bias, H, out);
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  __syncthreads();
  if (abort_flag && threadIdx.x == 0) atomicExch(err, 1);
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(taddr, 2 * ncols);
}

}  // namespace hcran

// ------------------------------------------------------------------ host side

namespace hcran {
__device__ int g_tc_error;  // set when a bounded tensor-core wait gave up

static int sm_count() {
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms;
}
constexpr int kOneCtaSmem = 120 * 1024;
static bool tc_dim_ok(int x) { return x >= 16 && x <= 256 && (x % 16) == 0; }
static bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

cudaError_t launch_dense(const void *A, const void *Bt, const float *bias, const void *H, int64_t T, int Q, int P,
                         int epi, void *out, cudaStream_t st) {
  int *err = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_tc_error);
  if (e != cudaSuccess) return e;
  // at least 120 KB: one CTA per SM, so the TMEM allocation (up to all 512
  // columns) never waits on another CTA
  const int need = P * Q * 2 + kStages * kTile * dense_kc(Q) * 2;
  const int smem = need > kOneCtaSmem ? need : kOneCtaSmem;
  e = cudaFuncSetAttribute(dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (T + kTile - 1) / kTile;
  const int grid = (int)(ntiles < sm_count() ? ntiles : sm_count());
  dense_kernel<<<grid, kPipeThreads, smem, st>>>(static_cast<const __nv_bfloat16 *>(A),
                                                static_cast<const __nv_bfloat16 *>(Bt), bias,
                                                static_cast<const __nv_bfloat16 *>(H), T, Q, P, epi, out, err);
  return cudaGetLastError();
}
}  // namespace hcran

extern "C" int hcran_mlp_dense(const void *A, const void *Bt, const float *bias, const void *H, int64_t T,
                               int32_t Q, int32_t P, int32_t epi, void *out, void *stream) {
  using namespace hcran;
  if (!A || !Bt || !out || T < 1 || !hcran::tc_dim_ok(Q) || !hcran::tc_dim_ok(P) || epi < 0 || epi > 3)
    return HCRAN_MLP_EINVAL;
  if (!hcran::al16(A) || !hcran::al16(Bt) || !hcran::al16(out) || (epi == kEpiReluMask && (!H || !hcran::al16(H))))
    return HCRAN_MLP_EINVAL;
  return launch_dense(A, Bt, bias, H, T, Q, P, epi, out, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? HCRAN_MLP_OK
             : HCRAN_MLP_ECUDA;
}

extern "C" int hcran_mlp_tc_status(int32_t *failed) {
  if (!failed) return HCRAN_MLP_EINVAL;
  int v = 0, zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(&v, hcran::g_tc_error, sizeof(int)) != cudaSuccess ||
      cudaMemcpyToSymbol(hcran::g_tc_error, &zero, sizeof(int)) != cudaSuccess)
    return HCRAN_MLP_ECUDA;
  *failed = v;
  return HCRAN_MLP_OK;
}

// ------------------------------------------------------------------ weight gradients

namespace hcran {

// transposed fill: rows t0.. of X [T][R] (BF16, row-major) become the K = t
// columns of the core layout of Xt [R][128] at smem base (t >= T: zero)
__device__ __forceinline__ void fill_core_t(unsigned char *base, const __nv_bfloat16 *X, int64_t t0, int64_t T,
                                            int R) {
  const int per_t = R >> 3;  // 16-byte chunks of one row of X
  for (int i = threadIdx.x; i < kTile * per_t; i += kTcThreads) {
    const int t = i / per_t, j = i - t * per_t;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (t0 + t < T) v = *reinterpret_cast<const uint4 *>(X + (t0 + t) * R + 8 * j);
    const uint16_t *h = reinterpret_cast<const uint16_t *>(&v);
#pragma unroll
    for (int e = 0; e < 8; e++)
      *reinterpret_cast<uint16_t *>(base + tc::core_off(8 * j + e, t, kTile)) = h[e];
  }
}

// partial[cta][r][s] = sum over the CTA's row tiles of X[t][r] * Y[t][s]
// (R = 256: two M = 128 halves; S in [16, 256]); every CTA writes its slice
__global__ void __launch_bounds__(kTcThreads, 1)
    wgrad_kernel(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ Y, int64_t T, int S,
                 float *__restrict__ partial, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  constexpr int R = 256;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *sX = smem;               // Xt [256][128] core layout (64 KB)
  unsigned char *sY = smem + R * kTile * 2;  // Yt [S][128] core layout
  const uint32_t ncols = S <= 16 ? 32u : (S <= 64 ? 128u : (S <= 128 ? 256u : 512u));  // two halves of S columns
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = tslot;
  const uint32_t idesc = tc::idesc_bf16(kTile, S);
  const uint32_t sbo = (uint32_t)(kTile >> 3) << 7;  // 128 K-columns per row block
  const int64_t ntiles = (T + kTile - 1) / kTile;
  uint32_t phase = 0;
  bool failed = false, any = false;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    fill_core_t(sX, X, tile * kTile, T, R);
    fill_core_t(sY, Y, tile * kTile, T, S);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::tc_fence_after();
      for (int h = 0; h < 2; h++)
        for (int s = 0; s < (kTile >> 4); s++) {
          // rows 128h.. of Xt start at row block 16h
          const uint64_t ad = tc::sdesc(tc::saddr(sX) + (uint32_t)(16 * h) * sbo + 256u * s, 128u, sbo);
          const uint64_t bd = tc::sdesc(tc::saddr(sY) + 256u * s, 128u, sbo);
          tc::mma_bf16(taddr + (uint32_t)(h * S), ad, bd, idesc, (any || s > 0) ? 1u : 0u);
        }
      tc::mma_commit(&bar);
    }
    any = true;
    const bool ok = tc::mbar_wait(&bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
  }
  tc::tc_fence_after();
  float *dst = partial + (size_t)blockIdx.x * R * S;
  if (!failed) {
    for (int h = 0; h < 2; h++) {
      const int r = 128 * h + 32 * warp + lane;
      for (int c0 = 0; c0 < S; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(h * S + c0), v);
#pragma unroll
        for (int i = 0; i < 16; i++) dst[(size_t)r * S + c0 + i] = any ? v[i] : 0.f;
      }
    }
  } else {
    if (threadIdx.x == 0) atomicExch(err, 1);
    tc::mbar_wait(&bar, phase ^ 1u);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

// dW[r][s] (transposed: dW[s][r]) = sum over the nparts slices, in slice order
__global__ void wgrad_reduce(const float *__restrict__ partial, int nparts, int S, int transpose, float *__restrict__ dW) {
  const int R = 256;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R * S; i += gridDim.x * blockDim.x) {
    float t = 0.f;
    for (int q = 0; q < nparts; q++) t += partial[(size_t)q * R * S + i];
    const int r = i / S, s = i - r * S;
    dW[transpose ? (size_t)s * R + r : (size_t)i] = t;
  }
}

// db[p] = sum over rows of Dz[t][p] (BF16), per-block partial sums then a
// fixed-order reduction
__global__ void bias_grad_partial(const __nv_bfloat16 *__restrict__ Dz, int64_t T, int P, float *__restrict__ part) {
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float t = 0.f;
    for (int64_t r = blockIdx.x; r < T; r += gridDim.x) t += __bfloat162float(Dz[r * P + p]);
    part[(size_t)blockIdx.x * P + p] = t;
  }
}
__global__ void bias_grad_reduce(const float *__restrict__ part, int nparts, int P, float *__restrict__ db) {
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float t = 0.f;
    for (int q = 0; q < nparts; q++) t += part[(size_t)q * P + p];
    db[p] = t;
  }
}

}  // namespace hcran

// ------------------------------------------------------------------ elementwise

namespace hcran {

// W16[p][q] = bf16(W32[p][q]), W16t[q][p] = the same value
__global__ void to_bf16_pair(const float *__restrict__ W, int P, int Q, __nv_bfloat16 *__restrict__ W16,
                             __nv_bfloat16 *__restrict__ W16t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P * Q; i += gridDim.x * blockDim.x) {
    const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
    const int p = i / Q, q = i - p * Q;
    W16[i] = v;
    W16t[(size_t)q * P + p] = v;
  }
}

// Adam (bias-corrected), FP32 master values
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// masked squared error over the first nout outputs: dOut (BF16 [T][16]) =
// 2 mask (out - target) / norm, per-block loss partial sums
__global__ void mse_grad_kernel(const float *__restrict__ out, const float *__restrict__ tgt,
                                const float *__restrict__ mask, int64_t T, int nout, float inv_norm,
                                __nv_bfloat16 *__restrict__ dout, float *__restrict__ part) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T * 16; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & 15);
    float d = 0.f;
    if (j < nout) {
      const float w = mask[i];
      const float e = out[i] - tgt[i];
      d = 2.f * w * e * inv_norm;
      acc += w * e * e * inv_norm;
    }
    dout[i] = __float2bfloat16_rn(d);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void sum_kernel(const float *__restrict__ part, int n, float *__restrict__ total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < n; i++) t += part[i];
    *total = t;
  }
}

}  // namespace hcran

// ------------------------------------------------------------------ the network object

namespace hcran {

cudaError_t launch_wgrad(const void *X, const void *Y, int64_t T, int S, float *partial, int grid, int *err,
                         cudaStream_t st) {
  const int need = 256 * kTile * 2 + S * kTile * 2;
  const int smem = need > kOneCtaSmem ? need : kOneCtaSmem;
  cudaError_t e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  wgrad_kernel<<<grid, kTcThreads, smem, st>>>(static_cast<const __nv_bfloat16 *>(X),
                                              static_cast<const __nv_bfloat16 *>(Y), T, S, partial, err);
  return cudaGetLastError();
}

}  // namespace hcran

using namespace hcran;

struct hcran_mlp_s {
  static constexpr int L = 4;
  int dims[L + 1] = {HCRAN_MLP_IN, HCRAN_MLP_HIDDEN, HCRAN_MLP_HIDDEN, HCRAN_MLP_HIDDEN, HCRAN_MLP_OUT};
  int64_t tmax = 0;
  int grid = 1;
  int64_t step = 0;
  float *W[L] = {}, *b[L] = {}, *gW[L] = {}, *gb[L] = {}, *mW[L] = {}, *vW[L] = {}, *mb[L] = {}, *vb[L] = {};
  __nv_bfloat16 *W16[L] = {}, *W16t[L] = {};
  __nv_bfloat16 *H[3] = {}, *dZ[2] = {}, *dOut = nullptr;
  float *partial = nullptr, *bpart = nullptr, *lpart = nullptr;
  std::vector<void *> owned;
  int P(int i) const { return dims[i + 1]; }
  int Q(int i) const { return dims[i]; }
  template <typename T>
  bool alloc(T **p, size_t n) {
    void *q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) return false;
    owned.push_back(q);
    *p = static_cast<T *>(q);
    return cudaMemset(q, 0, n * sizeof(T)) == cudaSuccess;
  }
  ~hcran_mlp_s() {
    for (void *q : owned) cudaFree(q);
  }
};

static int mlp_err_ptr(int **err) {
  return cudaGetSymbolAddress(reinterpret_cast<void **>(err), g_tc_error) == cudaSuccess ? 0 : 1;
}

// FP32 master weights -> BF16 copies (and transposes) of every layer
static cudaError_t mlp_sync_bf16(hcran_mlp_t h, cudaStream_t st) {
  for (int i = 0; i < hcran_mlp_s::L; i++) {
    to_bf16_pair<<<64, 256, 0, st>>>(h->W[i], h->P(i), h->Q(i), h->W16[i], h->W16t[i]);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// splitmix64 stream -> standard normal pairs (Box-Muller), host side
static double mlp_normal(uint64_t &s) {
  auto next = [&]() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  const double u1 = ((next() >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

extern "C" int hcran_mlp_create(hcran_mlp_t *out, uint64_t seed, int64_t max_rows) {
  if (!out || max_rows < 1 || max_rows > (int64_t(1) << 28)) return HCRAN_MLP_EINVAL;
  *out = nullptr;
  hcran_mlp_s *h = new (std::nothrow) hcran_mlp_s();
  if (!h) return HCRAN_MLP_ENOMEM;
  h->tmax = max_rows;
  h->grid = sm_count();
  bool ok = true;
  for (int i = 0; i < hcran_mlp_s::L && ok; i++) {
    const size_t n = (size_t)h->P(i) * h->Q(i), p = (size_t)h->P(i);
    ok = h->alloc(&h->W[i], n) && h->alloc(&h->b[i], p) && h->alloc(&h->gW[i], n) && h->alloc(&h->gb[i], p) &&
         h->alloc(&h->mW[i], n) && h->alloc(&h->vW[i], n) && h->alloc(&h->mb[i], p) && h->alloc(&h->vb[i], p) &&
         h->alloc(&h->W16[i], n) && h->alloc(&h->W16t[i], n);
  }
  for (int i = 0; i < 3 && ok; i++) ok = h->alloc(&h->H[i], (size_t)max_rows * HCRAN_MLP_HIDDEN);
  for (int i = 0; i < 2 && ok; i++) ok = h->alloc(&h->dZ[i], (size_t)max_rows * HCRAN_MLP_HIDDEN);
  ok = ok && h->alloc(&h->dOut, (size_t)max_rows * HCRAN_MLP_OUT) &&
       h->alloc(&h->partial, (size_t)h->grid * 256 * 256) && h->alloc(&h->bpart, (size_t)h->grid * 256) &&
       h->alloc(&h->lpart, (size_t)h->grid);
  if (!ok) {
    delete h;
    return HCRAN_MLP_ENOMEM;
  }
  // He initialisation: the first layer sees 4 nonzero features, the output
  // layer starts small
  uint64_t s = seed;
  for (int i = 0; i < hcran_mlp_s::L; i++) {
    const int P = h->P(i), Q = h->Q(i);
    const double fan = i == 0 ? (double)HCRAN_MLP_FEATURES : (double)Q;
    const double sd = i == hcran_mlp_s::L - 1 ? 0.1 * sqrt(1.0 / fan) : sqrt(2.0 / fan);
    std::vector<float> w((size_t)P * Q);
    for (size_t k = 0; k < w.size(); k++) w[k] = (float)(sd * mlp_normal(s));
    if (cudaMemcpy(h->W[i], w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      delete h;
      return HCRAN_MLP_ECUDA;
    }
  }
  if (mlp_sync_bf16(h, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    delete h;
    return HCRAN_MLP_ECUDA;
  }
  *out = h;
  return HCRAN_MLP_OK;
}

extern "C" void hcran_mlp_destroy(hcran_mlp_t h) { delete h; }

extern "C" int hcran_mlp_param_count(hcran_mlp_t h, int64_t *n) {
  if (!h || !n) return HCRAN_MLP_EINVAL;
  int64_t t = 0;
  for (int i = 0; i < hcran_mlp_s::L; i++) t += (int64_t)h->P(i) * h->Q(i) + h->P(i);
  *n = t;
  return HCRAN_MLP_OK;
}

// packed FP32 [W1 b1 W2 b2 W3 b3 W4 b4] between host and device (which = 0:
// parameters, 1: gradients of the last backward)
static int mlp_copy(hcran_mlp_t h, float *host, const float *src_host, int which) {
  size_t o = 0;
  for (int i = 0; i < hcran_mlp_s::L; i++) {
    const size_t n = (size_t)h->P(i) * h->Q(i), p = (size_t)h->P(i);
    float *w = which ? h->gW[i] : h->W[i], *bb = which ? h->gb[i] : h->b[i];
    cudaError_t e;
    if (src_host) {
      e = cudaMemcpy(w, src_host + o, n * sizeof(float), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(bb, src_host + o + n, p * sizeof(float), cudaMemcpyHostToDevice);
    } else {
      e = cudaMemcpy(host + o, w, n * sizeof(float), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemcpy(host + o + n, bb, p * sizeof(float), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return HCRAN_MLP_ECUDA;
    o += n + p;
  }
  return HCRAN_MLP_OK;
}
extern "C" int hcran_mlp_get_params(hcran_mlp_t h, float *host) {
  if (!h || !host) return HCRAN_MLP_EINVAL;
  return cudaDeviceSynchronize() == cudaSuccess ? mlp_copy(h, host, nullptr, 0) : HCRAN_MLP_ECUDA;
}
extern "C" int hcran_mlp_set_params(hcran_mlp_t h, const float *host) {
  if (!h || !host) return HCRAN_MLP_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return HCRAN_MLP_ECUDA;
  const int rc = mlp_copy(h, nullptr, host, 0);
  if (rc != HCRAN_MLP_OK) return rc;
  return mlp_sync_bf16(h, nullptr) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess ? HCRAN_MLP_OK
                                                                                            : HCRAN_MLP_ECUDA;
}
extern "C" int hcran_mlp_get_grads(hcran_mlp_t h, float *host) {
  if (!h || !host) return HCRAN_MLP_EINVAL;
  return cudaDeviceSynchronize() == cudaSuccess ? mlp_copy(h, host, nullptr, 1) : HCRAN_MLP_ECUDA;
}

// forward of rows [r0, r0 + T) of x: hidden activations into h->H (kept for
// the backward), outputs (FP32) into out
static cudaError_t mlp_forward_rows(hcran_mlp_t h, const __nv_bfloat16 *x, int64_t T, float *out, cudaStream_t st) {
  cudaError_t e = launch_dense(x, h->W16[0], h->b[0], nullptr, T, h->Q(0), h->P(0), kEpiBiasRelu, h->H[0], st);
  if (e == cudaSuccess)
    e = launch_dense(h->H[0], h->W16[1], h->b[1], nullptr, T, h->Q(1), h->P(1), kEpiBiasRelu, h->H[1], st);
  if (e == cudaSuccess)
    e = launch_dense(h->H[1], h->W16[2], h->b[2], nullptr, T, h->Q(2), h->P(2), kEpiBiasRelu, h->H[2], st);
  if (e == cudaSuccess)
    e = launch_dense(h->H[2], h->W16[3], h->b[3], nullptr, T, h->Q(3), h->P(3), kEpiBiasF32, out, st);
  return e;
}

extern "C" int hcran_mlp_forward(hcran_mlp_t h, const void *x, int64_t T, float *out, void *stream) {
  if (!h || !x || !out || T < 1 || !al16(x) || !al16(out)) return HCRAN_MLP_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const __nv_bfloat16 *xb = static_cast<const __nv_bfloat16 *>(x);
  for (int64_t r0 = 0; r0 < T; r0 += h->tmax) {  // chunks of at most tmax rows
    const int64_t n = T - r0 < h->tmax ? T - r0 : h->tmax;
    if (mlp_forward_rows(h, xb + r0 * HCRAN_MLP_IN, n, out + r0 * HCRAN_MLP_OUT, st) != cudaSuccess)
      return HCRAN_MLP_ECUDA;
  }
  return HCRAN_MLP_OK;
}

extern "C" int hcran_mlp_loss_grad(hcran_mlp_t h, const float *out, const float *target, const float *mask,
                                   int64_t T, int32_t nout, float *loss, void *stream) {
  if (!h || !out || !target || !mask || !loss || T < 1 || T > h->tmax || nout < 1 || nout > HCRAN_MLP_OUT)
    return HCRAN_MLP_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = h->grid;
  mse_grad_kernel<<<nb, 256, 0, st>>>(out, target, mask, T, nout, 1.f / (float)T, h->dOut, h->lpart);
  sum_kernel<<<1, 32, 0, st>>>(h->lpart, nb, loss);
  return cudaGetLastError() == cudaSuccess ? HCRAN_MLP_OK : HCRAN_MLP_ECUDA;
}

// gradient of the bias of a layer (column sums of its dZ)
static cudaError_t mlp_bias_grad(hcran_mlp_t h, const __nv_bfloat16 *dz, int64_t T, int P, float *gb,
                                 cudaStream_t st) {
  const int nb = (int)(T < h->grid ? T : h->grid);
  bias_grad_partial<<<nb, 256, 0, st>>>(dz, T, P, h->bpart);
  bias_grad_reduce<<<1, 256, 0, st>>>(h->bpart, nb, P, gb);
  return cudaGetLastError();
}

// weight gradient sum_t X[t][r] Y[t][s] (R = 256) into dW, transposed when
// the 256-wide side is the layer's input
static cudaError_t mlp_weight_grad(hcran_mlp_t h, const __nv_bfloat16 *X, const __nv_bfloat16 *Y, int64_t T, int S,
                                   int transpose, float *dW, int *err, cudaStream_t st) {
  const int64_t ntiles = (T + kTile - 1) / kTile;
  const int grid = (int)(ntiles < h->grid ? ntiles : h->grid);
  cudaError_t e = launch_wgrad(X, Y, T, S, h->partial, grid, err, st);
  if (e != cudaSuccess) return e;
  wgrad_reduce<<<64, 256, 0, st>>>(h->partial, grid, S, transpose, dW);
  return cudaGetLastError();
}

extern "C" int hcran_mlp_backward(hcran_mlp_t h, const void *x, int64_t T, void *stream) {
  if (!h || !x || T < 1 || T > h->tmax || !al16(x)) return HCRAN_MLP_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *err = nullptr;
  if (mlp_err_ptr(&err)) return HCRAN_MLP_ECUDA;
  const __nv_bfloat16 *xb = static_cast<const __nv_bfloat16 *>(x);
  cudaError_t e = cudaSuccess;
  // output layer: dZ4 = dOut; dW4 = dOut^T H3 (formed as H3^T dOut, transposed)
  e = mlp_weight_grad(h, h->H[2], h->dOut, T, h->P(3), 1, h->gW[3], err, st);
  if (e == cudaSuccess) e = mlp_bias_grad(h, h->dOut, T, h->P(3), h->gb[3], st);
  if (e == cudaSuccess)
    e = launch_dense(h->dOut, h->W16t[3], nullptr, h->H[2], T, h->P(3), h->Q(3), kEpiReluMask, h->dZ[0], st);
  // hidden layers 3, 2: dW = dZ^T H_prev; dZ_prev = (dZ W) * (H_prev > 0)
  int cur = 0;
  for (int i = 2; i >= 1 && e == cudaSuccess; i--) {
    e = mlp_weight_grad(h, h->dZ[cur], h->H[i - 1], T, h->Q(i), 0, h->gW[i], err, st);
    if (e == cudaSuccess) e = mlp_bias_grad(h, h->dZ[cur], T, h->P(i), h->gb[i], st);
    if (e == cudaSuccess)
      e = launch_dense(h->dZ[cur], h->W16t[i], nullptr, h->H[i - 1], T, h->P(i), h->Q(i), kEpiReluMask,
                       h->dZ[cur ^ 1], st);
    cur ^= 1;
  }
  // input layer: dW1 = dZ1^T x
  if (e == cudaSuccess) e = mlp_weight_grad(h, h->dZ[cur], xb, T, h->Q(0), 0, h->gW[0], err, st);
  if (e == cudaSuccess) e = mlp_bias_grad(h, h->dZ[cur], T, h->P(0), h->gb[0], st);
  return e == cudaSuccess ? HCRAN_MLP_OK : HCRAN_MLP_ECUDA;
}

extern "C" int hcran_mlp_adam(hcran_mlp_t h, float lr, float beta1, float beta2, float eps, void *stream) {
  if (!h || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return HCRAN_MLP_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->step++;
  const float c1 = 1.f - powf(beta1, (float)h->step), c2 = 1.f - powf(beta2, (float)h->step);
  for (int i = 0; i < hcran_mlp_s::L; i++) {
    adam_kernel<<<64, 256, 0, st>>>(h->W[i], h->gW[i], h->mW[i], h->vW[i], h->P(i) * h->Q(i), lr, beta1, beta2,
                                    eps, c1, c2);
    adam_kernel<<<1, 256, 0, st>>>(h->b[i], h->gb[i], h->mb[i], h->vb[i], h->P(i), lr, beta1, beta2, eps, c1, c2);
  }
  return mlp_sync_bf16(h, st) == cudaSuccess ? HCRAN_MLP_OK : HCRAN_MLP_ECUDA;
}
