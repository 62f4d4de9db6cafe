// mlp_kernels.cu -- tensor-core kernels of the warm-start network (BF16
// operands, FP32 accumulation in TMEM) and its elementwise pieces.
//
//   dense_kernel   out[t][p] = epi( sum_q A[t][q] * Bt[p][q] )   (M = 128 rows
//                  per tile, N = P <= 256, K = Q in steps of 16): the forward
//                  of a layer (A = activations, Bt = weights [out][in]) and
//                  the gradient of its input (A = dZ, Bt = weights^T)
//   wgrad_kernel   partial[cta][p][q] = sum_t Dz[t][p] * H[t][q] over the
//                  CTA's row tiles (the gradient of a weight matrix), then
//   wgrad_reduce   dW = sum over CTAs in a fixed order
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

// 16-byte rows chunks of a [rows][Kt] BF16 matrix (global, row stride ld
// elements) into the core-matrix layout at smem base; rows >= nrows are zero
__device__ __forceinline__ void fill_core(unsigned char *base, const __nv_bfloat16 *g, int64_t row0, int64_t nrows,
                                          int rows, int Kt, int64_t ld) {
  const int per_row = Kt >> 3;
  for (int i = threadIdx.x; i < rows * per_row; i += kTcThreads) {
    const int r = i / per_row, j = i - r * per_row;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (row0 + r < nrows) v = *reinterpret_cast<const uint4 *>(g + (row0 + r) * ld + 8 * j);
    *reinterpret_cast<uint4 *>(base + tc::core_off(r, 8 * j, Kt)) = v;
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    dense_kernel(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ Bt,
                 const float *__restrict__ bias, const __nv_bfloat16 *__restrict__ H, int64_t T, int Q, int P,
                 int epi, void *__restrict__ out, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *sA = smem;                      // [128][Q] core layout
  unsigned char *sB = smem + kTile * Q * 2;      // [P][Q] core layout
  const uint32_t ncols = P <= 32 ? 32u : (P <= 64 ? 64u : (P <= 128 ? 128u : 256u));
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fill_core(sB, Bt, 0, P, P, Q, Q);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = tslot;
  const uint32_t idesc = tc::idesc_bf16(kTile, P);
  const uint32_t sbo = (uint32_t)(Q >> 3) << 7;
  const int64_t ntiles = (T + kTile - 1) / kTile;
  uint32_t phase = 0;
  bool failed = false;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTile;
    fill_core(sA, A, row0, T, kTile, Q, Q);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::tc_fence_after();
      for (int s = 0; s < (Q >> 4); s++) {
        const uint64_t ad = tc::sdesc(tc::saddr(sA) + 256u * s, 128u, sbo);
        const uint64_t bd = tc::sdesc(tc::saddr(sB) + 256u * s, 128u, sbo);
        tc::mma_bf16(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
      }
      tc::mma_commit(&bar);
    }
    const bool ok = tc::mbar_wait(&bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {  // block-uniform: every thread leaves together
      failed = true;
      break;
    }
    tc::tc_fence_after();
    const int r = 32 * warp + lane;
    const int64_t row = row0 + r;
    for (int c0 = 0; c0 < P; c0 += 16) {
      float v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
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
    tc::tc_fence_before();
    __syncthreads();  // TMEM and the A tile are free for the next tile
  }
  if (failed) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    tc::mbar_wait(&bar, phase ^ 1u);  // let an MMA still in flight finish (bounded)
    __syncthreads();
  }
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
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
  // at least 120 KB: one CTA per SM, so a TMEM allocation never waits on another CTA
  const int need = kTile * Q * 2 + P * Q * 2;
  const int smem = need > kOneCtaSmem ? need : kOneCtaSmem;
  e = cudaFuncSetAttribute(dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (T + kTile - 1) / kTile;
  const int grid = (int)(ntiles < sm_count() ? ntiles : sm_count());
  dense_kernel<<<grid, kTcThreads, smem, st>>>(static_cast<const __nv_bfloat16 *>(A),
                                              static_cast<const __nv_bfloat16 *>(Bt), bias,
                                              static_cast<const __nv_bfloat16 *>(H), T, Q, P, epi, out, err);
  return cudaGetLastError();
}
}  // namespace hcran

#include "../../include/hcran_mlp.h"

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
