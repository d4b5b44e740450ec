// Forward pass of the learned-guess MLP (8 -> 256 -> 256 -> 1, ReLU) for inference, fused in one
// persistent kernel with the 256 x 256 layer on the 5th-generation tensor cores (tcgen05,
// kind::f16 with bfloat16 operands and FP32 accumulators in tensor memory).  Same rounding points
// as the training path (learned.cu): h1 = relu(x W1 + b1) in FP32, rounded to bfloat16; W2 rounded
// to bfloat16; FP32 accumulation; h2 = relu(acc + b2) and the output layer in FP32.
//
// Per CTA (one per SM): W2 is staged once as the B operand (N = 256 output neurons x K = 256,
// K-major, 128 KB), W1, b1, b2, W3 in shared memory.  Per tile of 128 rows: the 8 warps form h1
// straight into the A operand (128 x 256 bfloat16, 64 KB; each warp fills whole 8 x 16-byte core
// matrices, so the stores are conflict-free), one thread issues the 16 MMAs (M = 128, N = 256,
// K = 16 each) into 256 tensor-memory columns and commits to an mbarrier, and after the
// (bounded) wait every thread reads the accumulators of its row (warp w: lanes 32 (w % 4) ..,
// columns half w / 4) and reduces relu(acc + b2) . W3 in registers; the two halves are added
// in a fixed order.  No atomics: the result is reproducible run to run.
#include <algorithm>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "tcgen05.cuh"

namespace fp {
namespace {

constexpr int NIN = 8, NH = 256, TILE = 128, THREADS = 256;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t LBO_A = TILE * 16, LBO_B = NH * 16;        // K-direction core-matrix strides
constexpr uint32_t IDESC = tc::idesc_f32acc(1u, 128u, 256u);  // kind::f16, BF16 x BF16 -> FP32

// byte offset of element (r, k) (bfloat16) in a K-major operand whose K-direction core-matrix
// stride is lbo: core matrices of 8 rows x 8 elements
__device__ __forceinline__ uint32_t off_bf16(int r, int k, uint32_t lbo) {
  return (uint32_t)(k >> 3) * lbo + (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2;
}

}  // namespace

// Shared memory (dynamic): [control 1 KB] [B: W2^T bf16, 128 KB] [A: h1 bf16, 64 KB]
// [W1 8 x 256, b1, b2, W3 FP32] [x tile 128 x 8 FP32] [two partial-sum rows].
__global__ void __launch_bounds__(THREADS, 1) k_mlp_forward_tc(long long M, const float *X, const float *P,
                                                               float *out, int *status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 64);
  int *s_abort = reinterpret_cast<int *>(sm + 128);
  unsigned char *Bop = sm + 1024;
  unsigned char *Aop = Bop + NH * NH * 2;
  float *w1 = reinterpret_cast<float *>(Aop + TILE * NH * 2);
  float *b1 = w1 + NIN * NH, *b2 = b1 + NH, *w3 = b2 + NH;
  float *xt = w3 + NH;               // TILE x NIN
  float *part = xt + TILE * NIN;     // 2 x TILE
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init1(bar);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tslot, TMEM_COLS);
  // constants: W1, b1, b2, W3 in FP32; W2 as B[j][k] = bf16(W2[k][j]) (thread: 2 adjacent k)
  for (int e = tid; e < NIN * NH; e += THREADS) w1[e] = P[OFF_W1 + e];
  for (int e = tid; e < NH; e += THREADS) {
    b1[e] = P[OFF_B1 + e];
    b2[e] = P[OFF_B2 + e];
    w3[e] = P[OFF_W3 + e];
  }
  for (int idx = tid; idx < NH * NH / 2; idx += THREADS) {
    const int cm = idx >> 5, within = idx & 31;  // core matrix (32 k-groups x 32 row groups)
    const int j = (cm & 31) * 8 + (within >> 2), k = (cm >> 5) * 8 + 2 * (within & 3);
    const __nv_bfloat162 v = __floats2bfloat162_rn(P[OFF_W2 + k * NH + j], P[OFF_W2 + (k + 1) * NH + j]);
    *reinterpret_cast<__nv_bfloat162 *>(Bop + off_bf16(j, k, LBO_B)) = v;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const float b3 = P[OFF_B3];
  uint32_t phase = 0;
  bool pending = false;
  const long long ntile = (M + TILE - 1) / TILE;
  for (long long t = blockIdx.x; t < ntile && !*s_abort; t += gridDim.x) {
    const long long row0 = t * TILE;
    for (int e = tid; e < TILE * NIN; e += THREADS) {
      const long long r = row0 + e / NIN;
      xt[e] = r < M ? X[row0 * NIN + e] : 0.0f;
    }
    __syncthreads();
    // A operand: h1 = relu(b1 + sum_k x_k W1[k][j]) rounded to bfloat16 (the order of k_mlp_l1)
    for (int idx = tid; idx < TILE * NH / 2; idx += THREADS) {
      const int cm = idx >> 5, within = idx & 31;  // 32 k-groups x 16 row groups
      const int r = (cm & 15) * 8 + (within >> 2), j = (cm >> 4) * 8 + 2 * (within & 3);
      float v0 = b1[j], v1 = b1[j + 1];
#pragma unroll
      for (int k = 0; k < NIN; ++k) {
        const float xk = xt[r * NIN + k];
        v0 += xk * w1[k * NH + j];
        v1 += xk * w1[k * NH + j + 1];
      }
      *reinterpret_cast<__nv_bfloat162 *>(Aop + off_bf16(r, j, LBO_A)) =
          __floats2bfloat162_rn(fmaxf(v0, 0.0f), fmaxf(v1, 0.0f));
    }
    tc::proxy_fence();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int ks = 0; ks < NH / 16; ++ks) {
        const uint64_t ad = tc::smem_desc(tc::s_addr(Aop) + 2 * ks * LBO_A, LBO_A, 128);
        const uint64_t bd = tc::smem_desc(tc::s_addr(Bop) + 2 * ks * LBO_B, LBO_B, 128);
        tc::mma_f16(tmem, ad, bd, IDESC, ks > 0 ? 1u : 0u);
      }
      tc::mma_commit(bar);
    }
    pending = true;
    const bool ok = tc::mbar_wait_bounded(bar, phase);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) { set_status(status, DS_TIMEOUT); *s_abort = 1; }
      __syncthreads();
      break;
    }
    pending = false;
    phase ^= 1;
    tc::fence_after();
    // epilogue: row 32 (w % 4) + lane, columns [128 (w / 4), + 128)
    const int q = warp & 3, half = warp >> 2, r = 32 * q + lane;
    float acc = 0.0f;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float v[32];
      const int j0 = 128 * half + 32 * c;
      tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + j0, v);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) acc += fmaxf(v[jj] + b2[j0 + jj], 0.0f) * w3[j0 + jj];
    }
    part[half * TILE + r] = acc;
    tc::fence_before();
    __syncthreads();
    if (tid < TILE && row0 + tid < M) out[row0 + tid] = (part[tid] + part[TILE + tid]) + b3;
  }
  if (pending) {
    const bool ok = tc::mbar_wait_bounded(bar, phase);
    if (!ok && tid == 0) set_status(status, DS_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_free(tmem, TMEM_COLS);
}

size_t mlp_forward_tc_smem() {
  return 1024 + (size_t)NH * NH * 2 + (size_t)TILE * NH * 2 + sizeof(float) * ((size_t)NIN * NH + 3 * NH) +
         sizeof(float) * (TILE * NIN + 2 * TILE);
}

cudaError_t launch_mlp_forward_tc(long long rows, const float *X, const float *P, float *out, int num_sms,
                                  int *status, cudaStream_t st) {
  if (rows < 1) return cudaSuccess;
  const size_t smem = mlp_forward_tc_smem();
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ntile = (rows + TILE - 1) / TILE;
  const int grid = (int)std::min<long long>(num_sms, ntile);
  k_mlp_forward_tc<<<grid, THREADS, smem, st>>>(rows, X, P, out, status);
  return cudaGetLastError();
}

}  // namespace fp
