// Banded LDL^T factorisation in FP32 with the trailing updates on the 5th-generation tensor
// cores (tcgen05): the local Neumann / Dirichlet factorisations of Sec. 3.2 (K_s = L D L^T,
// no pivoting: K_s is symmetric quasi-definite in the 3-field form), same cyclic column band
// layout and same result convention as k_band_factor (slot j mod LD of column j holds 1/d_j,
// the other slots the unit-lower factor).
//
// Right-looking, panels of 32 columns.  A panel is factorised in shared memory on the CUDA
// cores (32 dependent column steps).  The trailing update of the next m <= b rows and columns,
//     A[T0 + i][T0 + j] -= sum_c L[T0 + i][J + c] d_c L[T0 + j][J + c],   j <= i < m,
// is a dense (m x 32) x (32 x m) product: it runs as tcgen05.mma kind::tf32 tiles of 128 x 128
// (K = 8 per instruction) with FP32 accumulators in tensor memory.  TF32 keeps 10 mantissa
// bits, so each operand is split x = hi + lo (hi = x rounded to TF32, lo = x - hi) and the
// product is hi*hi + hi*lo + lo*hi (the "3xTF32" error-compensated split; the lo*lo term is
// below FP32 rounding), which brings the update to about FP32 accuracy.
//
// Tiles: the lower-triangular 128 x 128 blocks (mt >= nt) of the m x m update.  Pass nt stages
// the B operand (rows of column block nt, d_c L, hi/lo) and issues the tiles mt = nt .. MT - 1
// into tensor-memory columns 128 (mt - nt); one commit to an mbarrier, a bounded wait, then the
// 8 warps read the accumulators (tcgen05.ld, warp w reads lanes 32 (w % 4) .., columns half
// w / 4) and subtract them from the band in global memory (coalesced: consecutive rows are
// consecutive slots of a column).  The A operand (all m rows, hi/lo) is staged once per panel.
//
// Shared-memory operand layout: K-major, no swizzle, "core matrices" of 8 rows x 16 bytes;
// element (row r, k) at byte (k / 4) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % 4) * 4 with
// LBO = rows * 16.  Every wait is bounded (~1 s of SM clock); on timeout the kernel sets
// DS_TIMEOUT, waits once more (bounded) for its own MMAs, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"
#include "tcgen05.cuh"

namespace fp {
namespace {

constexpr int TC_NB = 32;          // panel width = K of the trailing update
constexpr int TC_THREADS = 256;    // 8 warps
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t IDESC_TF32_128x128 = tc::idesc_f32acc(2u, 128u, 128u);  // kind::tf32, M = N = 128

using tc::fence_after;
using tc::fence_before;
using tc::mbar_init1;
using tc::mbar_wait_bounded;
using tc::proxy_fence;
using tc::s_addr;
using tc::smem_desc;
using tc::tmem_ld32;
using tc::to_tf32;
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t accum) {
  tc::mma_tf32(d, a, b, IDESC_TF32_128x128, accum);
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) { tc::mma_commit(bar); }
__device__ __forceinline__ void tc_fence_before() { fence_before(); }
__device__ __forceinline__ void tc_fence_after() { fence_after(); }

}  // namespace

// Shared memory (dynamic): [control 1024 B: mbarrier, tensor-memory address] [B hi, B lo: 128 x 32
// each] [A hi, A lo: MP x 32 each] [panel: 32 x (LD + 8)] [d: 32].  MP = 128 ceil(b / 128).
__global__ void __launch_bounds__(TC_THREADS, 1) k_band_factor_tc(const BandTask *tasks, int ntask, float *base,
                                                                  int MP, int *counter, int *status) {
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_tc);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_tc + 64);
  int *s_task = reinterpret_cast<int *>(smem_tc + 128);
  int *s_abort = reinterpret_cast<int *>(smem_tc + 132);
  unsigned char *Bh = smem_tc + 1024;
  unsigned char *Bl = Bh + 128 * TC_NB * 4;
  unsigned char *Ah = Bl + 128 * TC_NB * 4;
  unsigned char *Al = Ah + (size_t)MP * TC_NB * 4;
  float *pan = reinterpret_cast<float *>(Al + (size_t)MP * TC_NB * 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    mbar_init1(bar);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  bool pending = false;  // MMAs issued whose completion was not observed
  for (;;) {
    if (tid == 0) *s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int task = *s_task;
    if (task >= ntask || *s_abort) break;
    const BandTask tk = tasks[task];
    float *A = base + tk.fac_off;
    const int n = tk.n, LD = tk.LD, b = tk.b;
    // panel rows are stored at stride PS = LD + 8 (PS = 8 mod 32): the operand staging below
    // reads 4 columns x 8 consecutive slots per warp from 32 different banks
    const int PS = LD + 8;
    float *dpan = pan + TC_NB * PS;
    for (int J = 0; J < n && !*s_abort; J += TC_NB) {
      const int nbw = min(TC_NB, n - J);
      // J and LD are multiples of 32: slot (J + c) mod LD = jl + c for c < 32, and a row r of the
      // panel's window (J <= r < J + 32 + b) sits in slot jl + (r - J), minus LD once past it
      const int jl = J % LD;
      auto slot = [&](int r) { const int v = jl + (r - J); return v >= LD ? v - LD : v; };
      for (int c = warp; c < nbw; c += TC_THREADS / 32)
        for (int sl = lane; sl < LD; sl += 32) pan[c * PS + sl] = A[(long long)(J + c) * LD + sl];
      __syncthreads();
      // ---- panel factorisation (CUDA cores) ----
      for (int c = 0; c < nbw; ++c) {
        const int j = J + c;
        float *colc = pan + c * PS;
        const float d = colc[jl + c];
        const float dinv = 1.0f / d;
        if (tid == 0) {
          dpan[c] = d;
          if (!(d != 0.0f) || !isfinite(d)) set_status(status, DS_ZERO_PIVOT);
        }
        const int rmax = min(n - 1, j + b);
        // rows of the panel below the pivot: row r updates the panel columns c2 > c whose
        // diagonal lies at or above it (J + c2 <= r)
        for (int r = j + 1 + tid; r <= rmax; r += TC_THREADS) {
          const int sr = slot(r);
          const float lrj = colc[sr] * dinv;
          const int c2max = min(nbw - 1, r - J);
          float *pr = pan + (c + 1) * PS + sr;
          const float *pc = colc + jl + c + 1;
          for (int c2 = c + 1; c2 <= c2max; ++c2, pr += PS, ++pc) *pr -= lrj * *pc;
        }
        __syncthreads();
        for (int r = j + 1 + tid; r <= rmax; r += TC_THREADS) colc[slot(r)] *= dinv;
        if (tid == 0) colc[jl + c] = dinv;
        __syncthreads();
      }
      for (int c = warp; c < nbw; c += TC_THREADS / 32)
        for (int sl = lane; sl < LD; sl += 32) A[(long long)(J + c) * LD + sl] = pan[c * PS + sl];
      // ---- trailing update of rows / columns [T0, T0 + m) on the tensor cores ----
      const int T0 = J + nbw, m = min(n, J + nbw + b) - T0;
      if (m > 0) {
        const int MT = (m + 127) >> 7, RG = 16 * MT;  // 8-row groups of the A operand
        // A operand: L[T0 + r][J + k] (hi, lo) for r < 128 MT, zero outside the band / panel.
        // Thread idx writes element (within & 3, within >> 2) of core matrix cm = idx >> 5: a warp
        // fills one 128-byte core matrix (conflict-free)
        for (int idx = tid; idx < 128 * MT * TC_NB; idx += TC_THREADS) {
          const int cm = idx >> 5, within = idx & 31;
          const int r = (cm % RG) * 8 + (within >> 2), k = (cm / RG) * 4 + (within & 3);
          const int row = T0 + r, col = J + k;
          float x = 0.0f;
          if (r < m && k < nbw && row - col <= b) x = pan[k * PS + slot(row)];
          const uint32_t h = to_tf32(x);
          const float lo = x - __uint_as_float(h);
          const uint32_t off = (uint32_t)cm * 128 + within * 4;  // the offset of (r, k) in the layout above
          *reinterpret_cast<uint32_t *>(Ah + off) = h;
          *reinterpret_cast<uint32_t *>(Al + off) = to_tf32(lo);
        }
        for (int nt = 0; nt < MT && !*s_abort; ++nt) {
          // B operand: d_k L[T0 + 128 nt + r][J + k] (hi, lo), the same conflict-free order
          for (int idx = tid; idx < 128 * TC_NB; idx += TC_THREADS) {
            const int cm = idx >> 5, within = idx & 31;
            const int r = (cm % 16) * 8 + (within >> 2), k = (cm / 16) * 4 + (within & 3);
            const int rr = 128 * nt + r, row = T0 + rr, col = J + k;
            float x = 0.0f;
            if (rr < m && k < nbw && row - col <= b) x = dpan[k] * pan[k * PS + slot(row)];
            const uint32_t h = to_tf32(x);
            const float lo = x - __uint_as_float(h);
            const uint32_t off = (uint32_t)cm * 128 + within * 4;  // the offset of (r, k) in the layout above
            *reinterpret_cast<uint32_t *>(Bh + off) = h;
            *reinterpret_cast<uint32_t *>(Bl + off) = to_tf32(lo);
          }
          proxy_fence();
          tc_fence_before();
          __syncthreads();
          if (tid == 0) {
            tc_fence_after();
            const uint32_t lboA = 128 * MT * 16, lboB = 128 * 16;
            for (int mt = nt; mt < MT; ++mt) {
              const uint32_t d = tmem + 128 * (mt - nt);
#pragma unroll
              for (int ks = 0; ks < TC_NB / 8; ++ks) {
                const uint32_t ka = 2 * ks * lboA + mt * 16 * 128, kb = 2 * ks * lboB;
                const uint64_t ah = smem_desc(s_addr(Ah) + ka, lboA, 128);
                const uint64_t al = smem_desc(s_addr(Al) + ka, lboA, 128);
                const uint64_t bh = smem_desc(s_addr(Bh) + kb, lboB, 128);
                const uint64_t bl = smem_desc(s_addr(Bl) + kb, lboB, 128);
                mma_tf32(d, ah, bh, ks > 0 ? 1u : 0u);
                mma_tf32(d, ah, bl, 1u);
                mma_tf32(d, al, bh, 1u);
              }
            }
            mma_commit(bar);
          }
          pending = true;
          const bool ok = mbar_wait_bounded(bar, phase);
          if (!__syncthreads_and(ok)) {
            if (tid == 0) { set_status(status, DS_TIMEOUT); *s_abort = 1; }
            __syncthreads();
            break;
          }
          pending = false;
          phase ^= 1;
          tc_fence_after();
          // epilogue: subtract the accumulators from the band (lower triangle only)
          const int q = warp & 3, half = warp >> 2;
          for (int mt = nt; mt < MT; ++mt) {
            const int i = 128 * mt + 32 * q + lane;
#pragma unroll 1
            for (int ch = 0; ch < 2; ++ch) {
              float v[32];
              const int j0 = 128 * nt + 64 * half + 32 * ch;
              tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 128 * (mt - nt) + 64 * half + 32 * ch, v);
              if (i < m) {
                // all loads first, then all stores: the 32 read-modify-writes are independent
                float *Ai = A + (T0 + i) % LD;
                float a[32];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                  a[jj] = (j0 + jj <= i) ? Ai[(long long)(T0 + j0 + jj) * LD] : 0.0f;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                  if (j0 + jj <= i) Ai[(long long)(T0 + j0 + jj) * LD] = a[jj] - v[jj];
              }
            }
          }
          tc_fence_before();
          __syncthreads();
        }
      }
      __syncthreads();
    }
  }
  // ---- teardown: observe outstanding MMAs (bounded), free tensor memory ----
  if (pending) {
    const bool ok = mbar_wait_bounded(bar, phase);
    if (!ok && tid == 0) set_status(status, DS_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Shared memory of the kernel for the widest band: the layout above plus, where it fits, a
// zero-filled margin so that every operand descriptor's reach stays inside the allocation.
size_t band_factor_tc_smem(int ldmax, int bmax) {
  const int MP = 128 * ((bmax + 127) / 128);
  const size_t need = 1024 + 2 * 128 * TC_NB * 4 + 2 * (size_t)MP * TC_NB * 4 + (size_t)TC_NB * (ldmax + 8) * 4 +
                      TC_NB * 4;
  const size_t cap = 227 * 1024;
  return need > cap ? need : std::min(cap, need + 64 * 1024);
}

// One persistent CTA per SM (the shared memory admits only one; each holds all 512 tensor-
// memory columns) over a work queue of the tasks.
cudaError_t launch_band_factor_tc(const BandTask *tasks, int ntask, float *base, int ldmax, int bmax, int num_sms,
                                  int *counter, int *status, cudaStream_t stream) {
  const size_t smem = band_factor_tc_smem(ldmax, bmax);
  if (smem > 227 * 1024 || bmax > 511) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_band_factor_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const int MP = 128 * ((bmax + 127) / 128);
  k_band_factor_tc<<<std::min(num_sms, ntask), TC_THREADS, smem, stream>>>(tasks, ntask, base, MP, counter, status);
  return cudaGetLastError();
}

}  // namespace fp
