// Batched banded LDL^T factorisation and solves for the local systems K_s (Sec. 3.2:
// K_A needs K_s^{-1} applied to interface data, no nested iteration) and for the coarse
// matrix G^T G.
//
// Storage ("cyclic column layout"): a band matrix of order n and half bandwidth b is stored
// as n columns of LD >= b + 1 slots (LD a multiple of 32).  Column j keeps entry (r, j),
// j <= r <= j + b, in slot r mod LD; the other slots are zero.  After factorisation slot
// j mod LD holds 1/d_j and the other slots the unit-lower factor L.  With this layout a
// warp solving one system keeps the moving window of pending rows in registers indexed by
// slot, so the window never moves between lanes: lane l owns slots l, l+32, ...
//
// Factorisation: right-looking, panels of NB columns staged in shared memory, trailing
// update of the (b x b) triangle in 4x4 register tiles.  One CTA per matrix.
// Solve: one warp per system (dynamic work queue, tasks pre-sorted by cost), forward
// sweep (axpy form), diagonal, backward sweep (dot form with warp reductions).  Factor
// columns are streamed through a per-warp ring of shared-memory stages filled by TMA bulk
// copies (cp.async.bulk + mbarrier), with bounded waits that report DS_TIMEOUT.
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace fp {

// ============================ factorisation ============================================
template <typename T>
__global__ void __launch_bounds__(256) k_band_factor(const BandTask *tasks, int ntask, T *base, int NB,
                                                     int *status) {
  const int task = blockIdx.x;
  if (task >= ntask) return;
  const BandTask tk = tasks[task];
  T *A = base + tk.fac_off;
  const int n = tk.n, LD = tk.LD, b = tk.b;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *pan = reinterpret_cast<T *>(smem_raw);
  T *dpan = pan + (size_t)NB * LD;
  for (int J = 0; J < n; J += NB) {
    const int nbw = min(NB, n - J);
    for (int e = threadIdx.x; e < nbw * LD; e += blockDim.x) pan[e] = A[(long long)J * LD + e];
    __syncthreads();
    for (int c = 0; c < nbw; ++c) {
      const int j = J + c;
      const T d = pan[c * LD + j % LD];
      const T dinv = T(1) / d;
      if (threadIdx.x == 0) {
        dpan[c] = d;
        if (!(d != T(0)) || !isfinite((double)d)) set_status(status, DS_ZERO_PIVOT);
      }
      const int rmax = min(n - 1, j + b);
      const int ncols = nbw - c - 1;
      const int span = b + 1;
      for (int idx = threadIdx.x; idx < ncols * span; idx += blockDim.x) {
        const int c2 = c + 1 + idx / span;
        const int r = J + c2 + idx % span;
        if (r > rmax) continue;
        const T lrj = pan[c * LD + r % LD] * dinv;
        const T a_c2j = pan[c * LD + (J + c2) % LD];
        pan[c2 * LD + r % LD] -= lrj * a_c2j;
      }
      __syncthreads();
      for (int r = j + 1 + threadIdx.x; r <= rmax; r += blockDim.x) pan[c * LD + r % LD] *= dinv;
      if (threadIdx.x == 0) pan[c * LD + j % LD] = dinv;
      __syncthreads();
    }
    for (int e = threadIdx.x; e < nbw * LD; e += blockDim.x) A[(long long)J * LD + e] = pan[e];
    // trailing update of rows/columns [T0, T1)
    const int T0 = J + nbw, T1 = min(n, J + nbw + b);
    const int m = T1 - T0;
    if (m > 0) {
      const int nt = (m + 3) / 4;
      const int npairs = nt * (nt + 1) / 2;
      for (int pidx = threadIdx.x; pidx < npairs; pidx += blockDim.x) {
        int ti = (int)((sqrtf(8.0f * pidx + 1.0f) - 1.0f) * 0.5f);  // FP32 estimate, corrected exactly
        while (ti * (ti + 1) / 2 > pidx) --ti;
        while ((ti + 1) * (ti + 2) / 2 <= pidx) ++ti;
        const int tj = pidx - ti * (ti + 1) / 2;
        const int i0 = T0 + 4 * ti, j0 = T0 + 4 * tj;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[a][q] = T(0);
        for (int c = 0; c < nbw; ++c) {
          const int jc = J + c;
          const T dc = dpan[c];
          T li[4], lj[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = i0 + q;
            li[q] = (r < T1 && r - jc <= b) ? pan[c * LD + r % LD] : T(0);
            const int r2 = j0 + q;
            lj[q] = (r2 < T1 && r2 - jc <= b) ? pan[c * LD + r2 % LD] * dc : T(0);
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[a][q] += li[a] * lj[q];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = i0 + a, jj = j0 + q;
            if (i < T1 && jj < T1 && i >= jj) A[(long long)jj * LD + i % LD] -= acc[a][q];
          }
      }
    }
    __syncthreads();
  }
}

template __global__ void k_band_factor<double>(const BandTask *, int, double *, int, int *);
template __global__ void k_band_factor<float>(const BandTask *, int, float *, int, int *);

// ============================ TMA ring helpers ==========================================
namespace {
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2^31 SM cycles (about a second).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1LL << 31)) return false;
  }
  return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
}  // namespace

// Opaque select: keeps a register-array pick such as "xw[M - 1]" from being folded into a
// dynamically indexed (local-memory) access.
__device__ __forceinline__ float opaque_sel(bool p, float a, float b) {
  float r;
  asm("{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n selp.f32 %0, %1, %2, q;\n}\n"
      : "=f"(r) : "f"(a), "f"(b), "r"((unsigned)p));
  return r;
}
__device__ __forceinline__ double opaque_sel(bool p, double a, double b) {
  double r;
  asm("{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n selp.f64 %0, %1, %2, q;\n}\n"
      : "=d"(r) : "d"(a), "d"(b), "r"((unsigned)p));
  return r;
}

constexpr int SOLVE_STAGES = 3;
constexpr int CHUNK_BYTES = 16384;

// Per-warp ring of SOLVE_STAGES stages.  Requests are numbered per warp (seq); request q
// lives in stage q % S and completes phase (q / S) & 1 of that stage's mbarrier.
struct Ring {
  unsigned char *buf;
  uint64_t *bar;
  uint32_t seq0;  // global number of the current task's request 0
};

template <typename T>
struct TaskStream {
  const T *fac;
  int n, LD, C, nc;
  __device__ __forceinline__ int chunk_of_req(int r) const { return r < nc ? r : 2 * nc - 1 - r; }
  __device__ __forceinline__ void issue(const Ring &rg, int r) const {
    const int c = chunk_of_req(r);
    const int c0 = c * C;
    const int cols = min(C, n - c0);
    const uint32_t bytes = (uint32_t)cols * LD * sizeof(T);
    const uint32_t q = rg.seq0 + r;
    const int st = q % SOLVE_STAGES;
    mbar_expect_tx(&rg.bar[st], bytes);
    bulk_g2s(rg.buf + (size_t)st * CHUNK_BYTES, fac + (long long)c0 * LD, bytes, &rg.bar[st]);
  }
};

template <typename T, int MMAX>
__global__ void __launch_bounds__(128) k_band_solve(const BandTask *tasks, int ntask, const T *fbase,
                                                    double *xbase, int *counter, int *status,
                                                    const int *done) {
  if (done && *done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  extern __shared__ __align__(128) unsigned char smem[];
  Ring rg;
  rg.buf = smem + (size_t)warp * SOLVE_STAGES * CHUNK_BYTES;
  rg.bar = reinterpret_cast<uint64_t *>(smem + (size_t)nwarps * SOLVE_STAGES * CHUNK_BYTES) + warp * SOLVE_STAGES;
  if (lane == 0)
    for (int st = 0; st < SOLVE_STAGES; ++st) mbar_init(&rg.bar[st], 1);
  fence_mbar_init();
  __syncwarp();
  rg.seq0 = 0;
  bool abort = false;
  uint32_t inflight_lo = 0, inflight_hi = 0;  // requests [lo, hi) issued and not consumed
  while (!abort) {
    int task = 0;
    if (lane == 0) task = atomicAdd(counter, 1);
    task = __shfl_sync(FULL, task, 0);
    if (task >= ntask) break;
    const BandTask tk = tasks[task];
    TaskStream<T> ts;
    ts.fac = fbase + tk.fac_off;
    ts.n = tk.n;
    ts.LD = tk.LD;
    ts.C = max(1, CHUNK_BYTES / (int)(tk.LD * sizeof(T)));
    ts.nc = (ts.n + ts.C - 1) / ts.C;
    double *x = xbase + tk.x_off;
    const int n = ts.n, LD = ts.LD, M = LD / 32, C = ts.C;
    const int R = 2 * ts.nc;
    if (lane == 0)
      for (int r = 0; r < min(SOLVE_STAGES, R); ++r) ts.issue(rg, r);
    inflight_lo = rg.seq0;
    inflight_hi = rg.seq0 + min(SOLVE_STAGES, R);
    // wait for request r: returns false on timeout (uniform over the warp)
    auto wait_req = [&](int r) -> bool {
      const uint32_t q = rg.seq0 + r;
      const bool ok = mbar_wait(&rg.bar[q % SOLVE_STAGES], (q / SOLVE_STAGES) & 1);
      return __all_sync(FULL, ok);
    };
    auto release_req = [&](int r) {
      __syncwarp();
      inflight_lo = rg.seq0 + r + 1;
      if (r + SOLVE_STAGES < R) {
        if (lane == 0) {
          fence_proxy_async();
          ts.issue(rg, r + SOLVE_STAGES);
        }
        inflight_hi = rg.seq0 + r + SOLVE_STAGES + 1;
      }
    };
    const int nblk = (n + 31) / 32;
    // ---------------- forward sweep: L y = x, z = D^{-1} y --------------------------
    T w[MMAX];
#pragma unroll
    for (int m = 0; m < MMAX; ++m) {
      const int row = m * 32 + lane;
      w[m] = (m < M && row < n) ? T(x[row]) : T(0);
    }
    int cur = -1, cstart = 0, cend = 0;
    const T *cb = nullptr;
    for (int q = 0; q < nblk && !abort; ++q) {
      const int j0 = q * 32;
      const int g = q % M;
      int offs[MMAX];
#pragma unroll
      for (int m = 0; m < MMAX; ++m) offs[m] = (m < M) ? ((g + m) % M) * 32 + lane : 0;
      const int rr = j0 + LD + lane;
      const T refill = rr < n ? T(x[rr]) : T(0);
      T zout = T(0);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = j0 + i;
        if (j >= n) break;
        if (j >= cend) {
          if (cur >= 0) release_req(cur);
          cur = j / C;
          if (!wait_req(cur)) { abort = true; break; }
          cb = reinterpret_cast<const T *>(rg.buf + (size_t)((rg.seq0 + cur) % SOLVE_STAGES) * CHUNK_BYTES);
          cstart = cur * C;
          cend = min(n, cstart + C);
        }
        const T *col = cb + (size_t)(j - cstart) * LD;
        const T yj = __shfl_sync(FULL, w[0], i);
        const T c0 = col[offs[0]];
        if (lane == i) zout = yj * c0;
        w[0] -= c0 * yj;
#pragma unroll
        for (int m = 1; m < MMAX; ++m)
          if (m < M) w[m] -= col[offs[m]] * yj;
        if (lane == i) w[0] = refill;
      }
      if (abort) break;
      if (j0 + lane < n) x[j0 + lane] = double(zout);
      const T t0 = w[0];
      // rotate the window by one slot group (select form keeps w in registers)
#pragma unroll
      for (int m = 0; m + 1 < MMAX; ++m) w[m] = opaque_sel(m < M - 1, w[m + 1], opaque_sel(m == M - 1, t0, w[m]));
      if (M == MMAX) w[MMAX - 1] = t0;
    }
    if (abort) break;
    release_req(cur);
    // ---------------- backward sweep: L^T x = z --------------------------------------
    T xw[MMAX];
#pragma unroll
    for (int m = 0; m < MMAX; ++m) xw[m] = T(0);
    int curb = -1;
    cstart = n;
    for (int q = nblk - 1; q >= 0 && !abort; --q) {
      const int j0 = q * 32;
      const int g = q % M;
      int offs[MMAX];
#pragma unroll
      for (int m = 0; m < MMAX; ++m) offs[m] = (m < M) ? ((g + m) % M) * 32 + lane : 0;
      const T zin = (j0 + lane < n) ? T(x[j0 + lane]) : T(0);
      T xout = T(0);
#pragma unroll
      for (int i = 31; i >= 0; --i) {
        const int j = j0 + i;
        if (j >= n) continue;
        if (j < cstart) {
          if (curb >= 0) release_req(curb);
          const int c = j / C;
          curb = 2 * ts.nc - 1 - c;
          if (!wait_req(curb)) { abort = true; break; }
          cb = reinterpret_cast<const T *>(rg.buf + (size_t)((rg.seq0 + curb) % SOLVE_STAGES) * CHUNK_BYTES);
          cstart = c * C;
        }
        const T *col = cb + (size_t)(j - cstart) * LD;
        T part = (lane == i) ? T(0) : col[offs[0]] * xw[0];
#pragma unroll
        for (int m = 1; m < MMAX; ++m)
          if (m < M) part += col[offs[m]] * xw[m];
        part = warp_sum(part);
        if (lane == i) {
          xw[0] = zin - part;
          xout = xw[0];
        }
      }
      if (abort) break;
      if (j0 + lane < n) x[j0 + lane] = double(xout);
      // rotate the window back by one slot group; registers m >= M are never read, so the
      // shift is unconditional (keeps xw in registers)
      T tl = xw[0];
#pragma unroll
      for (int m = 1; m < MMAX; ++m) tl = opaque_sel(m == M - 1, xw[m], tl);
#pragma unroll
      for (int m = MMAX - 1; m >= 1; --m) xw[m] = xw[m - 1];
      xw[0] = tl;
    }
    if (abort) break;
    release_req(curb);
    rg.seq0 += R;
    inflight_lo = inflight_hi = rg.seq0;
  }
  if (abort) {
    if (lane == 0) set_status(status, DS_TIMEOUT);
    // wait (bounded) for copies still in flight before the CTA may exit
    for (uint32_t q = inflight_lo; q < inflight_hi; ++q) mbar_wait(&rg.bar[q % SOLVE_STAGES], (q / SOLVE_STAGES) & 1);
  }
}

#define FP_SOLVE_INST(T, MM)                                                                           \
  template __global__ void k_band_solve<T, MM>(const BandTask *, int, const T *, double *, int *, int *, \
                                               const int *);
FP_SOLVE_INST(double, 4)
FP_SOLVE_INST(double, 8)
FP_SOLVE_INST(double, 12)
FP_SOLVE_INST(double, 16)
FP_SOLVE_INST(float, 4)
FP_SOLVE_INST(float, 8)
FP_SOLVE_INST(float, 12)
FP_SOLVE_INST(float, 16)

// ============================ blocked sweeps ===========================================
// Inverse of every unit-lower 32 x 32 diagonal block of L (used by the explicit operator build,
// whose multi-right-hand-side sweeps apply them as 32 x 32 products), in FP64 from the stored factor,
// stored row-major (Linv[r][c], zero above the diagonal; identity beyond row n - 1 of a
// partial last block).  One CTA per task, one warp per block, lane c computes column c by
// forward substitution x_r = [r == c] - sum_{k<r} L[r][k] x_k.
template <typename T>
__global__ void k_band_linv(const BandTask *tasks, int ntask, const T *fbase, T *lbase) {
  const int task = blockIdx.x;
  if (task >= ntask) return;
  const BandTask tk = tasks[task];
  const T *fac = fbase + tk.fac_off;
  T *linv = lbase + tk.linv_off;
  const int n = tk.n, LD = tk.LD, b = tk.b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nblk = (n + 31) / 32;
  for (int q = warp; q < nblk; q += nw) {
    const int j0 = 32 * q, nb = min(32, n - j0);
    double x[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      double acc = (r == lane) ? 1.0 : 0.0;
      if (r < nb) {
#pragma unroll
        for (int k = 0; k < r; ++k) {
          const double l = (r - k <= b) ? double(fac[(long long)(j0 + k) * LD + (j0 + r) % LD]) : 0.0;
          acc -= l * x[k];
        }
      }
      x[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) linv[(long long)q * 1024 + r * 32 + lane] = T(x[r]);
  }
}

// Per-warp request stream of the blocked solve: the column chunks of block q, forward in
// ascending order, backward in descending order.  Request q of the warp lives in
// ring stage q % SOLVE_STAGES and completes phase (q / SOLVE_STAGES) & 1 of its mbarrier.
template <typename T>
struct BlkStream {
  unsigned char *ring;
  uint64_t *bar;
  const T *fac;
  int chunk;                 // bytes per ring stage
  int n, LD, C, nblk, total;
  uint32_t seq, issued, seq_task;
  int idir, iq, ik;  // issue cursor (meaningful in lane 0)
  bool abort;
  __device__ __forceinline__ int cpb(int q) const { return (min(32, n - 32 * q) + C - 1) / C; }
  __device__ __forceinline__ void issue_one() {
    const int st = issued % SOLVE_STAGES;
    const int c0 = 32 * iq + ik * C;
    const void *src = fac + (long long)c0 * LD;
    const uint32_t bytes = (uint32_t)min(C, n - c0) * LD * sizeof(T);
    mbar_expect_tx(&bar[st], bytes);
    bulk_g2s(ring + (size_t)st * chunk, src, bytes, &bar[st]);
    ++issued;
    if (idir == 0) {
      if (ik + 1 < cpb(iq)) ++ik;
      else if (iq + 1 < nblk) { ++iq; ik = 0; }
      else { idir = 1; iq = nblk - 1; ik = cpb(iq) - 1; }
    } else {
      if (ik > 0) --ik;
      else if (iq > 0) { --iq; ik = cpb(iq) - 1; }
      else idir = 2;
    }
  }
  __device__ __forceinline__ void top_up(int lane) {
    if (lane == 0)
      while ((int)(issued - seq_task) < total && issued - seq < SOLVE_STAGES) issue_one();
    issued = __shfl_sync(FULL, issued, 0);
  }
  __device__ __forceinline__ const T *acquire() {
    const bool ok = mbar_wait(&bar[seq % SOLVE_STAGES], (seq / SOLVE_STAGES) & 1);
    if (!__all_sync(FULL, ok)) { abort = true; return nullptr; }
    return reinterpret_cast<const T *>(ring + (size_t)(seq % SOLVE_STAGES) * chunk);
  }
  __device__ __forceinline__ void release(int lane) {
    __syncwarp();
    ++seq;
    if (lane == 0) fence_proxy_async();
    top_up(lane);
  }
};

// Blocked sweeps of L D L^T x = b, one warp per system from the work queue.  The window of
// pending rows stays in registers by slot (lane l, register m: slot group (q + m) mod M of block
// q), and the factor streams through the warp's ring in chunks of C columns, each byte read once
// per sweep.  The 32 columns of a block are applied one by one: the forward sweep in axpy form
// (one shuffle per column), the backward sweep in dot form (one warp reduction per column).
template <typename T, int MMAX>
__global__ void __launch_bounds__(256, 1) k_band_solve_blk(const BandTask *tasks, int ntask, const T *fbase,
                                                        double *xbase, int *counter, int *status, const int *done,
                                                        int chunk) {
  if (done && *done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  extern __shared__ __align__(128) unsigned char smem[];
  BlkStream<T> S;
  S.chunk = chunk;
  S.ring = smem + (size_t)warp * SOLVE_STAGES * chunk;
  S.bar = reinterpret_cast<uint64_t *>(smem + (size_t)nwarps * SOLVE_STAGES * chunk) + warp * SOLVE_STAGES;
  if (lane == 0)
    for (int st = 0; st < SOLVE_STAGES; ++st) mbar_init(&S.bar[st], 1);
  fence_mbar_init();
  __syncwarp();
  S.seq = 0;
  S.issued = 0;
  S.abort = false;
  while (!S.abort) {
    int task = 0;
    if (lane == 0) task = atomicAdd(counter, 1);
    task = __shfl_sync(FULL, task, 0);
    if (task >= ntask) break;
    const BandTask tk = tasks[task];
    S.fac = fbase + tk.fac_off;
    double *x = xbase + tk.x_off;
    const int n = tk.n, LD = tk.LD, M = LD / 32;
    int C = 32;
    while (C > 1 && C * LD * (int)sizeof(T) > chunk) C >>= 1;
    const int nblk = (n + 31) / 32;
    S.n = n; S.LD = LD; S.C = C; S.nblk = nblk;
    S.total = 0;
    for (int q = 0; q < nblk; ++q) S.total += 2 * S.cpb(q);
    S.seq_task = S.seq;
    S.idir = 0; S.iq = 0; S.ik = 0;
    S.top_up(lane);
    // ------------------------------- forward ------------------------------------
    T w[MMAX];
#pragma unroll
    for (int m = 0; m < MMAX; ++m) {
      const int row = m * 32 + lane;
      w[m] = (m < M && row < n) ? T(x[row]) : T(0);
    }
    for (int q = 0; q < nblk; ++q) {
      const int j0 = 32 * q, g = q % M;
      int offs[MMAX];
#pragma unroll
      for (int m = 0; m < MMAX; ++m) offs[m] = (m < M) ? ((g + m) % M) * 32 + lane : 0;
      const int rr = j0 + LD + lane;
      const T refill = rr < n ? T(x[rr]) : T(0);
      // column by column (axpy form): y_cc is lane cc's pending value once the columns before
      // it are applied.  Column cc's slot of lane l in the first slot group holds L[j0 + l][j0 + cc]
      // for l > cc (the in-block part), 1/d for l == cc, and the row j0 + LD + l of the next
      // window for l < cc; the other slot groups hold the rows of the window.
      T wq = w[0], zout = T(0), corr0 = T(0);
      const int ncol = min(32, n - j0);
      for (int c0c = 0; c0c < ncol && !S.abort; c0c += C) {
        if (c0c) S.release(lane);
        const T *cb = S.acquire();
        if (S.abort) break;
        const int cend = min(ncol, c0c + C);
#pragma unroll 2
        for (int cc = c0c; cc < cend; ++cc) {
          const T *col = cb + (size_t)(cc - c0c) * LD;
          const T c0 = col[offs[0]];
          const T yc = __shfl_sync(FULL, wq, cc);
          if (lane > cc) wq -= c0 * yc;
          else if (lane == cc) zout = yc * c0;
          else corr0 += c0 * yc;
#pragma unroll
          for (int m = 1; m < MMAX; ++m)
            if (m < M) w[m] -= col[offs[m]] * yc;
        }
      }
      if (S.abort) break;
      S.release(lane);
      if (j0 + lane < n) x[j0 + lane] = double(zout);
      w[0] = refill - corr0;
      const T t0 = w[0];
      // rotate the window by one slot group (select form keeps w in registers)
#pragma unroll
      for (int m = 0; m + 1 < MMAX; ++m) w[m] = opaque_sel(m < M - 1, w[m + 1], opaque_sel(m == M - 1, t0, w[m]));
      if (M == MMAX) w[MMAX - 1] = t0;
    }
    if (S.abort) break;
    // ------------------------------- backward -----------------------------------
    T xw[MMAX];
#pragma unroll
    for (int m = 0; m < MMAX; ++m) xw[m] = T(0);
    for (int q = nblk - 1; q >= 0; --q) {
      const int j0 = 32 * q, g = q % M;
      int offs[MMAX];
#pragma unroll
      for (int m = 0; m < MMAX; ++m) offs[m] = (m < M) ? ((g + m) % M) * 32 + lane : 0;
      const T zin = (j0 + lane < n) ? T(x[j0 + lane]) : T(0);
      const int ncol = min(32, n - j0);
      // columns in descending order (dot form): x_cc = z_cc - sum_{r > cc} L[r][j0 + cc] x_r, the
      // rows of the block below cc (x of lanes > cc, final by then) and of the window
      T xc = T(0);
      for (int kc = (ncol - 1) / C; kc >= 0 && !S.abort; --kc) {
        if (kc != (ncol - 1) / C) S.release(lane);
        const T *cb = S.acquire();
        if (S.abort) break;
        const int c0c = kc * C, cend = min(ncol, c0c + C);
#pragma unroll 4
        for (int cc = cend - 1; cc >= c0c; --cc) {
          const T *col = cb + (size_t)(cc - c0c) * LD;
          T sacc = col[offs[0]] * (lane < cc ? xw[0] : (lane > cc ? xc : T(0)));
#pragma unroll
          for (int m = 1; m < MMAX; ++m)
            if (m < M) sacc += col[offs[m]] * xw[m];
          sacc = warp_sum(sacc);
          if (lane == cc) xc = zin - sacc;
        }
      }
      if (S.abort) break;
      S.release(lane);
      xw[0] = xc;
      if (j0 + lane < n) x[j0 + lane] = double(xc);
      // rotate the window back by one slot group; registers m >= M are never read, so the
      // shift is unconditional (keeps xw in registers)
      T tl = xw[0];
#pragma unroll
      for (int m = 1; m < MMAX; ++m) tl = opaque_sel(m == M - 1, xw[m], tl);
#pragma unroll
      for (int m = MMAX - 1; m >= 1; --m) xw[m] = xw[m - 1];
      xw[0] = tl;
    }
  }
  if (S.abort) {
    if (lane == 0) set_status(status, DS_TIMEOUT);
    for (uint32_t q = S.seq; q < S.issued; ++q) mbar_wait(&S.bar[q % SOLVE_STAGES], (q / SOLVE_STAGES) & 1);
  }
}

size_t solve_smem_bytes(int warps_per_cta) {
  return (size_t)warps_per_cta * SOLVE_STAGES * CHUNK_BYTES + (size_t)warps_per_cta * SOLVE_STAGES * 8;
}

// Host launchers (template kernel stubs are not visible across translation units).
cudaError_t launch_band_factor(bool fp32, const BandTask *tasks, int ntask, void *base, int NB, int *status,
                               size_t smem, cudaStream_t stream) {
  cudaError_t e;
  if (fp32) {
    e = cudaFuncSetAttribute(k_band_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_band_factor<float><<<ntask, 256, smem, stream>>>(tasks, ntask, (float *)base, NB, status);
  } else {
    e = cudaFuncSetAttribute(k_band_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_band_factor<double><<<ntask, 256, smem, stream>>>(tasks, ntask, (double *)base, NB, status);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_solve_T(int mmax, int grid, int wpc, cudaStream_t stream, const BandTask *tasks,
                                  int ntask, const T *fac, double *x, int *counter, int *status, const int *done) {
  void (*kern)(const BandTask *, int, const T *, double *, int *, int *, const int *) = nullptr;
  switch (mmax) {
    case 4: kern = k_band_solve<T, 4>; break;
    case 8: kern = k_band_solve<T, 8>; break;
    case 12: kern = k_band_solve<T, 12>; break;
    default: kern = k_band_solve<T, 16>; break;
  }
  const size_t smem = solve_smem_bytes(wpc);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 32 * wpc, smem, stream>>>(tasks, ntask, fac, x, counter, status, done);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_solve_blk_T(int mmax, int grid, int wpc, int chunk, cudaStream_t stream,
                                      const BandTask *tasks, int ntask, const T *fac, double *x, int *counter,
                                      int *status, const int *done) {
  void (*kern)(const BandTask *, int, const T *, double *, int *, int *, const int *, int) = nullptr;
  switch (mmax) {
    case 4: kern = k_band_solve_blk<T, 4>; break;
    case 8: kern = k_band_solve_blk<T, 8>; break;
    case 12: kern = k_band_solve_blk<T, 12>; break;
    default: kern = k_band_solve_blk<T, 16>; break;
  }
  const size_t smem = (size_t)wpc * SOLVE_STAGES * (chunk + 8);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 32 * wpc, smem, stream>>>(tasks, ntask, fac, x, counter, status, done, chunk);
  return cudaGetLastError();
}

// chunk: bytes per ring stage (multiple of 1024, >= one factor column), wpc: warps per CTA (1..8).
cudaError_t launch_band_solve_blk(bool fp32, int mmax, int grid, int wpc, int chunk, cudaStream_t stream,
                                  const BandTask *tasks, int ntask, const void *fac, double *x, int *counter,
                                  int *status, const int *done) {
  if (fp32)
    return launch_solve_blk_T<float>(mmax, grid, wpc, chunk, stream, tasks, ntask, (const float *)fac, x, counter,
                                     status, done);
  return launch_solve_blk_T<double>(mmax, grid, wpc, chunk, stream, tasks, ntask, (const double *)fac, x, counter,
                                    status, done);
}

__global__ void k_round_to_float(const double *src, float *dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

cudaError_t launch_round_to_float(const double *src, float *dst, long long n, cudaStream_t stream) {
  k_round_to_float<<<2048, 256, 0, stream>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_band_linv(bool fp32, const BandTask *tasks, int ntask, const void *fac, void *linv,
                             cudaStream_t stream) {
  if (fp32) k_band_linv<float><<<ntask, 256, 0, stream>>>(tasks, ntask, (const float *)fac, (float *)linv);
  else k_band_linv<double><<<ntask, 256, 0, stream>>>(tasks, ntask, (const double *)fac, (double *)linv);
  return cudaGetLastError();
}

cudaError_t launch_band_solve(bool fp32, int mmax, int grid, int wpc, cudaStream_t stream, const BandTask *tasks,
                              int ntask, const void *fac, double *x, int *counter, int *status, const int *done) {
  if (fp32) return launch_solve_T<float>(mmax, grid, wpc, stream, tasks, ntask, (const float *)fac, x, counter, status, done);
  return launch_solve_T<double>(mmax, grid, wpc, stream, tasks, ntask, (const double *)fac, x, counter, status, done);
}

}  // namespace fp
