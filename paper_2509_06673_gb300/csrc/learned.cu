// Learned initial guess lambda_0 (a systems pattern of this library; not in the paper, whose
// Algorithm 1 starts from lambda^{n-1}).  A 3-layer MLP, 8 -> 256 -> 256 -> 1 with ReLU,
// maps per-multiplier features to the next increment of lambda in units of the last one.
// The 256 x 256 products run on tensor cores (mma.sync m16n8k16, bfloat16 operands, FP32
// accumulation); the thin first and last layers on CUDA cores in FP32.  Training (forward,
// backward, Adam) uses only these kernels.  Reductions are fixed-order (deterministic).
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.cuh"

namespace fp {

constexpr int MLP_NIN = 8, MLP_NH = 256;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_NIN * MLP_NH;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_NH;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_NH * MLP_NH;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_NH;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_NH;
constexpr int MLP_NPARAM = MLP_OFF_B3 + 1;

// ------------------------------- tensor-core GEMM ------------------------------------
// C[i][j] = epi( sum_k A(i,k) B(k,j) ), A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj],
// FP32 in memory, rounded to bfloat16 when staged in shared memory.  Epilogue:
// v = acc + bias[j] (bias may be null); if z: z[i*ldc + j] = v; if mask: v *= (mask[i*ldc+j] > 0);
// if relu: v = max(v, 0); C[i*ldc + j] = v.  Tiles 64 x 64 x 32, 4 warps of 32 x 32.
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const float *A, long long sai,
                                                   long long sak, const float *B, long long sbk, long long sbj,
                                                   float *C, int ldc, const float *bias, float *z, const float *mask,
                                                   int relu) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bt[GBN][GBK + GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const bool a_kfast = sak == 1, b_jfast = sbj == 1;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    // stage A (64 x 32) and B^T (64 x 32)
    for (int e = tid; e < GBM * GBK; e += 128) {
      const int ii = a_kfast ? e / GBK : e % GBM;
      const int kk = a_kfast ? e % GBK : e / GBM;
      const int gi = i0 + ii, gk = k0 + kk;
      const float v = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.f;
      As[ii][kk] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < GBN * GBK; e += 128) {
      const int jj = b_jfast ? e % GBN : e / GBK;
      const int kk = b_jfast ? e / GBN : e % GBK;
      const int gj = j0 + jj, gk = k0 + kk;
      const float v = (gj < N && gk < K) ? B[gk * sbk + gj * sbj] : 0.f;
      Bt[jj][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + 16 * a + g;
        af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * t]);
        af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * t]);
        af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * t + 8]);
        af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int cidx = wn + 8 * b + g;
        bf[b][0] = *reinterpret_cast<const uint32_t *>(&Bt[cidx][ks + 2 * t]);
        bf[b][1] = *reinterpret_cast<const uint32_t *>(&Bt[cidx][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
              : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bf[b][0]), "r"(bf[b][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = i0 + wm + 16 * a + g + (c >= 2 ? 8 : 0);
        const int j = j0 + wn + 8 * b + 2 * t + (c & 1);
        if (i >= M || j >= N) continue;
        float v = acc[a][b][c] + (bias ? bias[j] : 0.f);
        const long long o = (long long)i * ldc + j;
        if (z) z[o] = v;
        if (mask) v = mask[o] > 0.f ? v : 0.f;
        if (relu) v = fmaxf(v, 0.f);
        C[o] = v;
      }
}

// --------------------------- thin layers and reductions ------------------------------
// layer 1: z1 = x W1 + b1, h1 = relu(z1)  (x: M x 8)
__global__ void k_mlp_l1(int M, const float *x, const float *P, float *z1, float *h1) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)M * MLP_NH) return;
  const int i = (int)(e / MLP_NH), j = (int)(e % MLP_NH);
  float v = P[MLP_OFF_B1 + j];
#pragma unroll
  for (int k = 0; k < MLP_NIN; ++k) v += x[i * MLP_NIN + k] * P[MLP_OFF_W1 + k * MLP_NH + j];
  if (z1) z1[e] = v;
  h1[e] = fmaxf(v, 0.f);
}

// layer 3: out = h2 W3 + b3 (warp per row); with y: d_out = (out - y) / m, loss partials
__global__ void k_mlp_l3(int M, const float *h2, const float *P, float *out, const float *y, float *dout,
                         double *loss_rows, float inv_m) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= M) return;
  float acc = 0.f;
  for (int j = lane; j < MLP_NH; j += 32) acc += h2[(long long)row * MLP_NH + j] * P[MLP_OFF_W3 + j];
  acc = warp_sum(acc);
  if (lane == 0) {
    const float o = acc + P[MLP_OFF_B3];
    out[row] = o;
    if (y) {
      const float r = o - y[row];
      dout[row] = r * inv_m;
      loss_rows[row] = 0.5 * (double)r * r * inv_m;
    }
  }
}

// d2 = d_out (x) W3 * (z2 > 0)
__global__ void k_mlp_d2(int M, const float *dout, const float *P, const float *z2, float *d2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)M * MLP_NH) return;
  const int i = (int)(e / MLP_NH), j = (int)(e % MLP_NH);
  d2[e] = z2[e] > 0.f ? dout[i] * P[MLP_OFF_W3 + j] : 0.f;
}

// Column sums over the rows in fixed order: out[j] = sum_i A[i][j] * (w ? w[i] : 1).
// One block per column group of 32, threads stride rows, fixed-order combine.
__global__ void k_colsum(int M, int N, const float *A, int lda, const float *w, float *out) {
  __shared__ float sh[8][33];
  const int j = blockIdx.x * 32 + (threadIdx.x & 31), rg = threadIdx.x >> 5;  // 8 row groups
  float acc = 0.f;
  if (j < N)
    for (int i = rg; i < M; i += 8) acc += A[(long long)i * lda + j] * (w ? w[i] : 1.f);
  sh[rg][threadIdx.x & 31] = acc;
  __syncthreads();
  if (rg == 0 && j < N) {
    float s = 0.f;
    for (int q = 0; q < 8; ++q) s += sh[q][threadIdx.x & 31];
    out[j] = s;
  }
}

// dW1 = x^T d1 (8 x 256), fixed order over rows
__global__ void k_mlp_dw1(int M, const float *x, const float *d1, float *g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= MLP_NIN * MLP_NH) return;
  const int k = j / MLP_NH, c = j % MLP_NH;
  float acc = 0.f;
  for (int i = 0; i < M; ++i) acc += x[i * MLP_NIN + k] * d1[(long long)i * MLP_NH + c];
  g[MLP_OFF_W1 + j] = acc;
}

__global__ void k_sum_double(const double *v, int n, double *out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)blockDim.x; ++q) s += sh[q];
    *out += s;
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters
__global__ void k_adam(float *P, const float *G, float *m1, float *m2, int n, float lr, float b1, float b2, float eps,
                       int step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float v = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = v;
  const float ah = a / (1.f - powf(b1, (float)step)), vh = v / (1.f - powf(b2, (float)step));
  P[i] -= lr * ah / (sqrtf(vh) + eps);
}

// SplitMix64 (Steele, Lea & Flood 2014), counter-based: value i of stream seed
__device__ __forceinline__ double splitmix_u01(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return ((double)(z >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

// He-uniform W1, W2; zero output layer and biases, so the untrained network predicts no
// correction (the guess starts as the source-scaled extrapolation)
__global__ void k_mlp_init(float *P, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NPARAM) return;
  const double u = splitmix_u01(seed, i);
  float v = 0.f;
  if (i < MLP_OFF_B1) v = (float)((2.0 * u - 1.0) * sqrt(6.0 / MLP_NIN));
  else if (i >= MLP_OFF_W2 && i < MLP_OFF_B2) v = (float)((2.0 * u - 1.0) * sqrt(6.0 / MLP_NH));
  P[i] = v;
}

// ------------------------------- features and guess ----------------------------------
// Per multiplier r: [dl/s1, l1/s0, rho, rho*dl/s1, (dl/s1)(l1/s0), rho*l1/s0, kind, comp],
// dl = l1 - l2 (features are free of the node position, so nothing ties the network to the
// source location it was trained on),
// s1 = RMS(dl), s0 = RMS(l1) (from the sums of squares in sums[0], sums[1]).  The network
// inputs are clamped to [-FEAT_CLAMP, FEAT_CLAMP]: a localised source (a point load) makes
// the few rows near it hundreds of RMS units large, and such inputs made training diverge;
// the extrapolation itself (the skip connection) is computed from lambda directly.
constexpr float FEAT_CLAMP = 8.0f;
__device__ __forceinline__ float clampf(double v) { return (float)fmin(fmax(v, -FEAT_CLAMP), FEAT_CLAMP); }
__global__ void k_features(int n, const double *l1, const double *l2, const double *sums, const double *stepv,
                           const float *xy, const int *kind, const int *comp, float *X, float *scale_out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const double rho = stepv[ST_RHO];
  const double s1 = sqrt(sums[0] / n) + 1e-300, s0 = sqrt(sums[1] / n) + 1e-300;
  if (r == 0 && scale_out) scale_out[0] = (float)s1;
  if (r >= n) return;
  const double dl = (l1[r] - l2[r]) / s1;
  float *f = X + (long long)r * MLP_NIN;
  f[0] = clampf(dl);
  f[1] = clampf(l1[r] / s0);
  f[2] = clampf(rho);
  f[3] = clampf(rho * dl);
  f[4] = clampf(dl * (l1[r] / s0));
  f[5] = clampf(rho * (l1[r] / s0));
  f[6] = (float)kind[r];
  f[7] = (float)comp[r];
}

// The two directions of the learned guess from lambda^{n-1}: the source-scaled
// extrapolation dc = rho (l1 - l2) (the network's skip connection, in FP64 from lambda
// itself) and the network's correction db = s1 * out (s1 from the same sums).
__global__ void k_guess_dirs(int n, const double *l1, const double *l2, const float *out, const double *stepv,
                             const double *sums, double *dc, double *db) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double s1 = sqrt(sums[0] / n);
  dc[r] = stepv[ST_RHO] * (l1[r] - l2[r]);
  db[r] = s1 * (double)out[r];
}

// append samples (features, target = (l_new - l1 - rho (l1 - l2)) / s1: what the skip
// connection misses) for rows r0, r0+stride, ...
__global__ void k_record(int n, const float *X, const double *lnew, const double *l1, const double *l2,
                         const double *stepv, const double *sums, int r0, int stride, long long base, long long cap,
                         float *SX, float *SY) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long r = r0 + q * stride;
  if (r >= n) return;
  const long long d = base + q;
  if (d >= cap) return;
  const double s1 = sqrt(sums[0] / n) + 1e-300;
  for (int k = 0; k < MLP_NIN; ++k) SX[d * MLP_NIN + k] = X[r * MLP_NIN + k];
  SY[d] = (float)((lnew[r] - l1[r] - stepv[ST_RHO] * (l1[r] - l2[r])) / s1);
}

__global__ void k_gather_rows(int m, const int *idx, const float *SX, const float *SY, float *X, float *Y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * (MLP_NIN + 1)) return;
  const int i = e / (MLP_NIN + 1), k = e % (MLP_NIN + 1);
  const long long s = idx[i];
  if (k < MLP_NIN) X[(long long)i * MLP_NIN + k] = SX[s * MLP_NIN + k];
  else Y[i] = SY[s];
}

// The guess selector: lambda_0 = lambda_a + a tc + b tb with (a, b) minimising the true projected
// residual ||r_a - a u - b w||_2 (u = P F tc, w = P F tb; the residual is affine in lambda),
// from g = (u.u, u.w, w.w, u.r_a, w.r_a); (0, 0), the previous-step guess, is one of the
// candidates, so the result is never worse.  One thread.
__global__ void k_span_solve(const double *g, double *ab, int *flag) {
  const double uu = g[0], uw = g[1], ww = g[2], ur = g[3], wr = g[4];
  double a = 0.0, b = 0.0;
  const double det = uu * ww - uw * uw;
  if (uu > 0.0 && ww > 0.0 && det > 1e-10 * uu * ww) {
    a = (ur * ww - wr * uw) / det;
    b = (uu * wr - uw * ur) / det;
  } else if (uu > 0.0) {
    a = ur / uu;
  } else if (ww > 0.0) {
    b = wr / ww;
  }
  if (!isfinite(a) || !isfinite(b)) a = b = 0.0;
  ab[0] = a;
  ab[1] = b;
  *flag = (a != 0.0 || b != 0.0) ? 1 : 0;
}

__global__ void k_span_apply(int n, double *lam, double *r, const double *tc, const double *tb, const double *u,
                             const double *w, const double *ab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = ab[0], b = ab[1];
  lam[i] += a * tc[i] + b * tb[i];
  r[i] -= a * u[i] + b * w[i];
}

// ------------------------------------ launchers --------------------------------------
cudaError_t launch_gemm_bf16(cudaStream_t s, int M, int N, int K, const float *A, long long sai, long long sak,
                             const float *B, long long sbk, long long sbj, float *C, int ldc, const float *bias,
                             float *z, const float *mask, int relu) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  k_gemm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, bias, z, mask, relu);
  return cudaGetLastError();
}

}  // namespace fp
