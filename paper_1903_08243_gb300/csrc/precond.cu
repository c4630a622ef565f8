// Learned element-wise preconditioner: inference, loss gradient and training.
//
// Not in the paper (spec preconditioner for CG over the matrix-free
// operator).  For a residual r,
//
//   M(r) = D^{-1} r + sum_K R_K^T ( w_K * s_K * f(R_K r / s_K) ),
//   f(z) = W2 relu(W1 z + b1),   s_K = ||R_K r||_2,
//
// with R_K the gather of the cell's local dofs, w_K = 1 / (cells sharing the
// node) and D the operator diagonal.  W2 starts at zero, so the untrained
// preconditioner is Jacobi.  The linear mode drops the normalisation, the
// bias and the activation and ties W2 = W1^T:
//
//   M(r) = D^{-1} r + sum_K R_K^T w_K W1^T W1 (w_K R_K r),
//
// symmetric positive definite, so standard PCG applies.  Training minimises
// L = (M(r) - e)^T A (M(r) - e) / (e^T A e) over (residual, error) pairs.
//
// The per-cell MLP is a pair of dense contractions over a tile of 128 cells:
// [128 x 128] x [128 x 128] (the local dofs padded to 128), run on the tensor
// cores with BF16 operands and FP32 accumulation (mma.sync m16n8k16); each
// warp owns 16 cells of the tile.  The weight gradients reduce over cells:
// each warp accumulates 16 output rows of dW1 and dW2 across all its tiles
// in registers (operands loaded transposed with ldmatrix.trans) and adds
// them to the global gradient once.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "convert.cuh"
#include "mfa_internal.h"

namespace {

constexpr int kK = 128;          // padded local dofs
constexpr int kH = 128;          // hidden width
constexpr int kTile = 128;       // cells per tile
constexpr int kLd = kK + 8;      // smem row stride in bf16 (272 B: 16-byte aligned, conflict-free ldmatrix)
constexpr int kThreads = 256;    // 8 warps x 16 cells
constexpr int kW1 = 0;           // master layout: W1 [kH][kK], b1 [kH], W2 [kK][kH]
constexpr int kB1 = kH * kK;
constexpr int kW2 = kB1 + kH;
constexpr int kParams = kW2 + kK * kH;
constexpr int kMatBytes = kTile * kLd * 2;

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const bf16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment: rows r0..r0+15, k columns k0..k0+15 of a row-major [row][kLd] tile.
__device__ __forceinline__ void load_a(uint32_t* a, const bf16* A, int r0, int k0, int lane) {
  ldsm_x4(a, A + (r0 + (lane & 7) + ((lane >> 3) & 1) * 8) * kLd + k0 + (lane >> 4) * 8);
}
// A fragment of X^T: rows o0..o0+15 of X^T are columns of X [c][kLd]; k = c in c0..c0+15.
__device__ __forceinline__ void load_at(uint32_t* a, const bf16* X, int o0, int c0, int lane) {
  ldsm_x4_t(a, X + (c0 + (lane & 7) + (lane >> 4) * 8) * kLd + o0 + ((lane >> 3) & 1) * 8);
}
// B fragments of two n-tiles (n0, n0+8) when B(k, n) = W[n][k] (W row-major [n][kLd]).
__device__ __forceinline__ void load_b_nk(uint32_t* b, const bf16* W, int n0, int k0, int lane) {
  ldsm_x4(b, W + (n0 + (lane & 7) + (lane >> 4) * 8) * kLd + k0 + ((lane >> 3) & 1) * 8);
}
// B fragments of two n-tiles (n0, n0+8) when B(k, n) = Y[k][n] (Y row-major [k][kLd]).
__device__ __forceinline__ void load_b_kn(uint32_t* b, const bf16* Y, int n0, int k0, int lane) {
  ldsm_x4_t(b, Y + (k0 + (lane & 7) + ((lane >> 3) & 1) * 8) * kLd + n0 + (lane >> 4) * 8);
}

// acc[NT][4] (+)= A[r0.., :] * B over k in [0, 128), B(k, n) = W[n][k], n in [n0, n0 + 8 NT)
template <int NT>
__device__ __forceinline__ void gemm_awt(float (*acc)[4], const bf16* A, int r0, const bf16* W, int n0, int lane) {
#pragma unroll
  for (int k0 = 0; k0 < kK; k0 += 16) {
    uint32_t a[4];
    load_a(a, A, r0, k0, lane);
#pragma unroll
    for (int t = 0; t < NT; t += 2) {
      uint32_t b[4];
      load_b_nk(b, W, n0 + 8 * t, k0, lane);
      mma_bf16(acc[t], a, b);
      mma_bf16(acc[t + 1], a, b + 2);
    }
  }
}

// acc[NT][4] (+)= A[r0.., :] * Y[:, n0..], B(k, n) = Y[k][n]
template <int NT>
__device__ __forceinline__ void gemm_ay(float (*acc)[4], const bf16* A, int r0, const bf16* Y, int n0, int lane) {
#pragma unroll
  for (int k0 = 0; k0 < kK; k0 += 16) {
    uint32_t a[4];
    load_a(a, A, r0, k0, lane);
#pragma unroll
    for (int t = 0; t < NT; t += 2) {
      uint32_t b[4];
      load_b_kn(b, Y, n0 + 8 * t, k0, lane);
      mma_bf16(acc[t], a, b);
      mma_bf16(acc[t + 1], a, b + 2);
    }
  }
}

// acc[16][4] += X^T[o0.., :] * Y over the 128 tile rows: (X^T Y)[o][n] = sum_c X[c][o] Y[c][n]
__device__ __forceinline__ void gemm_xty(float (*acc)[4], const bf16* X, int o0, const bf16* Y, int lane) {
#pragma unroll 2
  for (int c0 = 0; c0 < kTile; c0 += 16) {
    uint32_t a[4];
    load_at(a, X, o0, c0, lane);
#pragma unroll
    for (int t = 0; t < 16; t += 2) {
      uint32_t b[4];
      load_b_kn(b, Y, 8 * t, c0, lane);
      mma_bf16(acc[t], a, b);
      mma_bf16(acc[t + 1], a, b + 2);
    }
  }
}

struct MlpArgs {
  const float* r;          // input vector (residual)
  float* y;                // forward: += network part; backward: unused
  const float* g;          // backward: dL/du = gscale * g
  const double* gscale;    // device scalar
  const int32_t* cell_node;
  const float* winv;       // partition-of-unity weights per node
  const bf16* w1;          // [kH][kK]
  const bf16* w2;          // [kK][kH]
  const float* b1;         // [kH]
  float* grad;             // master-layout gradient accumulator
  int64_t ncell;
  int nloc;
  int linear;              // 1: the tied linear variant
};

__device__ __forceinline__ void load_weights(bf16* W1s, bf16* W2s, float* b1s, const MlpArgs& a) {
  for (int i = threadIdx.x; i < kH * kK; i += kThreads) {
    const int r = i / kK, c = i % kK;
    W1s[r * kLd + c] = a.w1[i];
    W2s[r * kLd + c] = a.w2[i];
  }
  for (int i = threadIdx.x; i < kH; i += kThreads) b1s[i] = a.b1[i];
}

// Entries gathered or scattered per thread and round: the tile's node ids
// are read first (consecutive, coalesced), then every value they point to, so
// that kUnr dependent load pairs are in flight per thread instead of one.
constexpr int kUnr = 8;

// Gather r for the tile into F (float [kTile][kK]), then per-cell norms and
// the normalised BF16 inputs Z (zero-padded).  Ends with a block barrier.
__device__ __forceinline__ void gather_inputs(const MlpArgs& a, int64_t c0, int ncb, float* F, float* scale, bf16* Zs) {
  const int nloc = a.nloc;
  for (int i = threadIdx.x; i < kTile * kK; i += kThreads) F[i] = 0.0f;
  __syncthreads();
  const int total = ncb * nloc;
  const int32_t* cn = a.cell_node + c0 * nloc;  // the tile's rows of the map are consecutive
  for (int i0 = threadIdx.x; i0 < total; i0 += kThreads * kUnr) {
    int32_t nd[kUnr];
    float v[kUnr];
#pragma unroll
    for (int u = 0; u < kUnr; ++u) nd[u] = i0 + u * kThreads < total ? __ldg(cn + i0 + u * kThreads) : -1;
#pragma unroll
    for (int u = 0; u < kUnr; ++u)
      v[u] = nd[u] < 0 ? 0.0f : (a.linear ? __ldg(a.winv + nd[u]) * __ldg(a.r + nd[u]) : __ldg(a.r + nd[u]));
#pragma unroll
    for (int u = 0; u < kUnr; ++u) {
      const int i = i0 + u * kThreads;
      if (i < total) {
        const int c = i / nloc, k = i - c * nloc;
        F[c * kK + k] = v[u];
      }
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (a.linear) {  // z = w R r, no normalisation
    for (int c = warp * 16; c < warp * 16 + 16; ++c) {
      if (lane == 0) scale[c] = 1.0f;
      for (int k = lane; k < kK; k += 32) Zs[c * kLd + k] = __float2bfloat16_rn(F[c * kK + k]);
    }
    __syncthreads();
    return;
  }
  for (int c = warp * 16; c < warp * 16 + 16; ++c) {
    float ss = 0.0f;
    for (int k = lane; k < kK; k += 32) ss = fmaf(F[c * kK + k], F[c * kK + k], ss);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float s = sqrtf(ss);
    const float inv = s > 0.0f ? 1.0f / s : 0.0f;
    if (lane == 0) scale[c] = s;
    for (int k = lane; k < kK; k += 32) Zs[c * kLd + k] = __float2bfloat16_rn(F[c * kK + k] * inv);
  }
  __syncthreads();
}

// Hidden layer of this warp's 16 cells: Hs = relu(Z W1^T + b1) in BF16.
__device__ __forceinline__ void hidden_layer(const bf16* Zs, const bf16* W1s, const float* b1s, bf16* Hs, int r0,
                                             int lane, bool linear) {
  float acc[16][4];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
  gemm_awt<16>(acc, Zs, r0, W1s, 0, lane);
  const int row = r0 + (lane >> 2), col = (lane & 3) * 2;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int n = 8 * t + col;
    if (linear) {
      Hs[row * kLd + n] = __float2bfloat16_rn(acc[t][0]);
      Hs[row * kLd + n + 1] = __float2bfloat16_rn(acc[t][1]);
      Hs[(row + 8) * kLd + n] = __float2bfloat16_rn(acc[t][2]);
      Hs[(row + 8) * kLd + n + 1] = __float2bfloat16_rn(acc[t][3]);
    } else {
      Hs[row * kLd + n] = __float2bfloat16_rn(fmaxf(acc[t][0] + b1s[n], 0.0f));
      Hs[row * kLd + n + 1] = __float2bfloat16_rn(fmaxf(acc[t][1] + b1s[n + 1], 0.0f));
      Hs[(row + 8) * kLd + n] = __float2bfloat16_rn(fmaxf(acc[t][2] + b1s[n], 0.0f));
      Hs[(row + 8) * kLd + n + 1] = __float2bfloat16_rn(fmaxf(acc[t][3] + b1s[n + 1], 0.0f));
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kThreads, 1) mlp_forward_kernel(const MlpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* W1s = reinterpret_cast<bf16*>(smem);
  bf16* W2s = W1s + kTile * kLd;
  bf16* Zs = W2s + kTile * kLd;
  bf16* Hs = Zs + kTile * kLd;
  float* F = reinterpret_cast<float*>(Hs + kTile * kLd);  // [kTile][kK]
  float* scale = F + kTile * kK;
  float* b1s = scale + kTile;
  load_weights(W1s, W2s, b1s, a);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r0 = warp * 16;
  const int64_t ntile = (a.ncell + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t c0 = tile * kTile;
    const int ncb = (int)(a.ncell - c0 < kTile ? a.ncell - c0 : kTile);
    gather_inputs(a, c0, ncb, F, scale, Zs);
    hidden_layer(Zs, W1s, b1s, Hs, r0, lane, a.linear);
    float acc[16][4];
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
    if (a.linear) gemm_ay<16>(acc, Hs, r0, W1s, 0, lane);  // O = H W1 (tied)
    else gemm_awt<16>(acc, Hs, r0, W2s, 0, lane);          // O = H W2^T
    const int row = r0 + (lane >> 2), col = (lane & 3) * 2;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int n = 8 * t + col;
      F[row * kK + n] = acc[t][0] * scale[row];
      F[row * kK + n + 1] = acc[t][1] * scale[row];
      F[(row + 8) * kK + n] = acc[t][2] * scale[row + 8];
      F[(row + 8) * kK + n + 1] = acc[t][3] * scale[row + 8];
    }
    __syncthreads();
    {  // assemble with the partition-of-unity weights
      const int total = ncb * a.nloc;
      const int32_t* cn = a.cell_node + c0 * a.nloc;
      for (int i0 = threadIdx.x; i0 < total; i0 += kThreads * kUnr) {
        int32_t nd[kUnr];
        float w[kUnr];
#pragma unroll
        for (int u = 0; u < kUnr; ++u) nd[u] = i0 + u * kThreads < total ? __ldg(cn + i0 + u * kThreads) : -1;
#pragma unroll
        for (int u = 0; u < kUnr; ++u) w[u] = nd[u] < 0 ? 0.0f : __ldg(a.winv + nd[u]);
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
          const int i = i0 + u * kThreads;
          if (nd[u] >= 0) {
            const int c = i / a.nloc, k = i - c * a.nloc;
            atomicAdd(a.y + nd[u], w[u] * F[c * kK + k]);
          }
        }
      }
    }
    __syncthreads();
  }
}

// The linear mode's forward pass, M(r) = D^{-1} r + sum_K R_K^T w_K W1^T W1 (w_K R_K r): only W1 is needed
// and z = w R r is not normalised, so the tile is gathered straight into its BF16 operand Zs and the output
// goes back through the Zs / Hs region.  Three BF16 tiles (105 KB) instead of four tiles and an FP32 one
// (206 KB): two blocks per SM instead of one, so that one block's gather or scatter overlaps the other's
// products.  The padding columns of Zs (local dofs >= nloc) are zeroed once; rows past the last cell of a
// tile hold the previous tile's values and are never scattered.
__global__ void __launch_bounds__(kThreads, 2) mlp_linear_forward_kernel(const MlpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* W1s = reinterpret_cast<bf16*>(smem);
  bf16* Zs = W1s + kTile * kLd;
  bf16* Hs = Zs + kTile * kLd;
  float* F = reinterpret_cast<float*>(Zs);  // [kTile][kK] FP32 output, over Zs and Hs once both are consumed
  const int nloc = a.nloc;
  for (int i = threadIdx.x; i < kH * kK; i += kThreads) W1s[(i / kK) * kLd + i % kK] = a.w1[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r0 = warp * 16;
  const int64_t ntile = (a.ncell + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t c0 = tile * kTile;
    const int ncb = (int)(a.ncell - c0 < kTile ? a.ncell - c0 : kTile);
    const int total = ncb * nloc;
    for (int i = threadIdx.x; i < kTile * (kK - nloc); i += kThreads)  // padding columns (F overwrote them)
      Zs[(i / (kK - nloc)) * kLd + nloc + i % (kK - nloc)] = __float2bfloat16_rn(0.0f);
    const int32_t* cn = a.cell_node + c0 * nloc;
    for (int i0 = threadIdx.x; i0 < total; i0 += kThreads * kUnr) {  // gather z = w R r
      int32_t nd[kUnr];
      float v[kUnr];
#pragma unroll
      for (int u = 0; u < kUnr; ++u) nd[u] = i0 + u * kThreads < total ? __ldg(cn + i0 + u * kThreads) : -1;
#pragma unroll
      for (int u = 0; u < kUnr; ++u) v[u] = nd[u] < 0 ? 0.0f : __ldg(a.winv + nd[u]) * __ldg(a.r + nd[u]);
#pragma unroll
      for (int u = 0; u < kUnr; ++u) {
        const int i = i0 + u * kThreads;
        if (nd[u] >= 0) Zs[(i / nloc) * kLd + i % nloc] = __float2bfloat16_rn(v[u]);
      }
    }
    __syncthreads();
    hidden_layer(Zs, W1s, nullptr, Hs, r0, lane, true);  // H = Z W1^T, this warp's 16 cells
    float acc[16][4];
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
    gemm_ay<16>(acc, Hs, r0, W1s, 0, lane);  // O = H W1
    __syncthreads();  // every warp is done with Zs and Hs
    const int row = r0 + (lane >> 2), col = (lane & 3) * 2;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int n = 8 * t + col;
      F[row * kK + n] = acc[t][0];
      F[row * kK + n + 1] = acc[t][1];
      F[(row + 8) * kK + n] = acc[t][2];
      F[(row + 8) * kK + n + 1] = acc[t][3];
    }
    __syncthreads();
    for (int i0 = threadIdx.x; i0 < total; i0 += kThreads * kUnr) {  // assemble with the weights w
      int32_t nd[kUnr];
      float w[kUnr];
#pragma unroll
      for (int u = 0; u < kUnr; ++u) nd[u] = i0 + u * kThreads < total ? __ldg(cn + i0 + u * kThreads) : -1;
#pragma unroll
      for (int u = 0; u < kUnr; ++u) w[u] = nd[u] < 0 ? 0.0f : __ldg(a.winv + nd[u]);
#pragma unroll
      for (int u = 0; u < kUnr; ++u) {
        const int i = i0 + u * kThreads;
        if (nd[u] >= 0) atomicAdd(a.y + nd[u], w[u] * F[(i / nloc) * kK + i % nloc]);
      }
    }
    __syncthreads();  // the next tile's gather rewrites Zs (over F)
  }
}

__global__ void __launch_bounds__(kThreads, 1) mlp_backward_kernel(const MlpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* W1s = reinterpret_cast<bf16*>(smem);
  bf16* W2s = W1s + kTile * kLd;
  bf16* Zs = W2s + kTile * kLd;
  bf16* Hs = Zs + kTile * kLd;
  bf16* Ds = Hs + kTile * kLd;
  bf16* dHs = Ds + kTile * kLd;
  float* F = reinterpret_cast<float*>(Ds);  // aliases Ds and dHs while the inputs are gathered
  float* scale = reinterpret_cast<float*>(dHs + kTile * kLd);
  float* b1s = scale + kTile;
  load_weights(W1s, W2s, b1s, a);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, r0 = warp * 16;
  const float gs = mfa::d2f_bits(*a.gscale);
  float accW2[16][4], accW1[16][4];
#pragma unroll
  for (int t = 0; t < 16; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) accW2[t][j] = accW1[t][j] = 0.0f;
  float accb = 0.0f;
  const int64_t ntile = (a.ncell + kTile - 1) / kTile;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t c0 = tile * kTile;
    const int ncb = (int)(a.ncell - c0 < kTile ? a.ncell - c0 : kTile);
    gather_inputs(a, c0, ncb, F, scale, Zs);
    hidden_layer(Zs, W1s, b1s, Hs, r0, lane, a.linear);
    // Delta[c][o] = s_c w[node] dL/du[node]  (dL/dO), zero-padded
    for (int i = threadIdx.x; i < kTile * kLd; i += kThreads) Ds[i] = __float2bfloat16_rn(0.0f);
    __syncthreads();
    {
      const int total = ncb * a.nloc;
      const int32_t* cn = a.cell_node + c0 * a.nloc;
      for (int i0 = threadIdx.x; i0 < total; i0 += kThreads * kUnr) {
        int32_t nd[kUnr];
        float v[kUnr];
#pragma unroll
        for (int u = 0; u < kUnr; ++u) nd[u] = i0 + u * kThreads < total ? __ldg(cn + i0 + u * kThreads) : -1;
#pragma unroll
        for (int u = 0; u < kUnr; ++u) v[u] = nd[u] < 0 ? 0.0f : __ldg(a.winv + nd[u]) * __ldg(a.g + nd[u]);
#pragma unroll
        for (int u = 0; u < kUnr; ++u) {
          const int i = i0 + u * kThreads;
          if (nd[u] >= 0) {
            const int c = i / a.nloc, k = i - c * a.nloc;
            Ds[c * kLd + k] = __float2bfloat16_rn(scale[c] * v[u] * gs);
          }
        }
      }
    }
    __syncthreads();
    if (a.linear) {
      // O = W1^T W1 z: dW1 = H^T Delta + (Delta W1^T)^T Z, both reduced over the tile's cells
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float acc[8][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
        gemm_awt<8>(acc, Ds, r0, W1s, 64 * half, lane);  // P = Delta W1^T
        const int row = r0 + (lane >> 2), col = (lane & 3) * 2;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int n = 64 * half + 8 * t + col;
          dHs[row * kLd + n] = __float2bfloat16_rn(acc[t][0]);
          dHs[row * kLd + n + 1] = __float2bfloat16_rn(acc[t][1]);
          dHs[(row + 8) * kLd + n] = __float2bfloat16_rn(acc[t][2]);
          dHs[(row + 8) * kLd + n + 1] = __float2bfloat16_rn(acc[t][3]);
        }
      }
      __syncthreads();
      gemm_xty(accW1, Hs, r0, Ds, lane);   // + sum_c h_c delta_c^T
      gemm_xty(accW1, dHs, r0, Zs, lane);  // + sum_c p_c z_c^T
      __syncthreads();
      continue;
    }
    // dH = (Delta W2) * relu'(.) for this warp's cells, in two halves of 64 columns
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float acc[8][4];
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
      gemm_ay<8>(acc, Ds, r0, W2s, 64 * half, lane);
      const int row = r0 + (lane >> 2), col = (lane & 3) * 2;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int n = 64 * half + 8 * t + col;
        const float m00 = __bfloat162float(Hs[row * kLd + n]) > 0.0f ? 1.0f : 0.0f;
        const float m01 = __bfloat162float(Hs[row * kLd + n + 1]) > 0.0f ? 1.0f : 0.0f;
        const float m10 = __bfloat162float(Hs[(row + 8) * kLd + n]) > 0.0f ? 1.0f : 0.0f;
        const float m11 = __bfloat162float(Hs[(row + 8) * kLd + n + 1]) > 0.0f ? 1.0f : 0.0f;
        dHs[row * kLd + n] = __float2bfloat16_rn(acc[t][0] * m00);
        dHs[row * kLd + n + 1] = __float2bfloat16_rn(acc[t][1] * m01);
        dHs[(row + 8) * kLd + n] = __float2bfloat16_rn(acc[t][2] * m10);
        dHs[(row + 8) * kLd + n + 1] = __float2bfloat16_rn(acc[t][3] * m11);
      }
    }
    __syncthreads();
    gemm_xty(accW2, Ds, r0, Hs, lane);   // dW2[o][h] += sum_c Delta[c][o] H[c][h]
    gemm_xty(accW1, dHs, r0, Zs, lane);  // dW1[h][k] += sum_c dH[c][h] Z[c][k]
    if (threadIdx.x < kH)
      for (int c = 0; c < ncb; ++c) accb += __bfloat162float(dHs[c * kLd + threadIdx.x]);
    __syncthreads();
  }
  const int row = r0 + (lane >> 2), col = (lane & 3) * 2;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int n = 8 * t + col;
    atomicAdd(a.grad + kW2 + row * kH + n, accW2[t][0]);
    atomicAdd(a.grad + kW2 + row * kH + n + 1, accW2[t][1]);
    atomicAdd(a.grad + kW2 + (row + 8) * kH + n, accW2[t][2]);
    atomicAdd(a.grad + kW2 + (row + 8) * kH + n + 1, accW2[t][3]);
    atomicAdd(a.grad + kW1 + row * kK + n, accW1[t][0]);
    atomicAdd(a.grad + kW1 + row * kK + n + 1, accW1[t][1]);
    atomicAdd(a.grad + kW1 + (row + 8) * kK + n, accW1[t][2]);
    atomicAdd(a.grad + kW1 + (row + 8) * kK + n + 1, accW1[t][3]);
  }
  if (threadIdx.x < kH) atomicAdd(a.grad + kB1 + threadIdx.x, accb);
}

// Adam on the FP32 master weights; refreshes the BF16 copies and clears the
// gradient.  Entries outside the nloc x kH and kH x nloc blocks stay zero.
__global__ void adam_kernel(float* w, float* grad, float* m, float* v, bf16* w1, bf16* w2, float* b1, int nloc,
                            int linear, float lr, float beta1, float beta2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
    bool live = true;
    if (i < kB1) live = (i % kK) < nloc;
    else if (i >= kW2) live = !linear && ((i - kW2) / kH) < nloc;
    else live = !linear;
    float wi = w[i];
    if (live) {
      const float g = grad[i];
      const float mi = beta1 * m[i] + (1.0f - beta1) * g;
      const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
      m[i] = mi;
      v[i] = vi;
      wi -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    } else {
      wi = 0.0f;
    }
    w[i] = wi;
    grad[i] = 0.0f;
    if (i < kB1) w1[i] = __float2bfloat16_rn(wi);
    else if (i < kW2) b1[i - kB1] = wi;
    else w2[i - kW2] = __float2bfloat16_rn(wi);
  }
}

__global__ void refresh_kernel(const float* w, bf16* w1, bf16* w2, float* b1) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
    if (i < kB1) w1[i] = __float2bfloat16_rn(w[i]);
    else if (i < kW2) b1[i - kB1] = w[i];
    else w2[i - kW2] = __float2bfloat16_rn(w[i]);
  }
}

__global__ void jacobi32_kernel(const float* d, const float* r, float* z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = d[i] * r[i];
}

__global__ void sub32_kernel(float* u, const float* e, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] -= e[i];
}

__global__ void multiplicity_kernel(const int32_t* cell_node, int64_t count, float* mult) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(mult + cell_node[i], 1.0f);
}

__global__ void invert32_kernel(float* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = v[i] > 0.0f ? 1.0f / v[i] : 0.0f;
}

__global__ void inv_kernel(const double* den, double factor, double* out) { *out = factor / *den; }

unsigned grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// SplitMix64 (Steele, Lea and Flood 2014), counter based.
uint64_t splitmix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr int kFwdSmem = 4 * kMatBytes + (kTile * kK + kTile + kH) * 4;
constexpr int kLinSmem = 3 * kMatBytes;
static_assert(2 * kMatBytes >= kTile * kK * 4, "the FP32 output tile fits over Zs and Hs");
constexpr int kBwdSmem = 6 * kMatBytes + (kTile + kH) * 4;

}  // namespace

struct mfa_precond {
  mfa_ctx* ctx = nullptr;
  int device = 0;  // CUDA device of the handle's memory (destroy does not read ctx)
  mfa_form* form = nullptr;
  int nloc = 0;
  int64_t ncell = 0, ndof = 0;
  float *winv = nullptr, *dinv = nullptr, *w = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *b1 = nullptr;
  bf16 *w1 = nullptr, *w2 = nullptr;
  float *u = nullptr, *au = nullptr;
  double* scal = nullptr;  // [0] num, [1] den, [2] gscale, [3..] dot result
  double* partial = nullptr;
  int64_t adam_t = 0;
  int fwd_blocks = 0, bwd_blocks = 0, lin_blocks = 0;
  int linear = 0;
};

namespace {

MlpArgs mlp_args(mfa_precond* pc, const float* r, float* y, const float* g) {
  MlpArgs a{};
  a.r = r;
  a.y = y;
  a.g = g;
  a.gscale = pc->scal + 2;
  a.cell_node = pc->form->space->d_cell_node;
  a.winv = pc->winv;
  a.w1 = pc->w1;
  a.w2 = pc->w2;
  a.b1 = pc->b1;
  a.grad = pc->grad;
  a.ncell = pc->ncell;
  a.nloc = pc->nloc;
  a.linear = pc->linear;
  return a;
}

int check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MFA_OK;
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  return mfa::set_error(MFA_ERR_CUDA, msg);
}

int forward(mfa_precond* pc, const float* r, float* z, cudaStream_t s) {
  jacobi32_kernel<<<grid1(pc->ndof), 256, 0, s>>>(pc->dinv, r, z, pc->ndof);
  const int64_t ntile = (pc->ncell + kTile - 1) / kTile;
  if (ntile > 0) {
    if (pc->linear) {
      const int64_t grid = ntile < pc->lin_blocks ? ntile : pc->lin_blocks;
      mlp_linear_forward_kernel<<<(unsigned)grid, kThreads, kLinSmem, s>>>(mlp_args(pc, r, z, nullptr));
    } else {
      const int64_t grid = ntile < pc->fwd_blocks ? ntile : pc->fwd_blocks;
      mlp_forward_kernel<<<(unsigned)grid, kThreads, kFwdSmem, s>>>(mlp_args(pc, r, z, nullptr));
    }
  }
  return check(cudaGetLastError(), "mlp forward");
}

// loss of one pair into scal[0] / scal[1] and the gradient into pc->grad (accumulated)
int loss_grad(mfa_precond* pc, mfa_form* aform, const float* r, const float* e, cudaStream_t s) {
  mfa_ctx* ctx = pc->ctx;
  int rc = forward(pc, r, pc->u, s);  // u = M(r)
  if (rc) return rc;
  sub32_kernel<<<grid1(pc->ndof), 256, 0, s>>>(pc->u, e, pc->ndof);  // u = M(r) - e
  rc = mfa_apply_f32(ctx, aform, e, pc->au, 0);                      // A e for the denominator
  if (rc) return rc;
  rc = check(mfa::dot32_launch(e, pc->au, pc->ndof, pc->partial, pc->scal + 1, s), "dot");
  if (rc) return rc;
  rc = mfa_apply_f32(ctx, aform, pc->u, pc->au, 0);  // A u
  if (rc) return rc;
  rc = check(mfa::dot32_launch(pc->u, pc->au, pc->ndof, pc->partial, pc->scal + 0, s), "dot");
  if (rc) return rc;
  inv_kernel<<<1, 1, 0, s>>>(pc->scal + 1, 2.0, pc->scal + 2);  // dL/du = (2 / e.Ae) A u
  const int64_t ntile = (pc->ncell + kTile - 1) / kTile;
  if (ntile > 0) {
    const int64_t grid = ntile < pc->bwd_blocks ? ntile : pc->bwd_blocks;
    mlp_backward_kernel<<<(unsigned)grid, kThreads, kBwdSmem, s>>>(mlp_args(pc, r, nullptr, pc->au));
  }
  return check(cudaGetLastError(), "mlp backward");
}

}  // namespace

extern "C" {

int mfa_precond_create(mfa_ctx* ctx, mfa_form* form, int mode, uint64_t seed, mfa_precond** out) {
  if (!ctx || !form || !out) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_create: NULL argument");
  if (mode != MFA_PRECOND_MLP && mode != MFA_PRECOND_LINEAR)
    return mfa::set_error(MFA_ERR_ARG, "mfa_precond_create: unknown mode");
  *out = nullptr;
  mfa_space* sp = form->space;
  if (sp->mesh->cell_type != MFA_CELL_HEX8 || sp->ncomp != 1 || form->p.precision != MFA_PREC_FP64 ||
      form->p.kind > MFA_FORM_HELMHOLTZ || sp->nloc > kK)
    return mfa::set_error(MFA_ERR_UNSUPPORTED,
                          "mfa_precond_create: needs an FP64 scalar hex form with at most 128 local dofs (Q1-Q4)");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "cudaSetDevice");
  mfa_precond* pc = new mfa_precond();
  pc->ctx = ctx;
  pc->device = ctx->device;
  pc->form = form;
  pc->linear = mode == MFA_PRECOND_LINEAR;
  pc->nloc = sp->nloc;
  pc->ncell = sp->mesh->ncell;
  pc->ndof = sp->nnode;
  const int64_t n = pc->ndof > 0 ? pc->ndof : 1;
  bool ok = cudaMalloc((void**)&pc->winv, n * 4) == cudaSuccess && cudaMalloc((void**)&pc->dinv, n * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->u, n * 4) == cudaSuccess && cudaMalloc((void**)&pc->au, n * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->w, kParams * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->grad, kParams * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->m, kParams * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->v, kParams * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->b1, kH * 4) == cudaSuccess &&
            cudaMalloc((void**)&pc->w1, kH * kK * 2) == cudaSuccess &&
            cudaMalloc((void**)&pc->w2, kK * kH * 2) == cudaSuccess &&
            cudaMalloc((void**)&pc->scal, 16 * 8) == cudaSuccess &&
            cudaMalloc((void**)&pc->partial, mfa::dot_partials() * 8) == cudaSuccess;
  if (!ok) {
    mfa_precond_destroy(pc);
    return mfa::set_error(MFA_ERR_OOM, "mfa_precond_create: device buffers");
  }
  cudaStream_t s = ctx->stream;
  // partition-of-unity weights and the inverse diagonal, in float
  double* diag = nullptr;
  int rc = cudaMalloc((void**)&diag, n * 8) == cudaSuccess ? MFA_OK : mfa::set_error(MFA_ERR_OOM, "diag");
  if (!rc) rc = mfa_diagonal(ctx, form, diag);
  if (!rc) rc = check(mfa::reciprocal_launch(diag, diag, pc->ndof, s), "reciprocal");
  if (!rc) rc = check(mfa::convert_d2f_launch(diag, pc->dinv, pc->ndof, s), "convert");
  if (!rc) rc = check(cudaMemsetAsync(pc->winv, 0, n * 4, s), "memset");
  if (!rc) {
    multiplicity_kernel<<<grid1(pc->ncell * pc->nloc), 256, 0, s>>>(sp->d_cell_node, pc->ncell * pc->nloc, pc->winv);
    invert32_kernel<<<grid1(pc->ndof), 256, 0, s>>>(pc->winv, pc->ndof);
    rc = check(cudaGetLastError(), "weights");
  }
  // W1 ~ U(-a, a) from SplitMix64 with a = 1/sqrt(nloc) (MLP mode, where b1 = W2 = 0 makes the
  // untrained M Jacobi) or a = 0.01/sqrt(nloc) (linear mode: a small start next to Jacobi)
  std::vector<float> w(kParams, 0.0f);
  const float bound = (pc->linear ? 0.01f : 1.0f) / std::sqrt((float)pc->nloc);
  for (int h = 0; h < kH; ++h)
    for (int k = 0; k < pc->nloc; ++k) {
      const uint64_t z = splitmix(seed * 0x100000001B3ull + (uint64_t)(h * kK + k));
      const double u01 = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      w[kW1 + h * kK + k] = (float)((2.0 * u01 - 1.0) * bound);
    }
  if (!rc) rc = check(cudaMemcpy(pc->w, w.data(), kParams * 4, cudaMemcpyHostToDevice), "weights upload");
  if (!rc) rc = check(cudaMemset(pc->grad, 0, kParams * 4), "memset");
  if (!rc) rc = check(cudaMemset(pc->m, 0, kParams * 4), "memset");
  if (!rc) rc = check(cudaMemset(pc->v, 0, kParams * 4), "memset");
  if (!rc) {
    refresh_kernel<<<64, 256, 0, s>>>(pc->w, pc->w1, pc->w2, pc->b1);
    rc = check(cudaGetLastError(), "refresh");
  }
  if (!rc) rc = check(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem),
                      "smem attribute");
  if (!rc) rc = check(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem),
                      "smem attribute");
  if (!rc)
    rc = check(cudaFuncSetAttribute(mlp_linear_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLinSmem),
               "smem attribute");
  if (!rc) {
    int bf = 1, bb = 1, bl = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, mlp_forward_kernel, kThreads, kFwdSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, mlp_backward_kernel, kThreads, kBwdSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, mlp_linear_forward_kernel, kThreads, kLinSmem);
    pc->fwd_blocks = ctx->sm_count * (bf > 0 ? bf : 1);
    pc->bwd_blocks = ctx->sm_count * (bb > 0 ? bb : 1);
    pc->lin_blocks = ctx->sm_count * (bl > 0 ? bl : 1);
  }
  if (!rc) rc = check(cudaStreamSynchronize(s), "synchronize");
  cudaFree(diag);
  if (rc) {
    mfa_precond_destroy(pc);
    return rc;
  }
  *out = pc;
  return MFA_OK;
}

int mfa_precond_apply(mfa_ctx* ctx, mfa_precond* pc, const float* r, float* z) {
  if (!ctx || !pc || !r || !z || pc->ctx != ctx) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_apply: bad arguments");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "cudaSetDevice");
  return forward(pc, r, z, ctx->stream);
}

int mfa_precond_loss_grad(mfa_ctx* ctx, mfa_precond* pc, mfa_form* aform, const float* r, const float* e,
                          double* loss, float* grad_host) {
  if (!ctx || !pc || !aform || !r || !e || pc->ctx != ctx)
    return mfa::set_error(MFA_ERR_ARG, "mfa_precond_loss_grad: bad arguments");
  if (aform->space != pc->form->space || aform->p.precision == MFA_PREC_FP64)
    return mfa::set_error(MFA_ERR_ARG, "mfa_precond_loss_grad: needs an FP32/BF16 form on the same space");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = ctx->stream;
  int rc = check(cudaMemsetAsync(pc->grad, 0, kParams * 4, s), "memset");
  if (!rc) rc = loss_grad(pc, aform, r, e, s);
  double nd[2] = {0.0, 0.0};
  if (!rc) rc = check(cudaMemcpyAsync(nd, pc->scal, 16, cudaMemcpyDeviceToHost, s), "copy");
  if (!rc && grad_host) rc = check(cudaMemcpyAsync(grad_host, pc->grad, kParams * 4, cudaMemcpyDeviceToHost, s), "copy");
  if (!rc) rc = check(cudaStreamSynchronize(s), "synchronize");
  if (!rc) rc = check(cudaMemsetAsync(pc->grad, 0, kParams * 4, s), "memset");
  if (!rc && loss) *loss = nd[1] != 0.0 ? nd[0] / nd[1] : 0.0;
  return rc;
}

int mfa_precond_train(mfa_ctx* ctx, mfa_precond* pc, mfa_form* aform, int npairs, const float* const* rs,
                      const float* const* es, int steps, double lr, double* loss_first, double* loss_last) {
  if (!ctx || !pc || !aform || npairs <= 0 || !rs || !es || steps < 0 || !(lr > 0.0) || pc->ctx != ctx)
    return mfa::set_error(MFA_ERR_ARG, "mfa_precond_train: bad arguments");
  if (aform->space != pc->form->space || aform->p.precision == MFA_PREC_FP64)
    return mfa::set_error(MFA_ERR_ARG, "mfa_precond_train: needs an FP32/BF16 form on the same space");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = ctx->stream;
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  int rc = MFA_OK;
  double first = 0.0, last = 0.0;
  // mean loss over the pairs before training
  for (int j = 0; j < npairs && !rc; ++j) {
    double l = 0.0;
    rc = mfa_precond_loss_grad(ctx, pc, aform, rs[j], es[j], &l, nullptr);
    first += l / npairs;
  }
  for (int it = 0; it < steps && !rc; ++it) {
    const int j = it % npairs;
    rc = loss_grad(pc, aform, rs[j], es[j], s);
    if (rc) break;
    ++pc->adam_t;
    const float c1 = 1.0f / (1.0f - std::pow(beta1, (float)pc->adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(beta2, (float)pc->adam_t));
    adam_kernel<<<64, 256, 0, s>>>(pc->w, pc->grad, pc->m, pc->v, pc->w1, pc->w2, pc->b1, pc->nloc, pc->linear,
                                   (float)lr, beta1, beta2, eps, c1, c2);
    rc = check(cudaGetLastError(), "adam");
  }
  for (int j = 0; j < npairs && !rc; ++j) {
    double l = 0.0;
    rc = mfa_precond_loss_grad(ctx, pc, aform, rs[j], es[j], &l, nullptr);
    last += l / npairs;
  }
  if (loss_first) *loss_first = first;
  if (loss_last) *loss_last = last;
  return rc;
}

int mfa_precond_get_weights(const mfa_precond* pc, float* host) {
  if (!pc || !host) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_get_weights: NULL argument");
  if (cudaSetDevice(pc->ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "cudaSetDevice");
  if (cudaStreamSynchronize(pc->ctx->stream) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "synchronize");
  return check(cudaMemcpy(host, pc->w, kParams * 4, cudaMemcpyDeviceToHost), "mfa_precond_get_weights");
}

int mfa_precond_set_weights(mfa_precond* pc, const float* host) {
  if (!pc || !host) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_set_weights: NULL argument");
  if (cudaSetDevice(pc->ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "cudaSetDevice");
  std::vector<float> w(host, host + kParams);
  for (int i = 0; i < kParams; ++i) {  // keep the padding (and, in linear mode, b1 and W2) zero
    if (i < kB1 && (i % kK) >= pc->nloc) w[i] = 0.0f;
    if (i >= kW2 && ((i - kW2) / kH) >= pc->nloc) w[i] = 0.0f;
    if (pc->linear && i >= kB1) w[i] = 0.0f;
  }
  int rc = check(cudaMemcpy(pc->w, w.data(), kParams * 4, cudaMemcpyHostToDevice), "mfa_precond_set_weights");
  if (!rc) {
    refresh_kernel<<<64, 256, 0, pc->ctx->stream>>>(pc->w, pc->w1, pc->w2, pc->b1);
    rc = check(cudaStreamSynchronize(pc->ctx->stream), "refresh");
  }
  return rc;
}

int mfa_precond_save(const mfa_precond* pc, const char* path) {
  if (!pc || !path) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_save: NULL argument");
  std::vector<float> w(kParams);
  int rc = mfa_precond_get_weights(pc, w.data());
  if (rc) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_save: cannot open the file");
  const int32_t header[4] = {0x4D464150 /* 'MFAP' */, 1 + pc->linear /* version 1: MLP, 2: linear */, pc->nloc, kH};
  const bool ok = fwrite(header, sizeof(header), 1, f) == 1 && fwrite(w.data(), 4, kParams, f) == (size_t)kParams;
  fclose(f);
  return ok ? MFA_OK : mfa::set_error(MFA_ERR_ARG, "mfa_precond_save: write failed");
}

int mfa_precond_load(mfa_precond* pc, const char* path) {
  if (!pc || !path) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_load: NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return mfa::set_error(MFA_ERR_ARG, "mfa_precond_load: cannot open the file");
  int32_t header[4] = {0, 0, 0, 0};
  std::vector<float> w(kParams);
  const bool ok = fread(header, sizeof(header), 1, f) == 1 && fread(w.data(), 4, kParams, f) == (size_t)kParams;
  fclose(f);
  if (!ok || header[0] != 0x4D464150 || header[1] != 1 + pc->linear || header[2] != pc->nloc || header[3] != kH)
    return mfa::set_error(MFA_ERR_ARG, "mfa_precond_load: not a weight file of this preconditioner shape");
  return mfa_precond_set_weights(pc, w.data());
}

int mfa_precond_destroy(mfa_precond* pc) {
  if (!pc) return MFA_OK;
  cudaSetDevice(pc->device);
  void* all[] = {pc->winv, pc->dinv, pc->w, pc->grad, pc->m, pc->v, pc->b1, pc->w1, pc->w2, pc->u, pc->au,
                 pc->scal, pc->partial};
  for (void* p : all) cudaFree(p);
  delete pc;
  return MFA_OK;
}

}  // extern "C"

namespace mfa {
int precond_apply_f32(mfa_precond* pc, const float* r, float* z, cudaStream_t s) { return forward(pc, r, z, s); }
bool precond_is_linear(const mfa_precond* pc) { return pc->linear != 0; }
}  // namespace mfa
