// Sum-factorised hex action for FP32 arithmetic (FP32 and BF16 variants):
// one thread per 1D line of a cell, tables in the constant bank.
//
// The FP64 kernel (hex_kernels.cuh) is bound by the FP64 pipe and can spend
// two shared-memory loads per FMA.  In FP32 the same layout is bound by the
// load/store pipe, so this kernel changes the work split: a thread owns one
// line of n points in one direction, loads its n inputs once, and forms the
// n outputs with n^2 FMAs whose table coefficients are compile-time offsets
// into __constant__ memory (an FMA operand, no load instruction).  The same
// algorithm as the FP64 kernel: B sweeps in x, y, z; collocation derivatives
// D_x, D_y, D_z; pointwise G g (+ c0 w|J| u); transposed D and B sweeps;
// atomic scatter.  Double vectors are converted on the integer pipe.
//
// BF16 variant: the geometric factors, the largest stream, reach shared
// memory by one bulk copy per batch (cp.async.bulk, completion on an
// mbarrier), issued for the next batch as soon as the current one has
// consumed its factors, so the copy overlaps the transposed sweeps, the
// scatter and the next gather.  Each cell's factor block is padded to 16
// bytes for the copy (and further, see line_geom_stride).  Waits are bounded:
// on timeout the kernel sets error bit 4 and every thread leaves.  FP32
// stages its factors the same way by default; the form that reads them
// straight from global memory (on x-lines, coalesced; MFA_VARIANT_LINE) is
// compiled for both precisions, and the autotuner takes it where it is faster.
#pragma once

#include <cuda_bf16.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "convert.cuh"
#include "mfa_internal.h"

namespace mfa {
namespace hexl {

__host__ __device__ constexpr int tab_offset(int n) {  // B (n x n) then D (n x n) for n = 2, 3, ...
  int off = 0;
  for (int k = 2; k < n; ++k) off += 2 * k * k;
  return off;
}
constexpr int kTabFloats = tab_offset(10);

// One copy per translation unit; filled by upload_tables() of that unit.
static __constant__ float c_tab[2][kTabFloats];  // [0]: FP32 tables, [1]: tables rounded to bfloat16

constexpr int ceil32(int x) { return (x + 31) / 32 * 32; }

// Shared-memory layout of one plane: point (x, y, z) of the batch's cell c at
// c SC + x + SX y + SY z.  Unpadded for most n.  For n = 4 and n = 8 the lines
// of a warp would otherwise fall on the same banks (4-way and 8-way conflicts
// in the x sweeps, 4-way in the y sweeps: strides of 4 or 8 words with the
// default block sizes); the padded strides bring every sweep to 1.3-way on
// average, at 25% (n = 4) and 12.5% (n = 8) more shared memory.  For n = 7 the
// unpadded y sweeps are 3-way (a z-plane of 49 words starts 17 banks on); with
// a warp taking four whole rows of 7 lines (line_lanes) and z-planes of 56 words,
// cells of 392, the x and y sweeps are free of conflicts and the z sweeps
// conflict only where a warp spans two cells (14% more shared memory).
template <int N>
struct LLayout {
  static constexpr int SX = N == 8 ? 9 : N;
  static constexpr int SY = N == 4 ? 19 : (N == 8 ? 72 : (N == 7 ? 56 : N * N));
  static constexpr int SC = N == 4 ? 80 : (N == 8 ? 576 : (N == 7 ? 392 : N * N * N));
  static constexpr bool PADDED = SC != N * N * N;
  // plane offset of point i of the batch (cell i / n^3, local point i % n^3, x fastest)
  __host__ __device__ static constexpr int of(int i) {
    if constexpr (!PADDED) return i;
    const int c = i / (N * N * N), q = i - c * (N * N * N);
    return c * SC + q % N + SX * ((q / N) % N) + SY * (q / (N * N));
  }
};

// n >= 8: the scatter reads its node indices again (from L2) instead of holding them in registers through the
// batch, which lets those kernels reach four blocks per SM; below that the registers are there and the reload
// would only add its latency before the scatter.
template <int N>
__host__ __device__ constexpr bool line_reload_nodes() {
  return N >= 8;
}

template <int N, int CBX = 0>
struct LShape {
  static constexpr int L = N * N;         // lines per cell and direction
  static constexpr int P = N * N * N;     // points per cell
  static constexpr int PS = LLayout<N>::SC;  // floats per cell in a plane
  static constexpr int CB = CBX > 0 ? CBX : line_cb_for(N, 256);
  static constexpr int LANES = line_lanes(N);  // lanes of a warp that carry lines in the sweeps
  static constexpr int T = 32 * ((CB * L + LANES - 1) / LANES);
  static constexpr int SMEM = 4 * CB * PS * 4;  // planes U, V, F0, F1 (see line_batch)
  static constexpr int K = (CB * P + T - 1) / T;  // points per thread in the point-parallel phases
};

// Node of each of this thread's points of batch `batch` (-1 past the batch's end): requested a batch
// ahead, so the gather waits on one load instead of two (and for n < 8 the
// scatter reuses them; line_reload_nodes).
template <int N, int CBX>
__device__ __forceinline__ void line_load_nodes(const int32_t* cell_node, int64_t count, int64_t batch,
                                                int32_t (&node)[LShape<N, CBX>::K]) {
  using S = LShape<N, CBX>;
  const int64_t c0 = batch * S::CB;
  const int ncb = (int)(count - c0 < S::CB ? count - c0 : S::CB);
#pragma unroll
  for (int k = 0; k < S::K; ++k) {
    const int i = threadIdx.x + k * S::T;
    node[k] = i < ncb * S::P ? __ldg(cell_node + c0 * S::P + i) : -1;
  }
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One elected thread: announce `bytes` and start the bulk copy global -> shared.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t state;
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;\n"
               : "=l"(state)
               : "r"(saddr(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity`; false after the limit (the copy never landed).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_test(bar, parity)) return true;
  return false;
}

template <int KIND>
__host__ __device__ constexpr int geom_entries() {
  return KIND == MFA_FORM_MASS ? 1 : (KIND == MFA_FORM_LAPLACE ? 6 : 7);
}

// Plane offset (within a cell) of point m on line (a, b) in direction DIR (0: x, 1: y, 2: z).
template <int N, int DIR>
__device__ __forceinline__ int at(int a, int b, int m) {
  using Y = LLayout<N>;
  if constexpr (DIR == 0) return m + Y::SX * a + Y::SY * b;
  else if constexpr (DIR == 1) return a + Y::SX * m + Y::SY * b;
  else return a + Y::SX * b + Y::SY * m;
}

// out[line] = T[.][.] applied along DIR: out_r = sum_m Tab[r][m] in_m (TRANS: Tab[m][r]).
template <int N, int DIR, int TAB, bool TRANS, bool ACC, int variant>
__device__ __forceinline__ void sweep(const float* in, float* out, int a, int b) {
  constexpr int off = tab_offset(N) + (TAB == 0 ? 0 : N * N);
  float v[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = in[at<N, DIR>(a, b, m)];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = ACC ? out[at<N, DIR>(a, b, r)] : 0.0f;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][off + (TRANS ? m * N + r : r * N + m)], v[m], s);
    out[at<N, DIR>(a, b, r)] = s;
  }
}

// B along x, then D along x on the values just formed, for the thread's x-line
// (kept in registers in between): vout = B_x u, dout = D_x B_x u.  `dout` may
// alias `in` (the thread's own line is read before it is written).
template <int N, int variant>
__device__ __forceinline__ void sweep_bd_x(const float* in, float* vout, float* dout, int a, int b) {
  constexpr int offB = tab_offset(N), offD = tab_offset(N) + N * N;
  float v[N], vx[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = in[at<N, 0>(a, b, m)];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][offB + r * N + m], v[m], s);
    vx[r] = s;
    vout[at<N, 0>(a, b, r)] = s;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][offD + r * N + m], vx[m], s);
    dout[at<N, 0>(a, b, r)] = s;
  }
}

// The test side along z in one pass: out = B_z^T (acc + D_z^T f) for the
// thread's line, without writing the sum back first.  `out` may alias `f`.
template <int N, int variant>
__device__ __forceinline__ void sweep_dtbt_z(const float* f, const float* acc, float* out, int a, int b) {
  constexpr int offB = tab_offset(N), offD = tab_offset(N) + N * N;
  float v[N], w[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = f[at<N, 2>(a, b, m)];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = acc[at<N, 2>(a, b, r)];
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][offD + m * N + r], v[m], s);
    w[r] = s;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][offB + m * N + r], w[m], s);
    out[at<N, 2>(a, b, r)] = s;
  }
}

template <typename TX>
__device__ __forceinline__ float load_x(const TX* x, int32_t node, bool bf16) {
  float v;
  if constexpr (sizeof(TX) == 8) v = d2f_bits(__ldg(x + node));
  else v = __ldg(x + node);
  if (bf16) v = __bfloat162float(__float2bfloat16_rn(v));
  return v;
}

template <typename TY>
__device__ __forceinline__ void add_y(TY* y, int32_t node, float v) {
  if constexpr (sizeof(TY) == 8) atomicAdd(y + node, f2d_bits(v));
  else atomicAdd(y + node, v);
}

struct LineArgs {
  const void* x;  // double or float
  void* y;
  const int32_t* cell_node;
  const void* geom;     // float or bfloat16, [cell][geom_stride]
  int64_t count;
  int64_t gstride;      // elements per cell of `geom`
  int* err;
};

// Factor blocks: per cell, `gstride` elements holding NG entries of n^3
// points each, the points ordered with x slowest (point (x, y, z) at
// y + n z + n^2 x).  The pointwise step runs on x-lines, so at each point of
// the line the batch's threads read consecutive elements (one bank each from
// the shared stage, coalesced from global memory).
template <int PREC>
using GeoT = typename std::conditional<PREC == MFA_PREC_BF16, __nv_bfloat16, float>::type;

// Factor i of a batch: `p` is the shared-memory stage (SHARED) or global memory.
template <int PREC, bool SHARED>
__device__ __forceinline__ float geo_at(const void* p, int64_t i) {
  if constexpr (PREC == MFA_PREC_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  else if constexpr (SHARED) return static_cast<const float*>(p)[i];
  else return __ldg(static_cast<const float*>(p) + i);  // read-only path: global memory only
}

// The pointwise step on the thread's x-line, fused with D_x^T.  V and D0 hold
// the values and the x-derivative at the line's points (sweep_bd_x); F1 and F0
// hold the y- and z-derivatives there.  Per point, the fluxes
// f = G (d0, d1, d2) and the value term c0 w|J| u (Helmholtz); f1 and f2 go
// back to F1 and F0 for the transposed y and z sweeps, f0 stays in registers,
// and V receives r = c0 w|J| u + D_x^T f0.  `gs` is the batch's factor block
// (stage or global memory), `gc` the offset of the thread's cell in it.
template <int N, int KIND, int PREC, bool STG, int variant>
__device__ __forceinline__ void fused_x(const void* gs, int64_t gc, float* F0, float* F1, float* V, const float* D0,
                                        int a, int b) {
  constexpr int L = N * N, P = N * N * N, offD = tab_offset(N) + N * N;
  constexpr int NG = KIND == MFA_FORM_HELMHOLTZ ? 7 : 6;
  const int l = a + N * b;
  float f0[N], r0[N];
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const int j = at<N, 0>(a, b, m);
    const int64_t gi = gc + l + L * m;
    float g[NG];
#pragma unroll
    for (int e = 0; e < NG; ++e) g[e] = geo_at<PREC, STG>(gs, gi + (int64_t)e * P);
    const float d0 = D0[j], d1 = F1[j], d2 = F0[j];
    f0[m] = fmaf(g[0], d0, fmaf(g[3], d1, g[4] * d2));
    F1[j] = fmaf(g[3], d0, fmaf(g[1], d1, g[5] * d2));
    F0[j] = fmaf(g[4], d0, fmaf(g[5], d1, g[2] * d2));
    if constexpr (KIND == MFA_FORM_HELMHOLTZ) r0[m] = g[NG - 1] * V[j];
    else r0[m] = 0.0f;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = r0[r];
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][offD + m * N + r], f0[m], s);
    V[at<N, 0>(a, b, r)] = s;
  }
}

// Mass: B along x, the weight w|J| at each point of the line, and B^T along x
// in one pass over the thread's x-line (in registers).
template <int N, int PREC, bool STG, int variant>
__device__ __forceinline__ void fused_x_mass(const float* in, float* out, const void* gs, int64_t gc, int a, int b) {
  constexpr int L = N * N, offB = tab_offset(N);
  const int l = a + N * b;
  float v[N], u[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = in[at<N, 0>(a, b, m)];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < N; ++m) s = fmaf(c_tab[variant][offB + r * N + m], v[m], s);
    u[r] = s * geo_at<PREC, STG>(gs, gc + l + L * r);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int r = 0; r < N; ++r) s = fmaf(c_tab[variant][offB + r * N + k], u[r], s);
    out[at<N, 0>(a, b, k)] = s;
  }
}

// Shared staging of one batch's factors, and the barrier state.
struct Stage {
  unsigned char* buf;   // CB * gstride elements
  uint64_t* bar;
  uint32_t phase;
  int* abort;           // shared flag: a wait timed out
};

// Staged (bulk-copied) factors by default for both precisions: measured on
// 64^3, Q1-Q6, the autotuner picked the staged form for 11 of the 12 FP32
// operators once x is requested a batch ahead and the planes are four.
template <int PREC>
__host__ __device__ constexpr bool staged() {
  return true;
}

template <int N, int KIND, int PREC, bool STG = staged<PREC>(), int CBX = 0>
__device__ __forceinline__ void issue_factors(const LineArgs& a, int64_t batch, Stage& st) {
  if constexpr (!STG) return;
  using S = LShape<N, CBX>;
  const int64_t c0 = batch * S::CB;
  const int ncb = (int)(a.count - c0 < S::CB ? a.count - c0 : S::CB);
  const uint32_t bytes = (uint32_t)(ncb * a.gstride * (int64_t)sizeof(GeoT<PREC>));
  bulk_load(st.buf, static_cast<const GeoT<PREC>*>(a.geom) + c0 * a.gstride, bytes, st.bar);
}

// x at this thread's points of a batch (0 where node < 0), in registers.
template <typename TX, int K>
__device__ __forceinline__ void line_load_x(const void* xp, const int32_t (&node)[K], float (&xin)[K], bool bf16) {
  const TX* x = static_cast<const TX*>(xp);
#pragma unroll
  for (int k = 0; k < K; ++k) xin[k] = node[k] >= 0 ? load_x(x, node[k], bf16) : 0.0f;
}

// One batch of CB consecutive cells.  Contractions run line-parallel (a
// thread owns one line per direction; warps carry line_lanes(n) lines); the
// gather and the scatter run point-parallel over the whole batch, so
// consecutive threads read consecutive map and output addresses.  The sweep
// order ends the forward pass along x: B_z, B_y, then B_x and D_x on the
// thread's x-line in one pass, D_y and D_z from the values; the
// pointwise step and D_x^T run on the same x-line (fused_x), then D_y^T,
// D_z^T with B_z^T (sweep_dtbt_z), B_y^T and B_x^T.  The factors come from the
// bulk-copied stage (STG) or straight from global memory.  `next` >= 0: batch
// (of `an`) to prefetch afterwards.  `xin` holds x at this thread's points of
// this batch (requested during the previous batch); once the forward sweeps
// are done, the next batch's values are requested into it through
// `node_next`, so that they arrive while this batch finishes and the gather
// never waits on global memory.
template <int N, int KIND, int PREC, typename TX, bool STG = staged<PREC>(), int CBX = 0>
__device__ __forceinline__ bool line_batch(const LineArgs& a, int64_t batch, float* smem, Stage& st,
                                           const LineArgs* an, int64_t next,
                                           const int32_t (&node)[line_reload_nodes<N>() ? 1 : LShape<N, CBX>::K],
                                           const int32_t (&node_next)[LShape<N, CBX>::K],
                                           float (&xin)[LShape<N, CBX>::K]) {
  using S = LShape<N, CBX>;
  constexpr int L = S::L, CB = S::CB, T = S::T, K = S::K;
  constexpr int variant = PREC == MFA_PREC_BF16 ? 1 : 0;
  const int t = threadIdx.x;
  const int lane = t & 31;
  const int line = (t >> 5) * S::LANES + lane;  // the batch's lines, cell by cell
  const int cl = line / L, l = line - cl * L;
  const int la = l % N, lb = l / N;
  const int64_t c0 = batch * CB;
  const int ncb = (int)(a.count - c0 < CB ? a.count - c0 : CB);  // cells in this batch
  const bool valid = lane < S::LANES && cl < ncb;
  constexpr int PS = S::PS;
  using Y = LLayout<N>;
  // Four planes of CB cells (PS floats each, layout LLayout): U (gathered input, then B_y's output, then the
  // x-derivative, then the B^T results), V (values at the Gauss points, then the test-side accumulation), F0 and F1 (z- and
  // y-derivatives and their fluxes).  A thread without a line of this batch works on no plane.
  float* U0 = smem;
  float* V0 = U0 + CB * PS;
  float* F00 = V0 + CB * PS;
  float* F10 = F00 + CB * PS;
  const int cp = valid ? cl : 0;
  float* U = U0 + cp * PS;
  float* V = V0 + cp * PS;
  float* F0 = F00 + cp * PS;
  float* F1 = F10 + cp * PS;

  // gather, point-parallel: point i of the batch is local point i % P of cell c0 + i / P
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (t + k * T < ncb * S::P) U0[Y::of(t + k * T)] = xin[k];
  __syncthreads();
  if (valid) sweep<N, 2, 0, false, false, variant>(U, V, la, lb);  // B in z
  __syncthreads();
  if (valid) sweep<N, 1, 0, false, false, variant>(V, U, la, lb);  // B in y
  __syncthreads();
  if constexpr (KIND != MFA_FORM_MASS) {
    if (valid) sweep_bd_x<N, variant>(U, V, U, la, lb);  // B in x (values, into V), D in x (into U's plane)
    __syncthreads();
    if (valid) {
      sweep<N, 1, 1, false, false, variant>(V, F1, la, lb);  // D in y
      sweep<N, 2, 1, false, false, variant>(V, F0, la, lb);  // D in z
    }
  }
  // the next batch's x: its nodes were requested at the start of this batch and have arrived by now
  if (next >= 0) line_load_x<TX, K>(an->x, node_next, xin, variant == 1);
  // this batch's factors: from the stage (bulk copies) or straight from global memory
  if constexpr (STG) {
    if (!mbar_wait(st.bar, st.phase)) {
      atomicOr(a.err, 4);
      *st.abort = 1;
    }
    st.phase ^= 1u;
  }
  __syncthreads();
  if constexpr (STG) {
    if (*st.abort) return false;
  }
  const void* gs = STG ? static_cast<const void*>(st.buf)
                       : static_cast<const void*>(static_cast<const GeoT<PREC>*>(a.geom) + c0 * a.gstride);
  const int64_t gc = (int64_t)cp * a.gstride;
  if constexpr (KIND == MFA_FORM_MASS) {
    if (valid) fused_x_mass<N, PREC, STG, variant>(U, V, gs, gc, la, lb);  // B_x, w|J|, B_x^T: into V
  } else {
    if (valid) fused_x<N, KIND, PREC, STG, variant>(gs, gc, F0, F1, V, U, la, lb);  // r = c0 w|J| u + D_x^T f0
  }
  __syncthreads();
  // the stage is free: start the next batch's factors now
  if (t == 0 && next >= 0) issue_factors<N, KIND, PREC, STG, CBX>(*an, next, st);
  float* R0;  // plane of the result
  int32_t snode[K];  // nodes of this thread's points, for the scatter
  if constexpr (!line_reload_nodes<N>()) {
#pragma unroll
    for (int k = 0; k < K; ++k) snode[k] = node[k];
  }
  if constexpr (KIND != MFA_FORM_MASS) {
    if (valid) sweep<N, 1, 1, true, true, variant>(F1, V, la, lb);  // + D_y^T f1
    __syncthreads();
    if (valid) sweep_dtbt_z<N, variant>(F0, V, U, la, lb);          // B^T in z of (r + D_z^T f2)
    __syncthreads();
    if (valid) sweep<N, 1, 0, true, false, variant>(U, V, la, lb);  // B^T in y
    __syncthreads();
    if constexpr (line_reload_nodes<N>()) line_load_nodes<N, CBX>(a.cell_node, a.count, batch, snode);
    if (valid) sweep<N, 0, 0, true, false, variant>(V, U, la, lb);  // B^T in x
    R0 = U0;
  } else {
    if (valid) sweep<N, 1, 0, true, false, variant>(V, U, la, lb);  // B^T in y
    __syncthreads();
    if constexpr (line_reload_nodes<N>()) line_load_nodes<N, CBX>(a.cell_node, a.count, batch, snode);
    if (valid) sweep<N, 2, 0, true, false, variant>(U, V, la, lb);  // B^T in z
    R0 = V0;
  }
  __syncthreads();
  // scatter-add, point-parallel
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (snode[k] < 0) continue;
    if constexpr (sizeof(TX) == 8) add_y(static_cast<double*>(a.y), snode[k], R0[Y::of(t + k * T)]);
    else add_y(static_cast<float*>(a.y), snode[k], R0[Y::of(t + k * T)]);
  }
  __syncthreads();
  return true;
}

// The stage holds CB factor blocks of the largest stride line_geom_stride may choose (the launchers refuse a
// larger one).
template <int N, int PREC, int CBX = 0>
__host__ __device__ constexpr int stage_bytes(int ng) {
  return LShape<N, CBX>::CB * (int)line_geom_stride_max(N, ng, PREC == MFA_PREC_BF16 ? 2 : 4) *
         (PREC == MFA_PREC_BF16 ? 2 : 4);
}

// The stage starts 128-byte aligned (bulk copies need a 16-byte aligned destination).
template <int N, int CBX = 0>
__host__ __device__ constexpr int stage_offset() {
  return (LShape<N, CBX>::SMEM + 127) / 128 * 128;
}

template <int N, int KIND, int PREC, bool STG = staged<PREC>(), int CBX = 0>
__host__ __device__ constexpr int line_smem() {
  return STG ? stage_offset<N, CBX>() + stage_bytes<N, PREC, CBX>(geom_entries<KIND>()) + 16 : LShape<N, CBX>::SMEM;
}

// Blocks per SM that shared memory and the thread count allow, at most 4: the register budget of the grouped
// launches' __launch_bounds__, so that registers do not cut their occupancy below it (4 blocks of 256 threads:
// 64 registers; the 64-operator FP32 batch ran 12% faster with it, its Q7/Q8 groups going from 3 to 4 blocks
// per SM).  The single-operator kernel has no such bound: there it measured 1-10% slower on Q3-Q6, whose
// registers did not limit occupancy.
template <int N, int KIND, int PREC, bool STG = staged<PREC>(), int CBX = 0>
__host__ __device__ constexpr int line_min_blocks() {
  constexpr int by_smem = (228 * 1024) / (line_smem<N, KIND, PREC, STG, CBX>() + 1024);
  constexpr int by_threads = 2048 / LShape<N, CBX>::T;
  constexpr int m = by_smem < by_threads ? by_smem : by_threads;
  return m < 1 ? 1 : (m > 4 ? 4 : m);
}

template <int N, int KIND, int PREC, bool STG = staged<PREC>(), int CBX = 0>
__device__ __forceinline__ void stage_setup(float* smem, Stage& st, int* abort) {
  st.buf = reinterpret_cast<unsigned char*>(smem) + stage_offset<N, CBX>();
  st.bar = reinterpret_cast<uint64_t*>(st.buf + stage_bytes<N, PREC, CBX>(geom_entries<KIND>()));
  st.phase = 0;
  st.abort = abort;
  if (threadIdx.x == 0) {
    *abort = 0;
    if constexpr (STG) mbar_init(st.bar);
  }
  __syncthreads();
}

template <int N, int KIND, int PREC, typename TX, bool STG = staged<PREC>(), int CBX = 0>
__global__ void __launch_bounds__(LShape<N, CBX>::T) line_apply_kernel(const LineArgs a) {
  extern __shared__ __align__(128) float smem_l[];
  __shared__ int abort_flag;
  Stage st;
  stage_setup<N, KIND, PREC, STG, CBX>(smem_l, st, &abort_flag);
  using S = LShape<N, CBX>;
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if ((int64_t)blockIdx.x < nbatch && threadIdx.x == 0) issue_factors<N, KIND, PREC, STG, CBX>(a, blockIdx.x, st);
  int32_t node[line_reload_nodes<N>() ? 1 : S::K], nodes_next[S::K];
  float xin[S::K];
  if ((int64_t)blockIdx.x < nbatch) {
    line_load_nodes<N, CBX>(a.cell_node, a.count, blockIdx.x, nodes_next);
    line_load_x<TX, S::K>(a.x, nodes_next, xin, PREC == MFA_PREC_BF16);
  }
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int64_t next = batch + gridDim.x < nbatch ? batch + gridDim.x : -1;
    if constexpr (!line_reload_nodes<N>()) {
#pragma unroll
      for (int k = 0; k < S::K; ++k) node[k] = nodes_next[k];
    }
    if (next >= 0) line_load_nodes<N, CBX>(a.cell_node, a.count, next, nodes_next);
    if (!line_batch<N, KIND, PREC, TX, STG, CBX>(a, batch, smem_l, st, &a, next, node, nodes_next, xin)) return;
  }
}

// The grouped launches have no tuner: FP32 groups read their factors straight from global memory (coalesced on
// x-lines; the 64-operator batch measured that faster than staging, whose FP32 blocks cost occupancy); BF16
// groups stage them.
template <int PREC>
__host__ __device__ constexpr bool group_staged() {
  return PREC == MFA_PREC_BF16;
}

template <int N, int KIND, int PREC>
__global__ void __launch_bounds__(LShape<N>::T, (line_min_blocks<N, KIND, PREC, group_staged<PREC>()>()))
    line_group_kernel(const HexApplyArgs* __restrict__ items,
                                                                  const int64_t* __restrict__ first, int nitems) {
  extern __shared__ __align__(128) float smem_l[];
  __shared__ int abort_flag;
  constexpr bool STG = group_staged<PREC>();
  Stage st;
  stage_setup<N, KIND, PREC, STG>(smem_l, st, &abort_flag);
  const int64_t total = first[nitems];
  auto args_of = [&](int k) {
    const HexApplyArgs h = items[k];
    return LineArgs{h.x, h.y, h.cell_node, h.geom, h.count, h.geom_stride, h.err};
  };
  constexpr int K = LShape<N>::K;
  int32_t node[line_reload_nodes<N>() ? 1 : K], nodes_next[K];
  float xin[K];
  int k = 0;
  if ((int64_t)blockIdx.x < total) {
    while (k + 1 < nitems && (int64_t)blockIdx.x >= first[k + 1]) ++k;
    const LineArgs a0 = args_of(k);
    if (threadIdx.x == 0) issue_factors<N, KIND, PREC, STG>(a0, blockIdx.x - first[k], st);
    line_load_nodes<N, 0>(a0.cell_node, a0.count, blockIdx.x - first[k], nodes_next);
    line_load_x<double, K>(a0.x, nodes_next, xin, PREC == MFA_PREC_BF16);
  }
  for (int64_t gb = blockIdx.x; gb < total; gb += gridDim.x) {
    while (k + 1 < nitems && gb >= first[k + 1]) ++k;
    const LineArgs a = args_of(k);
    const int64_t gn = gb + gridDim.x;
    int kn = k;
    while (kn + 1 < nitems && gn >= first[kn + 1]) ++kn;
    const LineArgs an = args_of(kn < nitems ? kn : k);
    const int64_t next = gn < total ? gn - first[kn] : -1;
    if constexpr (!line_reload_nodes<N>()) {
#pragma unroll
      for (int j = 0; j < K; ++j) node[j] = nodes_next[j];
    }
    if (next >= 0) line_load_nodes<N, 0>(an.cell_node, an.count, next, nodes_next);
    if (!line_batch<N, KIND, PREC, double, STG>(a, gb - first[k], smem_l, st, &an, next, node, nodes_next, xin))
      return;
  }
}

template <typename Kern>
int occupancy(Kern kern, int threads, int smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int b = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem) != cudaSuccess || b < 1) b = 1;
  return b;
}

template <int N, int KIND, int PREC, typename TX, bool STG = staged<PREC>(), int CBX = 0>
cudaError_t launch_line(const LineArgs& a, GridBudget budget, cudaStream_t s) {
  using S = LShape<N, CBX>;
  constexpr int smem = line_smem<N, KIND, PREC, STG, CBX>();
  auto kern = line_apply_kernel<N, KIND, PREC, TX, STG, CBX>;
  if (a.gstride < (int64_t)(N * N * N) * geom_entries<KIND>() ||
      a.gstride > line_geom_stride_max(N, geom_entries<KIND>(), PREC == MFA_PREC_BF16 ? 2 : 4))
    return cudaErrorInvalidValue;
  static int bps = -1;
  if (bps < 0) bps = occupancy(kern, S::T, smem);
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t cap = budget.cap(bps);
  kern<<<(unsigned)(nbatch < cap ? nbatch : cap), S::T, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N, int KIND, int PREC>
cudaError_t launch_line_group(const HexApplyArgs* items, const int64_t* first, int nitems, int64_t total,
                              GridBudget budget, cudaStream_t s) {
  using S = LShape<N>;
  constexpr int smem = line_smem<N, KIND, PREC, group_staged<PREC>()>();
  auto kern = line_group_kernel<N, KIND, PREC>;
  static int bps = -1;
  if (bps < 0) bps = occupancy(kern, S::T, smem);
  if (total == 0) return cudaSuccess;
  const int64_t cap = budget.cap(bps);
  kern<<<(unsigned)(total < cap ? total : cap), S::T, smem, s>>>(items, first, nitems);
  return cudaGetLastError();
}

namespace {  // one copy per translation unit, like c_tab

std::mutex g_tab_mutex;
bool g_tab_ready[64] = {false};

// B (GLL basis at the Gauss points) and D (collocation derivative at the Gauss
// points) for every n, in float and rounded to bfloat16, into this unit's
// constant bank on the current device.
inline cudaError_t upload_tables() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  if (g_tab_ready[dev]) return cudaSuccess;
  std::vector<float> tab(2 * kTabFloats, 0.0f);
  for (int n = 2; n <= 9; ++n) {
    double gll[kMaxN], xg[kMaxN], wg[kMaxN], B[kMaxN * kMaxN], D[kMaxN * kMaxN];
    gll01(n, gll);
    gauss_legendre01(n, xg, wg);
    lagrange_matrix(n, gll, n, xg, B);
    collocation_derivative(n, xg, D);
    const int off = tab_offset(n);
    for (int i = 0; i < n * n; ++i) {
      tab[off + i] = (float)B[i];
      tab[off + n * n + i] = (float)D[i];
      tab[kTabFloats + off + i] = __bfloat162float(__double2bfloat16(B[i]));
      tab[kTabFloats + off + n * n + i] = __bfloat162float(__double2bfloat16(D[i]));
    }
  }
  e = cudaMemcpyToSymbol(c_tab, tab.data(), sizeof(float) * 2 * kTabFloats);
  if (e == cudaSuccess) g_tab_ready[dev] = true;
  return e;
}

}  // namespace

}  // namespace hexl
}  // namespace mfa
