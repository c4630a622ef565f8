// FP64 sum-factorised hex action with even-odd split 1D contractions.
//
// The FP64 pipe bounds the hex action on GB300, so the only way to go faster
// is fewer FP64 instructions.  The GLL nodes and the Gauss points are both
// symmetric about 1/2, hence the 1D matrices have a mirror symmetry:
// B[i][j] = B[n-1-i][n-1-j] (centrosymmetric) and D[i][j] = -D[n-1-i][n-1-j]
// (anti-centrosymmetric), and so do their transposes.  Writing the input of a
// line as even and odd parts e_j = v_j + v_{n-1-j}, o_j = v_j - v_{n-1-j}
// (j < n/2), an n x n product splits into two (n/2) x (n/2) products:
//
//   pe_i = sum_j E[i][j] e_j (+ S[i][mid] v_mid),  po_i = sum_j O[i][j] o_j,
//   out_i = pe_i + po_i,  out_{n-1-i} = sigma (pe_i - po_i),
//
// with E = (S[i][j] + S[i][n-1-j]) / 2, O = (S[i][j] - S[i][n-1-j]) / 2 and
// sigma = +1 for B, -1 for D.  The odd products accumulate onto pe_i, which
// gives out_i without an addition, and the mirror output is then one FMA,
// sigma (2 pe_i - out_i).  For n = 5 this is 19 instead of 25 FP64
// instructions per line, for n = 7 34 instead of 49, for n = 9 53 instead of 81.
// The FP64 pipe retires one warp instruction per SM sub-partition only every
// few dozen cycles, so instruction count, not dependency depth, sets the time.
// The sweep order and the pointwise physics are those of hex_kernels.cuh;
// one thread owns one line per direction, the table entries are
// compile-time offsets into __constant__ memory (FMA operands), and the
// gather, the geometric-factor reads and the scatter run point-parallel.
#pragma once

#include <mutex>
#include <vector>

#include "mfa_internal.h"

namespace mfa {
namespace hexeo {

// Split table of one n x n matrix: E [h][h], O [h][h], Mc [h] = S[i][mid],
// Mr [h+1] = (S[mid][j], j < h; S[mid][mid]).
__host__ __device__ constexpr int split_size(int n) { return 2 * (n / 2) * (n / 2) + (n / 2) + (n / 2) + 1; }
// Six matrices per n, n = 5..9: 0: B, 1: B^T, 2: D, 3: D^T, 4: D for the fused B/D sweep along z (E, O and
// Mr doubled, Mc as for D), 5: D^T for the fused D^T/B^T sweep along z (E, O and Mc doubled, Mr as for D^T).
constexpr int kMats = 6;
__host__ __device__ constexpr int tab_offset(int n, int mat) {
  int off = 0;
  for (int k = 5; k < n; ++k) off += kMats * split_size(k);
  return off + mat * split_size(n);
}
constexpr int kTabDoubles = tab_offset(10, 0);

static __constant__ double c_eo[kTabDoubles];

constexpr int ceil32(int x) { return (x + 31) / 32 * 32; }

// Cells per block for a target block size (the default targets 256 threads).
constexpr int eo_cb_for(int n, int target) { return cells_for_target(n * n, target); }

template <int N, int CBX = 0>
struct EShape {
  static constexpr int L = N * N;
  static constexpr int P = N * N * N;
  static constexpr int CB = CBX > 0 ? CBX : eo_cb_for(N, 256);
  static constexpr int T = ceil32(CB * L);
  static constexpr int SMEM = 4 * CB * P * 8;
  static constexpr int K = (CB * P + T - 1) / T;  // points per thread in the point-parallel phases
  // blocks per SM that shared memory allows (228 KB per SM, 1 KB reserved per block): the register
  // budget of __launch_bounds__, so that registers never cut occupancy below it
  static constexpr int MINB0 = (228 * 1024) / (SMEM + 1024);
  static constexpr int MINB = MINB0 < 1 ? 1 : (MINB0 * T > 2048 ? 2048 / T : MINB0);
};

// Node of each of this thread's points of batch `batch` (-1 past the batch's end).
template <int N, int CBX>
__device__ __forceinline__ void eo_load_nodes(const HexApplyArgs& a, int64_t batch, int32_t (&node)[EShape<N, CBX>::K]) {
  using S = EShape<N, CBX>;
  const int64_t c0 = batch * S::CB;
  const int ncb = (int)(a.count - c0 < S::CB ? a.count - c0 : S::CB);
#pragma unroll
  for (int k = 0; k < S::K; ++k) {
    const int i = threadIdx.x + k * S::T;
    node[k] = -1;
    if (i < ncb * S::P) {
      const int c = i / S::P, q = i - c * S::P;
      const int64_t cell = a.cell_list ? (int64_t)__ldg(a.cell_list + c0 + c) : c0 + c;
      node[k] = __ldg(a.cell_node + cell * S::P + q);
    }
  }
}

template <int KIND>
__host__ __device__ constexpr int geom_entries() {
  return KIND == MFA_FORM_MASS ? 1 : (KIND == MFA_FORM_LAPLACE ? 6 : 7);
}

template <int N, int DIR>
__device__ __forceinline__ int at(int a, int b, int m) {
  if constexpr (DIR == 0) return m + N * (a + N * b);
  else if constexpr (DIR == 1) return a + N * (m + N * b);
  else return a + N * (b + N * m);
}

// out (+)= S v along direction DIR of line (a, b); MAT selects S, SIGMA its mirror sign.
template <int N, int DIR, int MAT, int SIGMA, bool ACC>
__device__ __forceinline__ void eo_sweep(const double* in, double* out, int a, int b) {
  constexpr int H = N / 2;
  constexpr bool ODD = (N & 1) != 0;
  constexpr int base = tab_offset(N, MAT);
  constexpr int oE = base, oO = base + H * H, oMc = base + 2 * H * H, oMr = oMc + H;
  double v[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = in[at<N, DIR>(a, b, m)];
  double e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j] + v[N - 1 - j];
    o[j] = v[j] - v[N - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double pe = 0.0;
    if constexpr (ODD) pe = c_eo[oMc + i] * v[H];
#pragma unroll
    for (int j = 0; j < H; ++j) pe = fma(c_eo[oE + i * H + j], e[j], pe);
    double lo = pe;  // pe + po
#pragma unroll
    for (int j = 0; j < H; ++j) lo = fma(c_eo[oO + i * H + j], o[j], lo);
    const double hi = SIGMA > 0 ? fma(2.0, pe, -lo) : fma(-2.0, pe, lo);  // sigma (pe - po)
    if constexpr (ACC) {
      out[at<N, DIR>(a, b, i)] += lo;
      out[at<N, DIR>(a, b, N - 1 - i)] += hi;
    } else {
      out[at<N, DIR>(a, b, i)] = lo;
      out[at<N, DIR>(a, b, N - 1 - i)] = hi;
    }
  }
  if constexpr (ODD) {
    double s = SIGMA > 0 ? c_eo[oMr + H] * v[H] : 0.0;  // the middle diagonal of D is zero
#pragma unroll
    for (int j = 0; j < H; ++j) s = fma(c_eo[oMr + j], SIGMA > 0 ? e[j] : o[j], s);
    if constexpr (ACC) out[at<N, DIR>(a, b, H)] += s;
    else out[at<N, DIR>(a, b, H)] = s;
  }
}

// B then D along z on the thread's own z-line: vout = B u (values at the Gauss points), dout = D B u.  The
// even and odd parts of B u along z are 2 pe and 2 po of the B product (and its middle value), so the D
// product starts from them with the doubled split table (matrix 4) and needs no additions of its own before
// its products.  `dout` may alias `in`.
template <int N>
__device__ __forceinline__ void eo_sweep_bd_z(const double* in, double* vout, double* dout, int a, int b) {
  constexpr int H = N / 2;
  constexpr bool ODD = (N & 1) != 0;
  constexpr int bB = tab_offset(N, 0), bD = tab_offset(N, 4);
  constexpr int oEB = bB, oOB = bB + H * H, oMcB = bB + 2 * H * H, oMrB = oMcB + H;
  constexpr int oED = bD, oOD = bD + H * H, oMcD = bD + 2 * H * H, oMrD = oMcD + H;
  double v[N];
#pragma unroll
  for (int m = 0; m < N; ++m) v[m] = in[at<N, 2>(a, b, m)];
  double e[H], o[H], pe[H], po[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j] + v[N - 1 - j];
    o[j] = v[j] - v[N - 1 - j];
  }
  double mid = 0.0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double se = 0.0, so = 0.0;
    if constexpr (ODD) se = c_eo[oMcB + i] * v[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      se = fma(c_eo[oEB + i * H + j], e[j], se);
      so = fma(c_eo[oOB + i * H + j], o[j], so);
    }
    pe[i] = se;
    po[i] = so;
    vout[at<N, 2>(a, b, i)] = se + so;
    vout[at<N, 2>(a, b, N - 1 - i)] = se - so;
  }
  if constexpr (ODD) {
    double sm = c_eo[oMrB + H] * v[H];
#pragma unroll
    for (int j = 0; j < H; ++j) sm = fma(c_eo[oMrB + j], e[j], sm);
    mid = sm;
    vout[at<N, 2>(a, b, H)] = sm;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {  // D (anti-centrosymmetric): out_i = se + so, out_{n-1-i} = so - se
    double se = 0.0;
    if constexpr (ODD) se = c_eo[oMcD + i] * mid;
#pragma unroll
    for (int j = 0; j < H; ++j) se = fma(c_eo[oED + i * H + j], pe[j], se);
    double lo = se;
#pragma unroll
    for (int j = 0; j < H; ++j) lo = fma(c_eo[oOD + i * H + j], po[j], lo);
    dout[at<N, 2>(a, b, i)] = lo;
    dout[at<N, 2>(a, b, N - 1 - i)] = fma(-2.0, se, lo);
  }
  if constexpr (ODD) {  // the middle diagonal of D is zero
    double sm = 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j) sm = fma(c_eo[oMrD + j], po[j], sm);
    dout[at<N, 2>(a, b, H)] = sm;
  }
}

// The test side along z in one pass: out = B^T (acc + D^T f) on the thread's own z-line.  With lo, hi the
// D^T product's outputs (lo = pe + po, hi = po - pe), the even and odd parts of acc + D^T f are
// (acc_j + acc_{n-1-j}) + 2 po_j and (acc_j - acc_{n-1-j}) + 2 pe_j.  The D^T table with E, O and Mc
// doubled (matrix 5) lets each product chain start from the accumulator's sum or difference: one addition
// per half, where adding, recombining and splitting take six operations per pair.  `out` may alias `f`.
template <int N>
__device__ __forceinline__ void eo_sweep_dtbt_z(const double* f, const double* acc, double* out, int a, int b) {
  constexpr int H = N / 2;
  constexpr bool ODD = (N & 1) != 0;
  constexpr int bT = tab_offset(N, 5), bB = tab_offset(N, 1);
  constexpr int oET = bT, oOT = bT + H * H, oMcT = bT + 2 * H * H, oMrT = oMcT + H;
  constexpr int oEB = bB, oOB = bB + H * H, oMcB = bB + 2 * H * H, oMrB = oMcB + H;
  double v[N], ac[N];
#pragma unroll
  for (int m = 0; m < N; ++m) {
    v[m] = f[at<N, 2>(a, b, m)];
    ac[m] = acc[at<N, 2>(a, b, m)];
  }
  double e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[j] + v[N - 1 - j];
    o[j] = v[j] - v[N - 1 - j];
  }
  double te[H], to[H], tmid = 0.0;  // even and odd parts of t = acc + D^T f
#pragma unroll
  for (int i = 0; i < H; ++i) {
    double od = ac[i] - ac[N - 1 - i];  // + 2 pe_i
    if constexpr (ODD) od = fma(c_eo[oMcT + i], v[H], od);
#pragma unroll
    for (int j = 0; j < H; ++j) od = fma(c_eo[oET + i * H + j], e[j], od);
    double ev = ac[i] + ac[N - 1 - i];  // + 2 po_i
#pragma unroll
    for (int j = 0; j < H; ++j) ev = fma(c_eo[oOT + i * H + j], o[j], ev);
    te[i] = ev;
    to[i] = od;
  }
  if constexpr (ODD) {  // middle of D^T f: the middle diagonal of D^T is zero
    double sm = ac[H];
#pragma unroll
    for (int j = 0; j < H; ++j) sm = fma(c_eo[oMrT + j], o[j], sm);
    tmid = sm;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {  // B^T (centrosymmetric) on t
    double se = 0.0;
    if constexpr (ODD) se = c_eo[oMcB + i] * tmid;
#pragma unroll
    for (int j = 0; j < H; ++j) se = fma(c_eo[oEB + i * H + j], te[j], se);
    double lo = se;
#pragma unroll
    for (int j = 0; j < H; ++j) lo = fma(c_eo[oOB + i * H + j], to[j], lo);
    out[at<N, 2>(a, b, i)] = lo;
    out[at<N, 2>(a, b, N - 1 - i)] = fma(2.0, se, -lo);
  }
  if constexpr (ODD) {
    double sm = c_eo[oMrB + H] * tmid;
#pragma unroll
    for (int j = 0; j < H; ++j) sm = fma(c_eo[oMrB + j], te[j], sm);
    out[at<N, 2>(a, b, H)] = sm;
  }
}

// Four shared-memory planes of CB x n^3 doubles: U (gathered input, then the z-derivative and its flux, then
// the B^T results), V (values at the Gauss points, then the test-side accumulation), F0 and F1 (x- and
// y-derivatives and their fluxes).
// `node` holds the nodes of this thread's points (eo_load_nodes), loaded ahead
// of time: the gather and the scatter then wait on one load, not two.
template <int N, int KIND, bool COLOUR, int CBX = 0>
__device__ __forceinline__ void eo_batch(const HexApplyArgs& a, int64_t batch, double* smem,
                                         const int32_t (&node)[EShape<N, CBX>::K]) {
  using S = EShape<N, CBX>;
  constexpr int L = S::L, P = S::P, CB = S::CB, T = S::T, K = S::K, NG = geom_entries<KIND>();
  const int t = threadIdx.x;
  const int cl = t / L, l = t - cl * L;
  const int la = l % N, lb = l / N;
  const int64_t c0 = batch * CB;
  const int ncb = (int)(a.count - c0 < CB ? a.count - c0 : CB);
  const bool valid = cl < ncb;
  double* U0 = smem;
  double* V0 = U0 + CB * P;
  double* F00 = V0 + CB * P;
  double* F10 = F00 + CB * P;
  double* U = U0 + cl * P;
  double* V = V0 + cl * P;
  double* F0 = F00 + cl * P;
  double* F1 = F10 + cl * P;
  const double* geom = static_cast<const double*>(a.geom);
  auto cell_of = [&](int c) -> int64_t { return a.cell_list ? (int64_t)__ldg(a.cell_list + c0 + c) : c0 + c; };

#pragma unroll
  for (int k = 0; k < K; ++k)  // gather, point-parallel
    if (node[k] >= 0) U0[t + k * T] = __ldg(a.x + node[k]);
  __syncthreads();
  if (valid) eo_sweep<N, 0, 0, 1, false>(U, V, la, lb);  // B in x
  __syncthreads();
  if (valid) eo_sweep<N, 1, 0, 1, false>(V, U, la, lb);  // B in y
  __syncthreads();
  if constexpr (KIND == MFA_FORM_MASS) {
    if (valid) eo_sweep<N, 2, 0, 1, false>(U, V, la, lb);  // B in z: values at the Gauss points
    __syncthreads();
    for (int i = t; i < ncb * P; i += T) {
      const int c = i / P, q = i - c * P;
      V0[i] *= __ldg(geom + cell_of(c) * P + q);
    }
    __syncthreads();
    if (valid) eo_sweep<N, 2, 1, 1, false>(V, U, la, lb);  // B^T in z
  } else {
    if (valid) eo_sweep_bd_z<N>(U, V, U, la, lb);  // B in z (values, into V), D in z (into U's plane)
    __syncthreads();
    if (valid) {
      eo_sweep<N, 0, 2, -1, false>(V, F0, la, lb);  // D in x
      eo_sweep<N, 1, 2, -1, false>(V, F1, la, lb);  // D in y
    }
    __syncthreads();
    for (int i = t; i < ncb * P; i += T) {  // pointwise physics, point-parallel
      const int c = i / P, q = i - c * P;
      const double* gc = geom + cell_of(c) * (int64_t)NG * P + q;
      double g[NG];
#pragma unroll
      for (int e = 0; e < NG; ++e) g[e] = __ldg(gc + (int64_t)e * P);
      const double d0 = F00[i], d1 = F10[i], d2 = U0[i];
      F00[i] = fma(g[0], d0, fma(g[3], d1, g[4] * d2));
      F10[i] = fma(g[3], d0, fma(g[1], d1, g[5] * d2));
      U0[i] = fma(g[4], d0, fma(g[5], d1, g[2] * d2));
      if constexpr (KIND == MFA_FORM_HELMHOLTZ) V0[i] *= g[6];
      else V0[i] = 0.0;
    }
    __syncthreads();
    if (valid) eo_sweep<N, 0, 3, -1, true>(F0, V, la, lb);  // + D_x^T f0
    __syncthreads();
    if (valid) eo_sweep<N, 1, 3, -1, true>(F1, V, la, lb);  // + D_y^T f1
    __syncthreads();
    if (valid) eo_sweep_dtbt_z<N>(U, V, U, la, lb);       // B^T in z of (r + D_z^T f2)
  }
  __syncthreads();
  if (valid) eo_sweep<N, 1, 1, 1, false>(U, V, la, lb);  // B^T in y
  __syncthreads();
  if (valid) eo_sweep<N, 0, 1, 1, false>(V, U, la, lb);  // B^T in x
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {  // scatter-add, point-parallel
    if (node[k] < 0) continue;
    if constexpr (COLOUR) a.y[node[k]] += U0[t + k * T];  // no other cell of this colour touches the node
    else atomicAdd(a.y + node[k], U0[t + k * T]);
  }
  __syncthreads();
}

template <int N, int KIND, bool COLOUR, int CBX = 0>
__global__ void __launch_bounds__(EShape<N, CBX>::T, EShape<N, CBX>::MINB) eo_apply_kernel(const HexApplyArgs a) {
  extern __shared__ __align__(16) double smem_eo[];
  using S = EShape<N, CBX>;
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  // the next batch's nodes are requested before this batch's work, so they arrive during it.  (Prefetching
  // the next batch's geometric factors into L2 as well gained 0.5% and raised DRAM reads by a quarter:
  // not done.)
  int32_t node[S::K], next[S::K];
  if (blockIdx.x < nbatch) eo_load_nodes<N, CBX>(a, blockIdx.x, next);
  for (int64_t batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
#pragma unroll
    for (int k = 0; k < S::K; ++k) node[k] = next[k];
    if (batch + gridDim.x < nbatch) eo_load_nodes<N, CBX>(a, batch + gridDim.x, next);
    eo_batch<N, KIND, COLOUR, CBX>(a, batch, smem_eo, node);
  }
}

template <int N, int KIND>
__global__ void __launch_bounds__(EShape<N>::T, EShape<N>::MINB) eo_group_kernel(const HexApplyArgs* __restrict__ items,
                                                                const int64_t* __restrict__ first, int nitems) {
  extern __shared__ __align__(16) double smem_eo[];
  const int64_t total = first[nitems];
  int k = 0;
  for (int64_t gb = blockIdx.x; gb < total; gb += gridDim.x) {
    while (k + 1 < nitems && gb >= first[k + 1]) ++k;
    const HexApplyArgs h = items[k];
    int32_t node[EShape<N>::K];
    eo_load_nodes<N, 0>(h, gb - first[k], node);
    eo_batch<N, KIND, false>(h, gb - first[k], smem_eo, node);
  }
}

namespace {  // one copy per translation unit, like c_eo

template <typename Kern>
int occupancy(Kern kern, int threads, int smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int b = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem) != cudaSuccess || b < 1) b = 1;
  return b;
}

template <int N, int KIND, bool COLOUR, int CBX = 0>
cudaError_t launch(const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  using S = EShape<N, CBX>;
  auto kern = eo_apply_kernel<N, KIND, COLOUR, CBX>;
  static int bps = -1;
  if (bps < 0) bps = occupancy(kern, S::T, S::SMEM);
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t cap = budget.cap(bps);
  kern<<<(unsigned)(nbatch < cap ? nbatch : cap), S::T, S::SMEM, s>>>(a);
  return cudaGetLastError();
}

std::mutex g_mutex;
bool g_ready[64] = {false};

// Split tables of B, B^T, D, D^T and the two doubled variants for n = 5..9 into this unit's constant bank.
inline cudaError_t upload_tables() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_ready[dev]) return cudaSuccess;
  std::vector<double> tab(kTabDoubles, 0.0);
  for (int n = 5; n <= 9; ++n) {
    double gll[kMaxN], xg[kMaxN], wg[kMaxN], B[kMaxN * kMaxN], D[kMaxN * kMaxN];
    gll01(n, gll);
    gauss_legendre01(n, xg, wg);
    lagrange_matrix(n, gll, n, xg, B);  // B[q][a]
    collocation_derivative(n, xg, D);   // D[q][r]
    const int h = n / 2;
    for (int mat = 0; mat < kMats; ++mat) {
      auto S = [&](int i, int j) {
        const double* M = (mat < 2) ? B : D;
        return (mat == 1 || mat == 3 || mat == 5) ? M[j * n + i] : M[i * n + j];  // 1, 3, 5: transposes
      };
      // matrix 4: D fed with the halves of an even-odd split (its middle input is whole); matrix 5: D^T whose
      // mirror-pair outputs are wanted doubled (its middle output is not)
      const double s_eo = mat >= 4 ? 2.0 : 1.0, s_mc = mat == 5 ? 2.0 : 1.0, s_mr = mat == 4 ? 2.0 : 1.0;
      double* o = tab.data() + tab_offset(n, mat);
      for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) {
          o[i * h + j] = s_eo * 0.5 * (S(i, j) + S(i, n - 1 - j));          // E
          o[h * h + i * h + j] = s_eo * 0.5 * (S(i, j) - S(i, n - 1 - j));  // O
        }
      if (n & 1) {
        for (int i = 0; i < h; ++i) o[2 * h * h + i] = s_mc * S(i, h);      // Mc
        for (int j = 0; j <= h; ++j) o[2 * h * h + h + j] = s_mr * S(h, j); // Mr
      }
    }
  }
  e = cudaMemcpyToSymbol(c_eo, tab.data(), sizeof(double) * kTabDoubles);
  if (e == cudaSuccess) g_ready[dev] = true;
  return e;
}

}  // namespace

}  // namespace hexeo
}  // namespace mfa
