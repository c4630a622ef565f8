// Dispatch of the FP32 and BF16 hex action to the line-per-thread kernels
// (hex_lines.cuh), split over two translation units by degree.
#include <algorithm>
#include <vector>

#include "hex_lines.cuh"

namespace mfa {

cudaError_t hex_line_apply_a(int n, int kind, int prec, bool f32vec, const hexl::LineArgs& a, GridBudget budget,
                             cudaStream_t s);
cudaError_t hex_line_apply_b(int n, int kind, int prec, bool f32vec, const hexl::LineArgs& a, GridBudget budget,
                             cudaStream_t s);
cudaError_t hex_line_group_a(int n, int kind, int prec, const HexApplyArgs* items, const int64_t* first, int nitems,
                             int64_t total, GridBudget budget, cudaStream_t s);
cudaError_t hex_line_group_b(int n, int kind, int prec, const HexApplyArgs* items, const int64_t* first, int nitems,
                             int64_t total, GridBudget budget, cudaStream_t s);

cudaError_t hex_line_tuned_a(int n, int kind, int prec, bool stg, int cb, const hexl::LineArgs& a, GridBudget budget,
                             cudaStream_t s);
cudaError_t hex_line_tuned_b(int n, int kind, int prec, bool stg, int cb, const hexl::LineArgs& a, GridBudget budget,
                             cudaStream_t s);

// The factor block's stride: the line kernels' pointwise step reads, at each
// point x = m of a thread's x-line, element (cell c, entry e) at
// c stride + e n^3 + l + n^2 m (l: the line within its cell), the lines of a
// warp going cell by cell, line_lanes(n) to a warp.  For each candidate stride
// (the base plus 0..kLineGeomPadMax 16-byte units) this counts, over a run of
// cells and every entry and point, the 4-byte shared-memory words each warp
// load touches in its busiest bank, and keeps the stride with the fewest (the
// smallest on ties).  Deterministic: the same n, ng and element size always
// give the same stride.
int64_t line_geom_stride(int n, int ng, int esz) {
  const int64_t base = line_geom_stride_base(n, ng, esz), unit = 16 / esz;
  const int P = n * n * n, L = n * n, lanes = line_lanes(n), cells = 32;
  int64_t best = base, best_cost = -1;
  std::vector<int64_t> words;
  int count[32];
  for (int k = 0; k <= kLineGeomPadMax; ++k) {
    const int64_t gsd = base + k * unit;
    int64_t cost = 0;
    for (int w0 = 0; w0 < cells * L; w0 += lanes)
      for (int e = 0; e < ng; ++e)
        for (int m = 0; m < n; ++m) {
          words.clear();
          for (int j = 0; j < lanes && w0 + j < cells * L; ++j) {
            const int line = w0 + j, c = line / L, l = line - c * L;
            words.push_back((c * gsd + (int64_t)e * P + l + (int64_t)L * m) * esz / 4);
          }
          std::sort(words.begin(), words.end());
          words.erase(std::unique(words.begin(), words.end()), words.end());
          for (int& v : count) v = 0;
          int busiest = 0;
          for (int64_t wd : words) busiest = std::max(busiest, ++count[wd % 32]);
          cost += busiest;
        }
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = gsd;
    }
  }
  return best;
}

// Default (256-thread target), then the 512-thread target (hex_lines_tune_*.cu).
int hex_line_cb_options(int n, int* out) {
  if (n < 2 || n > 9) return 0;
  out[0] = line_cb_for(n, 256);
  out[1] = line_cb_for(n, 512);
  return 2;
}

cudaError_t hex_apply_launch_mixed(int n, int nq, int kind, int prec, bool colour, const LaunchConfig& lc,
                                   const HexTables&, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  if (nq != n || colour || a.cell_list) return cudaErrorInvalidValue;
  const int variant = lc.variant == MFA_VARIANT_AUTO ? hex_default_variant(n, nq, prec) : lc.variant;
  if (variant != MFA_VARIANT_LINE && variant != MFA_VARIANT_LINE_STAGED) return cudaErrorInvalidValue;
  const bool stg = variant == MFA_VARIANT_LINE_STAGED;
  const bool stg_default = prec == MFA_PREC_BF16 ? hexl::staged<MFA_PREC_BF16>() : hexl::staged<MFA_PREC_FP32>();
  const hexl::LineArgs la{a.x, a.y, a.cell_node, a.geom, a.count, a.geom_stride, a.err};
  if (stg == stg_default && (lc.cb == 0 || lc.cb == line_cb_for(n, 256)))
    return n <= 5 ? hex_line_apply_a(n, kind, prec, false, la, budget, s)
                  : hex_line_apply_b(n, kind, prec, false, la, budget, s);
  const int cb = lc.cb == 0 ? line_cb_for(n, 256) : lc.cb;
  return n <= 5 ? hex_line_tuned_a(n, kind, prec, stg, cb, la, budget, s)
                : hex_line_tuned_b(n, kind, prec, stg, cb, la, budget, s);
}

cudaError_t hex_apply_launch_f32(int n, int kind, int prec, const float* x, float* y, const int32_t* cell_node,
                                 const void* geom, int64_t count, int64_t gstride, int* err, GridBudget budget,
                                 cudaStream_t s) {
  const hexl::LineArgs la{x, y, cell_node, geom, count, gstride, err};
  return n <= 5 ? hex_line_apply_a(n, kind, prec, true, la, budget, s)
                : hex_line_apply_b(n, kind, prec, true, la, budget, s);
}

cudaError_t hex_group_launch_mixed(int n, int kind, int prec, const HexTables&, const HexApplyArgs* items,
                                   const int64_t* first, int nitems, int64_t total, GridBudget budget, cudaStream_t s) {
  return n <= 5 ? hex_line_group_a(n, kind, prec, items, first, nitems, total, budget, s)
                : hex_line_group_b(n, kind, prec, items, first, nitems, total, budget, s);
}

}  // namespace mfa
