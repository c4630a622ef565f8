// Locality-restoring renumbering of cells and nodes (reverse Cuthill-McKee).
//
// The paper's global assembly gathers and scatters through the cell->node
// map (Section 2.2); its cost depends on how close the nodes of consecutive
// cells are in memory.  Meshes from generators or partitioners often come in
// an arbitrary order.  This orders the cells by reverse Cuthill-McKee on the
// cell graph (two cells are adjacent when they share a vertex), then numbers
// the nodes in order of first touch along the new cell order, so that a
// block of consecutive cells reads and writes a compact window of x and y.
#include <algorithm>
#include <vector>

#include "mfa_internal.h"

namespace {

struct Csr {
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
};

// vertex -> cells
Csr vertex_cells(int64_t ncell, int nv, const int32_t* cell_vert, int64_t nvert) {
  Csr g;
  g.ptr.assign(nvert + 1, 0);
  for (int64_t i = 0; i < ncell * nv; ++i) g.ptr[cell_vert[i] + 1]++;
  for (int64_t v = 0; v < nvert; ++v) g.ptr[v + 1] += g.ptr[v];
  g.idx.resize(ncell * nv);
  std::vector<int64_t> pos(g.ptr.begin(), g.ptr.end() - 1);
  for (int64_t c = 0; c < ncell; ++c)
    for (int k = 0; k < nv; ++k) g.idx[pos[cell_vert[c * nv + k]]++] = (int32_t)c;
  return g;
}

// cell -> distinct neighbouring cells (sharing a vertex), sorted
Csr cell_graph(int64_t ncell, int nv, const int32_t* cell_vert, const Csr& vc) {
  Csr g;
  g.ptr.assign(ncell + 1, 0);
  std::vector<int32_t> mark(ncell, -1), nb;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int64_t c = 0; c < ncell; ++c) g.ptr[c + 1] += g.ptr[c];
      g.idx.resize(g.ptr[ncell]);
      std::fill(mark.begin(), mark.end(), -1);
    }
    for (int64_t c = 0; c < ncell; ++c) {
      nb.clear();
      for (int k = 0; k < nv; ++k) {
        const int32_t v = cell_vert[c * nv + k];
        for (int64_t e = vc.ptr[v]; e < vc.ptr[v + 1]; ++e) {
          const int32_t d = vc.idx[e];
          if (d != c && mark[d] != (int32_t)c) {
            mark[d] = (int32_t)c;
            nb.push_back(d);
          }
        }
      }
      if (pass == 0) {
        g.ptr[c + 1] = (int64_t)nb.size();
      } else {
        std::sort(nb.begin(), nb.end());
        std::copy(nb.begin(), nb.end(), g.idx.begin() + g.ptr[c]);
      }
    }
  }
  return g;
}

// Breadth-first order from `start` over the cells of its component not yet
// placed (done[c] == 0), neighbours by increasing degree (Cuthill-McKee).
// Cells met in this sweep get stamp[c] = id.  Returns the minimum-degree cell
// of the last level (a pseudo-peripheral candidate).
int32_t bfs(const Csr& g, int32_t start, const std::vector<char>& done, std::vector<int32_t>& stamp, int32_t id,
            std::vector<int32_t>& out) {
  auto seen = [&](int32_t c) { return done[c] || stamp[c] == id; };
  const size_t first = out.size();
  out.push_back(start);
  stamp[start] = id;
  std::vector<int32_t> nb;
  size_t head = first, level_begin = first;
  while (head < out.size()) {
    const size_t level_end = out.size();
    level_begin = head;
    for (; head < level_end; ++head) {
      const int32_t c = out[head];
      nb.clear();
      for (int64_t e = g.ptr[c]; e < g.ptr[c + 1]; ++e)
        if (!seen(g.idx[e])) nb.push_back(g.idx[e]);
      std::stable_sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
        return g.ptr[a + 1] - g.ptr[a] < g.ptr[b + 1] - g.ptr[b];
      });
      for (int32_t d : nb) {
        stamp[d] = id;
        out.push_back(d);
      }
    }
  }
  int32_t best = out[level_begin];
  for (size_t i = level_begin; i < out.size(); ++i)
    if (g.ptr[out[i] + 1] - g.ptr[out[i]] < g.ptr[best + 1] - g.ptr[best]) best = out[i];
  return best;
}

}  // namespace

extern "C" int mfa_order_rcm(int64_t ncell, int nv, const int32_t* cell_vert, int64_t nvert, int nloc,
                             const int32_t* cell_node, int64_t nnode, int32_t* cell_order, int32_t* node_perm) {
  if (ncell < 0 || nvert < 0 || nnode < 0 || (nv != 4 && nv != 8) || nloc < 1 || ncell >= (int64_t)1 << 31 ||
      nnode >= (int64_t)1 << 31 || (ncell > 0 && (!cell_vert || !cell_node || !cell_order)) ||
      (nnode > 0 && !node_perm))
    return mfa::set_error(MFA_ERR_ARG, "mfa_order_rcm: bad argument");
  for (int64_t i = 0; i < ncell * nv; ++i)
    if (cell_vert[i] < 0 || cell_vert[i] >= nvert) return mfa::set_error(MFA_ERR_RANGE, "mfa_order_rcm: vertex index");
  for (int64_t i = 0; i < ncell * nloc; ++i)
    if (cell_node[i] < 0 || cell_node[i] >= nnode) return mfa::set_error(MFA_ERR_RANGE, "mfa_order_rcm: node index");
  const Csr vc = vertex_cells(ncell, nv, cell_vert, nvert);
  const Csr g = cell_graph(ncell, nv, cell_vert, vc);
  std::vector<char> done(ncell, 0);
  std::vector<int32_t> stamp(ncell, -1), order, comp;
  order.reserve(ncell);
  int32_t id = 0;
  for (int64_t c0 = 0; c0 < ncell; ++c0) {
    if (done[c0]) continue;
    // start of this component: its minimum-degree cell, refined by two BFS sweeps
    comp.clear();
    bfs(g, (int32_t)c0, done, stamp, id++, comp);
    int32_t start = comp[0];
    for (int32_t c : comp)
      if (g.ptr[c + 1] - g.ptr[c] < g.ptr[start + 1] - g.ptr[start]) start = c;
    for (int sweep = 0; sweep < 2; ++sweep) {
      comp.clear();
      start = bfs(g, start, done, stamp, id++, comp);
    }
    const size_t before = order.size();
    bfs(g, start, done, stamp, id++, order);
    for (size_t i = before; i < order.size(); ++i) done[order[i]] = 1;
  }
  std::reverse(order.begin(), order.end());
  for (int64_t i = 0; i < ncell; ++i) cell_order[i] = order[i];
  // nodes by first touch along the new cell order
  std::fill(node_perm, node_perm + nnode, -1);
  int32_t next = 0;
  for (int64_t i = 0; i < ncell; ++i)
    for (int a = 0; a < nloc; ++a) {
      const int32_t v = cell_node[(int64_t)order[i] * nloc + a];
      if (node_perm[v] < 0) node_perm[v] = next++;
    }
  for (int64_t v = 0; v < nnode; ++v)
    if (node_perm[v] < 0) node_perm[v] = next++;  // nodes of no cell keep a place at the end
  return MFA_OK;
}
