// Cell -> node maps built from the vertex connectivity alone, and node
// positions.
//
// Section 2.2's global assembly reads the dofs of a cell through the
// cell2dof map.  For continuous Q_p (hex) and P_p (tet) spaces a node that
// lies on a vertex, edge or face is shared by every cell around it, and each
// cell sees it through its own local vertex order.  Each local node is given
// a key that does not depend on that order: the global ids of the vertices of
// its entity and its position measured in a frame fixed by those ids (edge:
// from the lower id; hex face: origin at the lowest id, first axis towards
// its lower-id neighbour; tet face: barycentric weights listed by increasing
// id).  Nodes are numbered by first appearance along the cell order, vertex
// nodes first as the mesh vertices.
#include <algorithm>
#include <array>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "mfa_internal.h"

namespace {

struct KeyHash {
  size_t operator()(const std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t>& k) const {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](int64_t v) {
      h ^= (uint64_t)v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    };
    mix(std::get<0>(k));
    mix(std::get<1>(k));
    mix(std::get<2>(k));
    mix(std::get<3>(k));
    mix(std::get<4>(k));
    return (size_t)h;
  }
};
using Key = std::tuple<int64_t, int64_t, int64_t, int64_t, int64_t>;

struct Numbering {
  std::unordered_map<Key, int32_t, KeyHash> ids;
  int32_t next;
  explicit Numbering(int32_t first) : next(first) {}
  int32_t get(const Key& k) {
    auto it = ids.find(k);
    if (it != ids.end()) return it->second;
    ids.emplace(k, next);
    return next++;
  }
};

// Q_p node (i, j, k) of a hex whose local vertex v sits at reference corner (v & 1, v >> 1 & 1, v >> 2 & 1).
int32_t hex_node_id(const int32_t* cv, int p, int i, int j, int k, int64_t cell, Numbering& num) {
  const int idx[3] = {i, j, k};
  int fixed = 0, bits = 0;
  for (int d = 0; d < 3; ++d)
    if (idx[d] == 0 || idx[d] == p) {
      ++fixed;
      if (idx[d] == p) bits |= 1 << d;
    }
  if (fixed == 3) return cv[bits];  // a vertex: its mesh id
  if (fixed == 2) {                 // an edge along the free axis f
    const int f = (idx[0] != 0 && idx[0] != p) ? 0 : ((idx[1] != 0 && idx[1] != p) ? 1 : 2);
    const int32_t A = cv[bits], B = cv[bits | (1 << f)];
    const int t = idx[f];
    return A < B ? num.get(Key{1, A, B, t, 0}) : num.get(Key{1, B, A, p - t, 0});
  }
  if (fixed == 1) {  // a face with free axes u < w
    int u = -1, w = -1;
    for (int d = 0; d < 3; ++d)
      if (idx[d] != 0 && idx[d] != p) {
        if (u < 0) u = d;
        else w = d;
      }
    // the four face vertices by their (bu, bw) bits
    int32_t V[2][2];
    for (int bu = 0; bu < 2; ++bu)
      for (int bw = 0; bw < 2; ++bw) V[bu][bw] = cv[bits | (bu << u) | (bw << w)];
    int ou = 0, ow = 0;  // origin: the lowest id
    for (int bu = 0; bu < 2; ++bu)
      for (int bw = 0; bw < 2; ++bw)
        if (V[bu][bw] < V[ou][ow]) ou = bu, ow = bw;
    int a = ou ? p - idx[u] : idx[u];  // coordinates from the origin
    int b = ow ? p - idx[w] : idx[w];
    const int32_t nu = V[1 - ou][ow], nw = V[ou][1 - ow];  // neighbours of the origin along u and w
    if (nw < nu) std::swap(a, b);                           // first axis towards the lower-id neighbour
    return num.get(Key{2, V[ou][ow], std::min(nu, nw), std::max(nu, nw), (int64_t)a * (p + 1) + b});
  }
  return num.get(Key{3, cell, i, j, k});  // interior
}

// Q_p node (i, j) of a quadrilateral whose local vertex v sits at reference corner (v & 1, v >> 1 & 1).
int32_t quad_node_id(const int32_t* cv, int p, int i, int j, int64_t cell, Numbering& num) {
  const bool ei = i == 0 || i == p, ej = j == 0 || j == p;
  if (ei && ej) return cv[(i == p ? 1 : 0) | (j == p ? 2 : 0)];
  if (ei || ej) {  // an edge along the free axis
    const int f = ei ? 1 : 0, fixed_bit = ei ? (i == p ? 1 : 0) : (j == p ? 2 : 0);
    const int32_t A = cv[fixed_bit], B = cv[fixed_bit | (1 << f)];
    const int tt = f == 0 ? i : j;
    return A < B ? num.get(Key{1, A, B, tt, 0}) : num.get(Key{1, B, A, p - tt, 0});
  }
  return num.get(Key{3, cell, i, j, 0});
}

// P_p node with barycentric weights b[3] (sum p) on the triangle's local vertices.
int32_t tri_node_id(const int32_t* cv, const int b[3], int64_t cell, Numbering& num) {
  int support[3], ns = 0;
  for (int s = 0; s < 3; ++s)
    if (b[s] > 0) support[ns++] = s;
  if (ns == 1) return cv[support[0]];
  if (ns == 3) return num.get(Key{3, cell, b[1], b[2], 0});
  std::pair<int32_t, int> sv[2] = {{cv[support[0]], b[support[0]]}, {cv[support[1]], b[support[1]]}};
  if (sv[1].first < sv[0].first) std::swap(sv[0], sv[1]);
  return num.get(Key{1, sv[0].first, sv[1].first, sv[0].second, 0});
}

// P_p node with barycentric weights b[4] (sum p) on the tet's local vertices.
int32_t tet_node_id(const int32_t* cv, int p, const int b[4], int64_t cell, Numbering& num) {
  int support[4], ns = 0;
  for (int s = 0; s < 4; ++s)
    if (b[s] > 0) support[ns++] = s;
  if (ns == 1) return cv[support[0]];
  if (ns == 4) return num.get(Key{3, cell, b[1], b[2], b[3]});
  // edge or face: the support vertices by increasing global id, with their weights
  std::pair<int32_t, int> sv[3];
  for (int r = 0; r < ns; ++r) sv[r] = {cv[support[r]], b[support[r]]};
  std::sort(sv, sv + ns);
  if (ns == 2) return num.get(Key{1, sv[0].first, sv[1].first, sv[0].second, 0});
  return num.get(Key{2, sv[0].first, sv[1].first, sv[2].first, (int64_t)sv[0].second * (p + 1) + sv[1].second});
}

// local P1/P2 order: vertices, then edges (0,1), (0,2), (0,3), (1,2), (1,3), (2,3); P3+: lattice (i, j, k)/p
void tet_local_weights(int p, std::vector<std::array<int, 4>>& out) {
  out.clear();
  if (p <= 2) {
    for (int v = 0; v < 4; ++v) {
      std::array<int, 4> b{0, 0, 0, 0};
      b[v] = p;
      out.push_back(b);
    }
    if (p == 2) {
      static const int ed[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
      for (auto& e : ed) {
        std::array<int, 4> b{0, 0, 0, 0};
        b[e[0]] = 1;
        b[e[1]] = 1;
        out.push_back(b);
      }
    }
    return;
  }
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j <= p - k; ++j)
      for (int i = 0; i <= p - k - j; ++i) out.push_back({p - i - j - k, i, j, k});
}

}  // namespace

extern "C" int mfa_build_cell_node(int cell_type, int degree, int64_t ncell, const int32_t* cell_vert, int64_t nvert,
                                   int32_t* cell_node, int64_t* nnode) {
  if ((cell_type != MFA_CELL_HEX8 && cell_type != MFA_CELL_TET4 && cell_type != MFA_CELL_TRI3 &&
       cell_type != MFA_CELL_QUAD4) ||
      ncell < 0 || nvert < 0 || !nnode || (ncell > 0 && (!cell_vert || !cell_node)))
    return mfa::set_error(MFA_ERR_ARG, "mfa_build_cell_node: bad argument");
  const bool hex = cell_type == MFA_CELL_HEX8, tensor = hex || cell_type == MFA_CELL_QUAD4;
  if ((tensor && (degree < 1 || degree > 8)) || (!tensor && (degree < 1 || degree > mfa::kTetMaxP)))
    return mfa::set_error(MFA_ERR_UNSUPPORTED, "mfa_build_cell_node: degree");
  const int nv = mfa::verts_of(cell_type);
  for (int64_t i = 0; i < ncell * nv; ++i)
    if (cell_vert[i] < 0 || cell_vert[i] >= nvert)
      return mfa::set_error(MFA_ERR_RANGE, "mfa_build_cell_node: vertex index outside [0, nvert)");
  Numbering num((int32_t)nvert);
  const int p = degree;
  if (hex) {
    const int n = p + 1, nl = n * n * n;
    for (int64_t c = 0; c < ncell; ++c) {
      const int32_t* cv = cell_vert + 8 * c;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) cell_node[c * nl + i + n * (j + n * k)] = hex_node_id(cv, p, i, j, k, c, num);
    }
  } else if (cell_type == MFA_CELL_QUAD4) {
    const int n = p + 1, nl = n * n;
    for (int64_t c = 0; c < ncell; ++c)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) cell_node[c * nl + i + n * j] = quad_node_id(cell_vert + 4 * c, p, i, j, c, num);
  } else if (cell_type == MFA_CELL_TRI3) {
    const int nl = mfa::tri_lattice_size(p);
    for (int64_t c = 0; c < ncell; ++c) {
      int a = 0;
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p - j; ++i, ++a) {
          const int b[3] = {p - i - j, i, j};
          cell_node[c * nl + a] = tri_node_id(cell_vert + 3 * c, b, c, num);
        }
    }
  } else {
    std::vector<std::array<int, 4>> w;
    tet_local_weights(p, w);
    const int nl = (int)w.size();
    for (int64_t c = 0; c < ncell; ++c)
      for (int a = 0; a < nl; ++a) cell_node[c * nl + a] = tet_node_id(cell_vert + 4 * c, p, w[a].data(), c, num);
  }
  if ((int64_t)num.next >= ((int64_t)1 << 31)) return mfa::set_error(MFA_ERR_RANGE, "mfa_build_cell_node: too many nodes");
  *nnode = num.next;
  return MFA_OK;
}

extern "C" int mfa_node_coords(int cell_type, int degree, int64_t ncell, const int32_t* cell_vert, const double* coords,
                               const int32_t* cell_node, int64_t nnode, double* out) {
  if ((cell_type != MFA_CELL_HEX8 && cell_type != MFA_CELL_TET4 && cell_type != MFA_CELL_TRI3 &&
       cell_type != MFA_CELL_QUAD4) ||
      ncell < 0 || nnode < 0 || (ncell > 0 && (!cell_vert || !coords || !cell_node)) || (nnode > 0 && !out))
    return mfa::set_error(MFA_ERR_ARG, "mfa_node_coords: bad argument");
  const int p = degree;
  const bool hex = cell_type == MFA_CELL_HEX8, tensor = hex || cell_type == MFA_CELL_QUAD4;
  if ((tensor && (p < 1 || p > 8)) || (!tensor && (p < 1 || p > mfa::kTetMaxP)))
    return mfa::set_error(MFA_ERR_UNSUPPORTED, "mfa_node_coords: degree");
  std::fill(out, out + 3 * nnode, 0.0);
  if (cell_type == MFA_CELL_QUAD4) {
    const int n = p + 1, nl = n * n;
    double s[mfa::kMaxN];
    mfa::gll01(n, s);
    for (int64_t c = 0; c < ncell; ++c)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const int32_t node = cell_node[c * nl + i + n * j];
          if (node < 0 || node >= nnode) return mfa::set_error(MFA_ERR_RANGE, "mfa_node_coords: node index");
          for (int d = 0; d < 3; ++d) {
            double x = 0.0;
            for (int v = 0; v < 4; ++v)
              x += ((v & 1) ? s[i] : 1.0 - s[i]) * ((v & 2) ? s[j] : 1.0 - s[j]) *
                   coords[3 * (int64_t)cell_vert[4 * c + v] + d];
            out[3 * (int64_t)node + d] = x;
          }
        }
    return MFA_OK;
  }
  if (cell_type == MFA_CELL_TRI3) {
    const int nl = mfa::tri_lattice_size(p);
    for (int64_t c = 0; c < ncell; ++c) {
      int a = 0;
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p - j; ++i, ++a) {
          const int32_t node = cell_node[c * nl + a];
          if (node < 0 || node >= nnode) return mfa::set_error(MFA_ERR_RANGE, "mfa_node_coords: node index");
          const double b[3] = {(double)(p - i - j) / p, (double)i / p, (double)j / p};
          for (int d = 0; d < 3; ++d) {
            double x = 0.0;
            for (int s = 0; s < 3; ++s) x += b[s] * coords[3 * (int64_t)cell_vert[3 * c + s] + d];
            out[3 * (int64_t)node + d] = x;
          }
        }
    }
    return MFA_OK;
  }
  if (hex) {
    const int n = p + 1, nl = n * n * n;
    double s[mfa::kMaxN];
    mfa::gll01(n, s);
    for (int64_t c = 0; c < ncell; ++c)
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int32_t node = cell_node[c * nl + i + n * (j + n * k)];
            if (node < 0 || node >= nnode) return mfa::set_error(MFA_ERR_RANGE, "mfa_node_coords: node index");
            const double xi[3] = {s[i], s[j], s[k]};
            for (int d = 0; d < 3; ++d) {
              double x = 0.0;
              for (int v = 0; v < 8; ++v) {
                double wv = 1.0;
                for (int e = 0; e < 3; ++e) wv *= ((v >> e) & 1) ? xi[e] : 1.0 - xi[e];
                x += wv * coords[3 * (int64_t)cell_vert[8 * c + v] + d];
              }
              out[3 * (int64_t)node + d] = x;
            }
          }
  } else {
    std::vector<std::array<int, 4>> w;
    tet_local_weights(p, w);
    const int nl = (int)w.size();
    for (int64_t c = 0; c < ncell; ++c)
      for (int a = 0; a < nl; ++a) {
        const int32_t node = cell_node[c * nl + a];
        if (node < 0 || node >= nnode) return mfa::set_error(MFA_ERR_RANGE, "mfa_node_coords: node index");
        for (int d = 0; d < 3; ++d) {
          double x = 0.0;
          for (int s = 0; s < 4; ++s) x += (double)w[a][s] / p * coords[3 * (int64_t)cell_vert[4 * c + s] + d];
          out[3 * (int64_t)node + d] = x;
        }
      }
  }
  return MFA_OK;
}
