// Host-side set-up of libtem: mesh ingest, Whitney element matrices, PEC,
// nested-dissection ordering, assembly tree (supernodal fronts), index maps
// for the device kernels, transmitter sources, the observation operator and
// the RT0 regulariser root.  Runs once per mesh; nothing here is timed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "tem_internal.h"

namespace tem {

namespace {

const int kLocalEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

inline void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Barycentric gradients of a tetrahedron (vertex rows p[4][3]) via the
// adjugate of the edge matrix; returns the signed 6*volume.
double bary_gradients(const double p[4][3], double g[4][3]) {
  double e1[3], e2[3], e3[3];
  for (int d = 0; d < 3; d++) {
    e1[d] = p[1][d] - p[0][d];
    e2[d] = p[2][d] - p[0][d];
    e3[d] = p[3][d] - p[0][d];
  }
  double c23[3], c31[3], c12[3];
  cross3(e2, e3, c23);
  cross3(e3, e1, c31);
  cross3(e1, e2, c12);
  double det = dot3(e1, c23);
  // grad lambda_1 = (e2 x e3)/det, etc.: rows of the inverse-transpose
  for (int d = 0; d < 3; d++) {
    g[1][d] = c23[d] / det;
    g[2][d] = c31[d] / det;
    g[3][d] = c12[d] / det;
    g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  }
  return det;
}

// Element matrices of the Whitney edge basis N_ab = l_a grad l_b - l_b grad l_a.
void element_matrices(const double p[4][3], double *Ke, double *Me, double &vol) {
  double g[4][3];
  double det = bary_gradients(p, g);
  vol = std::fabs(det) / 6.0;
  double G[4][4];
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) G[a][b] = dot3(g[a], g[b]);
  double curl[6][3];
  for (int i = 0; i < 6; i++) {
    cross3(g[kLocalEdge[i][0]], g[kLocalEdge[i][1]], curl[i]);
    for (int d = 0; d < 3; d++) curl[i][d] *= 2.0;
  }
  for (int i = 0; i < 6; i++) {
    int a = kLocalEdge[i][0], b = kLocalEdge[i][1];
    for (int j = 0; j < 6; j++) {
      int c = kLocalEdge[j][0], d = kLocalEdge[j][1];
      Ke[i * 6 + j] = vol / kMu0 * dot3(curl[i], curl[j]);
      // int l_a l_c = vol (1 + [a==c]) / 20
      auto I = [&](int x, int y) { return (x == y ? 2.0 : 1.0); };
      Me[i * 6 + j] = vol / 20.0 *
                      (I(a, c) * G[b][d] - I(a, d) * G[b][c] - I(b, c) * G[a][d] + I(b, d) * G[a][c]);
    }
  }
}

struct NDNode {
  std::vector<int32_t> piv;  // old interior indices
  int32_t child[kMaxChild] = {-1, -1, -1, -1};
  int32_t nchild = 0;
  bool merged = false;       // amalgamated into its parent
};

struct NDState {
  const Mesh *m;
  const std::vector<double> *cent;   // [nt*3]
  const std::vector<int64_t> *inc_ptr;
  const std::vector<int32_t> *inc_tet;
  std::vector<int8_t> side;
  std::vector<NDNode> nodes;
  int32_t leaf_max;
};

// Nested dissection by plane cuts.  A subdomain is a set of tetrahedra and
// the unknowns all of whose tetrahedra lie in it.  The tetrahedra are split
// by centroid at a vertex coordinate near the median along the longest
// extent; unknowns touching both halves form the separator.  On tensor grids
// the cut plane passes through mesh vertices, so the separator is exactly
// the edges lying in that plane.
int32_t nd_recurse(NDState &st, std::vector<int32_t> &dofs, std::vector<int32_t> &tets) {
  const Mesh &m = *st.m;
  const std::vector<double> &cent = *st.cent;
  auto make_leaf = [&]() {
    NDNode nd;
    nd.piv.swap(dofs);
    st.nodes.push_back(std::move(nd));
    return (int32_t)st.nodes.size() - 1;
  };
  if ((int64_t)dofs.size() <= st.leaf_max || tets.size() < 2) return make_leaf();
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int32_t t : tets)
    for (int d = 0; d < 3; d++) {
      lo[d] = std::min(lo[d], cent[3 * t + d]);
      hi[d] = std::max(hi[d], cent[3 * t + d]);
    }
  int ax = 0;
  for (int d = 1; d < 3; d++)
    if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
  std::vector<double> cc(tets.size());
  for (size_t i = 0; i < tets.size(); i++) cc[i] = cent[3 * tets[i] + ax];
  std::nth_element(cc.begin(), cc.begin() + cc.size() / 2, cc.end());
  double med = cc[cc.size() / 2];
  // snap the cut to the vertex coordinate closest to the median
  double best = med, bestd = 1e300;
  for (int32_t t : tets)
    for (int v = 0; v < 4; v++) {
      double x = m.xyz[3 * m.tv[4 * t + v] + ax];
      double dd = std::fabs(x - med);
      if (dd < bestd) { bestd = dd; best = x; }
    }
  double cut = best;
  auto count_left = [&](double c) {
    size_t nl = 0;
    for (int32_t t : tets) nl += cent[3 * t + ax] < c;
    return nl;
  };
  size_t nl = count_left(cut);
  if (nl == 0 || nl == tets.size()) {
    cut = med;
    nl = count_left(cut);
    if (nl == 0 || nl == tets.size()) return make_leaf();
  }
  std::vector<int32_t> tl, tr;
  tl.reserve(nl);
  tr.reserve(tets.size() - nl);
  for (int32_t t : tets) {
    bool l = cent[3 * t + ax] < cut;
    st.side[t] = l ? 0 : 1;
    (l ? tl : tr).push_back(t);
  }
  std::vector<int32_t> dl, dr, sep;
  const auto &ip = *st.inc_ptr;
  const auto &it = *st.inc_tet;
  for (int32_t d : dofs) {
    bool hl = false, hr = false;
    for (int64_t q = ip[d]; q < ip[d + 1]; q++) {
      if (st.side[it[q]] == 0) hl = true; else hr = true;
    }
    if (hl && hr) sep.push_back(d);
    else if (hl) dl.push_back(d);
    else dr.push_back(d);
  }
  std::vector<int32_t>().swap(dofs);
  std::vector<int32_t>().swap(tets);
  NDNode nd;
  if (!dl.empty()) nd.child[nd.nchild++] = nd_recurse(st, dl, tl);
  if (!dr.empty()) nd.child[nd.nchild++] = nd_recurse(st, dr, tr);
  nd.piv.swap(sep);
  if (nd.piv.empty() && nd.nchild == 1) {
    // nothing separated: splice the only child in
    return nd.child[0];
  }
  st.nodes.push_back(std::move(nd));
  return (int32_t)st.nodes.size() - 1;
}

}  // namespace

// Ordering (nested dissection by plane cuts), full symmetric pattern and
// assembly tree (fronts, relative maps, levels, update-arena plan, original
// entries -> factor positions, extend-add tasks) of a symmetric matrix whose
// unknowns sit on the tetrahedra: `per` slots per tetrahedron (its 6 edges or
// its 4 vertices) hold the unknown there (-1: none).
std::string build_symbolic(const SymIn &in, SymOut &out, Symbolic &s) {
  const Mesh &m = *in.m;
  const int64_t nt = m.nt, N = in.N;
  const int per = in.per;
  const std::vector<int32_t> &tu = *in.tunk;
  const int32_t leaf_max = in.leaf_max;
  if (N <= 0) return "no unknowns";
  // ---- old unknown -> incident tets ----
  std::vector<int64_t> ip(N + 1, 0);
  for (int64_t q = 0; q < per * nt; q++) {
    int32_t d = tu[q];
    if (d >= 0) ip[d + 1]++;
  }
  for (int64_t d = 0; d < N; d++) ip[d + 1] += ip[d];
  std::vector<int32_t> itet(ip[N]);
  {
    std::vector<int64_t> pos(ip.begin(), ip.end() - 1);
    for (int64_t q = 0; q < per * nt; q++) {
      int32_t d = tu[q];
      if (d >= 0) itet[pos[d]++] = int32_t(q / per);
    }
  }
  // ---- nested dissection ----
  NDState st;
  st.m = &m;
  st.cent = &m.cent;
  st.inc_ptr = &ip;
  st.inc_tet = &itet;
  st.side.assign(nt, 0);
  st.leaf_max = leaf_max > 0 ? leaf_max : 128;
  {
    std::vector<int32_t> dofs(N), tt(nt);
    std::iota(dofs.begin(), dofs.end(), 0);
    std::iota(tt.begin(), tt.end(), 0);
    nd_recurse(st, dofs, tt);
  }
  // ---- amalgamation: a child separator of at most amalg_max unknowns is
  //      merged into its parent front (its pivots first, in child order), and
  //      its own children become the parent's, while the parent keeps at most
  //      kMaxChild children.  Tiny separators (the planes between two leaf
  //      boxes) otherwise make a level of fronts that fill a fraction of the
  //      device tiles; merged, their unknowns cost some explicit zeros in the
  //      parent's dense front instead. ----
  if (in.amalg_max > 0) {
    std::vector<NDNode> &nd = st.nodes;
    for (size_t i = 0; i < nd.size(); i++) {   // postorder: every child is final before its parent
      NDNode &P = nd[i];
      int32_t kids[kMaxChild], nk = 0;
      std::vector<int32_t> piv;
      for (int q = 0; q < P.nchild; q++) {
        NDNode &C = nd[P.child[q]];
        const int rest = P.nchild - q - 1;   // later children, one slot each if kept
        const bool merge = C.nchild > 0 && (int64_t)C.piv.size() <= in.amalg_max && nk + C.nchild + rest <= kMaxChild;
        if (!merge) {
          kids[nk++] = P.child[q];
          continue;
        }
        piv.insert(piv.end(), C.piv.begin(), C.piv.end());
        for (int g = 0; g < C.nchild; g++) kids[nk++] = C.child[g];
        std::vector<int32_t>().swap(C.piv);
        C.nchild = 0;
        C.merged = true;
      }
      if (piv.empty()) continue;
      piv.insert(piv.end(), P.piv.begin(), P.piv.end());
      P.piv.swap(piv);
      P.nchild = nk;
      for (int q = 0; q < nk; q++) P.child[q] = kids[q];
    }
    // drop the merged nodes; postorder is kept
    std::vector<int32_t> remap(nd.size(), -1);
    std::vector<NDNode> keep;
    keep.reserve(nd.size());
    for (size_t i = 0; i < nd.size(); i++)
      if (!nd[i].merged) {
        remap[i] = (int32_t)keep.size();
        keep.push_back(std::move(nd[i]));
      }
    for (NDNode &x : keep)
      for (int q = 0; q < x.nchild; q++) x.child[q] = remap[x.child[q]];
    nd.swap(keep);
  }
  std::vector<NDNode> &nodes = st.nodes;  // postorder: children precede parents
  const int32_t nn = (int32_t)nodes.size();
  out.perm.resize(N);
  out.iperm.assign(N, -1);
  std::vector<int32_t> node_c0(nn), owner(N);
  {
    int32_t pos = 0;
    for (int32_t i = 0; i < nn; i++) {
      node_c0[i] = pos;
      for (int32_t d : nodes[i].piv) {
        out.perm[pos] = d;
        out.iperm[d] = pos;
        owner[pos] = i;
        pos++;
      }
    }
    if (pos != N) return "internal: ordering lost unknowns";
  }
  out.tunk.resize(per * nt);
  for (int64_t q = 0; q < per * nt; q++) {
    int32_t d = tu[q];
    out.tunk[q] = d >= 0 ? out.iperm[d] : -1;
  }
  // ---- full symmetric pattern (elimination numbering) ----
  {
    std::vector<int64_t> pk;
    pk.reserve(size_t(per) * per * nt);
    for (int64_t t = 0; t < nt; t++)
      for (int a = 0; a < per; a++) {
        int32_t r = out.tunk[per * t + a];
        if (r < 0) continue;
        for (int b = 0; b < per; b++) {
          int32_t c = out.tunk[per * t + b];
          if (c >= 0) pk.push_back(int64_t(r) * N + c);
        }
      }
    std::sort(pk.begin(), pk.end());
    pk.erase(std::unique(pk.begin(), pk.end()), pk.end());
    out.rp.assign(N + 1, 0);
    out.ci.resize(pk.size());
    for (size_t q = 0; q < pk.size(); q++) {
      out.rp[pk[q] / N + 1]++;
      out.ci[q] = int32_t(pk[q] % N);
    }
    for (int64_t r = 0; r < N; r++) out.rp[r + 1] += out.rp[r];
  }
  // ---- assembly tree: update rows of every node (postorder) ----
  std::vector<std::vector<int32_t>> upd(nn);
  std::vector<int32_t> height(nn, 0), stamp(N, -1);
  for (int32_t i = 0; i < nn; i++) {
    const int32_t c0 = node_c0[i], k = (int32_t)nodes[i].piv.size();
    const int32_t last = c0 + k - 1;
    std::vector<int32_t> &u = upd[i];
    for (int32_t r = c0; r < c0 + k; r++)
      for (int64_t z = out.rp[r]; z < out.rp[r + 1]; z++) {
        int32_t c = out.ci[z];
        if (c > last && stamp[c] != i) { stamp[c] = i; u.push_back(c); }
      }
    for (int q = 0; q < nodes[i].nchild; q++) {
      int32_t ch = nodes[i].child[q];
      height[i] = std::max(height[i], height[ch] + 1);
      for (int32_t c : upd[ch])
        if (c > last && stamp[c] != i) { stamp[c] = i; u.push_back(c); }
    }
    std::sort(u.begin(), u.end());
  }
  // ---- storage order: by height, then postorder ----
  std::vector<int32_t> order(nn);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return height[a] < height[b]; });
  std::vector<int32_t> slot(nn);
  for (int32_t q = 0; q < nn; q++) slot[order[q]] = q;
  s.fronts.assign(nn, Front());
  s.rows.clear();
  s.flops = 0;
  s.nnz_l = 0;
  s.nnz_l11 = 0;
  s.max_front = 0;
  int64_t lofs = 0;
  int32_t H = 0;
  for (int32_t q = 0; q < nn; q++) {
    int32_t i = order[q];
    Front &F = s.fronts[q];
    F.k = (int32_t)nodes[i].piv.size();
    F.n = F.k + (int32_t)upd[i].size();
    F.ld = F.n + (F.n & 1);   // even: every column starts on a 16-byte boundary
    F.c0 = node_c0[i];
    F.height = height[i];
    F.nchild = nodes[i].nchild;
    for (int c = 0; c < F.nchild; c++) F.child[c] = slot[nodes[i].child[c]];
    F.rows_off = (int64_t)s.rows.size();
    s.rows.insert(s.rows.end(), upd[i].begin(), upd[i].end());
    F.lofs = lofs;
    lofs += int64_t(F.ld) * F.k;
    H = std::max(H, F.height);
    s.max_front = std::max(s.max_front, F.n);
    const int64_t b = F.n - F.k;
    s.nnz_l += int64_t(F.k) * (F.k + 1) / 2 + int64_t(F.k) * b;
    s.nnz_l11 += int64_t(F.k) * (F.k + 1) / 2;
    for (int64_t j = 0; j < F.k; j++) {
      double t = double(F.n - j - 1);
      s.flops += t + t * (t + 1) / 2;
    }
  }
  for (int32_t q = 0; q < nn; q++)
    for (int c = 0; c < s.fronts[q].nchild; c++) s.fronts[s.fronts[q].child[c]].parent = q;
  s.ltotal = lofs;
  // ---- relative maps child update rows -> parent rows ----
  s.rel.clear();
  for (int32_t q = 0; q < nn; q++) {
    Front &F = s.fronts[q];
    F.rel_off = (int64_t)s.rel.size();
    if (F.parent < 0) continue;
    const Front &P = s.fronts[F.parent];
    const int32_t *prow = s.rows.data() + P.rows_off;
    const int32_t pb = P.n - P.k;
    for (int32_t r = 0; r < F.n - F.k; r++) {
      int32_t g = s.rows[F.rows_off + r];
      int32_t loc;
      if (g >= P.c0 && g < P.c0 + P.k) {
        loc = g - P.c0;
      } else {
        const int32_t *it = std::lower_bound(prow, prow + pb, g);
        if (it == prow + pb || *it != g) return "internal: child row missing from parent";
        loc = P.k + int32_t(it - prow);
      }
      s.rel.push_back(loc);
    }
  }
  // ---- levels ----
  s.levels.assign(H + 1, Level());
  for (int32_t q = 0; q < nn; q++) s.levels[s.fronts[q].height].fronts.push_back(q);
  for (Level &L : s.levels) {
    std::stable_sort(L.fronts.begin(), L.fronts.end(),
                     [&](int32_t a, int32_t b) { return s.fronts[a].k > s.fronts[b].k; });
    L.lbeg = INT64_MAX;
    L.lend = 0;
    L.max_k = 0;
    for (int32_t f : L.fronts) {
      const Front &F = s.fronts[f];
      L.lbeg = std::min(L.lbeg, F.lofs);
      L.lend = std::max(L.lend, F.lofs + int64_t(F.ld) * F.k);
      L.max_k = std::max(L.max_k, F.k);
    }
  }
  // ---- update arena plan (first fit; a block lives from its front's level
  //      until its parent's level has been assembled) ----
  {
    std::vector<std::pair<int64_t, int64_t>> freel;  // (offset, size), sorted by offset
    int64_t top = 0;
    auto alloc = [&](int64_t sz) -> int64_t {
      for (size_t i = 0; i < freel.size(); i++)
        if (freel[i].second >= sz) {
          int64_t o = freel[i].first;
          freel[i].first += sz;
          freel[i].second -= sz;
          if (freel[i].second == 0) freel.erase(freel.begin() + i);
          return o;
        }
      int64_t o = top;
      top += sz;
      return o;
    };
    auto release = [&](int64_t o, int64_t sz) {
      freel.push_back({o, sz});
      std::sort(freel.begin(), freel.end());
      std::vector<std::pair<int64_t, int64_t>> mg;
      for (auto &p : freel) {
        if (!mg.empty() && mg.back().first + mg.back().second == p.first) mg.back().second += p.second;
        else mg.push_back(p);
      }
      if (!mg.empty() && mg.back().first + mg.back().second == top) {
        top = mg.back().first;
        mg.pop_back();
      }
      freel.swap(mg);
    };
    int64_t peak = 0;
    for (Level &L : s.levels) {
      for (int32_t f : L.fronts) {
        Front &F = s.fronts[f];
        int64_t b = F.n - F.k;
        if (b > 0) F.uofs = alloc(b * b);
        peak = std::max(peak, top);
      }
      for (int32_t f : L.fronts) {
        Front &F = s.fronts[f];
        for (int c = 0; c < F.nchild; c++) {
          Front &C = s.fronts[F.child[c]];
          int64_t b = C.n - C.k;
          if (b > 0) release(C.uofs, b * b);
        }
      }
    }
    s.utotal = std::max<int64_t>(peak, 1);
  }
  // ---- original entries of A (lower triangle) -> factor positions ----
  {
    std::vector<int32_t> fslot_of_node(nn);
    for (int32_t i = 0; i < nn; i++) fslot_of_node[i] = slot[i];
    std::vector<std::vector<std::pair<int64_t, int64_t>>> per_level(H + 1);
    for (int32_t c = 0; c < N; c++) {
      const int32_t f = fslot_of_node[owner[c]];
      const Front &F = s.fronts[f];
      const int32_t *urow = s.rows.data() + F.rows_off;
      const int32_t b = F.n - F.k;
      for (int64_t z = out.rp[c]; z < out.rp[c + 1]; z++) {
        int32_t r = out.ci[z];
        if (r < c) continue;
        int32_t loc;
        if (r < F.c0 + F.k) {
          loc = r - F.c0;
        } else {
          const int32_t *it = std::lower_bound(urow, urow + b, r);
          if (it == urow + b || *it != r) return "internal: entry outside its front";
          loc = F.k + int32_t(it - urow);
        }
        int64_t dst = F.lofs + int64_t(c - F.c0) * F.ld + loc;
        per_level[F.height].push_back({z, dst});
      }
    }
    s.orig_nz.clear();
    s.orig_dst.clear();
    for (int32_t h = 0; h <= H; h++) {
      s.levels[h].obeg = (int64_t)s.orig_nz.size();
      for (auto &p : per_level[h]) {
        s.orig_nz.push_back(p.first);
        s.orig_dst.push_back(p.second);
      }
      s.levels[h].oend = (int64_t)s.orig_nz.size();
    }
  }
  // ---- extend-add task lists (child slots kept apart: one launch each) ----
  s.ea_child.clear();
  s.ea_col.clear();
  for (Level &L : s.levels)
    for (int sl = 0; sl < kMaxChild; sl++) {
      L.ea_beg[sl] = (int64_t)s.ea_child.size();
      for (int32_t f : L.fronts) {
        const Front &F = s.fronts[f];
        if (sl >= F.nchild) continue;
        const Front &C = s.fronts[F.child[sl]];
        for (int32_t j = 0; j < C.n - C.k; j++) {
          s.ea_child.push_back(F.child[sl]);
          s.ea_col.push_back(j);
        }
      }
      L.ea_end[sl] = (int64_t)s.ea_child.size();
    }
  return "";
}

std::string build_mesh(Mesh &m, int64_t nv, const double *xyz, int64_t nt, const int32_t *tets,
                       const double *sigma, const uint8_t *is_param, const SymOpts &opt,
                       Symbolic &s) {
  if (nv <= 0 || nt <= 0) return "empty mesh";
  if (nv >= (int64_t(1) << 21)) return "more than 2^21 vertices are not supported";
  if (nt * 36 >= (int64_t(1) << 32)) return "too many tetrahedra";
  m.nv = nv;
  m.nt = nt;
  m.xyz.assign(xyz, xyz + 3 * nv);
  m.tv.resize(4 * nt);
  for (int64_t t = 0; t < nt; t++) {
    int32_t v[4];
    for (int a = 0; a < 4; a++) {
      v[a] = tets[4 * t + a];
      if (v[a] < 0 || v[a] >= nv) return "tet vertex id out of range";
    }
    std::sort(v, v + 4);
    if (v[0] == v[1] || v[1] == v[2] || v[2] == v[3]) return "tet with repeated vertex";
    for (int a = 0; a < 4; a++) m.tv[4 * t + a] = v[a];
  }
  // ---- edges ----
  std::vector<int64_t> keys(6 * nt);
  for (int64_t t = 0; t < nt; t++)
    for (int i = 0; i < 6; i++)
      keys[6 * t + i] = int64_t(m.tv[4 * t + kLocalEdge[i][0]]) * nv + m.tv[4 * t + kLocalEdge[i][1]];
  m.ekey = keys;
  std::sort(m.ekey.begin(), m.ekey.end());
  m.ekey.erase(std::unique(m.ekey.begin(), m.ekey.end()), m.ekey.end());
  m.ne = (int64_t)m.ekey.size();
  m.ev.resize(2 * m.ne);
  for (int64_t e = 0; e < m.ne; e++) {
    m.ev[2 * e] = int32_t(m.ekey[e] / nv);
    m.ev[2 * e + 1] = int32_t(m.ekey[e] % nv);
  }
  m.tedge.resize(6 * nt);
  for (int64_t q = 0; q < 6 * nt; q++)
    m.tedge[q] = int32_t(std::lower_bound(m.ekey.begin(), m.ekey.end(), keys[q]) - m.ekey.begin());
  std::vector<int64_t>().swap(keys);
  // ---- faces; PEC on edges of faces that belong to one tetrahedron ----
  const int lf[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  std::vector<int64_t> fk(4 * nt);
  const int64_t nv2 = nv * nv;
  for (int64_t t = 0; t < nt; t++)
    for (int f = 0; f < 4; f++)
      fk[4 * t + f] = int64_t(m.tv[4 * t + lf[f][0]]) * nv2 + int64_t(m.tv[4 * t + lf[f][1]]) * nv +
                      m.tv[4 * t + lf[f][2]];
  std::sort(fk.begin(), fk.end());
  std::vector<uint8_t> pec(m.ne, 0);
  m.vbnd.assign(nv, 0);
  m.faces.clear();
  for (size_t i = 0; i < fk.size();) {
    size_t j = i;
    while (j < fk.size() && fk[j] == fk[i]) j++;
    int32_t a = int32_t(fk[i] / nv2), b = int32_t((fk[i] / nv) % nv), c = int32_t(fk[i] % nv);
    m.faces.push_back(a);
    m.faces.push_back(b);
    m.faces.push_back(c);
    if (j - i == 1) {
      int32_t fv[3] = {a, b, c};
      m.vbnd[a] = m.vbnd[b] = m.vbnd[c] = 1;
      for (int q = 0; q < 3; q++)
        for (int r = q + 1; r < 3; r++) {
          int64_t key = int64_t(fv[q]) * nv + fv[r];
          int64_t e = std::lower_bound(m.ekey.begin(), m.ekey.end(), key) - m.ekey.begin();
          pec[e] = 1;
        }
    } else if (j - i > 2) {
      return "non-manifold face shared by more than two tetrahedra";
    }
    i = j;
  }
  m.dof_old.assign(m.ne, -1);
  int64_t N = 0;
  for (int64_t e = 0; e < m.ne; e++)
    if (!pec[e]) m.dof_old[e] = int32_t(N++);
  m.N = N;
  if (N == 0) return "no interior edges";
  // ---- element matrices ----
  m.vol.resize(nt);
  m.Ke.resize(36 * nt);
  m.Me1.resize(36 * nt);
  m.cent.assign(3 * nt, 0.0);
  for (int64_t t = 0; t < nt; t++) {
    double p[4][3];
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) p[a][d] = m.xyz[3 * m.tv[4 * t + a] + d];
    element_matrices(p, &m.Ke[36 * t], &m.Me1[36 * t], m.vol[t]);
    if (!(m.vol[t] > 0)) return "degenerate tetrahedron";
    for (int d = 0; d < 3; d++) m.cent[3 * t + d] = 0.25 * (p[0][d] + p[1][d] + p[2][d] + p[3][d]);
  }
  m.sigma.assign(sigma, sigma + nt);
  m.is_param.assign(is_param, is_param + nt);
  m.pidx.assign(nt, -1);
  m.ptet.clear();
  for (int64_t t = 0; t < nt; t++)
    if (m.is_param[t]) {
      m.pidx[t] = int32_t(m.ptet.size());
      m.ptet.push_back(int32_t(t));
    }
  m.P = (int64_t)m.ptet.size();
  // ---- ordering and assembly tree of A (unknowns on the interior edges) ----
  {
    std::vector<int32_t> tu(6 * nt);
    for (int64_t q = 0; q < 6 * nt; q++) tu[q] = m.dof_old[m.tedge[q]];
    SymIn in{&m, N, 6, &tu, opt.leaf_max, opt.amalg_max};
    SymOut so;
    const std::string e = build_symbolic(in, so, s);
    if (!e.empty()) return e;
    m.perm.swap(so.perm);
    m.iperm.swap(so.iperm);
    m.tdof.swap(so.tunk);
    m.rp.swap(so.rp);
    m.ci.swap(so.ci);
  }
  const int64_t nnz = m.rp[N];
  auto find_nz = [&](int32_t r, int32_t c) -> int64_t {
    auto b = m.ci.begin() + m.rp[r], e = m.ci.begin() + m.rp[r + 1];
    return std::lower_bound(b, e, c) - m.ci.begin();
  };
  m.kval.assign(nnz, 0.0);
  m.mc_ptr.assign(nnz + 1, 0);
  for (int64_t t = 0; t < nt; t++)
    for (int a = 0; a < 6; a++) {
      int32_t r = m.tdof[6 * t + a];
      if (r < 0) continue;
      for (int b = 0; b < 6; b++) {
        int32_t c = m.tdof[6 * t + b];
        if (c < 0) continue;
        int64_t z = find_nz(r, c);
        m.kval[z] += m.Ke[36 * t + 6 * a + b];
        m.mc_ptr[z + 1]++;
      }
    }
  for (int64_t z = 0; z < nnz; z++) m.mc_ptr[z + 1] += m.mc_ptr[z];
  m.mc_idx.resize(m.mc_ptr[nnz]);
  {
    std::vector<int64_t> pos(m.mc_ptr.begin(), m.mc_ptr.end() - 1);
    for (int64_t t = 0; t < nt; t++)
      for (int a = 0; a < 6; a++) {
        int32_t r = m.tdof[6 * t + a];
        if (r < 0) continue;
        for (int b = 0; b < 6; b++) {
          int32_t c = m.tdof[6 * t + b];
          if (c < 0) continue;
          int64_t z = find_nz(r, c);
          m.mc_idx[pos[z]++] = uint32_t(36 * t + 6 * a + b);
        }
      }
  }
  // ---- dof (new) -> incident (tet, local) ----
  m.inc_ptr.assign(N + 1, 0);
  for (int64_t q = 0; q < 6 * nt; q++)
    if (m.tdof[q] >= 0) m.inc_ptr[m.tdof[q] + 1]++;
  for (int64_t d = 0; d < N; d++) m.inc_ptr[d + 1] += m.inc_ptr[d];
  m.inc_tet.resize(m.inc_ptr[N]);
  m.inc_loc.resize(m.inc_ptr[N]);
  {
    std::vector<int64_t> pos(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
    for (int64_t q = 0; q < 6 * nt; q++) {
      int32_t d = m.tdof[q];
      if (d < 0) continue;
      m.inc_tet[pos[d]] = int32_t(q / 6);
      m.inc_loc[pos[d]] = int8_t(q % 6);
      pos[d]++;
    }
  }
  // ---- regulariser root W over parameter cells (two-point RT0 form) ----
  {
    std::vector<std::pair<int64_t, int32_t>> ft;  // (face key, tet)
    ft.reserve(4 * nt);
    for (int64_t t = 0; t < nt; t++) {
      if (!m.is_param[t]) continue;
      for (int f = 0; f < 4; f++) {
        int64_t key = int64_t(m.tv[4 * t + lf[f][0]]) * nv2 + int64_t(m.tv[4 * t + lf[f][1]]) * nv +
                      m.tv[4 * t + lf[f][2]];
        ft.push_back({key, int32_t(t)});
      }
    }
    std::sort(ft.begin(), ft.end());
    std::vector<int32_t> fa, fb;
    std::vector<double> wv;
    for (size_t i = 0; i + 1 < ft.size(); i++) {
      if (ft[i].first != ft[i + 1].first) continue;
      int32_t a = ft[i].second, b = ft[i + 1].second;
      int64_t key = ft[i].first;
      int32_t v0 = int32_t(key / nv2), v1 = int32_t((key / nv) % nv), v2 = int32_t(key % nv);
      double e1[3], e2[3], cr[3], dc[3];
      for (int d = 0; d < 3; d++) {
        e1[d] = m.xyz[3 * v1 + d] - m.xyz[3 * v0 + d];
        e2[d] = m.xyz[3 * v2 + d] - m.xyz[3 * v0 + d];
        dc[d] = m.cent[3 * a + d] - m.cent[3 * b + d];
      }
      cross3(e1, e2, cr);
      double area = 0.5 * std::sqrt(dot3(cr, cr));
      double dist = std::sqrt(dot3(dc, dc));
      fa.push_back(m.pidx[a]);
      fb.push_back(m.pidx[b]);
      wv.push_back(std::sqrt(area / dist));
      i++;
    }
    m.nf = (int64_t)fa.size();
    m.w_rp.assign(m.nf + 1, 0);
    m.w_ci.resize(2 * m.nf);
    m.w_val.resize(2 * m.nf);
    for (int64_t f = 0; f < m.nf; f++) {
      m.w_rp[f + 1] = 2 * (f + 1);
      m.w_ci[2 * f] = fa[f];
      m.w_val[2 * f] = wv[f];
      m.w_ci[2 * f + 1] = fb[f];
      m.w_val[2 * f + 1] = -wv[f];
    }
    // transpose
    m.wt_rp.assign(m.P + 1, 0);
    for (int64_t q = 0; q < 2 * m.nf; q++) m.wt_rp[m.w_ci[q] + 1]++;
    for (int64_t p = 0; p < m.P; p++) m.wt_rp[p + 1] += m.wt_rp[p];
    m.wt_ci.resize(2 * m.nf);
    m.wt_val.resize(2 * m.nf);
    std::vector<int64_t> pos(m.wt_rp.begin(), m.wt_rp.end() - 1);
    for (int64_t f = 0; f < m.nf; f++)
      for (int64_t q = m.w_rp[f]; q < m.w_rp[f + 1]; q++) {
        int32_t p = m.w_ci[q];
        m.wt_ci[pos[p]] = int32_t(f);
        m.wt_val[pos[p]] = m.w_val[q];
        pos[p]++;
      }
  }
  return "";
}

std::string build_nodal(const Mesh &m, const SymOpts &opt, NodalMesh &nm, Symbolic &s) {
  const int64_t nt = m.nt, nv = m.nv;
  // interior vertices: the hat functions whose gradients are interior edge fields
  std::vector<int32_t> vold(nv, -1), vert_of;
  for (int64_t v = 0; v < nv; v++)
    if (!m.vbnd[v]) {
      vold[v] = int32_t(vert_of.size());
      vert_of.push_back(int32_t(v));
    }
  const int64_t N = (int64_t)vert_of.size();
  if (N == 0) return "no interior vertices";
  std::vector<int32_t> tu(4 * nt);
  for (int64_t q = 0; q < 4 * nt; q++) tu[q] = vold[m.tv[q]];
  SymIn in{&m, N, 4, &tu, opt.leaf_max, opt.amalg_max};
  SymOut so;
  const std::string e = build_symbolic(in, so, s);
  if (!e.empty()) return e;
  nm.N = N;
  nm.perm.resize(N);
  for (int64_t i = 0; i < N; i++) nm.perm[i] = vert_of[so.perm[i]];
  nm.tnode.swap(so.tunk);
  nm.rp.swap(so.rp);
  nm.ci.swap(so.ci);
  // P1 stiffness of every tetrahedron: S_t[a][b] = vol grad l_a . grad l_b
  nm.S.resize(16 * nt);
  for (int64_t t = 0; t < nt; t++) {
    double p[4][3], g[4][3];
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) p[a][d] = m.xyz[3 * m.tv[4 * t + a] + d];
    bary_gradients(p, g);
    for (int a = 0; a < 4; a++)
      for (int b = 0; b < 4; b++) nm.S[16 * t + 4 * a + b] = m.vol[t] * dot3(g[a], g[b]);
  }
  // contributions of the tetrahedra to each Laplacian entry
  auto find_nz = [&](int32_t r, int32_t c) -> int64_t {
    auto b = nm.ci.begin() + nm.rp[r], e2 = nm.ci.begin() + nm.rp[r + 1];
    return std::lower_bound(b, e2, c) - nm.ci.begin();
  };
  const int64_t nnz = nm.rp[N];
  nm.mc_ptr.assign(nnz + 1, 0);
  for (int64_t t = 0; t < nt; t++)
    for (int a = 0; a < 4; a++) {
      const int32_t r = nm.tnode[4 * t + a];
      if (r < 0) continue;
      for (int b = 0; b < 4; b++) {
        const int32_t c = nm.tnode[4 * t + b];
        if (c >= 0) nm.mc_ptr[find_nz(r, c) + 1]++;
      }
    }
  for (int64_t z = 0; z < nnz; z++) nm.mc_ptr[z + 1] += nm.mc_ptr[z];
  nm.mc_idx.resize(nm.mc_ptr[nnz]);
  {
    std::vector<int64_t> pos(nm.mc_ptr.begin(), nm.mc_ptr.end() - 1);
    for (int64_t t = 0; t < nt; t++)
      for (int a = 0; a < 4; a++) {
        const int32_t r = nm.tnode[4 * t + a];
        if (r < 0) continue;
        for (int b = 0; b < 4; b++) {
          const int32_t c = nm.tnode[4 * t + b];
          if (c >= 0) nm.mc_idx[pos[find_nz(r, c)]++] = uint32_t(16 * t + 4 * a + b);
        }
      }
  }
  // gradient incidence: edge unknown d (lower -> higher vertex) and its end nodes
  std::vector<int32_t> vnew(nv, -1);
  for (int64_t i = 0; i < N; i++) vnew[nm.perm[i]] = int32_t(i);
  std::vector<int64_t> edge_of_old(m.N);
  for (int64_t ed = 0; ed < m.ne; ed++)
    if (m.dof_old[ed] >= 0) edge_of_old[m.dof_old[ed]] = ed;
  nm.e_lo.resize(m.N);
  nm.e_hi.resize(m.N);
  nm.g_ptr.assign(N + 1, 0);
  for (int64_t d = 0; d < m.N; d++) {
    const int64_t ed = edge_of_old[m.perm[d]];
    nm.e_lo[d] = vnew[m.ev[2 * ed]];
    nm.e_hi[d] = vnew[m.ev[2 * ed + 1]];
    if (nm.e_lo[d] >= 0) nm.g_ptr[nm.e_lo[d] + 1]++;
    if (nm.e_hi[d] >= 0) nm.g_ptr[nm.e_hi[d] + 1]++;
  }
  for (int64_t i = 0; i < N; i++) nm.g_ptr[i + 1] += nm.g_ptr[i];
  nm.g_edge.resize(nm.g_ptr[N]);
  nm.g_sign.resize(nm.g_ptr[N]);
  {
    std::vector<int64_t> pos(nm.g_ptr.begin(), nm.g_ptr.end() - 1);
    for (int64_t d = 0; d < m.N; d++) {
      if (nm.e_lo[d] >= 0) {
        const int64_t q = pos[nm.e_lo[d]]++;
        nm.g_edge[q] = int32_t(d);
        nm.g_sign[q] = -1;
      }
      if (nm.e_hi[d] >= 0) {
        const int64_t q = pos[nm.e_hi[d]]++;
        nm.g_edge[q] = int32_t(d);
        nm.g_sign[q] = 1;
      }
    }
  }
  // C = M(sigma) G through the edge unknowns' incident (tet, local edge) pairs
  nm.B.resize(24 * nt);
  for (int64_t t = 0; t < nt; t++)
    for (int a = 0; a < 4; a++)
      for (int l = 0; l < 6; l++)
        nm.B[24 * t + 6 * a + l] =
            0.25 * (nm.S[16 * t + 4 * a + kLocalEdge[l][1]] - nm.S[16 * t + 4 * a + kLocalEdge[l][0]]);
  nm.c_rp.assign(m.N + 1, 0);
  nm.c_ci.clear();
  nm.c_mc_ptr.assign(1, 0);
  nm.c_mc_idx.clear();
  std::vector<std::pair<int32_t, uint32_t>> row;   // (node, contribution)
  for (int64_t d = 0; d < m.N; d++) {
    row.clear();
    for (int64_t q = m.inc_ptr[d]; q < m.inc_ptr[d + 1]; q++) {
      const int32_t t = m.inc_tet[q], l = m.inc_loc[q];
      for (int a = 0; a < 4; a++) {
        const int32_t nd = nm.tnode[4 * int64_t(t) + a];
        if (nd >= 0) row.push_back({nd, uint32_t(24 * int64_t(t) + 6 * a + l)});
      }
    }
    std::sort(row.begin(), row.end());
    for (size_t i = 0; i < row.size();) {
      size_t j = i;
      while (j < row.size() && row[j].first == row[i].first) nm.c_mc_idx.push_back(row[j++].second);
      nm.c_ci.push_back(row[i].first);
      nm.c_mc_ptr.push_back((int64_t)nm.c_mc_idx.size());
      i = j;
    }
    nm.c_rp[d + 1] = (int64_t)nm.c_ci.size();
  }
  return "";
}

std::string build_sources(const Mesh &m, int32_t n_tx, const int64_t *loop_ptr,
                          const int32_t *loop_verts, int32_t n_rx, const double *rx,
                          std::vector<double> &f, std::vector<int64_t> &q_rp,
                          std::vector<int32_t> &q_ci, std::vector<double> &q_val,
                          std::vector<int32_t> &qt_dof, std::vector<int64_t> &qt_rp,
                          std::vector<int32_t> &qt_ci, std::vector<double> &qt_val) {
  const int64_t N = m.N, nv = m.nv;
  auto edge_of = [&](int32_t p, int32_t q) -> int64_t {
    int64_t a = std::min(p, q), b = std::max(p, q);
    int64_t key = a * nv + b;
    auto it = std::lower_bound(m.ekey.begin(), m.ekey.end(), key);
    if (it == m.ekey.end() || *it != key) return -1;
    return it - m.ekey.begin();
  };
  // ---- sources: f_k = int_loop N_k . dl = +-1 on the loop's edges ----
  f.assign(N * n_tx, 0.0);
  for (int32_t x = 0; x < n_tx; x++) {
    int64_t b = loop_ptr[x], e = loop_ptr[x + 1];
    if (e - b < 3) return "a loop needs at least three vertices";
    for (int64_t s = b; s < e; s++) {
      int32_t p = loop_verts[s], q = loop_verts[s + 1 < e ? s + 1 : b];
      if (p < 0 || p >= nv || q < 0 || q >= nv) return "loop vertex out of range";
      int64_t ed = edge_of(p, q);
      if (ed < 0) return "loop segment is not a mesh edge";
      int32_t d = m.dof_old[ed];
      if (d < 0) return "loop runs on the PEC boundary";
      f[int64_t(m.iperm[d]) * n_tx + x] += (p < q) ? 1.0 : -1.0;
    }
  }
  // ---- observation operator: -(curl e)_z by Stokes on surface triangles ----
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < nv; v++)
    for (int d = 0; d < 3; d++) {
      lo[d] = std::min(lo[d], m.xyz[3 * v + d]);
      hi[d] = std::max(hi[d], m.xyz[3 * v + d]);
    }
  double scale = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  double tol = 1e-9 * scale;
  const int64_t nfc = (int64_t)m.faces.size() / 3;
  q_rp.assign(n_rx + 1, 0);
  q_ci.clear();
  q_val.clear();
  for (int32_t r = 0; r < n_rx; r++) {
    const double *p = rx + 3 * r;
    std::vector<std::pair<int32_t, double>> circ;  // (new dof, signed count)
    double area = 0;
    for (int64_t fi = 0; fi < nfc; fi++) {
      int32_t v[3] = {m.faces[3 * fi], m.faces[3 * fi + 1], m.faces[3 * fi + 2]};
      const double *A = &m.xyz[3 * v[0]], *B = &m.xyz[3 * v[1]], *C = &m.xyz[3 * v[2]];
      if (std::fabs(A[2] - p[2]) > tol || std::fabs(B[2] - p[2]) > tol || std::fabs(C[2] - p[2]) > tol)
        continue;
      double a2 = (B[0] - A[0]) * (C[1] - A[1]) - (B[1] - A[1]) * (C[0] - A[0]);
      if (a2 < 0) {
        std::swap(v[1], v[2]);
        std::swap(B, C);
        a2 = -a2;
      }
      if (a2 <= 0) continue;
      // closure test with the three edge functions
      const double *P3[3] = {A, B, C};
      bool inside = true;
      for (int k = 0; k < 3; k++) {
        const double *U = P3[(k + 1) % 3], *W = P3[(k + 2) % 3];
        double lam = ((W[0] - U[0]) * (p[1] - U[1]) - (W[1] - U[1]) * (p[0] - U[0])) / a2;
        if (lam < -1e-9) { inside = false; break; }
      }
      if (!inside) continue;
      area += 0.5 * a2;
      for (int k = 0; k < 3; k++) {
        int32_t s0 = v[k], s1 = v[(k + 1) % 3];
        int64_t ed = edge_of(s0, s1);
        int32_t d = ed >= 0 ? m.dof_old[ed] : -1;
        if (d < 0) continue;
        circ.push_back({m.iperm[d], s0 < s1 ? 1.0 : -1.0});
      }
    }
    if (area <= 0) return "receiver lies on no horizontal mesh face";
    std::sort(circ.begin(), circ.end());
    for (size_t i = 0; i < circ.size();) {
      size_t j = i;
      double c = 0;
      while (j < circ.size() && circ[j].first == circ[i].first) c += circ[j++].second;
      if (c != 0.0) {
        q_ci.push_back(circ[i].first);
        q_val.push_back(-c / area);
      }
      i = j;
    }
    q_rp[r + 1] = (int64_t)q_ci.size();
  }
  // transpose: column (dof) -> (receiver, value), only dofs that appear
  std::vector<std::pair<int32_t, std::pair<int32_t, double>>> tr;
  for (int32_t r = 0; r < n_rx; r++)
    for (int64_t z = q_rp[r]; z < q_rp[r + 1]; z++) tr.push_back({q_ci[z], {r, q_val[z]}});
  std::sort(tr.begin(), tr.end(), [](const auto &a, const auto &b) {
    return a.first < b.first || (a.first == b.first && a.second.first < b.second.first);
  });
  // Q^T as a list of the distinct dofs Q touches, each with its receivers
  qt_dof.clear();
  qt_rp.clear();
  qt_ci.clear();
  qt_val.clear();
  for (size_t i = 0; i < tr.size();) {
    size_t j = i;
    qt_dof.push_back(tr[i].first);
    qt_rp.push_back((int64_t)qt_ci.size());
    while (j < tr.size() && tr[j].first == tr[i].first) {
      qt_ci.push_back(tr[j].second.first);
      qt_val.push_back(tr[j].second.second);
      j++;
    }
    i = j;
  }
  qt_rp.push_back((int64_t)qt_ci.size());
  return "";
}

}  // namespace tem
