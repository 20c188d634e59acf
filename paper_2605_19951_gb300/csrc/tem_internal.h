// Internal host-side structures of libtem: mesh, ordering, assembly tree.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace tem {

constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr int kMaxChild = 4;       // children per front (two from the dissection, four after amalgamation)
constexpr int kAmalgDefault = 32;  // separators of at most this many unknowns merge into their parent

// Per-front description (one supernode of the assembly tree = one node of
// the nested-dissection tree: a separator or a leaf subdomain).
struct Front {
  int32_t k = 0;        // pivots (columns eliminated here)
  int32_t n = 0;        // order of the frontal matrix: k + b
  int32_t ld = 0;       // column stride of the factor block: n rounded up to even
  int32_t c0 = 0;       // first pivot in the elimination numbering
  int32_t parent = -1;  // parent front (-1 = root)
  int32_t height = 0;   // 0 = leaf
  int32_t nchild = 0;
  int32_t child[kMaxChild] = {-1, -1, -1, -1};
  int64_t rows_off = 0; // offset of the update-row list in Symbolic::rows
  int64_t lofs = 0;     // offset of the n x k factor block (elements)
  int64_t uofs = -1;    // offset of the b x b update block in the arena
  int64_t rel_off = 0;  // offset of this front's relative map into its parent
};

struct Level {
  std::vector<int32_t> fronts;  // sorted by k descending
  int64_t lbeg = 0, lend = 0;   // contiguous factor range [lbeg, lend)
  int64_t obeg = 0, oend = 0;   // original-entry range
  int64_t ea_beg[kMaxChild] = {}, ea_end[kMaxChild] = {};  // extend-add tasks per child slot
  int32_t max_k = 0;
};

struct Mesh {
  int64_t nv = 0, nt = 0, ne = 0, N = 0, P = 0;
  std::vector<double> xyz;          // [nv*3]
  std::vector<int32_t> tv;          // [nt*4] vertex ids sorted ascending
  std::vector<int32_t> ev;          // [ne*2] edge end points (lower first)
  std::vector<int64_t> ekey;        // [ne] sorted keys lo*nv + hi
  std::vector<int32_t> faces;       // [n_faces*3] unique triangles, sorted ids
  std::vector<int32_t> tedge;       // [nt*6] edge ids of local edges
  std::vector<int32_t> dof_old;     // [ne] interior index or -1 (PEC)
  std::vector<int32_t> tdof;        // [nt*6] elimination-numbered dof or -1
  std::vector<double> vol;          // [nt]
  std::vector<double> cent;         // [nt*3] tetrahedron centroids
  std::vector<uint8_t> vbnd;        // [nv] 1 = vertex of a boundary face (PEC)
  std::vector<double> Ke;           // [nt*36] curl-curl / mu0
  std::vector<double> Me1;          // [nt*36] unit-conductivity mass
  std::vector<double> sigma;        // [nt]
  std::vector<uint8_t> is_param;    // [nt]
  std::vector<int32_t> pidx;        // [nt] parameter index or -1
  std::vector<int32_t> ptet;        // [P] tet of each parameter
  // elimination numbering
  std::vector<int32_t> perm;        // new -> old interior index
  std::vector<int32_t> iperm;       // old -> new
  // full symmetric pattern of A in elimination numbering
  std::vector<int64_t> rp;          // [N+1]
  std::vector<int32_t> ci;          // [nnz]
  std::vector<double> kval;         // [nnz]
  std::vector<int64_t> mc_ptr;      // [nnz+1] contributions to M values
  std::vector<uint32_t> mc_idx;     // tet*36 + a*6 + b
  // dof -> incident (tet, local) pairs, elimination numbering
  std::vector<int64_t> inc_ptr;     // [N+1]
  std::vector<int32_t> inc_tet;     // tet id
  std::vector<int8_t> inc_loc;      // local edge 0..5
  // regulariser root W (faces x P) and its transpose
  int64_t nf = 0;
  std::vector<int64_t> w_rp;
  std::vector<int32_t> w_ci;
  std::vector<double> w_val;
  std::vector<int64_t> wt_rp;
  std::vector<int32_t> wt_ci;
  std::vector<double> wt_val;
};

struct Symbolic {
  std::vector<Front> fronts;            // storage order (by level)
  std::vector<Level> levels;
  std::vector<int32_t> rows;            // update rows of every front (elimination numbering)
  std::vector<int32_t> rel;             // child update row -> parent local row
  std::vector<int64_t> orig_nz;         // lower-triangle entries of A ...
  std::vector<int64_t> orig_dst;        // ... and their destination in the factor store
  std::vector<int32_t> ea_child;        // extend-add tasks: child front
  std::vector<int32_t> ea_col;          //                   child update column
  int64_t ltotal = 0;                   // factor elements per pole
  int64_t utotal = 0;                   // update arena elements per pole
  double flops = 0;                     // complex MACs per pole
  int64_t nnz_l = 0;                    // meaningful factor entries per pole
  int64_t nnz_l11 = 0;                  // of which in the pivot blocks
  int32_t max_front = 0;
};

// Input of the ordering / assembly-tree builder: unknowns sitting on the
// tetrahedra of a mesh, `per` slots per tetrahedron (6 edges or 4 vertices).
struct SymIn {
  const Mesh *m;                     // vertices, tetrahedra and their centroids
  int64_t N;                         // unknowns, numbered 0..N-1 ("old" numbering)
  int per;                           // slots per tetrahedron
  const std::vector<int32_t> *tunk;  // [nt*per] old unknown of each slot, -1 = none
  int32_t leaf_max;                  // largest leaf of the dissection (0 = default)
  int32_t amalg_max;                 // separators of at most this many unknowns merge into their parent (0: none)
};

// Options of the dissection and assembly tree.
struct SymOpts {
  int32_t leaf_max = 0;              // largest leaf of the dissection (0 = default, 128)
  int32_t amalg_max = kAmalgDefault; // amalgamation threshold (0: none)
};
struct SymOut {
  std::vector<int32_t> perm, iperm;  // new -> old, old -> new
  std::vector<int32_t> tunk;         // [nt*per] elimination-numbered unknown of each slot, -1 = none
  std::vector<int64_t> rp;           // full symmetric pattern, elimination numbering
  std::vector<int32_t> ci;
};

// Gradient space of the edge unknowns (auxiliary nodal space of the FP32
// refinement): the interior vertices (not on a boundary face) and the
// sigma-weighted P1 Laplacian G^T M(sigma) G = sum_t sigma_t S_t on them,
// S_t[a][b] = vol_t grad l_a . grad l_b.
struct NodalMesh {
  int64_t N = 0;                    // interior vertices
  std::vector<int32_t> perm;        // elimination index -> vertex id
  std::vector<int32_t> tnode;       // [nt*4] elimination-numbered node of each tet vertex, -1 on the boundary
  std::vector<double> S;            // [nt*16] vol grad l_a . grad l_b (a, b = sorted local vertices)
  std::vector<int64_t> rp;          // pattern of the Laplacian (elimination numbering)
  std::vector<int32_t> ci;
  std::vector<int64_t> mc_ptr;      // [nnz+1] contributions to each Laplacian entry ...
  std::vector<uint32_t> mc_idx;     // ... as t*16 + 4a + b
  std::vector<int32_t> e_lo, e_hi;  // [N_edge] nodes at the lower / higher end of each edge unknown (-1: boundary)
  std::vector<int64_t> g_ptr;       // [N+1] node -> incident edge unknowns ...
  std::vector<int32_t> g_edge;      // ... edge (elimination numbering)
  std::vector<int8_t> g_sign;       // ... +1 at its higher end, -1 at its lower end
  // C = M(sigma) G (edge unknowns x nodes): C[d][a] = sum_t sigma_t B_t[a][loc(d)],
  // B_t[a][(i,j)] = int_t N_ij . grad l_a = (S_t[a][j] - S_t[a][i]) / 4
  std::vector<double> B;            // [nt*24] at t*24 + 6a + local edge
  std::vector<int64_t> c_rp;        // [N_edge+1] rows of C (edge unknowns, elimination numbering)
  std::vector<int32_t> c_ci;        // node of each entry
  std::vector<int64_t> c_mc_ptr;    // contributions to each entry ...
  std::vector<uint32_t> c_mc_idx;   // ... as t*24 + 6a + local edge
};

// Host builders (host.cpp).  Return "" on success or an error message.
std::string build_symbolic(const SymIn &in, SymOut &out, Symbolic &s);
std::string build_nodal(const Mesh &m, const SymOpts &opt, NodalMesh &nm, Symbolic &s);
std::string build_mesh(Mesh &m, int64_t nv, const double *xyz, int64_t nt,
                       const int32_t *tets, const double *sigma,
                       const uint8_t *is_param, const SymOpts &opt, Symbolic &s);
std::string build_sources(const Mesh &m, int32_t n_tx, const int64_t *loop_ptr,
                          const int32_t *loop_verts, int32_t n_rx, const double *rx,
                          std::vector<double> &f,          // [N][n_tx] elimination order
                          std::vector<int64_t> &q_rp, std::vector<int32_t> &q_ci,
                          std::vector<double> &q_val,
                          std::vector<int32_t> &qt_dof,   // distinct dofs of Q
                          std::vector<int64_t> &qt_rp,    // [n_qdof+1]
                          std::vector<int32_t> &qt_ci,    // receiver
                          std::vector<double> &qt_val);

}  // namespace tem
