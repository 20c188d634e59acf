// Internal interface between the C-ABI layer (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace tem {

constexpr int kNB = 32;        // pivot block width of the blocked LDL^T and the solves
constexpr int kPanelRT = 128;  // panel rows per CTA
constexpr int kSB = 256;       // super-block of the solves' pivot blocks (multiple of kNB)
constexpr int kSplitK = 512;   // inner-dimension chunk of one super-block product task
constexpr int kKB = 128;       // FP32 factor: columns of one block of the tensor-core trailing update

template <typename R>
struct UpdateTile;
template <>
struct UpdateTile<float> {
  static constexpr int TM = 64;
};
template <>
struct UpdateTile<double> {
  static constexpr int TM = 32;
};
template <typename R>
struct SolveTile;
template <>
struct SolveTile<float> {
  static constexpr int RT = 64;   // pivot rows per CTA in a forward step
  static constexpr int CT = 32;   // pivot columns per CTA in a backward step
  static constexpr int BM = 128;  // update rows per CTA of the forward L21 product
  static constexpr int BN = 64;   // pivot columns per CTA of the backward L21 product
  static constexpr int KC = 32;   // inner chunk of both products
};
template <>
struct SolveTile<double> {
  static constexpr int RT = 16;
  static constexpr int CT = 16;
  static constexpr int BM = 64;
  static constexpr int BN = 64;
  static constexpr int KC = 16;
};

// Grid sizes of one pivot step of one level (host-computed).
struct StepDims {
  int nfronts;        // fronts of the level with k > step*NB (a prefix: sorted by k desc)
  int panel_tiles;
  int update_tiles;   // trailing update of the whole trailing triangle
  int update_tiles_blk;  // trailing update restricted to the step's kKB block (tensor-core factor)
  int fwd_tiles;
  int bwd_tiles;
};

// One output tile of a front product of the FP32 solves (host-built, per
// level and mode), tensor-core form.  A is read through the tensor map
// `map` (3-D: floats along a column, columns, poles; zero outside the block)
// at coordinates (x0, y0) + the chunk offset: column-major modes step the
// column y, row-major modes the float x.  B row kk is bbase + kk
// (contiguous) or rows[bbase + kk] (gathered); outputs are rows obase + m
// (stores) or rows[obase + m] (atomic subtraction).  Tiles start at even
// rows: output rows m < mfirst and inner indices kk < kfirst (B zero there)
// are padding of a front with an odd number of pivots.
struct TcTask {
  int32_t map, x0, y0;
  int32_t kdim;    // inner dimension (0: no product, the epilogue still runs)
  int32_t mrows;   // rows of the 64-row tile inside the block
  int32_t bbase;
  int32_t obase;
  int16_t mfirst, kfirst;
};
static_assert(sizeof(TcTask) == 32, "TcTask is loaded as two 16-byte vectors");

// The same tile for the SIMT kernel: A element (m, kk) at aoff + kk * lda + m
// (column-major modes) or aoff + m * lda + kk (row-major modes).
struct SimtTask {
  int64_t aoff;
  int32_t lda, kdim, mrows, bbase, obase;
  int16_t mfirst, kfirst;
};

// The four front products of the FP32 solves (explicit inverses T11 = L11^-1):
//   TRI_F  X[c0+i]      = sum_c T11[i][c] Y[c0+c]              (store)
//   FWD21  Y[rows_i]   -= sum_c L21[i][c] X[c0+c]              (atomic)
//   BWD21  Y[c0+c]      = Dinv_c X[c0+c] - sum_i L21[i][c] X[rows_i]   (store)
//   TRI_B  X[c0+c]      = sum_i T11[i][c] Y[c0+i]              (store)
enum ProdMode { PM_TRI_F = 0, PM_FWD21 = 1, PM_BWD21 = 2, PM_TRI_B = 3, PM_COUNT = 4 };
// The same kernel's trailing update of the FP32 factorisation (Algorithm 1, factorise):
//   F[r][s] -= sum_c L[r][j0 + c] D_c L[s][j0 + c],  c < kb (one kKB block), r >= s >= t0 = j0 + kb,
// into the factor block (s < k) or the update block (s >= k).  TcTask fields in this mode:
//   map = front, x0 = panel-copy row of front row 0 (A row = x0 + y0 + m), y0 = first row r0 of the
//   tile, kdim = kb, mrows = rows of the tile, bbase = first column s0 (even), obase = j0,
//   mfirst = t0 - s0 (leading columns left alone), kfirst = 0.
constexpr int PM_UPD = 4;

// The tensor-core trailing update after one kKB block of every front of a level.
struct UpdBlock {
  const TcTask *tasks = nullptr;   // 128-row x 32-column tiles (all fronts of the level)
  int ntask = 0;
  const int4 *copies = nullptr;    // (front, panel-copy row of front row 0, t0, kb): rows t0..n-1 copied
  int ncopy = 0;
  int copy_tiles = 0;              // 32-row tiles of the largest n - t0
};

// One tile task of the in-place inversion of L11 (merge of two diagonal
// blocks A = [a0, a0+s), C = [a0+s, a0+s+sc)): 64 x 64 tile (ti, tj) of the
// sc x s block; Y scratch of the pair at ybase (column-major, ld sc).
struct InvTask {
  int32_t front, a0, s, sc;
  int32_t ti, tj;
  int64_t ybase;
};

struct LevelDev {
  const int32_t *fronts = nullptr;  // device list, sorted by k descending
  int nf = 0;
  int h = 0;                        // level index (height in the assembly tree)
  const int2 *f21_tasks = nullptr;  // (front, row tile) of the forward L21 product
  int n_f21 = 0;
  const int2 *b21_tasks = nullptr;  // (front, column tile) of the backward L21 product
  int n_b21 = 0;
  int bwd_upd_tiles = 0;            // ceil(max k / 8)
  int64_t lbeg = 0, lend = 0, obeg = 0, oend = 0;
  int64_t ea_beg[4] = {}, ea_end[4] = {};   // extend-add tasks per child slot
  std::vector<StepDims> steps;
  struct SuperBlock {
    const int4 *fwd = nullptr;   // (front, row tile, k begin, k end) of k_fwd_sb
    int n_fwd = 0;
    const int4 *bwd = nullptr;   // (front, column tile, row begin, row end) of k_bwd_sb
    int n_bwd = 0;
  };
  std::vector<SuperBlock> sb;
  // FP32 solves: front-product tasks per mode
  const TcTask *prod[PM_COUNT] = {nullptr, nullptr, nullptr, nullptr};
  const SimtTask *prod_simt[PM_COUNT] = {nullptr, nullptr, nullptr, nullptr};
  int n_prod[PM_COUNT] = {0, 0, 0, 0};        // tensor-core tiles (128 columns wide for BWD21 / TRI_B)
  int n_prod_simt[PM_COUNT] = {0, 0, 0, 0};   // SIMT tiles (64 wide)
  // FP32 factorisation: inversion of L11, per merge stage (block size 32 * 2^stage)
  struct InvStage {
    const InvTask *tasks = nullptr;
    int n = 0;
  };
  std::vector<InvStage> inv;
  const int2 *inv_diag = nullptr;   // (front, 32-block) of every diagonal block
  int n_inv_diag = 0;
  // FP32 factorisation: (front, 0 = T11 / 1 = L21, 32-row block) of the row-major copies
  const int4 *rcopy = nullptr;
  int n_rcopy = 0;
  int max_k = 0;   // largest pivot count of the level's fronts
  // FP32 factorisation on the tensor cores: one entry per kKB block of pivots
  std::vector<UpdBlock> upd;
};

template <typename R>
struct FactorPlan {
  int m = 0;
  cx<R> *L = nullptr;
  int64_t lstride = 0;
  cx<R> *U = nullptr;
  int64_t ustride = 0;
  const FrontDev *F = nullptr;
  const int32_t *rel = nullptr;
  const int32_t *ea_child = nullptr;
  const int32_t *ea_col = nullptr;
  const int64_t *orig_nz = nullptr;
  const int64_t *orig_dst = nullptr;
  const double *kval = nullptr;
  const double *mval = nullptr;
  int64_t mstride = 0;              // pole stride of mval (0: one M for all poles)
  const double2 *xi = nullptr;
  cx<R> *dscr = nullptr;            // [max fronts per level][m][NB*NB]
  cx<R> *linv = nullptr;            // [m][inv blocks][NB*NB] diagonal-block inverses (output)
  int64_t istride = 0;
  DevStatus *status = nullptr;
  // FP32: L11 is replaced by its inverse after each level; D^-1 goes to dinv
  cx<R> *dinv = nullptr;            // [m][N]
  int64_t N = 0;
  cx<R> *yscr = nullptr;            // inversion scratch [m][yscr_stride]
  int64_t yscr_stride = 0;
  cx<R> *T11R = nullptr, *L21T = nullptr;   // row-major copies for the tensor-core products
  int64_t t11r_stride = 0, l21t_stride = 0;
  const int64_t *t11r_ofs = nullptr, *l21t_ofs = nullptr;   // per front
  // FP32 trailing updates on the tensor cores (kKB blocks): row-major panel copies and tensor maps
  bool tc_update = false;
  cx<R> *Pc = nullptr;              // [m][prows][kKB] panel copy
  int64_t pstride = 0;              // prows * kKB
  const void *cmaps = nullptr;      // per front: column blocks of the factor store (B operand)
  const void *pcmap = nullptr;      // the panel copy (A operand)
  void level(int h, const LevelDev &lv, cudaStream_t s);
  void invert_level(const LevelDev &lv, cudaStream_t s);
};

template <>
void FactorPlan<float>::invert_level(const LevelDev &lv, cudaStream_t s);
template <>
void FactorPlan<double>::invert_level(const LevelDev &lv, cudaStream_t s);

template <typename R>
struct SolvePlan {
  int m = 0;
  int nrhs = 0;
  const cx<R> *L = nullptr;
  int64_t lstride = 0;
  const cx<R> *Linv = nullptr;
  int64_t istride = 0;
  const FrontDev *F = nullptr;
  const int32_t *rows = nullptr;
  cx<R> *Y = nullptr;   // [m][N][nrhs] right-hand sides in, work space
  cx<R> *X = nullptr;   // [m][N][nrhs] solution out
  int64_t vstride = 0;  // N * nrhs
  const int *pmap = nullptr;  // device list of the poles to solve (nullptr: all)
  int np = 0;                 // poles solved
  bool use_tc = false;        // FP32: front products on the tensor cores
  const cx<R> *dinv = nullptr;  // FP32: [m][N] inverse pivots
  const void *tmaps = nullptr;  // FP32: 4 tensor maps per front (one per product mode)
  const void *vmaps = nullptr;  // FP32: tensor maps of Y and X, and the row-gather map of X (nullptr for an odd nrhs)
  int64_t N = 0;
  DevStatus *status = nullptr;
  void forward_level(const LevelDev &lv, cudaStream_t s);
  void backward_level(const LevelDev &lv, cudaStream_t s);
};

// FP32 front products (solve_tc.cu): tensor cores (P.use_tc) or SIMT.
void launch_prod(int mode, const SolvePlan<float> &P, const LevelDev &lv, cudaStream_t s);
// Tensor-core trailing update of one kKB block of a level's fronts (solve_tc.cu).
void launch_tc_update(const FactorPlan<float> &P, const UpdBlock &ub, cudaStream_t s);

// Resident CTAs per SM of the tensor-core product kernel (0 before its first launch).
int tc_ctas_per_sm();
// Limits of the tensor-core pipeline waits (library-wide; defaults 2^26 polls, 1 s).
void set_tc_wait_limit(uint32_t polls, uint64_t ns);
// FP32 solve-product launches on the tensor cores (true) or the FP32 pipes, library-wide.
int64_t prod_launches(bool tensor_cores);
// Tensor-core trailing-update launches of the FP32 factorisations, library-wide.
int64_t update_launches();
// Tensor maps of every front's factor block (4 per front, index 4 f + mode)
// in a new device array (*out, cudaFree by the caller); "" on success.
struct FrontGeom {
  int64_t lofs, t11r_ofs, l21t_ofs;
  int32_t n, k, ld, ld2;
};
// The factor store and its row-major copies (FP32 mode), pole strides in elements.
struct FactorViews {
  const c64 *L;
  int64_t lstride;
  const c64 *T11R;     // per front k x ld2, row i = T11[i][0..k) (zero above the diagonal)
  int64_t t11r_stride;
  const c64 *L21T;     // per front b x ld2, row i = L21[i][0..k)
  int64_t l21t_stride;
};
std::string build_tensor_maps(const std::vector<FrontGeom> &fronts, const FactorViews &v, int m, void **out);
// Maps over [pole][rows][nrhs] complex vectors (pole stride rows * nrhs), in
// order (boxes of 16 rows x 32 right-hand sides), then one row-gather map
// over bufs[gather] seen as m * rows rows of nrhs values (boxes of one row x
// 32 right-hand sides, for tile::gather4 loads).
struct VecBuf {
  const c64 *base;
  int64_t rows;
};
std::string build_vector_maps(const std::vector<VecBuf> &bufs, int gather, int nrhs, int m, void **out);
// Maps for it: per front a map over its column-major factor block (boxes of 32 complex rows x 16
// columns), and one over the panel copy [m][prows][kKB] (boxes of 128 rows x 16 complex).
std::string build_update_maps(const std::vector<FrontGeom> &fronts, const c64 *L, int64_t lstride, const c64 *Pc,
                              int64_t prows, int m, void **cmaps, void **pcmap);

void launch_sigma(const double *logs, const int32_t *ptet, int64_t P, double *sigma, cudaStream_t s);
// mval[z] = sum over the contributions idx of entry z: sigma[idx / per] * me1[idx]
void launch_mvals(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                  const double *me1, int per, int64_t nnz, double *mval, cudaStream_t s);
void launch_mvals(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                  const double *me1, int per, int64_t nnz, float *mval, cudaStream_t s);   // FP32 result
void launch_mvals_floor(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                        const double *tetfloor, const double *me1, const double2 *xi, double tau, int m,
                        int64_t nnz, double *mval, cudaStream_t s);

// ---- ops.cu ----
// b (c128, pole stride bstride elements, may be 0) -> Y (R) scaled per (pole, rhs) column
// by 1/colmax; colmax [m][nrhs] written (FP32 mode).  With scale == false a plain copy.
// All four take a pole map (device, np entries; nullptr = poles 0..np-1).
template <typename R>
void launch_rhs_to_work(const c128 *b, int64_t bstride, cx<R> *Y, double *colmax, int np, const int *pmap,
                        int64_t N, int nrhs, bool scale, cudaStream_t s);
// x (c128) (+)= colmax * X (R)
template <typename R>
void launch_accumulate(const cx<R> *X, const double *colmax, c128 *x, int np, const int *pmap, int64_t N,
                       int nrhs, bool add, cudaStream_t s);
// r = b - (K - xi_p M) x,  FP64
void launch_residual(const int64_t *rp, const int32_t *ci, const double *kv, const double *mv,
                     const double2 *xi, const c128 *b, int64_t bstride, const c128 *x, c128 *r,
                     int np, const int *pmap, int64_t N, int nrhs, cudaStream_t s);
// Refinement progress of each mapped pole over the masked unknowns:
// num[p] = max |colmax * X|, den[p] = max |x| (double bits, max-accumulated).
template <typename R>
void launch_progress(const cx<R> *X, const double *colmax, const c128 *x, const uint8_t *mask, double *num,
                     double *den, int np, const int *pmap, int64_t N, int nrhs, cudaStream_t s);
// ---- refine.cu: FP32-mode refinement in double-float pairs ----
void launch_split_real(const double *v, float2 *out, int64_t n, cudaStream_t s);   // v -> (hi, lo)
void launch_split_cx(const c128 *v, float4 *out, int64_t n, cudaStream_t s);       // (re.hi, re.lo, im.hi, im.lo)
void launch_join_cx(const float4 *v, c128 *out, int64_t n, cudaStream_t s);        // hi + lo in FP64
// r (FP32) = b - K x + xi_p (M x) with b, x, K, M as pairs
void launch_residual_df(const int64_t *rp, const int32_t *ci, const float2 *kdf, const float2 *mdf,
                        const double2 *xi, const float4 *bdf, int64_t bstride, const float4 *xdf, c64 *r, int np,
                        const int *pmap, int64_t N, int nrhs, cudaStream_t s);
// colmax (FP32) = column maxima of v, Y = v / colmax; v complex FP32 or pairs (hi parts)
template <typename T>
void launch_scale_to_work(const T *v, int64_t vstride, c64 *Y, float *colmax, int np, const int *pmap, int64_t N,
                          int nrhs, cudaStream_t s);
// The gradient-space part of a refinement step's x update (Xn == nullptr: none):
// x_p[d] += -(psi[e_hi[d]] - psi[e_lo[d]]) * ninv_xi[p], psi = colmax_n * Xn ([Nn][ncol]).
struct NodalPart {
  const c64 *Xn = nullptr;
  const float *colmax_n = nullptr;
  const int32_t *e_lo = nullptr, *e_hi = nullptr;
  const float2 *ninv_xi = nullptr;   // -1 / xi_p
  int ncol = 0;
};
// x (+)= colmax X in pairs (plus the nodal part)
void launch_accumulate_df(const c64 *X, const float *colmax, float4 *x, int np, const int *pmap, int64_t N, int nrhs,
                          bool add, cudaStream_t s, const NodalPart &nd = NodalPart());
// Gradient-space correction (refine.cu): Yn[a][p nrhs + j] = (G^T r_p)[a][j] for the
// mapped poles (Yn [Nn][m nrhs], other poles' columns zeroed when pmap is set) ...
void launch_nodal_rhs(const int64_t *g_ptr, const int32_t *g_edge, const int8_t *g_sign, const c64 *r, c64 *Yn,
                      int64_t Nn, int np, const int *pmap, int m, int64_t N, int nrhs, cudaStream_t s);
// ... and with psi = colmax_n Xn: r_p -= M(sigma) G psi_p (C = M G in CSR, FP32 values)
void launch_nodal_apply(const int64_t *c_rp, const int32_t *c_ci, const float *c_val, const c64 *Xn,
                        const float *colmax_n, c64 *r, int np, const int *pmap, int m, int64_t N, int nrhs,
                        cudaStream_t s);
void launch_progress_df(const c64 *X, const float *colmax, const float4 *x, const uint8_t *mask, double *num,
                        double *den, int np, const int *pmap, int64_t N, int nrhs, cudaStream_t s);
// F (real [N][nrhs]) -> c128 b
void launch_real_to_c128(const double *f, c128 *b, int64_t count, cudaStream_t s);
// d[x][r][j] = 2 Re sum_p alpha_pj (Q y_p)[r][x] for x < ntx (vector rows of nrhs >= ntx)
void launch_residue(const int64_t *q_rp, const int32_t *q_ci, const double *q_val,
                    const double2 *alpha, const c128 *y, double *d, int m, int64_t N, int nrhs,
                    int ntx, int n_rx, int K, cudaStream_t s);
// the same from the refined iterate's double-float pairs [m][N][nrhs] (FP32 mode, no FP64 copy)
void launch_residue(const int64_t *q_rp, const int32_t *q_ci, const double *q_val,
                    const double2 *alpha, const float4 *y, double *d, int m, int64_t N, int nrhs,
                    int ntx, int n_rx, int K, cudaStream_t s);
// rhs_p[dof][x] = sum_r Qt[dof][r] sum_j alpha_pj w[x][r][j], x < ntx (zeroes rhs first)
void launch_qt_rhs(const int32_t *qt_dof, const int64_t *qt_rp, const int32_t *qt_ci,
                   const double *qt_val, int n_qdof, const double2 *alpha, const double *w, c128 *rhs,
                   int m, int64_t N, int nrhs, int ntx, int n_rx, int K, cudaStream_t s);
// the same as the double-float pairs of the FP32 refinement
void launch_qt_rhs(const int32_t *qt_dof, const int64_t *qt_rp, const int32_t *qt_ci,
                   const double *qt_val, int n_qdof, const double2 *alpha, const double *w, float4 *rhs,
                   int m, int64_t N, int nrhs, int ntx, int n_rx, int K, cudaStream_t s);
// h_p[d][x] = xi_p sum_{(t,a) at d} v_t sigma_t sum_b M1_t[a][b] g_p[tdof_t[b]][x]
void launch_dm_apply(const int64_t *inc_ptr, const int32_t *inc_tet, const int8_t *inc_loc,
                     const int32_t *tdof, const int32_t *pidx, const double *v, const double *sigma,
                     const double *me1, const double2 *xi, const c128 *g, c128 *h, int m, int64_t N,
                     int nrhs, cudaStream_t s);
// grad[p] = 2 Re sum_i xi_i sigma_t sum_x (P z_ix)^T M1_t (P g_ix), t = ptet[p] (FP64)
void launch_bilinear(const int32_t *ptet, int64_t P, const int32_t *tdof, const double *sigma,
                     const double *me1, const double2 *xi, const c128 *g, const c128 *z, double *grad,
                     int m, int64_t N, int nrhs, cudaStream_t s);
// the same from pairs (g, z float4 [m][N][nrhs], M1 float2 [nt][36]) in double-float
// arithmetic; part: scratch [m][P] of per-pole cell sums
void launch_bilinear_df(const int32_t *ptet, int64_t P, const int32_t *tdof, const double *sigma,
                        const float2 *me1df, const double2 *xi, const float4 *gdf, const float4 *zdf, double *grad,
                        int m, int64_t N, int nrhs, double *part, cudaStream_t s);
// J v right-hand sides from pairs (vs: scratch [nt] for v_t sigma_t as pairs)
void launch_dm_apply_df(const int64_t *inc_ptr, const int32_t *inc_tet, const int8_t *inc_loc, const int32_t *tdof,
                        const int32_t *ptet, int64_t P, const double *v, const double *sigma, float2 *vs, int64_t nt,
                        const float2 *me1df, const double2 *xi, const float4 *gdf, float4 *h, int m, int64_t N,
                        int nrhs, cudaStream_t s);
// sparse y = A x (CSR) and y = A^T x via the transpose CSR; beta-scaled accumulate
void launch_csr_mv(const int64_t *rp, const int32_t *ci, const double *val, const double *x, double *y,
                   int64_t rows, double alpha, double beta, cudaStream_t s);

// Gauss-Newton bookkeeping: t = wd (d - d_obs), t2 = wd^2 (d - d_obs); *out += x . y; out = m + eta dm
void launch_gn_res(const double *d, const double *d_obs, const double *wd, double *t, double *t2, int64_t n,
                   cudaStream_t s);
void launch_dot(const double *x, const double *y, int64_t n, double *out, cudaStream_t s);
void launch_axpy(const double *m, const double *dm, double eta, double *out, int64_t n, cudaStream_t s);

// residues of the rational approximant for new observation times (rational.cu):
// basis + Householder QR of the penalised least-squares matrix, then one solve per time
void launch_fit_qr(const double2 *xi, int m, int64_t nz, double lz0, double lz1, double mu, double *B,
                   double *rdiag, double *cf, cudaStream_t s);
void launch_fit_solve(const double *B, int m, int64_t nz, double lz0, double lz1, const double *rdiag,
                      const double *cf, const double *t, int K, double *Y, double2 *alpha, cudaStream_t s,
                      double *coef = nullptr, double *tail_sq = nullptr);
// variable projection: Kaufman Jacobian tails T [K][2m][rows] and the normal
// equations G [2m][2m + 1] (J^T J | J^T r up to sign) of the pole fit
void launch_vp_normal(const double *B, int m, int64_t nz, double lz0, double lz1, double mu, const double2 *xi,
                      const double *cf, const double *coef, int K, const double *Y, double *T, double *G,
                      cudaStream_t s);

// status words before a factorisation (a kernel, so that the call stays capturable)
void launch_status_init(DevStatus *st, cudaStream_t s);

// ---- LSQR helpers (ops.cu) ----
struct LsqrScalars {
  double alpha, beta, rhobar, phibar, rho, c, sn, theta, phi;
  double sumsq;  // reduction target
};
void launch_sumsq(const double *x, int64_t n, double *out, cudaStream_t s);   // *out += sum x^2
// element-wise LSQR steps (op codes in ops.cu), scalars read on the device
void launch_lsqr_kernel(int op, LsqrScalars *sc, double *a, const double *b, const double *c,
                        const double *wd, int64_t n, cudaStream_t s);
void launch_lsqr_scalars(LsqrScalars *sc, int which, cudaStream_t s);

// Kernel classes that can be timed individually with CUDA events.
enum KernelClass {
  KC_UPDATE = 0, KC_PANEL, KC_FWD, KC_BWD, KC_BWD_UPD, KC_EXTEND_ADD, KC_FWD21, KC_FWD_SB, KC_BWD_SB, KC_INVERT, KC_RESIDUAL, KC_REFINE_VEC, KC_JACOBIAN,
  KC_NODAL, KC_NODAL_RHS, KC_NODAL_SWEEP, KC_NODAL_APPLY, KC_UPDATE_TC,
  KC_COUNT
};
struct Profiler {
  bool on = false;
  bool muted = false;                  // inside a timed composite (the nodal correction)
  int cls = -1;                        // class being timed
  int level = -1;                      // tree level being timed (-1: all)
  int cur_level = -1;                  // level of the launches being issued
  std::vector<cudaEvent_t> pool;       // start/stop pairs
  int used = 0;
  double total_ms = 0;
  int64_t launches = 0;
  void begin(int c, cudaStream_t s);
  void end(int c, cudaStream_t s);
  void collect();                      // after a stream synchronise
  void release();
};
extern thread_local Profiler *g_prof;   // set by the API layer around a call

// Kernel launches issued by this library (all threads), for reporting.
int64_t launch_total();
void count_launch();

}  // namespace tem
