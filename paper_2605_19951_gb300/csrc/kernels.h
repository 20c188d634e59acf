// Internal interface between the C-ABI layer (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace tem {

constexpr int kNB = 32;        // pivot block width of the blocked LDL^T and the solves
constexpr int kPanelRT = 128;  // panel rows per CTA
constexpr int kSB = 256;       // super-block of the solves' pivot blocks (multiple of kNB)
constexpr int kSplitK = 512;   // inner-dimension chunk of one super-block product task

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
  int update_tiles;
  int fwd_tiles;
  int bwd_tiles;
};

struct LevelDev {
  const int32_t *fronts = nullptr;  // device list, sorted by k descending
  int nf = 0;
  int h = 0;                        // level index (height in the assembly tree)
  const int2 *f21_tasks = nullptr;  // (front, row tile) of the forward L21 product
  int n_f21 = 0;
  const int2 *b21_tasks = nullptr;  // (front, column tile) of the backward L21 product
  int n_b21 = 0;
  const int2 *f21tc_tasks = nullptr;  // the same for the tensor-core kernels (64-row / 64-column tiles)
  int n_f21tc = 0;
  const int2 *b21tc_tasks = nullptr;
  int n_b21tc = 0;
  int bwd_upd_tiles = 0;            // ceil(max k / 8)
  int64_t lbeg = 0, lend = 0, obeg = 0, oend = 0;
  int64_t ea_beg[2] = {0, 0}, ea_end[2] = {0, 0};
  std::vector<StepDims> steps;
  struct SuperBlock {
    const int4 *fwd = nullptr;   // (front, row tile, k begin, k end) of k_fwd_sb
    int n_fwd = 0;
    const int4 *bwd = nullptr;   // (front, column tile, row begin, row end) of k_bwd_sb
    int n_bwd = 0;
  };
  std::vector<SuperBlock> sb;
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
  void level(int h, const LevelDev &lv, cudaStream_t s);
};

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
  bool use_tc = false;        // FP32: update-row products on the tensor cores
  DevStatus *status = nullptr;
  void forward_level(const LevelDev &lv, cudaStream_t s);
  void backward_level(const LevelDev &lv, cudaStream_t s);
};

void launch_fwd_l21_tc(const SolvePlan<float> &P, const LevelDev &lv, DevStatus *st, cudaStream_t s);
void launch_bwd_l21_tc(const SolvePlan<float> &P, const LevelDev &lv, DevStatus *st, cudaStream_t s);

void launch_sigma(const double *logs, const int32_t *ptet, int64_t P, double *sigma, cudaStream_t s);
void launch_mvals(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                  const double *me1, int64_t nnz, double *mval, cudaStream_t s);
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
// F (real [N][nrhs]) -> c128 b
void launch_real_to_c128(const double *f, c128 *b, int64_t count, cudaStream_t s);
// d[x][r][j] = 2 Re sum_p alpha_pj coef_p (Q y_p)[r][x]; coef = 1 (forward) or xi_p
void launch_residue(const int64_t *q_rp, const int32_t *q_ci, const double *q_val,
                    const double2 *alpha, const c128 *y, double *d, int m, int64_t N, int nrhs,
                    int n_rx, int K, cudaStream_t s);
// rhs_p[dof][x] = sum_r Qt[dof][r] sum_j alpha_pj w[x][r][j] (zeroes rhs first)
void launch_qt_rhs(const int32_t *qt_dof, const int64_t *qt_rp, const int32_t *qt_ci,
                   const double *qt_val, int n_qdof, const double2 *alpha, const double *w, c128 *rhs,
                   int m, int64_t N, int nrhs, int n_rx, int K, cudaStream_t s);
// h_p[d][x] = xi_p sum_{(t,a) at d} v_t sigma_t sum_b M1_t[a][b] g_p[tdof_t[b]][x]
void launch_dm_apply(const int64_t *inc_ptr, const int32_t *inc_tet, const int8_t *inc_loc,
                     const int32_t *tdof, const int32_t *pidx, const double *v, const double *sigma,
                     const double *me1, const double2 *xi, const c128 *g, c128 *h, int m, int64_t N,
                     int nrhs, cudaStream_t s);
// grad[p] = 2 Re sum_i xi_i sigma_t sum_x (P z_ix)^T M1_t (P g_ix), t = ptet[p]
void launch_bilinear(const int32_t *ptet, int64_t P, const int32_t *tdof, const double *sigma,
                     const double *me1, const double2 *xi, const c128 *g, const c128 *z, double *grad,
                     int m, int64_t N, int nrhs, cudaStream_t s);
// sparse y = A x (CSR) and y = A^T x via the transpose CSR; beta-scaled accumulate
void launch_csr_mv(const int64_t *rp, const int32_t *ci, const double *val, const double *x, double *y,
                   int64_t rows, double alpha, double beta, cudaStream_t s);

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
  KC_UPDATE = 0, KC_PANEL, KC_FWD, KC_BWD, KC_BWD_UPD, KC_EXTEND_ADD, KC_FWD21, KC_FWD_SB, KC_BWD_SB, KC_COUNT
};
struct Profiler {
  bool on = false;
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
