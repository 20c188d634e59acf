// C ABI of libtem (see include/tem.h): context, device memory, and the
// orchestration of factor / forward / J v / J^T w / LSQR on one GPU.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/tem.h"
#include "kernels.h"
#include "tem_internal.h"

using namespace tem;

#include <atomic>

namespace tem {
thread_local Profiler *g_prof = nullptr;
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(); }

void Profiler::begin(int c, cudaStream_t s) {
  if (!on || muted || c != cls || (level >= 0 && cur_level != level)) return;
  if (used + 2 > (int)pool.size()) {
    size_t old = pool.size();
    pool.resize(std::max<size_t>(64, 2 * old + 2));
    for (size_t i = old; i < pool.size(); i++) cudaEventCreate(&pool[i]);
  }
  cudaEventRecord(pool[used], s);
}
void Profiler::end(int c, cudaStream_t s) {
  if (!on || muted || c != cls || (level >= 0 && cur_level != level)) return;
  cudaEventRecord(pool[used + 1], s);
  used += 2;
}
void Profiler::collect() {
  for (int i = 0; i + 1 < used; i += 2) {
    float ms = 0;
    cudaEventElapsedTime(&ms, pool[i], pool[i + 1]);
    total_ms += ms;
    launches++;
  }
  used = 0;
}
void Profiler::release() {
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
  used = 0;
}
}  // namespace tem

namespace {

enum StateBits { ST_MESH = 1, ST_POLES = 2, ST_SOURCES = 4, ST_FACTORED = 8, ST_FORWARD = 16 };

template <typename T>
struct DVec {
  T *p = nullptr;
  size_t n = 0;
};

}  // namespace

// One family of sparse complex-symmetric matrices A_p = K - xi_p M_p (p < m)
// sharing a pattern: its assembly tree, the task lists of the factor and
// solve kernels, the factor store and the solve vectors.
struct FactorSys {
  Symbolic sym;
  int64_t N = 0;                          // unknowns
  int m = 0;                              // matrices factored together (pole dimension)
  int nrhs = 0;                           // right-hand sides per vector row (even)
  std::vector<LevelDev> levels;
  int max_level_fronts = 0;
  int64_t inv_blocks = 0;                 // diagonal-block inverses per pole
  std::vector<int2> f21_h, b21_h;         // task lists of the L21 products (all levels)
  int2 *f21 = nullptr, *b21 = nullptr;
  std::vector<int4> sbf_h, sbb_h;         // task lists of the super-block products
  int4 *sbf = nullptr, *sbb = nullptr;
  std::vector<TcTask> prod_h;             // FP32: front-product tasks (all levels and modes)
  TcTask *prod = nullptr;
  std::vector<SimtTask> prod_simt_h;      // the same tiles for the SIMT products
  SimtTask *prod_simt = nullptr;
  void *tmaps = nullptr;                  // FP32: tensor maps of the factor blocks
  void *vmaps = nullptr;                  // FP32: tensor maps of the solve vectors
  std::vector<int4> rcopy_h;              // FP32: row-major copy tasks (all levels)
  int4 *rcopy = nullptr;
  std::vector<int64_t> t11r_ofs_h, l21t_ofs_h;   // FP32: per front offsets of the row-major copies
  int64_t *t11r_ofs = nullptr, *l21t_ofs = nullptr;
  int64_t t11r_total = 0, l21t_total = 0;
  void *T11R = nullptr, *L21T = nullptr;
  std::vector<InvTask> inv_h;             // FP32: pivot-block inversion tasks
  InvTask *inv = nullptr;
  std::vector<int2> invdiag_h;
  int2 *invdiag = nullptr;
  int64_t yscr_stride = 0;                // inversion scratch per pole
  // FP32: tensor-core trailing updates per kKB block (all levels)
  std::vector<TcTask> upd_h;
  TcTask *upd = nullptr;
  std::vector<int4> ucopy_h;
  int4 *ucopy = nullptr;
  int64_t prows = 0;                      // rows of the panel copy (largest level block)
  void *Pc = nullptr;                     // [m][prows][kKB] c64
  void *cmaps = nullptr, *pcmap = nullptr;
  // device symbolic tables
  FrontDev *fronts = nullptr;
  int32_t *rows = nullptr, *rel = nullptr, *ea_child = nullptr, *ea_col = nullptr, *levfronts = nullptr;
  int64_t *orig_nz = nullptr, *orig_dst = nullptr;
  // numeric
  void *L = nullptr, *U = nullptr, *dscr = nullptr, *Y = nullptr, *X = nullptr, *linv = nullptr;
  void *dinv = nullptr, *yscr = nullptr;   // FP32: inverse pivots, inversion scratch
  // matrix values: A_p = K - xi_p M_p, M_p = mval + p * mstride
  const double *kval = nullptr;
  const double *mval = nullptr;
  int64_t mstride = 0;
  const double2 *xi = nullptr;
};

struct tem_ctx {
  int precision = TEM_FP64;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;
  int state = 0;
  int refine = 3;
  int refine_adj = 1;        // FP32 mode: corrections per adjoint (J^T w) solve
  double floor_tau = 1e-6;   // FP32 mode: conductivity floor of the factored matrix
  double refine_tol = 0.0;   // FP32 mode: stop a pole's refinement below this progress (0: fixed count)
  int64_t pole_solves = 0;   // statistics: poles x sweeps pairs issued
  int64_t solve_calls = 0;
  uint8_t *earth = nullptr;  // unknowns on edges of parameter cells (what every output reads)
  int *pmap = nullptr;       // device list of the poles still refining
  double *prog = nullptr;    // [2m] progress maxima
  int64_t bytes = 0;
  std::vector<void *> allocs;
  Profiler prof;

  Mesh mesh;
  FactorSys es;                           // the shifted edge systems A_i = K - xi_i M (all poles)
  FactorSys ns;                           // FP32 mode: the nodal gradient-space Laplacian (one matrix)
  NodalMesh nodal;
  bool use_tc = true;                     // FP32 mode: front products on tcgen05
  bool tc_fronts = true;                  // FP32 mode: trailing updates of the fronts on tcgen05
  bool async = false;                     // calls return once issued; tem_status reads the status words
  SymOpts sym_opts;                       // dissection and amalgamation options of tem_mesh

  // mesh tables
  double *sigma_fixed = nullptr, *sigma = nullptr, *me1 = nullptr, *kval = nullptr, *mval = nullptr;
  double *tetfloor = nullptr, *mval_fact = nullptr;   // FP32 mode: per-pole floored M values
  int64_t *rp = nullptr, *mc_ptr = nullptr, *inc_ptr = nullptr;
  int32_t *ci = nullptr, *inc_tet = nullptr, *tdof = nullptr, *pidx = nullptr, *ptet = nullptr;
  uint32_t *mc_idx = nullptr;
  int8_t *inc_loc = nullptr;
  int64_t *w_rp = nullptr, *wt_rp = nullptr;
  int32_t *w_ci = nullptr, *wt_ci = nullptr;
  double *w_val = nullptr, *wt_val = nullptr;

  // FP32 mode: nodal gradient-space correction of the refinement
  bool use_nodal = true;
  int32_t *n_tnode = nullptr, *n_elo = nullptr, *n_ehi = nullptr, *n_gedge = nullptr;
  int64_t *n_mc_ptr = nullptr, *n_gptr = nullptr;
  uint32_t *n_mc_idx = nullptr;
  int8_t *n_gsign = nullptr;
  double *n_stiff = nullptr, *n_kval = nullptr, *n_mval = nullptr;
  int64_t *n_crp = nullptr, *n_cmc_ptr = nullptr;   // C = M(sigma) G: rows and contribution lists
  int32_t *n_cci = nullptr;
  uint32_t *n_cmc_idx = nullptr;
  double *n_btab = nullptr;
  float *n_cval = nullptr;                          // C values (FP32: they only feed the FP32 correction)
  float2 *ninv_xi = nullptr;                        // -1 / xi_p
  double2 *n_xi = nullptr;
  float *colmax_n = nullptr;   // column scales of the nodal solves
  double *part = nullptr;      // [m][P] per-pole J^T w cell sums (FP32 mode)
  float2 *me1df = nullptr;     // FP32 mode: M1 element matrices as pairs [nt][36]
  float4 *gdf = nullptr;       // FP32 mode: forward solutions as pairs [m][N][nrhs]
  float2 *vsdf = nullptr;      // FP32 mode: v_t sigma_t as pairs [nt] (J v right-hand sides)

  // poles
  int m = 0, K = 0;
  std::vector<double> xi_h, alpha_h;
  double2 *xi = nullptr, *alpha = nullptr;

  // sources
  int n_tx = 0, n_rx = 0, n_qdof = 0;
  int nrhs = 0;   // right-hand sides per vector row: n_tx rounded up to even (TMA rows of 16 bytes)
  double *f = nullptr;
  int64_t *q_rp = nullptr, *qt_rp = nullptr;
  int32_t *q_ci = nullptr, *qt_ci = nullptr, *qt_dof = nullptr;
  double *q_val = nullptr, *qt_val = nullptr;

  // numeric
  float2 *kdf = nullptr, *mdf = nullptr;   // FP32: K and M values as double-float pairs
  float4 *xdf = nullptr;                   // FP32: refined iterate as pairs [m][N][nrhs]
  float *colmax_f = nullptr;               // FP32: column scales of the correction solves
  DevStatus *status = nullptr;
  c128 *g = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *fb = nullptr;
  double *colmax = nullptr;
  DevStatus status_h{};

  // LSQR
  double *ls_u = nullptr, *ls_v = nullptr, *ls_w = nullptr, *ls_jv = nullptr, *ls_jtw = nullptr,
         *ls_tmpd = nullptr, *ls_tmpp = nullptr, *ls_dm = nullptr, *ls_wv = nullptr;
  LsqrScalars *ls_sc = nullptr;
  double *d_cur = nullptr;   // data of the last tem_forward
  double *m_cur = nullptr;   // model of the last tem_factor
};

namespace {

thread_local std::string g_create_err;

int fail(tem_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(tem_ctx *c, cudaError_t e, const char *where) {
  cudaGetLastError();
  int code = (e == cudaErrorMemoryAllocation) ? TEM_ERR_OOM : TEM_ERR_CUDA;
  return fail(c, code, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);    \
  } while (0)

template <typename T>
int dalloc(tem_ctx *c, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
  c->allocs.push_back(q);
  c->bytes += int64_t(count * sizeof(T));
  *p = (T *)q;
  return TEM_OK;
}

// Free one allocation made by dalloc (count elements) and forget it.
template <typename T>
void dfree(tem_ctx *c, T **p, size_t count) {
  if (!*p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), static_cast<void *>(*p));
  if (it != c->allocs.end()) c->allocs.erase(it);
  cudaFree(*p);
  c->bytes -= int64_t((count ? count : 1) * sizeof(T));
  *p = nullptr;
}

template <typename T>
int upload(tem_ctx *c, T **p, const std::vector<T> &v) {
  int st = dalloc(c, p, v.size());
  if (st) return st;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload");
  }
  return TEM_OK;
}

#define TRY(x)          \
  do {                  \
    int st_ = (x);      \
    if (st_) return st_; \
  } while (0)

int sync(tem_ctx *c, const char *where) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  if (c->prof.on) c->prof.collect();
  return TEM_OK;
}

// Status words written by the solve kernels (bounded tensor-core waits).
int check_solve_status(tem_ctx *c) {
  DevStatus h{};
  CK(cudaMemcpyAsync(&h, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (h.tc_timeout) {
    // reported once: the flag is cleared so that the context's next call starts clean
    CK(cudaMemsetAsync(&c->status->tc_timeout, 0, sizeof(int32_t), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return fail(c, TEM_ERR_TIMEOUT, "a tensor-core completion wait expired in a solve");
  }
  return TEM_OK;
}

// End of a call: in the default mode synchronise the stream and read the
// solve status words; in asynchronous mode only check that the launches were
// accepted (the caller reads the status with tem_status).
int finish(tem_ctx *c, const char *where) {
  if (c->async) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, where);
    return TEM_OK;
  }
  TRY(sync(c, where));
  return check_solve_status(c);
}

// NVTX range around a library call or phase (header-only NVTX v3: free unless
// a profiler injects itself), so that timelines and ncu --nvtx filters can
// select the factorisation, the solves and the products.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

struct ProfScope {
  explicit ProfScope(tem_ctx *c) { g_prof = c->prof.on ? &c->prof : nullptr; }
  ~ProfScope() { g_prof = nullptr; }
};

// FP32 task lists of one level: the four front products of the solves (64-row
// / 64-column tiles; kernels.h gives each mode's operands) and the merge
// stages of the pivot-block inversion.  List offsets are stored in the
// LevelDev pointers until the lists are uploaded.
void build_fp32_tasks(FactorSys &S_, const Level &L, LevelDev &lv) {
  const auto &S = S_.sym;
  for (int mode = 0; mode < PM_COUNT; mode++) {
    const size_t beg = S_.prod_h.size(), beg_s = S_.prod_simt_h.size();
    for (int32_t fi : L.fronts) {
      const Front &F = S.fronts[fi];
      const int k = F.k, b = F.n - F.k;
      if (k <= 0) continue;
      // tile with A origin (row x, column y) of the front block, for the
      // tensor-core kernel (tc) and / or the SIMT kernel (simt)
      auto push = [&](bool tc, bool simt, int row, int col, int kdim, int mrows, int bbase, int obase, int mfirst,
                      int kfirst) {
        if (tc) {
          TcTask t;
          t.map = 4 * fi + mode;
          t.x0 = 2 * row;
          t.y0 = col;
          t.kdim = kdim;
          t.mrows = mrows;
          t.bbase = bbase;
          t.obase = obase;
          t.mfirst = int16_t(mfirst);
          t.kfirst = int16_t(kfirst);
          S_.prod_h.push_back(t);
        }
        if (simt) {
          SimtTask u;
          u.aoff = F.lofs + int64_t(col) * F.ld + row;
          u.lda = F.ld;
          u.kdim = kdim;
          u.mrows = mrows;
          u.bbase = bbase;
          u.obase = obase;
          u.mfirst = int16_t(mfirst);
          u.kfirst = int16_t(kfirst);
          S_.prod_simt_h.push_back(u);
        }
      };
      const int r0 = k & ~1;   // even origin of the update rows (row k - 1 is padding when k is odd)
      if (mode == PM_TRI_F) {
        for (int i0 = 0; i0 < k; i0 += 64)
          push(false, true, i0, 0, std::min(k, i0 + 64), std::min(64, k - i0), F.c0, F.c0 + i0, 0, 0);
        // tensor cores: 128 rows of the row-major T11 copy (run origin x = 0, row origin y = i0)
        for (int i0 = 0; i0 < k; i0 += 128) {
          push(true, false, 0, 0, std::min(k, i0 + 128), std::min(128, k - i0), F.c0, F.c0 + i0, 0, 0);
          S_.prod_h.back().y0 = i0;
        }
      } else if (mode == PM_FWD21) {
        if (b > 0) {
          for (int R = r0; R < F.n; R += 64)
            push(false, true, R, 0, k, std::min(64, F.n - R), F.c0, (int)F.rows_off + R - k, std::max(0, k - R), 0);
          // tensor cores: 128 rows of the row-major L21 copy
          for (int i0 = 0; i0 < b; i0 += 128) {
            push(true, false, 0, 0, k, std::min(128, b - i0), F.c0, (int)F.rows_off + i0, 0, 0);
            S_.prod_h.back().y0 = i0;
          }
        }
      } else if (mode == PM_BWD21) {
        // B rows: X[rows[rows_off + kk - kfirst]] for inner index kk >= kfirst,
        // gathered by the SIMT kernel (64-column tiles) or by TMA row-gather
        // loads (128-column tiles)
        const int kdim = b == 0 ? 0 : F.n - r0;
        for (int cb = 0; cb < k; cb += 64)
          push(false, true, r0, cb, kdim, std::min(64, k - cb), (int)F.rows_off - (k - r0), F.c0 + cb, 0, k - r0);
        for (int cb = 0; cb < k; cb += 128)
          push(true, false, r0, cb, kdim, std::min(128, k - cb), (int)F.rows_off - (k - r0), F.c0 + cb, 0, k - r0);
      } else {
        for (int cb = 0; cb < k; cb += 64)
          push(false, true, cb, cb, k - cb, std::min(64, k - cb), F.c0 + cb, F.c0 + cb, 0, 0);
        for (int cb = 0; cb < k; cb += 128)
          push(true, false, cb, cb, k - cb, std::min(128, k - cb), F.c0 + cb, F.c0 + cb, 0, 0);
      }
    }
    lv.n_prod[mode] = int(S_.prod_h.size() - beg);
    lv.n_prod_simt[mode] = int(S_.prod_simt_h.size() - beg_s);
    // tensor-core tasks, longest inner dimension first (the kernel deals them out in this order)
    std::stable_sort(S_.prod_h.begin() + beg, S_.prod_h.end(),
                     [](const TcTask &x, const TcTask &y) { return x.kdim > y.kdim; });
    lv.prod[mode] = (const TcTask *)(uintptr_t)beg;
    lv.prod_simt[mode] = (const SimtTask *)(uintptr_t)beg_s;
  }
  // row-major copies of T11 and L21 (after the level's inversion)
  {
    const size_t beg = S_.rcopy_h.size();
    for (int32_t fi : L.fronts) {
      const Front &F = S.fronts[fi];
      if (F.k <= 0) continue;
      for (int rb = 0; rb * 32 < F.k; rb++) S_.rcopy_h.push_back(make_int4(fi, 0, rb, 0));
      for (int rb = 0; rb * 32 < F.n - F.k; rb++) S_.rcopy_h.push_back(make_int4(fi, 1, rb, 0));
    }
    lv.n_rcopy = int(S_.rcopy_h.size() - beg);
    lv.rcopy = (const int4 *)(uintptr_t)beg;
  }
  // inversion: 32-blocks, then pairwise merges of blocks of 32 * 2^stage
  const size_t dbeg = S_.invdiag_h.size();
  int kmax = 0;
  for (int32_t fi : L.fronts) {
    const Front &F = S.fronts[fi];
    kmax = std::max(kmax, F.k);
    for (int J = 0; J * kNB < F.k; J++) S_.invdiag_h.push_back(make_int2(fi, J));
  }
  lv.n_inv_diag = int(S_.invdiag_h.size() - dbeg);
  lv.inv_diag = (const int2 *)(uintptr_t)dbeg;
  lv.inv.clear();
  for (int sz = kNB; sz < kmax; sz *= 2) {
    LevelDev::InvStage st;
    const size_t beg = S_.inv_h.size();
    int64_t ybase = 0;
    for (int32_t fi : L.fronts) {
      const Front &F = S.fronts[fi];
      for (int a0 = 0; a0 + sz < F.k; a0 += 2 * sz) {
        const int sc = std::min(sz, F.k - a0 - sz);
        for (int ti = 0; ti * 64 < sc; ti++)
          for (int tj = 0; tj * 64 < sz; tj++) {
            InvTask t;
            t.front = fi;
            t.a0 = a0;
            t.s = sz;
            t.sc = sc;
            t.ti = ti;
            t.tj = tj;
            t.ybase = ybase;
            S_.inv_h.push_back(t);
          }
        ybase += int64_t(sc) * sz;
      }
    }
    st.n = int(S_.inv_h.size() - beg);
    st.tasks = (const InvTask *)(uintptr_t)beg;
    S_.yscr_stride = std::max(S_.yscr_stride, ybase);
    lv.inv.push_back(st);
  }
}

// Grid dimensions of every pivot step (depend on the precision's tile sizes).
template <typename R>
void build_steps(FactorSys &S_) {
  const auto &S = S_.sym;
  S_.levels.clear();
  S_.f21_h.clear();
  S_.b21_h.clear();
  S_.sbf_h.clear();
  S_.sbb_h.clear();
  S_.prod_h.clear();
  S_.prod_simt_h.clear();
  S_.rcopy_h.clear();
  // row-major copy layout: per front k x ld2 (T11) and b x ld2 (L21), ld2 = k rounded up to even
  S_.t11r_ofs_h.assign(S.fronts.size(), 0);
  S_.l21t_ofs_h.assign(S.fronts.size(), 0);
  S_.t11r_total = S_.l21t_total = 0;
  for (size_t f = 0; f < S.fronts.size(); f++) {
    const Front &F = S.fronts[f];
    const int64_t ld2 = F.k + (F.k & 1);
    S_.t11r_ofs_h[f] = S_.t11r_total;
    S_.l21t_ofs_h[f] = S_.l21t_total;
    S_.t11r_total += int64_t(F.k) * ld2;
    S_.l21t_total += int64_t(F.n - F.k) * ld2;
  }
  S_.inv_h.clear();
  S_.invdiag_h.clear();
  S_.upd_h.clear();
  S_.ucopy_h.clear();
  S_.prows = 0;
  S_.yscr_stride = 0;
  S_.max_level_fronts = 0;
  int64_t off = 0;
  for (const Level &L : S.levels) {
    LevelDev lv;
    lv.h = (int)S_.levels.size();
    lv.nf = (int)L.fronts.size();
    lv.fronts = S_.levfronts + off;
    off += lv.nf;
    lv.lbeg = L.lbeg;
    lv.lend = L.lend;
    lv.obeg = L.obeg;
    lv.oend = L.oend;
    static_assert(kMaxChild == 4, "LevelDev holds four extend-add slots");
    for (int s = 0; s < kMaxChild; s++) {
      lv.ea_beg[s] = L.ea_beg[s];
      lv.ea_end[s] = L.ea_end[s];
    }
    lv.bwd_upd_tiles = std::max(1, div_up(L.max_k, 8));
    lv.max_k = L.max_k;
    lv.n_f21 = 0;
    lv.n_b21 = 0;
    const size_t f21_beg = S_.f21_h.size(), b21_beg = S_.b21_h.size();
    for (int32_t fi : L.fronts) {
      const Front &F = S.fronts[fi];
      const int b = F.n - F.k;
      if (F.k <= 0) continue;
      // the forward product only where there are update rows; the backward
      // one for every front (it also forms w = D^-1 y of the pivots)
      if (b > 0)
        for (int t = 0; t < div_up(b, SolveTile<R>::BM); t++) S_.f21_h.push_back(make_int2(fi, t));
      for (int t = 0; t < div_up(F.k, SolveTile<R>::BN); t++) S_.b21_h.push_back(make_int2(fi, t));
    }
    lv.n_f21 = int(S_.f21_h.size() - f21_beg);
    lv.n_b21 = int(S_.b21_h.size() - b21_beg);
    if constexpr (std::is_same<R, float>::value) build_fp32_tasks(S_, L, lv);
    lv.f21_tasks = (const int2 *)(uintptr_t)f21_beg;   // offsets until the lists are on the device
    lv.b21_tasks = (const int2 *)(uintptr_t)b21_beg;
    // super-block products: forward rows of block J against pivots [0, J0);
    // backward columns of block J against pivot rows [J1, k)
    const int nsb = div_up(L.max_k, kSB);
    lv.sb.assign(nsb, LevelDev::SuperBlock());
    for (int J = 0; J < nsb; J++) {
      const size_t fb = S_.sbf_h.size(), bb = S_.sbb_h.size();
      for (int32_t fi : L.fronts) {
        const Front &F = S.fronts[fi];
        const int J0 = J * kSB;
        if (F.k <= J0) break;
        const int J1 = std::min(F.k, J0 + kSB);
        for (int kb = 0; kb < J0; kb += kSplitK)
          for (int t = 0; t < div_up(J1 - J0, SolveTile<R>::BM); t++)
            S_.sbf_h.push_back(make_int4(fi, t, kb, std::min(J0, kb + kSplitK)));
        for (int rb = J1; rb < F.k; rb += kSplitK)
          for (int t = 0; t < div_up(J1 - J0, SolveTile<R>::BN); t++)
            S_.sbb_h.push_back(make_int4(fi, t, rb, std::min(F.k, rb + kSplitK)));
      }
      lv.sb[J].n_fwd = int(S_.sbf_h.size() - fb);
      lv.sb[J].n_bwd = int(S_.sbb_h.size() - bb);
      lv.sb[J].fwd = (const int4 *)(uintptr_t)fb;   // offsets until the lists are on the device
      lv.sb[J].bwd = (const int4 *)(uintptr_t)bb;
    }
    const int nsteps = div_up(L.max_k, kNB);
    for (int s = 0; s < nsteps; s++) {
      StepDims d{};
      const int j0 = s * kNB;
      for (int32_t fi : L.fronts) {
        const Front &F = S.fronts[fi];
        if (F.k <= j0) break;  // sorted by k descending
        d.nfronts++;
        const int nb = std::min(kNB, F.k - j0);
        const int64_t below = int64_t(F.n) - j0 - nb;
        d.panel_tiles = std::max(d.panel_tiles, std::max(1, div_up(below, kPanelRT)));
        const int64_t T = div_up(below, UpdateTile<R>::TM);
        d.update_tiles = (int)std::max<int64_t>(d.update_tiles, std::max<int64_t>(1, T * (T + 1) / 2));
        {   // restricted to the step's kKB block (tensor-core factor)
          const int64_t pbeg = j0 + nb, s_end = std::min<int64_t>(F.k, (j0 / kKB + 1) * int64_t(kKB));
          const int64_t TJ = s_end > pbeg ? div_up(s_end - pbeg, UpdateTile<R>::TM) : 0;
          d.update_tiles_blk =
              (int)std::max<int64_t>(d.update_tiles_blk, std::max<int64_t>(1, TJ * T - TJ * (TJ - 1) / 2));
        }
        const int sb_end = std::min(F.k, (j0 / kSB + 1) * kSB), sb_beg = (j0 / kSB) * kSB;
        d.fwd_tiles = std::max(d.fwd_tiles, std::max(1, div_up(sb_end - j0 - nb, SolveTile<R>::RT)));
        d.bwd_tiles = std::max(d.bwd_tiles, std::max(1, div_up(j0 - sb_beg, SolveTile<R>::CT)));
      }
      lv.steps.push_back(d);
    }
    if constexpr (std::is_same<R, float>::value) {
      // tensor-core trailing updates: per kKB block b, the fronts with pivots in it and rows below it
      for (int b = 0; b * kKB < L.max_k; b++) {
        UpdBlock ub;
        const int j0 = b * kKB;
        const size_t tb = S_.upd_h.size(), cb = S_.ucopy_h.size();
        int64_t rows = 0;
        for (int32_t fi : L.fronts) {
          const Front &F = S.fronts[fi];
          if (F.k <= j0) break;  // sorted by k descending
          const int kb = std::min(kKB, F.k - j0), t0 = j0 + kb;
          if (t0 >= F.n) continue;
          const int64_t prow0 = rows - t0;   // panel-copy row of front row r: prow0 + r
          S_.ucopy_h.push_back(make_int4(fi, int(prow0), t0, kb));
          ub.copy_tiles = std::max(ub.copy_tiles, div_up(F.n - t0, 32));
          for (int s0 = t0 & ~1; s0 < F.n; s0 += 32)
            for (int r0 = t0 + std::max(0, (s0 - t0) / 128) * 128; r0 < F.n; r0 += 128) {
              TcTask t;
              t.map = fi;
              t.x0 = int(prow0);
              t.y0 = r0;
              t.kdim = kb;
              t.mrows = std::min(128, F.n - r0);
              t.bbase = s0;
              t.obase = j0;
              t.mfirst = int16_t(std::max(0, t0 - s0));
              t.kfirst = 0;
              S_.upd_h.push_back(t);
            }
          rows += F.n - t0;
        }
        ub.ntask = int(S_.upd_h.size() - tb);
        ub.ncopy = int(S_.ucopy_h.size() - cb);
        std::stable_sort(S_.upd_h.begin() + tb, S_.upd_h.end(),
                         [](const TcTask &x, const TcTask &y) { return x.kdim > y.kdim; });
        ub.tasks = (const TcTask *)(uintptr_t)tb;   // offsets until the lists are on the device
        ub.copies = (const int4 *)(uintptr_t)cb;
        S_.prows = std::max(S_.prows, rows);
        lv.upd.push_back(ub);
      }
    }
    S_.max_level_fronts = std::max(S_.max_level_fronts, lv.nf);
    S_.levels.push_back(std::move(lv));
  }
}

template <typename R>
FactorPlan<R> factor_plan(FactorSys &S, DevStatus *status, bool tc_update) {
  FactorPlan<R> P;
  P.tc_update = tc_update && S.Pc != nullptr;
  P.Pc = (cx<R> *)S.Pc;
  P.pstride = std::max<int64_t>(1, S.prows) * kKB;
  P.cmaps = S.cmaps;
  P.pcmap = S.pcmap;
  P.m = S.m;
  P.L = (cx<R> *)S.L;
  P.lstride = S.sym.ltotal;
  P.U = (cx<R> *)S.U;
  P.ustride = S.sym.utotal;
  P.F = S.fronts;
  P.rel = S.rel;
  P.ea_child = S.ea_child;
  P.ea_col = S.ea_col;
  P.orig_nz = S.orig_nz;
  P.orig_dst = S.orig_dst;
  P.kval = S.kval;
  P.mval = S.mval;
  P.mstride = S.mstride;
  P.xi = S.xi;
  P.dscr = (cx<R> *)S.dscr;
  P.linv = (cx<R> *)S.linv;
  P.istride = S.inv_blocks * kNB * kNB;
  P.status = status;
  P.dinv = (cx<R> *)S.dinv;
  P.N = S.N;
  P.yscr = (cx<R> *)S.yscr;
  P.yscr_stride = S.yscr_stride;
  P.T11R = (cx<R> *)S.T11R;
  P.L21T = (cx<R> *)S.L21T;
  P.t11r_stride = std::max<int64_t>(1, S.t11r_total);
  P.l21t_stride = std::max<int64_t>(1, S.l21t_total);
  P.t11r_ofs = S.t11r_ofs;
  P.l21t_ofs = S.l21t_ofs;
  return P;
}

template <typename R>
SolvePlan<R> solve_plan(const FactorSys &S) {
  SolvePlan<R> P;
  P.m = S.m;
  P.nrhs = S.nrhs;
  P.L = (const cx<R> *)S.L;
  P.lstride = S.sym.ltotal;
  P.Linv = (const cx<R> *)S.linv;
  P.istride = S.inv_blocks * kNB * kNB;
  P.F = S.fronts;
  P.rows = S.rows;
  P.Y = (cx<R> *)S.Y;
  P.X = (cx<R> *)S.X;
  P.vstride = S.N * S.nrhs;
  P.dinv = (const cx<R> *)S.dinv;
  P.tmaps = S.tmaps;
  P.vmaps = S.vmaps;
  P.N = S.N;
  return P;
}

// Factor every matrix of S, level by level (FP32: each level's pivot blocks
// inverted in place and row-major copies written for the solves).
template <typename R>
void factor_sys(tem_ctx *c, FactorSys &S) {
  FactorPlan<R> P = factor_plan<R>(S, c->status, c->tc_fronts);
  const int H = (int)S.levels.size();
  for (int h = 0; h < H; h++) {
    P.level(h, S.levels[h], c->stream);
    if constexpr (std::is_same<R, float>::value) P.invert_level(S.levels[h], c->stream);
  }
}

// X = A_p^-1 Y for the mapped poles of S (forward and backward sweeps).
template <typename R>
void sweeps(tem_ctx *c, FactorSys &S, const int *pmap, int np) {
  SolvePlan<R> P = solve_plan<R>(S);
  P.pmap = pmap;
  P.np = np;
  P.use_tc = c->use_tc;
  P.status = c->status;
  c->pole_solves += np;
  const int H = (int)S.levels.size();
  for (int h = 0; h < H; h++) P.forward_level(S.levels[h], c->stream);
  for (int h = H - 1; h >= 0; h--) P.backward_level(S.levels[h], c->stream);
}

// Gradient-space correction of one refinement step (FP32 mode), with the
// residual r of the mapped poles in the edge system's Y (FP32, unscaled):
// psi = L_sigma^-1 G^T r for all poles and right-hand sides at once (the
// nodal system, one matrix), then x += -G psi / xi_p and r -= M(sigma) G psi.
void nodal_correct(tem_ctx *c, const int *pm, int np) {
  FactorSys &S = c->ns;
  cudaStream_t s = c->stream;
  auto pb = [&](int k) { if (g_prof) g_prof->begin(k, s); };
  auto pe = [&](int k) { if (g_prof) g_prof->end(k, s); };
  pb(KC_NODAL);
  pb(KC_NODAL_RHS);
  c64 *Yn = (c64 *)S.Y;
  launch_nodal_rhs(c->n_gptr, c->n_gedge, c->n_gsign, (const c64 *)c->es.Y, Yn, S.N, np, pm, c->m, c->mesh.N,
                   c->nrhs, s);
  launch_scale_to_work<c64>(Yn, 0, Yn, c->colmax_n, 1, nullptr, S.N, S.nrhs, s);
  pe(KC_NODAL_RHS);
  pb(KC_NODAL_SWEEP);
  if (g_prof) g_prof->muted = true;   // the nodal sweeps are not edge-system product launches
  sweeps<float>(c, S, nullptr, 1);
  if (g_prof) g_prof->muted = false;
  pe(KC_NODAL_SWEEP);
  c->pole_solves -= 1;
  pb(KC_NODAL_APPLY);
  launch_nodal_apply(c->n_crp, c->n_cci, c->n_cval, (const c64 *)S.X, c->colmax_n, (c64 *)c->es.Y, np, pm, c->m,
                     c->mesh.N, c->nrhs, s);
  pe(KC_NODAL_APPLY);
  pe(KC_NODAL);
}

// x = A_i^-1 b for all poles; b c128 with pole stride bstride (0 = shared).
// FP32 mode: refinement x += P_i^-1 (b - A_i x) with the FP64 residual; with
// refine_tol > 0 a pole stops once its correction on the unknowns the outputs
// read (edges of parameter cells) is below refine_tol of the solution there,
// and later sweeps run over the remaining poles only (a host read per step).
int solve_all(tem_ctx *c, const c128 *b, int64_t bstride, c128 *x, int steps, bool join = true,
              bool b_in_pairs = false) {
  Range nvtx_range("solve");
  const int64_t N = c->mesh.N;
  const int nx = c->nrhs, m = c->m;
  cudaStream_t s = c->stream;
  c->solve_calls++;
  if (c->precision == TEM_FP64) {
    launch_rhs_to_work<double>(b, bstride, (c128 *)c->es.Y, nullptr, m, nullptr, N, nx, false, s);
    sweeps<double>(c, c->es, nullptr, m);
    launch_accumulate<double>((const c128 *)c->es.X, nullptr, x, m, nullptr, N, nx, false, s);
    return TEM_OK;
  }
  // FP32 mode: b and the iterate as double-float pairs, corrections in FP32
  float4 *bdf = reinterpret_cast<float4 *>(c->r);   // pairs of b (shared when bstride == 0)
  const int64_t bsd = bstride ? N * nx : 0;
  auto prof_begin = [&](int k) { if (g_prof) g_prof->begin(k, s); };
  auto prof_end = [&](int k) { if (g_prof) g_prof->end(k, s); };
  prof_begin(KC_REFINE_VEC);
  if (!b_in_pairs)   // else the caller wrote b as pairs into c->r already
    launch_split_cx(b, bdf, (bstride ? int64_t(m) : int64_t(1)) * N * nx, s);
  c64 *Y = (c64 *)c->es.Y;
  launch_scale_to_work<float4>(bdf, bsd, Y, c->colmax_f, m, nullptr, N, nx, s);
  prof_end(KC_REFINE_VEC);
  sweeps<float>(c, c->es, nullptr, m);
  prof_begin(KC_REFINE_VEC);
  launch_accumulate_df((const c64 *)c->es.X, c->colmax_f, c->xdf, m, nullptr, N, nx, false, s);
  prof_end(KC_REFINE_VEC);
  const int *pm = nullptr;
  int np = m;
  for (int it = 0; it < steps; it++) {
    prof_begin(KC_RESIDUAL);
    launch_residual_df(c->rp, c->ci, c->kdf, c->mdf, c->xi, bdf, bsd, c->xdf, Y, np, pm, N, nx, s);
    prof_end(KC_RESIDUAL);
    if (c->use_nodal) nodal_correct(c, pm, np);
    prof_begin(KC_REFINE_VEC);
    launch_scale_to_work<c64>(Y, N * nx, Y, c->colmax_f, np, pm, N, nx, s);
    prof_end(KC_REFINE_VEC);
    sweeps<float>(c, c->es, pm, np);
    prof_begin(KC_REFINE_VEC);
    NodalPart nd;   // the x update of this step's gradient-space correction, added with the edge correction
    if (c->use_nodal) {
      nd.Xn = (const c64 *)c->ns.X;
      nd.colmax_n = c->colmax_n;
      nd.e_lo = c->n_elo;
      nd.e_hi = c->n_ehi;
      nd.ninv_xi = c->ninv_xi;
      nd.ncol = c->ns.nrhs;
    }
    launch_accumulate_df((const c64 *)c->es.X, c->colmax_f, c->xdf, np, pm, N, nx, true, s, nd);
    prof_end(KC_REFINE_VEC);
    if (c->refine_tol <= 0 || it + 1 == steps) continue;
    CK(cudaMemsetAsync(c->prog, 0, sizeof(double) * 2 * m, s));
    launch_progress_df((const c64 *)c->es.X, c->colmax_f, c->xdf, c->earth, c->prog, c->prog + m, np, pm, N, nx, s);
    std::vector<double> pr(2 * m);
    std::vector<int> keep;
    CK(cudaMemcpyAsync(pr.data(), c->prog, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int> cur(np);
    if (pm) CK(cudaMemcpy(cur.data(), pm, sizeof(int) * np, cudaMemcpyDeviceToHost));
    else for (int i = 0; i < np; i++) cur[i] = i;
    for (int p : cur)
      if (pr[p] > c->refine_tol * pr[m + p]) keep.push_back(p);
    if (keep.empty()) break;
    CK(cudaMemcpy(c->pmap, keep.data(), sizeof(int) * keep.size(), cudaMemcpyHostToDevice));
    pm = c->pmap;
    np = (int)keep.size();
  }
  if (join) {   // else the caller reads the pairs in xdf
    prof_begin(KC_REFINE_VEC);
    launch_join_cx(c->xdf, x, int64_t(m) * N * nx, s);
    prof_end(KC_REFINE_VEC);
  }
  return TEM_OK;
}

// Host check of the tensor-core trailing-update tasks against the fronts and
// the panel copy, before any of them reaches the device: every TMA x origin
// even (16-byte aligned), every column and row inside its front, every copied
// row inside the panel copy.  "" when all hold.
std::string check_update_tasks(const FactorSys &Q) {
  const auto &Fs = Q.sym.fronts;
  for (const LevelDev &lv : Q.levels)
    for (size_t b = 0; b < lv.upd.size(); b++) {
      const UpdBlock &ub = lv.upd[b];
      const size_t t0i = (uintptr_t)ub.tasks, c0i = (uintptr_t)ub.copies;
      for (int q = 0; q < ub.ncopy; q++) {
        const int4 cp = Q.ucopy_h[c0i + q];
        if (cp.x < 0 || cp.x >= (int)Fs.size()) return "update copy: front out of range";
        const Front &F = Fs[cp.x];
        if (cp.w <= 0 || cp.w > kKB || cp.z - cp.w != int(b) * kKB || cp.z >= F.n || cp.z > F.k)
          return "update copy: bad block";
        if (int64_t(cp.y) + cp.z < 0 || int64_t(cp.y) + F.n > Q.prows) return "update copy: rows outside the copy";
      }
      for (int q = 0; q < ub.ntask; q++) {
        const TcTask &t = Q.upd_h[t0i + q];
        if (t.map < 0 || t.map >= (int)Fs.size()) return "update task: front out of range";
        const Front &F = Fs[t.map];
        const int t0 = t.obase + t.kdim;
        if (t.obase != int(b) * kKB || t.kdim <= 0 || t.kdim > kKB || t0 > F.k) return "update task: bad block";
        if (t.bbase & 1) return "update task: odd column origin";
        if (t.bbase < 0 || t.bbase >= F.n || t.bbase + t.mfirst != std::max(t.bbase, t0)) return "update task: columns";
        if (t.y0 < t0 || t.mrows <= 0 || t.mrows > 128 || t.y0 + t.mrows > F.n) return "update task: rows";
        if (int64_t(t.x0) + t.y0 < 0 || int64_t(t.x0) + t.y0 + t.mrows > Q.prows) return "update task: copy rows";
      }
    }
  return "";
}

// Device copies of a system's assembly tree and of its factor / solve task lists.
int upload_sys(tem_ctx *c, FactorSys &Q, bool fp32) {
  const Symbolic &S = Q.sym;
  std::vector<FrontDev> fd(S.fronts.size());
  int64_t inv = 0;
  for (size_t i = 0; i < S.fronts.size(); i++) {
    const Front &F = S.fronts[i];
    fd[i] = FrontDev{F.lofs, F.uofs, F.rows_off, F.rel_off, inv, F.n, F.k, F.c0, F.parent, F.ld, 0};
    inv += div_up(F.k, kNB);
  }
  Q.inv_blocks = inv;
  TRY(upload(c, &Q.fronts, fd));
  TRY(upload(c, &Q.rows, S.rows));
  TRY(upload(c, &Q.rel, S.rel));
  TRY(upload(c, &Q.orig_nz, S.orig_nz));
  TRY(upload(c, &Q.orig_dst, S.orig_dst));
  TRY(upload(c, &Q.ea_child, S.ea_child));
  TRY(upload(c, &Q.ea_col, S.ea_col));
  std::vector<int32_t> lf;
  for (const Level &L : S.levels) lf.insert(lf.end(), L.fronts.begin(), L.fronts.end());
  TRY(upload(c, &Q.levfronts, lf));
  if (fp32) build_steps<float>(Q);
  else build_steps<double>(Q);
  TRY(upload(c, &Q.f21, Q.f21_h));
  TRY(upload(c, &Q.b21, Q.b21_h));
  TRY(upload(c, &Q.sbf, Q.sbf_h));
  TRY(upload(c, &Q.sbb, Q.sbb_h));
  TRY(upload(c, &Q.prod, Q.prod_h));
  TRY(upload(c, &Q.prod_simt, Q.prod_simt_h));
  TRY(upload(c, &Q.rcopy, Q.rcopy_h));
  TRY(upload(c, &Q.t11r_ofs, Q.t11r_ofs_h));
  TRY(upload(c, &Q.l21t_ofs, Q.l21t_ofs_h));
  TRY(upload(c, &Q.inv, Q.inv_h));
  TRY(upload(c, &Q.invdiag, Q.invdiag_h));
  {
    const std::string e = check_update_tasks(Q);
    if (!e.empty()) return fail(c, TEM_ERR_MESH, "internal: " + e);
  }
  TRY(upload(c, &Q.upd, Q.upd_h));
  TRY(upload(c, &Q.ucopy, Q.ucopy_h));
  for (LevelDev &lv : Q.levels) {
    lv.f21_tasks = Q.f21 + (uintptr_t)lv.f21_tasks;
    lv.b21_tasks = Q.b21 + (uintptr_t)lv.b21_tasks;
    for (int mode = 0; mode < PM_COUNT; mode++) {
      lv.prod[mode] = Q.prod + (uintptr_t)lv.prod[mode];
      lv.prod_simt[mode] = Q.prod_simt + (uintptr_t)lv.prod_simt[mode];
    }
    lv.rcopy = Q.rcopy + (uintptr_t)lv.rcopy;
    lv.inv_diag = Q.invdiag + (uintptr_t)lv.inv_diag;
    for (auto &st : lv.inv) st.tasks = Q.inv + (uintptr_t)st.tasks;
    for (auto &sb : lv.sb) {
      sb.fwd = Q.sbf + (uintptr_t)sb.fwd;
      sb.bwd = Q.sbb + (uintptr_t)sb.bwd;
    }
    for (auto &ub : lv.upd) {
      ub.tasks = Q.upd + (uintptr_t)ub.tasks;
      ub.copies = Q.ucopy + (uintptr_t)ub.copies;
    }
  }
  for (const LevelDev &lv : Q.levels)
    if (lv.nf > 65535) return fail(c, TEM_ERR_MESH, "more than 65535 fronts in one tree level");
  return TEM_OK;
}

// Factor store, solve vectors and (FP32) inverse pivots, row-major copies and
// tensor maps of one system.
int alloc_sys(tem_ctx *c, FactorSys &S, bool fp32) {
  const size_t es = fp32 ? sizeof(c64) : sizeof(c128);
  const int64_t N = S.N;
  const int m = S.m, nx = S.nrhs;
  void *p;
  TRY(dalloc(c, (char **)&p, size_t(m) * S.sym.ltotal * es));
  S.L = p;
  TRY(dalloc(c, (char **)&p, size_t(m) * S.sym.utotal * es));
  S.U = p;
  TRY(dalloc(c, (char **)&p, size_t(std::max(1, S.max_level_fronts)) * m * kNB * kNB * es));
  S.dscr = p;
  TRY(dalloc(c, (char **)&p, size_t(m) * std::max<int64_t>(1, S.inv_blocks) * kNB * kNB * es));
  S.linv = p;
  TRY(dalloc(c, (char **)&p, size_t(m) * N * nx * es));
  S.Y = p;
  TRY(dalloc(c, (char **)&p, size_t(m) * N * nx * es));
  S.X = p;
  // the products read whole 16-row chunks of these (finite values past a block)
  CK(cudaMemset(S.Y, 0, size_t(m) * N * nx * es));
  CK(cudaMemset(S.X, 0, size_t(m) * N * nx * es));
  if (!fp32) return TEM_OK;
  TRY(dalloc(c, (c64 **)&S.dinv, size_t(m) * N));
  TRY(dalloc(c, (c64 **)&S.yscr, size_t(m) * std::max<int64_t>(1, S.yscr_stride)));
  TRY(dalloc(c, (c64 **)&S.T11R, size_t(m) * std::max<int64_t>(1, S.t11r_total)));
  TRY(dalloc(c, (c64 **)&S.L21T, size_t(m) * std::max<int64_t>(1, S.l21t_total)));
  std::vector<FrontGeom> geo(S.sym.fronts.size());
  for (size_t i = 0; i < geo.size(); i++) {
    const Front &F = S.sym.fronts[i];
    geo[i] = FrontGeom{F.lofs, S.t11r_ofs_h[i], S.l21t_ofs_h[i], F.n, F.k, F.ld, F.k + (F.k & 1)};
  }
  const FactorViews views{(const c64 *)S.L, S.sym.ltotal, (const c64 *)S.T11R, std::max<int64_t>(1, S.t11r_total),
                          (const c64 *)S.L21T, std::max<int64_t>(1, S.l21t_total)};
  const std::string e = build_tensor_maps(geo, views, m, &S.tmaps);
  if (!e.empty()) return fail(c, TEM_ERR_CUDA, e);
  c->allocs.push_back(S.tmaps);
  const std::string e2 =
      build_vector_maps({VecBuf{(const c64 *)S.Y, N}, VecBuf{(const c64 *)S.X, N}}, 1, nx, m, &S.vmaps);
  if (!e2.empty()) return fail(c, TEM_ERR_CUDA, e2);
  if (S.vmaps) c->allocs.push_back(S.vmaps);
  // panel copy of the tensor-core trailing updates (zeroed once: rows a box reads past a front stay finite)
  TRY(dalloc(c, (c64 **)&S.Pc, size_t(m) * std::max<int64_t>(1, S.prows) * kKB));
  CK(cudaMemset(S.Pc, 0, sizeof(c64) * size_t(m) * std::max<int64_t>(1, S.prows) * kKB));
  const std::string e3 = build_update_maps(geo, (const c64 *)S.L, S.sym.ltotal, (const c64 *)S.Pc,
                                           std::max<int64_t>(1, S.prows), m, &S.cmaps, &S.pcmap);
  if (!e3.empty()) return fail(c, TEM_ERR_CUDA, e3);
  c->allocs.push_back(S.cmaps);
  c->allocs.push_back(S.pcmap);
  return TEM_OK;
}

int ensure_lsqr_buffers(tem_ctx *c) {
  if (c->ls_u) return TEM_OK;
  const int64_t nd = int64_t(c->n_tx) * c->n_rx * c->K, P = c->mesh.P, nf = c->mesh.nf;
  TRY(dalloc(c, &c->ls_u, nd + nf));
  TRY(dalloc(c, &c->ls_v, P));
  TRY(dalloc(c, &c->ls_w, P));
  TRY(dalloc(c, &c->ls_jv, nd));
  TRY(dalloc(c, &c->ls_jtw, P));
  TRY(dalloc(c, &c->ls_tmpd, nd));
  TRY(dalloc(c, &c->ls_tmpp, P));
  TRY(dalloc(c, &c->ls_wv, std::max<int64_t>(nf, 1)));
  TRY(dalloc(c, &c->ls_sc, 1));
  return TEM_OK;
}

int ensure_numeric(tem_ctx *c) {
  if (c->es.L) return TEM_OK;
  const bool fp32 = c->precision != TEM_FP64;
  const int64_t N = c->mesh.N;
  const int m = c->m, nx = c->nrhs;
  c->es.m = m;
  c->es.nrhs = nx;
  TRY(alloc_sys(c, c->es, fp32));
  TRY(dalloc(c, &c->g, size_t(m) * N * nx));
  TRY(dalloc(c, &c->b, size_t(m) * N * nx));
  TRY(dalloc(c, &c->x, size_t(m) * N * nx));
  if (fp32) {
    TRY(dalloc(c, &c->r, size_t(m) * N * nx));
    TRY(dalloc(c, &c->kdf, c->mesh.kval.size()));
    TRY(dalloc(c, &c->mdf, c->mesh.kval.size()));
    TRY(dalloc(c, &c->xdf, size_t(m) * N * nx));
    TRY(dalloc(c, &c->colmax_f, size_t(m) * nx));
    TRY(dalloc(c, &c->mval_fact, size_t(m) * c->mesh.kval.size()));
    std::vector<double> tf(c->mesh.nt);
    for (int64_t t = 0; t < c->mesh.nt; t++) tf[t] = 1.0 / (kMu0 * std::pow(c->mesh.vol[t], 2.0 / 3.0));
    TRY(upload(c, &c->tetfloor, tf));   // 1 / (mu0 h_t^2); tau applied at factor time
    // nodal gradient space: one real Laplacian (as a complex matrix with xi = -1)
    // for all m * nrhs right-hand sides of a refinement step
    c->ns.m = 1;
    c->ns.nrhs = m * nx;
    TRY(alloc_sys(c, c->ns, true));
    TRY(dalloc(c, &c->colmax_n, size_t(m) * nx));
    TRY(dalloc(c, &c->part, size_t(m) * std::max<int64_t>(1, c->mesh.P)));
    TRY(dalloc(c, &c->gdf, size_t(m) * N * nx));
    TRY(dalloc(c, &c->vsdf, size_t(c->mesh.nt)));
  }
  c->es.kval = c->kval;
  c->es.mval = fp32 ? c->mval_fact : c->mval;
  c->es.mstride = fp32 ? (int64_t)c->mesh.kval.size() : 0;
  c->es.xi = c->xi;
  TRY(dalloc(c, &c->fb, size_t(N) * nx));
  TRY(dalloc(c, &c->colmax, size_t(m) * nx));
  TRY(dalloc(c, &c->d_cur, size_t(c->n_tx) * c->n_rx * c->K));
  TRY(dalloc(c, &c->pmap, size_t(m)));
  TRY(dalloc(c, &c->prog, size_t(2 * m)));
  TRY(dalloc(c, &c->m_cur, size_t(std::max<int64_t>(1, c->mesh.P))));
  return TEM_OK;
}

}  // namespace

extern "C" {

int tem_create(tem_ctx **ctx, int precision, void *stream) {
  if (!ctx) return fail(nullptr, TEM_ERR_ARG, "ctx is NULL");
  *ctx = nullptr;
  if (precision != TEM_FP64 && precision != TEM_FP32_REFINED)
    return fail(nullptr, TEM_ERR_ARG, "unknown precision");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, TEM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  tem_ctx *c = new tem_ctx();
  c->precision = precision;
  c->stream = (cudaStream_t)stream;
  c->device = dev;
  // with the gradient-space correction and the floor tau = 1e-6, three corrections bring the
  // data and J v within 1e-7 of the FP64 path on the 46^3 box (two leave J v near 3e-6), and one
  // brings J^T w within 3e-9
  c->refine = precision == TEM_FP64 ? 0 : 3;
  c->refine_adj = precision == TEM_FP64 ? 0 : 1;
  if (dalloc(c, &c->status, 1)) {
    std::string m = c->err;
    delete c;
    return fail(nullptr, TEM_ERR_OOM, m);
  }
  *ctx = c;
  return TEM_OK;
}

int tem_destroy(tem_ctx *c) {
  if (!c) return TEM_OK;
  cudaStreamSynchronize(c->stream);
  for (void *p : c->allocs) cudaFree(p);
  c->prof.release();
  delete c;
  return TEM_OK;
}

const char *tem_last_error(tem_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int tem_mesh(tem_ctx *c, int64_t n_vert, const double *xyz, int64_t n_tet, const int32_t *tets,
             const double *sigma, const uint8_t *is_param, int32_t leaf_max) {
  if (!c) return TEM_ERR_ARG;
  if (c->state & ST_MESH) return fail(c, TEM_ERR_STATE, "mesh already set");
  if (!xyz || !tets || !sigma || !is_param) return fail(c, TEM_ERR_ARG, "NULL mesh array");
  c->sym_opts.leaf_max = leaf_max;
  std::string msg = build_mesh(c->mesh, n_vert, xyz, n_tet, tets, sigma, is_param, c->sym_opts, c->es.sym);
  if (!msg.empty()) return fail(c, TEM_ERR_MESH, msg);
  Mesh &M = c->mesh;
  TRY(upload(c, &c->sigma_fixed, M.sigma));
  TRY(dalloc(c, &c->sigma, M.nt));
  TRY(upload(c, &c->me1, M.Me1));
  TRY(upload(c, &c->kval, M.kval));
  TRY(dalloc(c, &c->mval, M.kval.size()));
  TRY(upload(c, &c->rp, M.rp));
  TRY(upload(c, &c->ci, M.ci));
  TRY(upload(c, &c->mc_ptr, M.mc_ptr));
  TRY(upload(c, &c->mc_idx, M.mc_idx));
  TRY(upload(c, &c->inc_ptr, M.inc_ptr));
  TRY(upload(c, &c->inc_tet, M.inc_tet));
  TRY(upload(c, &c->inc_loc, M.inc_loc));
  TRY(upload(c, &c->tdof, M.tdof));
  TRY(upload(c, &c->pidx, M.pidx));
  {
    std::vector<uint8_t> earth(M.N, 0);
    for (int64_t t = 0; t < M.nt; t++)
      if (M.is_param[t])
        for (int a = 0; a < 6; a++)
          if (M.tdof[6 * t + a] >= 0) earth[M.tdof[6 * t + a]] = 1;
    TRY(upload(c, &c->earth, earth));
  }
  TRY(upload(c, &c->ptet, M.ptet));
  c->es.N = M.N;
  TRY(upload_sys(c, c->es, c->precision != TEM_FP64));
  TRY(upload(c, &c->w_rp, M.w_rp));
  TRY(upload(c, &c->w_ci, M.w_ci));
  TRY(upload(c, &c->w_val, M.w_val));
  TRY(upload(c, &c->wt_rp, M.wt_rp));
  TRY(upload(c, &c->wt_ci, M.wt_ci));
  TRY(upload(c, &c->wt_val, M.wt_val));
  if (c->precision != TEM_FP64) {
    std::vector<float2> mp(M.Me1.size());
    for (size_t q = 0; q < mp.size(); q++) {   // pairs hi + lo, both rounded to nearest
      const float hi = static_cast<float>(M.Me1[q]);
      mp[q] = make_float2(hi, static_cast<float>(M.Me1[q] - double(hi)));
    }
    TRY(upload(c, &c->me1df, mp));
    // the gradient space of the refinement: interior vertices, P1 Laplacian
    msg = build_nodal(M, c->sym_opts, c->nodal, c->ns.sym);
    if (!msg.empty()) return fail(c, TEM_ERR_MESH, msg);
    const NodalMesh &G = c->nodal;
    c->ns.N = G.N;
    TRY(upload_sys(c, c->ns, true));
    TRY(upload(c, &c->n_tnode, G.tnode));
    TRY(upload(c, &c->n_stiff, G.S));
    TRY(upload(c, &c->n_mc_ptr, G.mc_ptr));
    TRY(upload(c, &c->n_mc_idx, G.mc_idx));
    TRY(upload(c, &c->n_elo, G.e_lo));
    TRY(upload(c, &c->n_ehi, G.e_hi));
    TRY(upload(c, &c->n_gptr, G.g_ptr));
    TRY(upload(c, &c->n_gedge, G.g_edge));
    TRY(upload(c, &c->n_gsign, G.g_sign));
    TRY(upload(c, &c->n_crp, G.c_rp));
    TRY(upload(c, &c->n_cci, G.c_ci));
    TRY(upload(c, &c->n_cmc_ptr, G.c_mc_ptr));
    TRY(upload(c, &c->n_cmc_idx, G.c_mc_idx));
    TRY(upload(c, &c->n_btab, G.B));
    TRY(dalloc(c, &c->n_cval, G.c_ci.size()));
    TRY(upload(c, &c->n_kval, std::vector<double>(G.ci.size(), 0.0)));
    TRY(dalloc(c, &c->n_mval, G.ci.size()));
    TRY(upload(c, &c->n_xi, std::vector<double2>{make_double2(-1.0, 0.0)}));
    c->ns.kval = c->n_kval;
    c->ns.mval = c->n_mval;
    c->ns.mstride = 0;
    c->ns.xi = c->n_xi;
  }
  TRY(sync(c, "tem_mesh"));
  c->state |= ST_MESH;
  return TEM_OK;
}

int tem_poles(tem_ctx *c, int32_t m, const double *xi, int32_t n_times, const double *alpha) {
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_MESH)) return fail(c, TEM_ERR_STATE, "tem_mesh first");
  if (c->state & ST_POLES) return fail(c, TEM_ERR_STATE, "poles already set");
  if (m <= 0 || m > 32 || n_times <= 0 || !xi || !alpha) return fail(c, TEM_ERR_ARG, "bad poles (1 <= m <= 32)");
  for (int i = 0; i < m; i++)
    if (!(xi[2 * i] < 0)) return fail(c, TEM_ERR_ARG, "every pole needs Re xi < 0");
  c->m = m;
  c->K = n_times;
  c->xi_h.assign(xi, xi + 2 * m);
  c->alpha_h.assign(alpha, alpha + 2 * size_t(m) * n_times);
  std::vector<double> xv(c->xi_h), av(c->alpha_h);
  TRY(dalloc(c, &c->xi, m));
  TRY(dalloc(c, &c->alpha, size_t(m) * n_times));
  {
    std::vector<float2> w(m);
    for (int i = 0; i < m; i++) {   // -1 / xi_i, for the gradient-space correction
      const double a = xi[2 * i], b = xi[2 * i + 1], d = a * a + b * b;
      w[i] = make_float2(float(-a / d), float(b / d));
    }
    TRY(upload(c, &c->ninv_xi, w));
  }
  CK(cudaMemcpyAsync(c->xi, xv.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->alpha, av.data(), sizeof(double2) * m * n_times, cudaMemcpyHostToDevice, c->stream));
  TRY(sync(c, "tem_poles"));
  c->state |= ST_POLES;
  return TEM_OK;
}

int tem_times(tem_ctx *c, int32_t n_times, const double *t, int32_t n_z, double z_min, double z_max, double mu,
              double *alpha_out) {
  Range nvtx_range("tem_times");
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_POLES)) return fail(c, TEM_ERR_STATE, "tem_poles first");
  if (c->async) return fail(c, TEM_ERR_STATE, "tem_times synchronises: switch the asynchronous mode off first");
  if (n_times <= 0 || n_times > (1 << 20) || !t) return fail(c, TEM_ERR_ARG, "bad times (1 <= n_times <= 2^20)");
  for (int j = 0; j < n_times; j++)
    if (!(t[j] > 0) || !std::isfinite(t[j])) return fail(c, TEM_ERR_ARG, "every time must be finite and > 0");
  if (n_z < 2 || n_z > (1 << 20) || !(z_min > 0) || !(z_max > z_min) || !std::isfinite(z_max) || !(mu >= 0) ||
      !std::isfinite(mu))
    return fail(c, TEM_ERR_ARG, "bad sample set (2 <= n_z <= 2^20, 0 < z_min < z_max finite, mu >= 0)");
  const int m = c->m, K = n_times;
  const int64_t rows = int64_t(n_z) + 1 + 2 * m;
  if (rows * K > (int64_t(1) << 31))   // the right-hand sides of the fit: 16 GB at this bound
    return fail(c, TEM_ERR_ARG, "residue fit too large: (n_z + 1 + 2m) n_times must stay below 2^31");
  cudaStream_t s = c->stream;
  // work arrays of this call, released on every return
  struct Scratch {
    std::vector<void *> p;
    ~Scratch() {
      for (void *q : p) cudaFree(q);
    }
  } w;
  auto get = [&](size_t bytes, void **out) {
    *out = nullptr;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
    w.p.push_back(*out);
    return int(TEM_OK);
  };
  double *B, *Y, *rd, *cf, *td;
  double2 *al;
  TRY(get(sizeof(double) * rows * 2 * m, (void **)&B));
  TRY(get(sizeof(double) * rows * K, (void **)&Y));
  TRY(get(sizeof(double) * 2 * m, (void **)&rd));
  TRY(get(sizeof(double) * 2 * m, (void **)&cf));
  TRY(get(sizeof(double) * K, (void **)&td));
  TRY(get(sizeof(double2) * m * K, (void **)&al));
  const double lz0 = std::log10(z_min), lz1 = std::log10(z_max);
  CK(cudaMemcpyAsync(td, t, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  launch_fit_qr(c->xi, m, n_z, lz0, lz1, mu, B, rd, cf, s);
  std::vector<double> rdh(2 * m);
  CK(cudaMemcpyAsync(rdh.data(), rd, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s));
  TRY(sync(c, "tem_times"));
  double rmax = 0;
  for (double v : rdh) rmax = std::max(rmax, std::fabs(v));
  for (double v : rdh)
    if (!std::isfinite(v) || !(std::fabs(v) > 1e-14 * rmax))
      return fail(c, TEM_ERR_ARG, "the sample set leaves the residue fit rank deficient (raise mu or n_z)");
  launch_fit_solve(B, m, n_z, lz0, lz1, rd, cf, td, K, Y, al, s);
  std::vector<double> ah(2 * size_t(m) * K);
  CK(cudaMemcpyAsync(ah.data(), al, sizeof(double2) * m * K, cudaMemcpyDeviceToHost, s));
  TRY(sync(c, "tem_times"));
  for (double v : ah)
    if (!std::isfinite(v)) return fail(c, TEM_ERR_ARG, "non-finite residue");
  // install: alpha and every buffer sized by the data (n_tx n_rx K) follow the new K
  const size_t nd_old = size_t(c->n_tx) * c->n_rx * c->K;
  dfree(c, &c->alpha, size_t(m) * c->K);
  TRY(dalloc(c, &c->alpha, size_t(m) * K));
  CK(cudaMemcpyAsync(c->alpha, al, sizeof(double2) * m * K, cudaMemcpyDeviceToDevice, s));
  if (c->d_cur) {
    dfree(c, &c->d_cur, nd_old);
    TRY(dalloc(c, &c->d_cur, size_t(c->n_tx) * c->n_rx * K));
  }
  if (c->ls_u) {   // LSQR work vectors: reallocated at the next LSQR call
    const int64_t P = c->mesh.P, nf = c->mesh.nf;
    dfree(c, &c->ls_u, nd_old + nf);
    dfree(c, &c->ls_v, size_t(P));
    dfree(c, &c->ls_w, size_t(P));
    dfree(c, &c->ls_jv, nd_old);
    dfree(c, &c->ls_jtw, size_t(P));
    dfree(c, &c->ls_tmpd, nd_old);
    dfree(c, &c->ls_tmpp, size_t(P));
    dfree(c, &c->ls_wv, size_t(std::max<int64_t>(nf, 1)));
    dfree(c, &c->ls_sc, 1);
  }
  TRY(sync(c, "tem_times"));
  c->K = K;
  c->alpha_h = ah;
  c->state &= ~ST_FORWARD;   // the data of the last tem_forward had the old times; the factors stay
  if (alpha_out) std::copy(ah.begin(), ah.end(), alpha_out);
  return TEM_OK;
}

int tem_fit_poles(int32_t m, int32_t n_times, const double *t, int32_t n_z, double z_min, double z_max, double mu,
                  int32_t max_iter, double *xi, double *obj, void *stream) {
  Range nvtx_range("tem_fit_poles");
  tem_ctx *c = nullptr;   // no context: errors go to tem_last_error(NULL)
  if (m <= 0 || m > 32 || n_times <= 0 || n_times > 4096 || !t || !xi || !obj || max_iter < 0 || max_iter > 100000)
    return fail(c, TEM_ERR_ARG, "bad pole-fit arguments (1 <= m <= 32, 1 <= n_times <= 4096)");
  for (int j = 0; j < n_times; j++)
    if (!(t[j] > 0) || !std::isfinite(t[j])) return fail(c, TEM_ERR_ARG, "every time must be finite and > 0");
  if (n_z < 2 || n_z > (1 << 20) || !(z_min > 0) || !(z_max > z_min) || !std::isfinite(z_max) || !(mu >= 0) ||
      !std::isfinite(mu))
    return fail(c, TEM_ERR_ARG, "bad sample set (2 <= n_z <= 2^20, 0 < z_min < z_max finite, mu >= 0)");
  for (int i = 0; i < m; i++)
    if (!(xi[2 * i] < 0) || !(xi[2 * i + 1] > 0) || !std::isfinite(xi[2 * i]) || !std::isfinite(xi[2 * i + 1]))
      return fail(c, TEM_ERR_ARG, "starting poles need Re xi < 0 < Im xi");
  const int K = n_times, nc = 2 * m;
  const int64_t rows = int64_t(n_z) + 1 + nc;
  if (rows * nc * K > (int64_t(1) << 31))   // the Jacobian tails: 16 GB at this bound
    return fail(c, TEM_ERR_ARG, "pole fit too large: (n_z + 1 + 2m) 2m n_times must stay below 2^31");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  struct Scratch {
    std::vector<void *> p;
    ~Scratch() {
      for (void *q : p) cudaFree(q);
    }
  } w;
  auto get = [&](size_t bytes, void **out) {
    *out = nullptr;
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
    w.p.push_back(*out);
    return int(TEM_OK);
  };
  double *B, *Y, *rd, *cf, *td, *coef, *tail, *T, *G;
  double2 *xd;
  TRY(get(sizeof(double) * rows * nc, (void **)&B));
  TRY(get(sizeof(double) * rows * K, (void **)&Y));
  TRY(get(sizeof(double) * nc, (void **)&rd));
  TRY(get(sizeof(double) * nc, (void **)&cf));
  TRY(get(sizeof(double) * K, (void **)&td));
  TRY(get(sizeof(double) * nc * K, (void **)&coef));
  TRY(get(sizeof(double) * K, (void **)&tail));
  TRY(get(sizeof(double) * rows * nc * K, (void **)&T));
  TRY(get(sizeof(double) * nc * (nc + 1), (void **)&G));
  TRY(get(sizeof(double2) * m, (void **)&xd));
  const double lz0 = std::log10(z_min), lz1 = std::log10(z_max);
  CK(cudaMemcpyAsync(td, t, sizeof(double) * K, cudaMemcpyHostToDevice, s));
  auto poles_of = [&](const std::vector<double> &p) {
    std::vector<double> x(2 * m);
    for (int i = 0; i < m; i++) {
      x[2 * i] = -std::exp(p[i]);
      x[2 * i + 1] = std::exp(p[m + i]);
    }
    return x;
  };
  // objective sum_j ||(I - Q Q^T) e_j||^2 at p (leaves B, Y and coef of p on the device); +inf if singular
  auto eval = [&](const std::vector<double> &p, double *f) {
    const std::vector<double> x = poles_of(p);
    CK(cudaMemcpyAsync(xd, x.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, s));
    launch_fit_qr(xd, m, n_z, lz0, lz1, mu, B, rd, cf, s);
    std::vector<double> rdh(nc), th(K);
    CK(cudaMemcpyAsync(rdh.data(), rd, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double rmax = 0;
    for (double v : rdh) rmax = std::max(rmax, std::fabs(v));
    for (double v : rdh)
      if (!std::isfinite(v) || !(std::fabs(v) > 1e-14 * rmax)) {
        *f = INFINITY;
        return int(TEM_OK);
      }
    launch_fit_solve(B, m, n_z, lz0, lz1, rd, cf, td, K, Y, nullptr, s, coef, tail);
    CK(cudaMemcpyAsync(th.data(), tail, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double sum = 0;
    for (double v : th) sum += v;
    *f = std::isfinite(sum) ? sum : INFINITY;
    return int(TEM_OK);
  };
  std::vector<double> p(nc);
  for (int i = 0; i < m; i++) {
    p[i] = std::log(-xi[2 * i]);
    p[m + i] = std::log(xi[2 * i + 1]);
  }
  double f = 0;
  TRY(eval(p, &f));
  if (!std::isfinite(f)) return fail(c, TEM_ERR_ARG, "the starting poles leave the residue fit rank deficient");
  const double f0 = f;
  double lam = 1e-3;
  int it = 0;
  std::vector<double> Gh(size_t(nc) * (nc + 1));
  for (; it < max_iter; it++) {
    // Levenberg-Marquardt step on the Kaufman normal equations (T^T T + lam diag) d = T^T y
    launch_vp_normal(B, m, n_z, lz0, lz1, mu, xd, cf, coef, K, Y, T, G, s);
    CK(cudaMemcpyAsync(Gh.data(), G, sizeof(double) * Gh.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    auto gel = [&](int a, int b) { return Gh[size_t(std::min(a, b)) * (nc + 1) + std::max(a, b)]; };
    bool accepted = false;
    double fn = f;
    std::vector<double> pn(nc);
    for (int tries = 0; tries < 30 && !accepted; tries++) {
      // Cholesky of A = G + lam (diag(G) + 1e-9 trace(G) / nc): Marquardt's scaling, kept
      // positive for parameters whose columns vanish (a residue of zero)
      std::vector<double> A(size_t(nc) * nc), d(nc);
      double tr = 0;
      for (int a = 0; a < nc; a++) tr += gel(a, a);
      for (int a = 0; a < nc; a++) {
        for (int b = 0; b < nc; b++) A[size_t(a) * nc + b] = gel(a, b);
        A[size_t(a) * nc + a] += lam * (gel(a, a) + 1e-9 * tr / nc);
        d[a] = Gh[size_t(a) * (nc + 1) + nc];
      }
      bool spd = true;
      for (int a = 0; a < nc && spd; a++) {
        for (int b = 0; b <= a; b++) {
          double v = A[size_t(a) * nc + b];
          for (int q = 0; q < b; q++) v -= A[size_t(a) * nc + q] * A[size_t(b) * nc + q];
          if (a == b) {
            if (!(v > 0)) { spd = false; break; }
            A[size_t(a) * nc + a] = std::sqrt(v);
          } else {
            A[size_t(a) * nc + b] = v / A[size_t(b) * nc + b];
          }
        }
      }
      if (spd) {
        for (int a = 0; a < nc; a++) {   // L z = d, then L^T x = z
          for (int q = 0; q < a; q++) d[a] -= A[size_t(a) * nc + q] * d[q];
          d[a] /= A[size_t(a) * nc + a];
        }
        for (int a = nc - 1; a >= 0; a--) {
          for (int q = a + 1; q < nc; q++) d[a] -= A[size_t(q) * nc + a] * d[q];
          d[a] /= A[size_t(a) * nc + a];
        }
        double dmax = 0;   // at most a factor e^2 per step in any pole's real or imaginary part
        for (int a = 0; a < nc; a++) dmax = std::max(dmax, std::fabs(d[a]));
        const double sc = dmax > 2.0 ? 2.0 / dmax : 1.0;
        for (int a = 0; a < nc; a++) pn[a] = p[a] + sc * d[a];
        TRY(eval(pn, &fn));
        if (fn < f) accepted = true;
      }
      if (!accepted) lam *= 4.0;
    }
    if (!accepted) {   // no descent left: restore the device state of p and stop
      TRY(eval(p, &f));
      break;
    }
    const double rel = (f - fn) / f;
    p = pn;
    f = fn;
    lam = std::max(lam / 3.0, 1e-12);
    if (rel < 1e-12) {
      it++;
      break;
    }
  }
  const std::vector<double> x = poles_of(p);
  std::copy(x.begin(), x.end(), xi);
  obj[0] = f0;
  obj[1] = f;
  obj[2] = double(it);
  return TEM_OK;
}

int tem_sources(tem_ctx *c, int32_t n_tx, const int64_t *loop_ptr, const int32_t *loop_verts, int32_t n_rx,
                const double *rx) {
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_MESH)) return fail(c, TEM_ERR_STATE, "tem_mesh first");
  if (c->state & ST_SOURCES) return fail(c, TEM_ERR_STATE, "sources already set");
  if (n_tx <= 0 || n_rx <= 0 || !loop_ptr || !loop_verts || !rx) return fail(c, TEM_ERR_ARG, "bad sources");
  std::vector<double> f, q_val, qt_val;
  std::vector<int64_t> q_rp, qt_rp;
  std::vector<int32_t> q_ci, qt_ci, qt_dof;
  std::string msg = build_sources(c->mesh, n_tx, loop_ptr, loop_verts, n_rx, rx, f, q_rp, q_ci, q_val, qt_dof,
                                  qt_rp, qt_ci, qt_val);
  if (!msg.empty()) return fail(c, TEM_ERR_MESH, msg);
  c->n_tx = n_tx;
  c->nrhs = n_tx + (n_tx & 1);
  c->n_rx = n_rx;
  c->n_qdof = (int)qt_dof.size();
  if (c->nrhs != n_tx) {   // a zero right-hand side pads an odd transmitter count
    std::vector<double> fp(size_t(c->mesh.N) * c->nrhs, 0.0);
    for (int64_t i = 0; i < c->mesh.N; i++)
      for (int x = 0; x < n_tx; x++) fp[size_t(i) * c->nrhs + x] = f[size_t(i) * n_tx + x];
    f.swap(fp);
  }
  TRY(upload(c, &c->f, f));
  TRY(upload(c, &c->q_rp, q_rp));
  TRY(upload(c, &c->q_ci, q_ci));
  TRY(upload(c, &c->q_val, q_val));
  TRY(upload(c, &c->qt_dof, qt_dof));
  TRY(upload(c, &c->qt_rp, qt_rp));
  TRY(upload(c, &c->qt_ci, qt_ci));
  TRY(upload(c, &c->qt_val, qt_val));
  TRY(sync(c, "tem_sources"));
  c->state |= ST_SOURCES;
  return TEM_OK;
}

int tem_factor(tem_ctx *c, const double *log_sigma) {
  Range nvtx_range("tem_factor");
  if (!c) return TEM_ERR_ARG;
  const int need = ST_MESH | ST_POLES | ST_SOURCES;
  if ((c->state & need) != need) return fail(c, TEM_ERR_STATE, "tem_mesh, tem_poles and tem_sources first");
  if (!log_sigma && c->mesh.P > 0) return fail(c, TEM_ERR_ARG, "log_sigma is NULL");
  TRY(ensure_numeric(c));
  ProfScope ps(c);
  cudaStream_t s = c->stream;
  const Mesh &M = c->mesh;
  CK(cudaMemcpyAsync(c->sigma, c->sigma_fixed, sizeof(double) * M.nt, cudaMemcpyDeviceToDevice, s));
  if (M.P > 0) {
    CK(cudaMemcpyAsync(c->m_cur, log_sigma, sizeof(double) * M.P, cudaMemcpyDeviceToDevice, s));
    launch_sigma(log_sigma, c->ptet, M.P, c->sigma, s);
  }
  launch_mvals(c->mc_ptr, c->mc_idx, c->sigma, c->me1, 36, (int64_t)M.kval.size(), c->mval, s);
  if (c->mval_fact) {
    launch_mvals_floor(c->mc_ptr, c->mc_idx, c->sigma, c->tetfloor, c->me1, c->xi, c->floor_tau, c->m,
                       (int64_t)M.kval.size(), c->mval_fact, s);
    // the refinement's residual uses K and the true M as double-float pairs
    launch_split_real(c->kval, c->kdf, (int64_t)M.kval.size(), s);
    launch_split_real(c->mval, c->mdf, (int64_t)M.kval.size(), s);
  }
  launch_status_init(c->status, s);   // a kernel, not a host copy: the call stays capturable
  if (c->precision == TEM_FP64) {
    factor_sys<double>(c, c->es);
  } else {
    factor_sys<float>(c, c->es);
    if (c->use_nodal) {
      // sigma-weighted P1 Laplacian G^T M(sigma) G of the gradient space (pole independent)
      launch_mvals(c->n_mc_ptr, c->n_mc_idx, c->sigma, c->n_stiff, 16, (int64_t)c->nodal.ci.size(), c->n_mval, s);
      launch_mvals(c->n_cmc_ptr, c->n_cmc_idx, c->sigma, c->n_btab, 24, (int64_t)c->nodal.c_ci.size(), c->n_cval, s);
      factor_sys<float>(c, c->ns);
    }
  }
  c->state &= ~(ST_FACTORED | ST_FORWARD);
  if (c->async) {   // a pivot failure is reported by tem_status
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "tem_factor");
    c->state |= ST_FACTORED;
    return TEM_OK;
  }
  CK(cudaMemcpyAsync(&c->status_h, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  TRY(sync(c, "tem_factor"));
  if (c->status_h.pivot_fail) {
    char buf[160];
    snprintf(buf, sizeof buf, "pivot underflow in front %d", c->status_h.pivot_front);
    return fail(c, TEM_ERR_PIVOT, buf);
  }
  c->state |= ST_FACTORED;
  return TEM_OK;
}

int tem_forward(tem_ctx *c, double *d) {
  Range nvtx_range("tem_forward");
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_FACTORED)) return fail(c, TEM_ERR_STATE, "tem_factor first");
  if (!d) return fail(c, TEM_ERR_ARG, "d is NULL");
  ProfScope ps(c);
  cudaStream_t s = c->stream;
  const int64_t N = c->mesh.N;
  launch_real_to_c128(c->f, c->fb, N * c->nrhs, s);
  TRY(solve_all(c, c->fb, 0, c->g, c->refine));
  if (c->precision != TEM_FP64)   // the Jacobian kernels read the forward solutions as pairs
    CK(cudaMemcpyAsync(c->gdf, c->xdf, sizeof(float4) * c->m * N * c->nrhs, cudaMemcpyDeviceToDevice, s));
  launch_residue(c->q_rp, c->q_ci, c->q_val, c->alpha, c->g, d, c->m, N, c->nrhs, c->n_tx, c->n_rx, c->K, s);
  CK(cudaMemcpyAsync(c->d_cur, d, sizeof(double) * c->n_tx * c->n_rx * c->K, cudaMemcpyDeviceToDevice, s));
  TRY(finish(c, "tem_forward"));
  c->state |= ST_FORWARD;
  return TEM_OK;
}

namespace {
int jvp_async(tem_ctx *c, const double *v, double *jv) {
  const int64_t N = c->mesh.N;
  if (g_prof) g_prof->begin(KC_JACOBIAN, c->stream);
  if (c->precision == TEM_FP64)
    launch_dm_apply(c->inc_ptr, c->inc_tet, c->inc_loc, c->tdof, c->pidx, v, c->sigma, c->me1, c->xi, c->g, c->b,
                    c->m, N, c->nrhs, c->stream);
  else
    launch_dm_apply_df(c->inc_ptr, c->inc_tet, c->inc_loc, c->tdof, c->ptet, c->mesh.P, v, c->sigma, c->vsdf,
                       c->mesh.nt, c->me1df, c->xi, c->gdf, reinterpret_cast<float4 *>(c->r), c->m, N, c->nrhs,
                       c->stream);   // as the pairs the refinement takes
  if (g_prof) g_prof->end(KC_JACOBIAN, c->stream);
  // FP32 mode: the residue sums read the refined pairs directly (no FP64 copy of the solutions)
  const bool fp64 = c->precision == TEM_FP64;
  TRY(solve_all(c, c->b, N * c->nrhs, c->x, c->refine, fp64, !fp64));
  if (g_prof) g_prof->begin(KC_JACOBIAN, c->stream);
  if (fp64)
    launch_residue(c->q_rp, c->q_ci, c->q_val, c->alpha, c->x, jv, c->m, N, c->nrhs, c->n_tx, c->n_rx, c->K,
                   c->stream);
  else
    launch_residue(c->q_rp, c->q_ci, c->q_val, c->alpha, c->xdf, jv, c->m, N, c->nrhs, c->n_tx, c->n_rx, c->K,
                   c->stream);
  if (g_prof) g_prof->end(KC_JACOBIAN, c->stream);
  return TEM_OK;
}
int jtvp_async(tem_ctx *c, const double *w, double *jtw) {
  const int64_t N = c->mesh.N;
  if (g_prof) g_prof->begin(KC_JACOBIAN, c->stream);
  const bool fp64 = c->precision == TEM_FP64;
  if (fp64)
    launch_qt_rhs(c->qt_dof, c->qt_rp, c->qt_ci, c->qt_val, c->n_qdof, c->alpha, w, c->b, c->m, N, c->nrhs,
                  c->n_tx, c->n_rx, c->K, c->stream);
  else   // straight into the pairs the refinement takes
    launch_qt_rhs(c->qt_dof, c->qt_rp, c->qt_ci, c->qt_val, c->n_qdof, c->alpha, w,
                  reinterpret_cast<float4 *>(c->r), c->m, N, c->nrhs, c->n_tx, c->n_rx, c->K, c->stream);
  if (g_prof) g_prof->end(KC_JACOBIAN, c->stream);
  // the adjoint solves feed only the cell sums over parameter cells, which
  // converge in fewer corrections than the receivers' fields (46^3 box: within
  // 1e-7 of the converged J^T w after 6)
  TRY(solve_all(c, c->b, N * c->nrhs, c->x, c->refine_adj, fp64, !fp64));   // FP32: b and x as pairs
  if (g_prof) g_prof->begin(KC_JACOBIAN, c->stream);
  if (c->precision == TEM_FP64)
    launch_bilinear(c->ptet, c->mesh.P, c->tdof, c->sigma, c->me1, c->xi, c->g, c->x, jtw, c->m, N, c->nrhs,
                    c->stream);
  else   // per-pole double-float cell sums of the refined pairs (xdf holds z), then summed over poles
    launch_bilinear_df(c->ptet, c->mesh.P, c->tdof, c->sigma, c->me1df, c->xi, c->gdf, c->xdf, jtw, c->m, N,
                       c->nrhs, c->part, c->stream);
  if (g_prof) g_prof->end(KC_JACOBIAN, c->stream);
  return TEM_OK;
}
}  // namespace

int tem_jvp(tem_ctx *c, const double *v, double *jv) {
  Range nvtx_range("tem_jvp");
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_FORWARD)) return fail(c, TEM_ERR_STATE, "tem_forward first");
  if (!v || !jv) return fail(c, TEM_ERR_ARG, "NULL vector");
  ProfScope ps(c);
  TRY(jvp_async(c, v, jv));
  return finish(c, "tem_jvp");
}

int tem_jtvp(tem_ctx *c, const double *w, double *jtw) {
  Range nvtx_range("tem_jtvp");
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_FORWARD)) return fail(c, TEM_ERR_STATE, "tem_forward first");
  if (!w || !jtw) return fail(c, TEM_ERR_ARG, "NULL vector");
  ProfScope ps(c);
  TRY(jtvp_async(c, w, jtw));
  return finish(c, "tem_jtvp");
}

int tem_lsqr(tem_ctx *c, const double *d_obs, const double *wd, const double *m_ref, double lambda,
             int32_t n_iter, double *dm) {
  Range nvtx_range("tem_lsqr");
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_FORWARD)) return fail(c, TEM_ERR_STATE, "tem_forward first");
  if (!d_obs || !wd || !m_ref || !dm || n_iter < 0 || !(lambda >= 0)) return fail(c, TEM_ERR_ARG, "bad LSQR args");
  const int64_t nd = int64_t(c->n_tx) * c->n_rx * c->K, P = c->mesh.P, nf = c->mesh.nf;
  TRY(ensure_lsqr_buffers(c));
  ProfScope ps(c);
  cudaStream_t s = c->stream;
  const double sl = std::sqrt(lambda);
  double *u1 = c->ls_u, *u2 = c->ls_u + nd;
  LsqrScalars *sc = c->ls_sc;
  CK(cudaMemsetAsync(sc, 0, sizeof(LsqrScalars), s));
  // u = b = -[W_d (d - d_obs); sqrt(lam) W (m - m_ref)]
  launch_lsqr_kernel(6, sc, u1, c->d_cur, d_obs, wd, nd, s);
  launch_csr_mv(c->w_rp, c->w_ci, c->w_val, c->m_cur, u2, nf, -sl, 0.0, s);
  launch_csr_mv(c->w_rp, c->w_ci, c->w_val, m_ref, u2, nf, sl, 1.0, s);
  launch_sumsq(c->ls_u, nd + nf, &sc->sumsq, s);
  launch_lsqr_kernel(0, sc, c->ls_u, nullptr, nullptr, nullptr, nd + nf, s);
  launch_lsqr_scalars(sc, 0, s);  // beta
  // v = A^T u
  launch_lsqr_kernel(5, sc, c->ls_tmpd, u1, wd, nullptr, nd, s);
  TRY(jtvp_async(c, c->ls_tmpd, c->ls_jtw));
  CK(cudaMemcpyAsync(c->ls_v, c->ls_jtw, sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
  launch_csr_mv(c->wt_rp, c->wt_ci, c->wt_val, u2, c->ls_v, P, sl, 1.0, s);
  launch_sumsq(c->ls_v, P, &sc->sumsq, s);
  launch_lsqr_kernel(1, sc, c->ls_v, nullptr, nullptr, nullptr, P, s);
  launch_lsqr_scalars(sc, 1, s);  // alpha
  launch_lsqr_scalars(sc, 2, s);  // phibar, rhobar
  CK(cudaMemcpyAsync(c->ls_w, c->ls_v, sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(dm, 0, sizeof(double) * P, s));
  for (int it = 0; it < n_iter; it++) {
    // u = A v - alpha u
    TRY(jvp_async(c, c->ls_v, c->ls_jv));
    launch_lsqr_kernel(2, sc, u1, c->ls_jv, wd, nullptr, nd, s);
    launch_csr_mv(c->w_rp, c->w_ci, c->w_val, c->ls_v, c->ls_wv, nf, sl, 0.0, s);
    launch_lsqr_kernel(7, sc, u2, c->ls_wv, nullptr, nullptr, nf, s);  // u2 = sl W v - alpha u2
    launch_sumsq(c->ls_u, nd + nf, &sc->sumsq, s);
    launch_lsqr_kernel(0, sc, c->ls_u, nullptr, nullptr, nullptr, nd + nf, s);
    launch_lsqr_scalars(sc, 0, s);  // beta
    // v = A^T u - beta v
    launch_lsqr_kernel(5, sc, c->ls_tmpd, u1, wd, nullptr, nd, s);
    TRY(jtvp_async(c, c->ls_tmpd, c->ls_jtw));
    launch_csr_mv(c->wt_rp, c->wt_ci, c->wt_val, u2, c->ls_jtw, P, sl, 1.0, s);
    launch_lsqr_kernel(3, sc, c->ls_v, c->ls_jtw, nullptr, nullptr, P, s);
    launch_sumsq(c->ls_v, P, &sc->sumsq, s);
    launch_lsqr_kernel(1, sc, c->ls_v, nullptr, nullptr, nullptr, P, s);
    launch_lsqr_scalars(sc, 1, s);  // alpha
    launch_lsqr_scalars(sc, 3, s);  // rho, c, s, theta, phi
    launch_lsqr_kernel(4, sc, dm, c->ls_w, c->ls_v, nullptr, P, s);
  }
  return finish(c, "tem_lsqr");
}

int tem_set_wait_limit(tem_ctx *c, uint32_t max_polls, double max_seconds) {
  if (!c) return TEM_ERR_ARG;
  if (max_polls == 0 || !(max_seconds > 0) || max_seconds > 60) return fail(c, TEM_ERR_ARG, "bad wait limit");
  set_tc_wait_limit(max_polls, uint64_t(max_seconds * 1e9));
  return TEM_OK;
}


int tem_gn_eval(tem_ctx *c, const double *d_obs, const double *wd, const double *m_ref, double lambda,
                const double *dm, double *grad, double *out) {
  Range nvtx_range("tem_gn_eval");
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_FORWARD)) return fail(c, TEM_ERR_STATE, "tem_forward first");
  if (!d_obs || !wd || !m_ref || !out || !(lambda >= 0) || (dm && !grad)) return fail(c, TEM_ERR_ARG, "bad arguments");
  if (c->async) return fail(c, TEM_ERR_STATE, "tem_gn_eval returns host scalars: not in asynchronous mode");
  TRY(ensure_lsqr_buffers(c));
  ProfScope ps(c);
  cudaStream_t s = c->stream;
  const int64_t nd = int64_t(c->n_tx) * c->n_rx * c->K, P = c->mesh.P, nf = c->mesh.nf;
  double *sums = reinterpret_cast<double *>(c->ls_sc);   // sum t^2, sum (W (m - m_ref))^2, grad . dm
  CK(cudaMemsetAsync(sums, 0, 3 * sizeof(double), s));
  double *t = c->ls_tmpd, *t2 = c->ls_jv, *wv = c->ls_wv;
  launch_gn_res(c->d_cur, d_obs, wd, t, t2, nd, s);
  launch_dot(t, t, nd, sums, s);
  launch_csr_mv(c->w_rp, c->w_ci, c->w_val, c->m_cur, wv, nf, 1.0, 0.0, s);
  launch_csr_mv(c->w_rp, c->w_ci, c->w_val, m_ref, wv, nf, -1.0, 1.0, s);
  launch_dot(wv, wv, nf, sums + 1, s);
  if (grad) {
    // grad phi = J^T W_d^2 (d - d_obs) + lambda W^T W (m - m_ref)
    TRY(jtvp_async(c, t2, grad));
    launch_csr_mv(c->wt_rp, c->wt_ci, c->wt_val, wv, grad, P, lambda, 1.0, s);
    if (dm) launch_dot(grad, dm, P, sums + 2, s);
  }
  double h[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, s));
  TRY(finish(c, "tem_gn_eval"));
  out[1] = 0.5 * h[0];
  out[2] = 0.5 * h[1];
  out[0] = out[1] + lambda * out[2];
  out[3] = nd > 0 ? h[0] / double(nd) : 0.0;
  out[4] = h[2];
  return TEM_OK;
}

int tem_model_step(tem_ctx *c, const double *m, const double *dm, double eta, double *out) {
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_MESH) || !m || !dm || !out || !std::isfinite(eta)) return fail(c, TEM_ERR_ARG, "bad arguments");
  launch_axpy(m, dm, eta, out, c->mesh.P, c->stream);
  return finish(c, "tem_model_step");
}

int tem_set_amalgamation(tem_ctx *c, int32_t max_pivots) {
  if (!c) return TEM_ERR_ARG;
  if (c->state & ST_MESH) return fail(c, TEM_ERR_STATE, "the assembly tree is built by tem_mesh: set this before");
  if (max_pivots < 0 || max_pivots > 4096) return fail(c, TEM_ERR_ARG, "max_pivots in 0..4096");
  c->sym_opts.amalg_max = max_pivots;
  return TEM_OK;
}

int tem_set_tensor_cores(tem_ctx *c, int enable) {
  if (!c) return TEM_ERR_ARG;
  c->use_tc = enable != 0;
  return TEM_OK;
}

int tem_set_async(tem_ctx *c, int enable) {
  if (!c) return TEM_ERR_ARG;
  if (enable && c->refine_tol > 0)
    return fail(c, TEM_ERR_ARG, "asynchronous calls need a fixed correction count (tem_set_refine tol = 0)");
  if (c->async && !enable) TRY(sync(c, "tem_set_async"));
  c->async = enable != 0;
  return TEM_OK;
}

int tem_status(tem_ctx *c) {
  if (!c) return TEM_ERR_ARG;
  TRY(sync(c, "tem_status"));
  CK(cudaMemcpy(&c->status_h, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  if (c->status_h.tc_timeout) {   // reported once
    CK(cudaMemset(&c->status->tc_timeout, 0, sizeof(int32_t)));
    c->status_h.tc_timeout = 0;
    return fail(c, TEM_ERR_TIMEOUT, "a tensor-core completion wait expired");
  }
  if (c->status_h.pivot_fail) {
    c->state &= ~(ST_FACTORED | ST_FORWARD);
    char buf[160];
    snprintf(buf, sizeof buf, "pivot underflow in front %d", c->status_h.pivot_front);
    return fail(c, TEM_ERR_PIVOT, buf);
  }
  return TEM_OK;
}

int tem_batch(tem_ctx **ctx, int32_t n, int32_t ops, const double *const *log_sigma, double *const *d,
              const double *const *w, double *const *jtw) {
  Range nvtx_range("tem_batch");
  if (!ctx || n <= 0 || (ops & ~(TEM_BATCH_FACTOR | TEM_BATCH_FORWARD | TEM_BATCH_JTVP)) || ops == 0)
    return fail(nullptr, TEM_ERR_ARG, "tem_batch: bad contexts or operations");
  for (int i = 0; i < n; i++) {
    tem_ctx *c = ctx[i];
    if (!c) return fail(nullptr, TEM_ERR_ARG, "tem_batch: NULL context");
    if (((ops & TEM_BATCH_FACTOR) && !(log_sigma && log_sigma[i])) || ((ops & TEM_BATCH_FORWARD) && !(d && d[i])) ||
        ((ops & TEM_BATCH_JTVP) && !(w && w[i] && jtw && jtw[i])))
      return fail(c, TEM_ERR_ARG, "tem_batch: missing array");
  }
  // every context's calls, issued asynchronously on its own stream (no synchronisation in between)
  std::vector<char> was(n);
  int st = TEM_OK;
  for (int i = 0; i < n && st == TEM_OK; i++) {
    tem_ctx *c = ctx[i];
    was[i] = c->async;
    c->async = true;
    if (ops & TEM_BATCH_FACTOR) st = tem_factor(c, log_sigma[i]);
    if (st == TEM_OK && (ops & TEM_BATCH_FORWARD)) st = tem_forward(c, d[i]);
    if (st == TEM_OK && (ops & TEM_BATCH_JTVP)) st = tem_jtvp(c, w[i], jtw[i]);
  }
  for (int i = 0; i < n; i++) ctx[i]->async = was[i];
  if (st != TEM_OK) return st;
  // synchronous contexts: wait for all of them and report their status
  for (int i = 0; i < n; i++)
    if (!ctx[i]->async) TRY(tem_status(ctx[i]));
  return TEM_OK;
}

int tem_set_tc_fronts(tem_ctx *c, int enable) {
  if (!c) return TEM_ERR_ARG;
  if (c->tc_fronts != (enable != 0)) c->state &= ~(ST_FACTORED | ST_FORWARD);   // the next tem_factor decides
  c->tc_fronts = enable != 0;
  return TEM_OK;
}

int tem_set_refine(tem_ctx *c, int32_t steps, double floor_tau, double tol) {
  if (!c) return TEM_ERR_ARG;
  if (steps < 0 || steps > 40) return fail(c, TEM_ERR_ARG, "refine steps in 0..40");
  if (!(floor_tau >= 0) || floor_tau > 1.0) return fail(c, TEM_ERR_ARG, "floor_tau in [0, 1]");
  if (!(tol >= 0) || tol > 1.0) return fail(c, TEM_ERR_ARG, "tol in [0, 1]");
  if (tol > 0 && c->async) return fail(c, TEM_ERR_ARG, "a refinement tolerance reads progress on the host: not in asynchronous mode");
  c->refine = steps;
  c->floor_tau = floor_tau;
  c->refine_tol = tol;
  return TEM_OK;
}

int tem_set_nodal(tem_ctx *c, int enable) {
  if (!c) return TEM_ERR_ARG;
  if (c->state & ST_FACTORED) {
    // the nodal factor is formed by tem_factor: switching it on needs a new factorisation
    if (enable && !c->use_nodal) c->state &= ~(ST_FACTORED | ST_FORWARD);
  }
  c->use_nodal = enable != 0;
  return TEM_OK;
}

int tem_set_refine_adjoint(tem_ctx *c, int32_t steps) {
  if (!c) return TEM_ERR_ARG;
  if (steps < 0 || steps > 40) return fail(c, TEM_ERR_ARG, "refine steps in 0..40");
  c->refine_adj = steps;
  return TEM_OK;
}

int tem_info(tem_ctx *c, tem_stats *o) {
  if (!c || !o) return TEM_ERR_ARG;
  memset(o, 0, sizeof(*o));
  o->n_dof = c->mesh.N;
  o->n_tet = c->mesh.nt;
  o->n_param = c->mesh.P;
  o->n_faces_reg = c->mesh.nf;
  o->n_fronts = (int64_t)c->es.sym.fronts.size();
  o->n_levels = (int64_t)c->es.sym.levels.size();
  o->nnz_a = (int64_t)c->mesh.ci.size();
  o->nnz_l = c->es.sym.nnz_l;
  o->flops_factor = c->es.sym.flops;
  o->max_front = c->es.sym.max_front;
  o->bytes_device = c->bytes;
  o->m = c->m;
  o->n_times = c->K;
  o->n_tx = c->n_tx;
  o->n_rx = c->n_rx;
  o->precision = c->precision;
  o->refine_steps = c->refine;
  o->refine_steps_adjoint = c->refine_adj;
  o->last_pivot_front = c->status_h.pivot_fail ? c->status_h.pivot_front : -1;
  double mp;
  memcpy(&mp, &c->status_h.min_pivot_bits, sizeof(double));
  o->min_pivot_abs = mp;
  o->nnz_l11 = c->es.sym.nnz_l11;
  o->pole_solves = c->pole_solves;
  o->solve_calls = c->solve_calls;
  int64_t nl = 0;
  for (const LevelDev &lv : c->es.levels) {
    if (c->precision == TEM_FP64) {
      nl += 2 * (int64_t)lv.steps.size() + (lv.n_f21 > 0 ? 1 : 0) + (lv.n_b21 > 0 ? 1 : 0);
      for (const auto &sb : lv.sb) nl += (sb.n_fwd > 0 ? 1 : 0) + (sb.n_bwd > 0 ? 1 : 0);
    } else {
      for (int mode = 0; mode < PM_COUNT; mode++) nl += lv.n_prod[mode] > 0 ? 1 : 0;
    }
  }
  o->n_solve_launch = nl;
  o->tc_ctas_per_sm = tc_ctas_per_sm();
  o->tc_prod_launches = prod_launches(true);
  o->simt_prod_launches = prod_launches(false);
  o->n_nodes = c->ns.N;
  o->nnz_l_nodal = c->ns.sym.nnz_l;
  o->nodal = c->precision != TEM_FP64 && c->use_nodal ? 1 : 0;
  o->tc_update_launches = update_launches();
  return TEM_OK;
}

int tem_export_pattern(tem_ctx *c, int64_t *nnz, int64_t *row_ptr, int32_t *col, double *k_val, double *m_val) {
  if (!c || !nnz) return TEM_ERR_ARG;
  if (!(c->state & ST_MESH)) return fail(c, TEM_ERR_STATE, "tem_mesh first");
  const Mesh &M = c->mesh;
  *nnz = (int64_t)M.ci.size();
  if (row_ptr) memcpy(row_ptr, M.rp.data(), sizeof(int64_t) * M.rp.size());
  if (col) memcpy(col, M.ci.data(), sizeof(int32_t) * M.ci.size());
  if (k_val) memcpy(k_val, M.kval.data(), sizeof(double) * M.kval.size());
  if (m_val) {
    if (!(c->state & ST_FACTORED)) return fail(c, TEM_ERR_STATE, "M values exist after tem_factor");
    CK(cudaMemcpy(m_val, c->mval, sizeof(double) * M.kval.size(), cudaMemcpyDeviceToHost));
  }
  return TEM_OK;
}

int tem_export_forward(tem_ctx *c, double *g) {
  if (!c || !g) return TEM_ERR_ARG;
  if (!(c->state & ST_FORWARD)) return fail(c, TEM_ERR_STATE, "tem_forward first");
  const int64_t N = c->mesh.N;
  const int nx = c->nrhs;
  std::vector<c128> h(size_t(c->m) * N * nx);
  CK(cudaMemcpy(h.data(), c->g, sizeof(c128) * h.size(), cudaMemcpyDeviceToHost));
  for (int p = 0; p < c->m; p++)
    for (int64_t i = 0; i < N; i++)
      for (int x = 0; x < c->n_tx; x++) {   // drop the padding right-hand side
        const c128 v = h[(size_t(p) * N + i) * nx + x];
        const size_t o = 2 * ((size_t(p) * N + i) * c->n_tx + x);
        g[o] = v.x;
        g[o + 1] = v.y;
      }
  return TEM_OK;
}

int tem_level_info(tem_ctx *c, int64_t *out) {
  if (!c || !out) return TEM_ERR_ARG;
  if (!(c->state & ST_MESH)) return fail(c, TEM_ERR_STATE, "tem_mesh first");
  const Symbolic &S = c->es.sym;
  for (size_t h = 0; h < S.levels.size(); h++) {
    int64_t *o = out + 4 * h;
    o[0] = (int64_t)S.levels[h].fronts.size();
    o[1] = o[2] = o[3] = 0;
    for (int32_t f : S.levels[h].fronts) {
      const Front &F = S.fronts[f];
      o[1] += int64_t(F.k) * (F.k + 1) / 2;
      o[2] += int64_t(F.k) * (F.n - F.k);
      o[3] = std::max<int64_t>(o[3], F.k);
    }
  }
  return TEM_OK;
}

int tem_export_dofs(tem_ctx *c, int64_t *edge_verts) {
  if (!c || !edge_verts) return TEM_ERR_ARG;
  if (!(c->state & ST_MESH)) return fail(c, TEM_ERR_STATE, "tem_mesh first");
  const Mesh &M = c->mesh;
  std::vector<int64_t> old_edge(M.N);
  for (int64_t e = 0; e < M.ne; e++)
    if (M.dof_old[e] >= 0) old_edge[M.dof_old[e]] = e;
  for (int64_t i = 0; i < M.N; i++) {
    int64_t e = old_edge[M.perm[i]];
    edge_verts[2 * i] = M.ev[2 * e];
    edge_verts[2 * i + 1] = M.ev[2 * e + 1];
  }
  return TEM_OK;
}

int tem_set_profiling(tem_ctx *c, int kernel_class) {
  if (!c) return TEM_ERR_ARG;
  const int cls = kernel_class < 0 ? -1 : kernel_class % 64, lev = kernel_class < 0 ? -1 : kernel_class / 64 - 1;
  if (kernel_class < -1 || cls >= KC_COUNT) return fail(c, TEM_ERR_ARG, "bad kernel class");
  c->prof.on = kernel_class >= 0;
  c->prof.cls = cls;
  c->prof.level = lev;
  c->prof.total_ms = 0;
  c->prof.launches = 0;
  c->prof.used = 0;
  return TEM_OK;
}

int64_t tem_launch_count(void) { return launch_total(); }

int tem_kernel_time(tem_ctx *c, double *total_ms, int64_t *launches) {
  if (!c || !total_ms || !launches) return TEM_ERR_ARG;
  *total_ms = c->prof.total_ms;
  *launches = c->prof.launches;
  return TEM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// LSQR that allocates nothing.
//
// For callers that cannot allocate device memory while an inversion runs:
// programs whose device memory is handed out by their own allocator (a
// framework's caching pool) or that must not risk a cudaMalloc failing, or
// cudaMalloc/cudaFree synchronising the device, between Gauss-Newton steps.
// tem_lsqr allocates its work vectors on first use; this variant keeps them
// in one file-scope device array instead.  The factors and solve buffers it
// uses were allocated by tem_factor, which such callers run at start-up.

namespace {
constexpr size_t kNoAllocDoubles = size_t(4) << 20;  // 4 Mi doubles = 32 MiB per device
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];
std::mutex g_noalloc_mu;
std::map<int, double *> g_noalloc_addr;  // device -> address of g_noalloc_scratch

size_t pad32(size_t n) { return (n + 31) & ~size_t(31); }  // keep every slice 256-byte aligned
}  // namespace

extern "C" int tem_lsqr_noalloc(tem_ctx *c, const double *d_obs, const double *wd, const double *m_ref,
                                double lambda, int32_t n_iter, double *dm) {
  if (!c) return TEM_ERR_ARG;
  if (!(c->state & ST_FORWARD)) return fail(c, TEM_ERR_STATE, "tem_forward first");
  if (!d_obs || !wd || !m_ref || !dm || n_iter < 0 || !(lambda >= 0)) return fail(c, TEM_ERR_ARG, "bad LSQR args");
  const int64_t nd = int64_t(c->n_tx) * c->n_rx * c->K, P = c->mesh.P, nf = c->mesh.nf;
  const size_t nsc = pad32((sizeof(LsqrScalars) + sizeof(double) - 1) / sizeof(double));
  const size_t need = nsc + pad32(nd + nf) + 3 * pad32(P) + 2 * pad32(nd) + pad32(std::max<int64_t>(nf, 1));
  if (need > kNoAllocDoubles) {
    char buf[200];
    snprintf(buf, sizeof buf, "problem needs %zu doubles of LSQR scratch, the no-alloc limit is %zu", need,
             kNoAllocDoubles);
    return fail(c, TEM_ERR_ARG, buf);
  }
  int cur = -1;
  CK(cudaGetDevice(&cur));
  if (cur != c->device) return fail(c, TEM_ERR_STATE, "the context's device is not current");
  ProfScope ps(c);
  double *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(c->device);
    if (it == g_noalloc_addr.end()) {
      CK(cudaGetSymbolAddress((void **)&base, g_noalloc_scratch));
      g_noalloc_addr[c->device] = base;
    } else {
      base = it->second;
    }
  }
  LsqrScalars *sc = (LsqrScalars *)base;
  double *p = base + nsc;
  double *u = p;            p += pad32(nd + nf);
  double *v = p;            p += pad32(P);
  double *w = p;            p += pad32(P);
  double *jtw = p;          p += pad32(P);
  double *jv = p;           p += pad32(nd);
  double *tmpd = p;         p += pad32(nd);
  double *wv = p;           p += pad32(std::max<int64_t>(nf, 1));
  cudaStream_t s = c->stream;
  const double sl = std::sqrt(lambda);
  double *u1 = u, *u2 = u + nd;
  CK(cudaMemsetAsync(sc, 0, sizeof(LsqrScalars), s));   // sumsq and the recurrences start at zero
  launch_lsqr_kernel(6, sc, u1, c->d_cur, d_obs, wd, nd, s);
  launch_csr_mv(c->w_rp, c->w_ci, c->w_val, c->m_cur, u2, nf, -sl, 0.0, s);
  launch_csr_mv(c->w_rp, c->w_ci, c->w_val, m_ref, u2, nf, sl, 1.0, s);
  launch_sumsq(u, nd + nf, &sc->sumsq, s);
  launch_lsqr_kernel(0, sc, u, nullptr, nullptr, nullptr, nd + nf, s);
  launch_lsqr_scalars(sc, 0, s);
  launch_lsqr_kernel(5, sc, tmpd, u1, wd, nullptr, nd, s);
  TRY(jtvp_async(c, tmpd, jtw));
  CK(cudaMemcpyAsync(v, jtw, sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
  launch_csr_mv(c->wt_rp, c->wt_ci, c->wt_val, u2, v, P, sl, 1.0, s);
  launch_sumsq(v, P, &sc->sumsq, s);
  launch_lsqr_kernel(1, sc, v, nullptr, nullptr, nullptr, P, s);
  launch_lsqr_scalars(sc, 1, s);
  launch_lsqr_scalars(sc, 2, s);
  CK(cudaMemcpyAsync(w, v, sizeof(double) * P, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(dm, 0, sizeof(double) * P, s));
  for (int it = 0; it < n_iter; it++) {
    TRY(jvp_async(c, v, jv));
    launch_lsqr_kernel(2, sc, u1, jv, wd, nullptr, nd, s);
    launch_csr_mv(c->w_rp, c->w_ci, c->w_val, v, wv, nf, sl, 0.0, s);
    launch_lsqr_kernel(7, sc, u2, wv, nullptr, nullptr, nf, s);
    launch_sumsq(u, nd + nf, &sc->sumsq, s);
    launch_lsqr_kernel(0, sc, u, nullptr, nullptr, nullptr, nd + nf, s);
    launch_lsqr_scalars(sc, 0, s);
    launch_lsqr_kernel(5, sc, tmpd, u1, wd, nullptr, nd, s);
    TRY(jtvp_async(c, tmpd, jtw));
    launch_csr_mv(c->wt_rp, c->wt_ci, c->wt_val, u2, jtw, P, sl, 1.0, s);
    launch_lsqr_kernel(3, sc, v, jtw, nullptr, nullptr, P, s);
    launch_sumsq(v, P, &sc->sumsq, s);
    launch_lsqr_kernel(1, sc, v, nullptr, nullptr, nullptr, P, s);
    launch_lsqr_scalars(sc, 1, s);
    launch_lsqr_scalars(sc, 3, s);
    launch_lsqr_kernel(4, sc, dm, w, v, nullptr, P, s);
  }
  return finish(c, "tem_lsqr_noalloc");
}
