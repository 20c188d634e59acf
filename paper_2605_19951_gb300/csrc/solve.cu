// Multi-right-hand-side supernodal solves with the stored LDL^T factors,
// A_i X = B for all poles at once (Algorithm 1: solve with the cached factors).
//
// Vectors are [pole][N][nrhs] in the elimination numbering, right-hand sides
// contiguous.  The grid's z dimension runs over (pole, chunk of 32 RHS); in a
// CTA each warp owns rows (or columns) and each lane one right-hand side.
//
// Forward (L y = b, assembly tree bottom-up): at pivot step j of a front the
// CTA solves the unit lower NB x NB diagonal block for y_j (redundantly, from
// untouched data), CTA 0 stores y_j, and every CTA subtracts L[rows, j] y_j
// from its RT rows below: pivot rows of the same front directly, update rows
// (ancestors, shared with other fronts of the level) with atomics.
// Backward (D z = y, L^T x = z, top-down): w = D^-1 y - L21^T x_upd for all
// pivots of the level's fronts, then reverse pivot steps solve L_jj^T x_j = w_j
// and subtract L[j rows, c]^T x_j from the pivot columns c left of the block.
#include "common.cuh"
#include "kernels.h"

namespace tem {

template <typename R, int NB, int RT>
__global__ void __launch_bounds__(256) k_fwd_step(const cx<R> *__restrict__ L, int64_t lstride,
                                                  const FrontDev *__restrict__ F,
                                                  const int32_t *__restrict__ lev,
                                                  const int32_t *__restrict__ rows, int step,
                                                  cx<R> *__restrict__ Y, cx<R> *__restrict__ X,
                                                  int64_t vstride, int nrhs, int nchunk) {
  const FrontDev f = F[lev[blockIdx.y]];
  const int p = blockIdx.z / nchunk, ch = blockIdx.z % nchunk;
  const int j0 = step * NB;
  if (j0 >= f.k) return;
  const int nb = min(NB, f.k - j0);
  const int64_t n = f.n;
  const int64_t rbeg = j0 + nb;
  const int tile = blockIdx.x;
  if (tile > 0 && rbeg + int64_t(tile) * RT >= n) return;
  const cx<R> *A = L + p * lstride + f.lofs;
  cx<R> *Yp = Y + p * vstride;
  cx<R> *Xp = X + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Ljj[NB][NB + 1];
  __shared__ cx<R> xs[NB][32];
  __shared__ cx<R> Lt[NB][RT];
  for (int idx = threadIdx.x; idx < NB * NB; idx += 256) {
    int r = idx % NB, c = idx / NB;
    if (r < nb && c < nb && r > c) Ljj[r][c] = A[(j0 + c) * n + j0 + r];
  }
  for (int i = warp; i < NB; i += 8)
    xs[i][lane] = (ok && i < nb) ? Yp[int64_t(f.c0 + j0 + i) * nrhs + rhs] : mk<R>(R(0), R(0));
  const int64_t r0 = rbeg + int64_t(tile) * RT;
  for (int idx = threadIdx.x; idx < NB * RT; idx += 256) {
    int c = idx / RT, i = idx % RT;
    Lt[c][i] = (c < nb && r0 + i < n) ? A[(j0 + c) * n + r0 + i] : mk<R>(R(0), R(0));
  }
  __syncthreads();
  if (warp == 0) {
    for (int c = 0; c < nb; c++) {
      const cx<R> xc = xs[c][lane];
      for (int i = c + 1; i < nb; i++) cfms(xs[i][lane], Ljj[i][c], xc);
    }
  }
  __syncthreads();
  if (tile == 0 && ok)
    for (int i = warp; i < nb; i += 8) Xp[int64_t(f.c0 + j0 + i) * nrhs + rhs] = xs[i][lane];
  if (!ok) return;
  const int32_t *urow = rows + f.rows_off;
  for (int i = warp; i < RT; i += 8) {
    const int64_t r = r0 + i;
    if (r >= n) break;
    cx<R> acc = mk<R>(R(0), R(0));
#pragma unroll 8
    for (int c = 0; c < NB; c++)
      if (c < nb) cfma(acc, Lt[c][i], xs[c][lane]);
    if (r < f.k) {
      cx<R> *y = Yp + int64_t(f.c0 + r) * nrhs + rhs;
      *y = *y - acc;
    } else {
      atomic_add_cx(Yp + int64_t(urow[r - f.k]) * nrhs + rhs, mk<R>(-acc.x, -acc.y));
    }
  }
}

// w_c = D_c^-1 y_c - sum_{i >= k} L[i][c] x[row_i]  for every pivot c of the level's fronts;
// y_c is read from X (forward result), x[row_i] from X (final values of the
// ancestors, solved earlier in the top-down sweep); w goes to Y.
template <typename R>
__global__ void __launch_bounds__(256) k_bwd_upd(const cx<R> *__restrict__ L, int64_t lstride,
                                                 const FrontDev *__restrict__ F,
                                                 const int32_t *__restrict__ lev,
                                                 const int32_t *__restrict__ rows,
                                                 cx<R> *__restrict__ Y, const cx<R> *__restrict__ X,
                                                 int64_t vstride, int nrhs, int nchunk) {
  const FrontDev f = F[lev[blockIdx.y]];
  const int p = blockIdx.z / nchunk, ch = blockIdx.z % nchunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 8 + warp;
  if (c >= f.k) return;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  const int64_t n = f.n;
  const cx<R> *col = L + p * lstride + f.lofs + int64_t(c) * n;
  const cx<R> *Xp = X + p * vstride;
  cx<R> *Yp = Y + p * vstride;
  const int32_t *urow = rows + f.rows_off;
  cx<R> acc = mk<R>(R(0), R(0));
  for (int64_t i0 = f.k; i0 < n; i0 += 32) {
    const int64_t i = i0 + lane;
    cx<R> l = mk<R>(R(0), R(0));
    int32_t ri = 0;
    if (i < n) {
      l = col[i];
      ri = urow[i - f.k];
    }
    const int cnt = int(n - i0 < 32 ? n - i0 : 32);
    for (int q = 0; q < cnt; q++) {
      cx<R> lq;
      lq.x = __shfl_sync(0xffffffffu, l.x, q);
      lq.y = __shfl_sync(0xffffffffu, l.y, q);
      const int32_t rq = __shfl_sync(0xffffffffu, ri, q);
      if (ok) cfma(acc, lq, Xp[int64_t(rq) * nrhs + rhs]);
    }
  }
  if (!ok) return;
  // the forward sweep left y_c (solution of L y = b) in X at the pivot rows
  const cx<R> d = col[c];
  const int64_t at = int64_t(f.c0 + c) * nrhs + rhs;
  Yp[at] = Xp[at] * crecip(d) - acc;
}

template <typename R, int NB, int CT>
__global__ void __launch_bounds__(256) k_bwd_step(const cx<R> *__restrict__ L, int64_t lstride,
                                                  const FrontDev *__restrict__ F,
                                                  const int32_t *__restrict__ lev, int step,
                                                  cx<R> *__restrict__ Y, cx<R> *__restrict__ X,
                                                  int64_t vstride, int nrhs, int nchunk) {
  const FrontDev f = F[lev[blockIdx.y]];
  const int p = blockIdx.z / nchunk, ch = blockIdx.z % nchunk;
  const int j0 = step * NB;
  if (j0 >= f.k) return;
  const int nb = min(NB, f.k - j0);
  const int tile = blockIdx.x;
  if (tile > 0 && tile * CT >= j0) return;
  const int64_t n = f.n;
  const cx<R> *A = L + p * lstride + f.lofs;
  cx<R> *Yp = Y + p * vstride;
  cx<R> *Xp = X + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Ljj[NB][NB + 1];
  __shared__ cx<R> ws[NB][32];
  __shared__ cx<R> Lb[CT][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += 256) {
    int r = idx % NB, c = idx / NB;
    if (r < nb && c < nb && r > c) Ljj[r][c] = A[(j0 + c) * n + j0 + r];
  }
  for (int i = warp; i < NB; i += 8)
    ws[i][lane] = (ok && i < nb) ? Yp[int64_t(f.c0 + j0 + i) * nrhs + rhs] : mk<R>(R(0), R(0));
  const int cbeg = tile * CT;
  for (int idx = threadIdx.x; idx < NB * CT; idx += 256) {
    int i = idx % NB, cc = idx / NB;
    Lb[cc][i] = (i < nb && cbeg + cc < j0) ? A[int64_t(cbeg + cc) * n + j0 + i] : mk<R>(R(0), R(0));
  }
  __syncthreads();
  if (warp == 0) {
    for (int c = nb - 1; c >= 0; c--) {
      const cx<R> xc = ws[c][lane];
      for (int i = 0; i < c; i++) cfms(ws[i][lane], Ljj[c][i], xc);
    }
  }
  __syncthreads();
  if (!ok) return;
  if (tile == 0)
    for (int i = warp; i < nb; i += 8) Xp[int64_t(f.c0 + j0 + i) * nrhs + rhs] = ws[i][lane];
  for (int cc = warp; cc < CT; cc += 8) {
    const int c = cbeg + cc;
    if (c >= j0) break;
    cx<R> acc = mk<R>(R(0), R(0));
#pragma unroll 8
    for (int i = 0; i < NB; i++)
      if (i < nb) cfma(acc, Lb[cc][i], ws[i][lane]);
    cx<R> *y = Yp + int64_t(f.c0 + c) * nrhs + rhs;
    *y = *y - acc;
  }
}

template <typename R>
void SolvePlan<R>::forward_level(const LevelDev &lv, cudaStream_t s) {
  const int nchunk = (nrhs + 31) / 32;
  for (int step = 0; step < (int)lv.steps.size(); step++) {
    const StepDims &sd = lv.steps[step];
    dim3 g(sd.fwd_tiles, sd.nfronts, m * nchunk);
    if (g_prof) g_prof->begin(KC_FWD, s);
    tem::count_launch();
    k_fwd_step<R, kNB, SolveTile<R>::RT><<<g, 256, 0, s>>>(L, lstride, F, lv.fronts, rows, step, Y, X,
                                                            vstride, nrhs, nchunk);
    if (g_prof) g_prof->end(KC_FWD, s);
  }
}

template <typename R>
void SolvePlan<R>::backward_level(const LevelDev &lv, cudaStream_t s) {
  const int nchunk = (nrhs + 31) / 32;
  if (lv.nf == 0) return;
  dim3 gu(lv.bwd_upd_tiles, lv.nf, m * nchunk);
  if (g_prof) g_prof->begin(KC_BWD_UPD, s);
  tem::count_launch();
  k_bwd_upd<R><<<gu, 256, 0, s>>>(L, lstride, F, lv.fronts, rows, Y, X, vstride, nrhs, nchunk);
  if (g_prof) g_prof->end(KC_BWD_UPD, s);
  for (int step = (int)lv.steps.size() - 1; step >= 0; step--) {
    const StepDims &sd = lv.steps[step];
    dim3 g(sd.bwd_tiles, sd.nfronts, m * nchunk);
    if (g_prof) g_prof->begin(KC_BWD, s);
    tem::count_launch();
    k_bwd_step<R, kNB, SolveTile<R>::CT><<<g, 256, 0, s>>>(L, lstride, F, lv.fronts, step, Y, X, vstride, nrhs,
                                                  nchunk);
    if (g_prof) g_prof->end(KC_BWD, s);
  }
}

template struct SolvePlan<float>;
template struct SolvePlan<double>;

}  // namespace tem
