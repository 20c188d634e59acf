// Multi-right-hand-side supernodal solves with the stored LDL^T factors,
// A_i X = B for all poles at once (Algorithm 1: solve with the cached factors).
// This file holds the FP64 path (substitution with the pivot blocks); the
// FP32 path, whose pivot blocks hold their explicit inverses, runs four front
// products per level pair (solve_tc.cu).
//
// Vectors are [pole][N][nrhs] in the elimination numbering, right-hand sides
// contiguous.  The grid's z dimension runs over (pole, chunk of 32 RHS); a
// lane owns one right-hand side.  The inverse of every unit-lower NB x NB
// diagonal block is stored by the factorisation (Linv), so each diagonal
// solve is a small product that all warps share.
//
// Forward (L y = b), assembly tree bottom-up, per level:
//   k_fwd_l11  per pivot step j: y_j = Linv_jj b_j (stored in X), then the
//              pivot rows below the block (L11 only) -= L[r, j] y_j;
//   k_fwd_l21  once: Y[update rows] -= L21 X_piv, a tiled GEMM per front
//              with atomic accumulation (fronts of a level share ancestors).
// Backward (D z = y, L^T x = z), top-down, per level:
//   k_bwd_l21  once: w = D^-1 y - L21^T x_upd (tiled GEMM, no atomics);
//   k_bwd_l11  reverse pivot steps: x_j = Linv_jj^T w_j, then the pivot
//              columns left of the block -= L[j rows, c]^T x_j.
// The pivot blocks are also grouped in super-blocks of kSB pivots: the step
// kernels only touch rows / columns inside their super-block, and the rest
// of the pivot-block work of a super-block is one split-K product
// (k_fwd_sb: y_J -= L[J, 0:J0] x; k_bwd_sb: w_J -= L[J1:k, J]^T x).
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace tem {

// y[i][lane] <- sum_c Inv(i, c) y[c][lane] for i < NB, in place; Inv is
// stored as Inv[c][i] (column c of the inverse); transpose applies Inv^T.
// Ends with a barrier.
template <typename R, int NB>
__device__ __forceinline__ void small_apply(const cx<R> (*Inv)[NB], cx<R> (*y)[32], int warp, int lane,
                                            bool transpose) {
  constexpr int PW = NB / 8;
  cx<R> out[PW];
#pragma unroll
  for (int q = 0; q < PW; q++) {
    const int i = warp + 8 * q;
    cx<R> acc = mk<R>(R(0), R(0));
#pragma unroll 8
    for (int c = 0; c < NB; c++) cfma(acc, transpose ? Inv[i][c] : Inv[c][i], y[c][lane]);
    out[q] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PW; q++) y[warp + 8 * q][lane] = out[q];
  __syncthreads();
}

template <typename R, int NB, int RT>
__global__ void __launch_bounds__(256) k_fwd_l11(const cx<R> *__restrict__ L, int64_t lstride,
                                                 const cx<R> *__restrict__ Linv, int64_t istride,
                                                 const FrontDev *__restrict__ F,
                                                 const int32_t *__restrict__ lev, int step,
                                                 cx<R> *__restrict__ Y, cx<R> *__restrict__ X,
                                                 int64_t vstride, int nrhs, int nchunk,
                                                 const int *__restrict__ pmap) {
  const FrontDev f = F[lev[blockIdx.y]];
  const int p = pole_of(blockIdx.z / nchunk, pmap), ch = blockIdx.z % nchunk;
  const int j0 = step * NB;
  if (j0 >= f.k) return;
  const int nb = min(NB, f.k - j0);
  const int64_t n = f.ld;   // column stride
  const int rbeg = j0 + nb;                       // pivot rows below the block ...
  const int rend = min(f.k, (j0 / kSB + 1) * kSB);  // ... inside its super-block
  const int tile = blockIdx.x;
  if (tile > 0 && rbeg + tile * RT >= rend) return;
  const cx<R> *A = L + p * lstride + f.lofs;
  const cx<R> *Iv = Linv + p * istride + (f.inv_off + step) * (NB * NB);
  cx<R> *Yp = Y + p * vstride;
  cx<R> *Xp = X + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Inv[NB][NB];
  __shared__ cx<R> xs[NB][32];
  __shared__ cx<R> Lt[NB][RT];
  for (int idx = threadIdx.x; idx < NB * NB; idx += 256) Inv[idx / NB][idx % NB] = Iv[idx];
  for (int i = warp; i < NB; i += 8)
    xs[i][lane] = (ok && i < nb) ? Yp[int64_t(f.c0 + j0 + i) * nrhs + rhs] : mk<R>(R(0), R(0));
  const int r0 = rbeg + tile * RT;
  for (int idx = threadIdx.x; idx < NB * RT; idx += 256) {
    int c = idx / RT, i = idx % RT;
    Lt[c][i] = (c < nb && r0 + i < rend) ? A[(j0 + c) * n + r0 + i] : mk<R>(R(0), R(0));
  }
  __syncthreads();
  small_apply<R, NB>(Inv, xs, warp, lane, false);   // y_j = Linv_jj b_j
  if (!ok) return;
  if (tile == 0)
    for (int i = warp; i < nb; i += 8) Xp[int64_t(f.c0 + j0 + i) * nrhs + rhs] = xs[i][lane];
  for (int i = warp; i < RT; i += 8) {
    const int r = r0 + i;
    if (r >= rend) break;
    cx<R> acc = mk<R>(R(0), R(0));
#pragma unroll 8
    for (int c = 0; c < NB; c++) cfma(acc, Lt[c][i], xs[c][lane]);
    cx<R> *y = Yp + int64_t(f.c0 + r) * nrhs + rhs;
    *y = *y - acc;
  }
}

// Y[rows_i] -= sum_c L21[i][c] X[c0 + c], one task = BM update rows of one front.
template <typename R, int BM, int KC>
__global__ void __launch_bounds__(256) k_fwd_l21(const cx<R> *__restrict__ L, int64_t lstride,
                                                 const FrontDev *__restrict__ F,
                                                 const int2 *__restrict__ tasks,
                                                 const int32_t *__restrict__ rows,
                                                 cx<R> *__restrict__ Y, const cx<R> *__restrict__ X,
                                                 int64_t vstride, int nrhs, int nchunk,
                                                 const int *__restrict__ pmap) {
  constexpr int RW = BM / 8;                      // rows per warp
  const int2 t = tasks[blockIdx.x];
  const FrontDev f = F[t.x];
  const int p = pole_of(blockIdx.y / nchunk, pmap), ch = blockIdx.y % nchunk;
  const int64_t n = f.ld;   // column stride
  const int b = f.n - f.k;
  const int i0 = t.y * BM;                        // first update row of the tile
  const cx<R> *A = L + p * lstride + f.lofs + f.k;   // L21 rows start at row k
  const cx<R> *Xp = X + p * vstride;
  cx<R> *Yp = Y + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Ls[KC][BM];
  __shared__ cx<R> Xs[KC][32];
  cx<R> acc[RW];
#pragma unroll
  for (int q = 0; q < RW; q++) acc[q] = mk<R>(R(0), R(0));
  for (int c0 = 0; c0 < f.k; c0 += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * BM; idx += 256) {
      int c = idx / BM, i = idx % BM;
      Ls[c][i] = (c0 + c < f.k && i0 + i < b) ? A[int64_t(c0 + c) * n + i0 + i] : mk<R>(R(0), R(0));
    }
    for (int c = warp; c < KC; c += 8)
      Xs[c][lane] = (ok && c0 + c < f.k) ? Xp[int64_t(f.c0 + c0 + c) * nrhs + rhs] : mk<R>(R(0), R(0));
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < KC; c++) {
      const cx<R> x = Xs[c][lane];
#pragma unroll
      for (int q = 0; q < RW; q++) cfma(acc[q], Ls[c][warp * RW + q], x);
    }
  }
  if (!ok) return;
  const int32_t *urow = rows + f.rows_off;
#pragma unroll
  for (int q = 0; q < RW; q++) {
    const int i = i0 + warp * RW + q;
    if (i < b) atomic_add_cx(Yp + int64_t(urow[i]) * nrhs + rhs, mk<R>(-acc[q].x, -acc[q].y));
  }
}

// w_c = D_c^-1 y_c - sum_i L21[i][c] x[rows_i]; one task = BN pivot columns of one front.
// y_c comes from X (forward result), x[rows_i] from X (final values of the
// ancestors, solved earlier in the top-down sweep); w goes to Y.
template <typename R, int BN, int KC>
__global__ void __launch_bounds__(256) k_bwd_l21(const cx<R> *__restrict__ L, int64_t lstride,
                                                 const FrontDev *__restrict__ F,
                                                 const int2 *__restrict__ tasks,
                                                 const int32_t *__restrict__ rows,
                                                 cx<R> *__restrict__ Y, const cx<R> *__restrict__ X,
                                                 int64_t vstride, int nrhs, int nchunk,
                                                 const int *__restrict__ pmap) {
  constexpr int CW = BN / 8;                      // columns per warp
  const int2 t = tasks[blockIdx.x];
  const FrontDev f = F[t.x];
  const int p = pole_of(blockIdx.y / nchunk, pmap), ch = blockIdx.y % nchunk;
  const int64_t n = f.ld;   // column stride
  const int b = f.n - f.k;
  const int cb = t.y * BN;                        // first pivot column of the tile
  const cx<R> *A = L + p * lstride + f.lofs;
  const cx<R> *Xp = X + p * vstride;
  cx<R> *Yp = Y + p * vstride;
  const int32_t *urow = rows + f.rows_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Ls[KC][BN + 1];
  __shared__ cx<R> Xs[KC][32];
  cx<R> acc[CW];
#pragma unroll
  for (int q = 0; q < CW; q++) acc[q] = mk<R>(R(0), R(0));
  for (int i0 = 0; i0 < b; i0 += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * BN; idx += 256) {
      int i = idx % KC, c = idx / KC;
      Ls[i][c] = (i0 + i < b && cb + c < f.k) ? A[int64_t(cb + c) * n + f.k + i0 + i] : mk<R>(R(0), R(0));
    }
    for (int i = warp; i < KC; i += 8)
      Xs[i][lane] = (ok && i0 + i < b) ? Xp[int64_t(urow[i0 + i]) * nrhs + rhs] : mk<R>(R(0), R(0));
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < KC; i++) {
      const cx<R> x = Xs[i][lane];
#pragma unroll
      for (int q = 0; q < CW; q++) cfma(acc[q], Ls[i][warp * CW + q], x);
    }
  }
  if (!ok) return;
#pragma unroll
  for (int q = 0; q < CW; q++) {
    const int c = cb + warp * CW + q;
    if (c >= f.k) break;
    const cx<R> d = A[int64_t(c) * n + c];
    const int64_t at = int64_t(f.c0 + c) * nrhs + rhs;
    Yp[at] = Xp[at] * crecip(d) - acc[q];
  }
}

template <typename R, int NB, int CT>
__global__ void __launch_bounds__(256) k_bwd_l11(const cx<R> *__restrict__ L, int64_t lstride,
                                                 const cx<R> *__restrict__ Linv, int64_t istride,
                                                 const FrontDev *__restrict__ F,
                                                 const int32_t *__restrict__ lev, int step,
                                                 cx<R> *__restrict__ Y, cx<R> *__restrict__ X,
                                                 int64_t vstride, int nrhs, int nchunk,
                                                 const int *__restrict__ pmap) {
  const FrontDev f = F[lev[blockIdx.y]];
  const int p = pole_of(blockIdx.z / nchunk, pmap), ch = blockIdx.z % nchunk;
  const int j0 = step * NB;
  if (j0 >= f.k) return;
  const int nb = min(NB, f.k - j0);
  const int tile = blockIdx.x;
  const int cfirst = (j0 / kSB) * kSB;           // columns left of the block inside its super-block
  if (tile > 0 && cfirst + tile * CT >= j0) return;
  const int64_t n = f.ld;   // column stride
  const cx<R> *A = L + p * lstride + f.lofs;
  const cx<R> *Iv = Linv + p * istride + (f.inv_off + step) * (NB * NB);
  cx<R> *Yp = Y + p * vstride;
  cx<R> *Xp = X + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Inv[NB][NB];
  __shared__ cx<R> xs[NB][32];
  __shared__ cx<R> Lb[CT][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += 256) Inv[idx / NB][idx % NB] = Iv[idx];
  for (int i = warp; i < NB; i += 8)
    xs[i][lane] = (ok && i < nb) ? Yp[int64_t(f.c0 + j0 + i) * nrhs + rhs] : mk<R>(R(0), R(0));
  const int cbeg = cfirst + tile * CT;
  for (int idx = threadIdx.x; idx < NB * CT; idx += 256) {
    int i = idx % NB, cc = idx / NB;
    Lb[cc][i] = (i < nb && cbeg + cc < j0) ? A[int64_t(cbeg + cc) * n + j0 + i] : mk<R>(R(0), R(0));
  }
  __syncthreads();
  small_apply<R, NB>(Inv, xs, warp, lane, true);   // x_j = Linv_jj^T w_j
  if (!ok) return;
  if (tile == 0)
    for (int i = warp; i < nb; i += 8) Xp[int64_t(f.c0 + j0 + i) * nrhs + rhs] = xs[i][lane];
  for (int cc = warp; cc < CT; cc += 8) {
    const int c = cbeg + cc;
    if (c >= j0) break;
    cx<R> acc = mk<R>(R(0), R(0));
#pragma unroll 8
    for (int i = 0; i < NB; i++) cfma(acc, Lb[cc][i], xs[i][lane]);
    cx<R> *y = Yp + int64_t(f.c0 + c) * nrhs + rhs;
    *y = *y - acc;
  }
}

// Super-block products of the pivot blocks (split over the inner dimension,
// atomically accumulated; every task owns one output tile and one K range).
// Forward: Y[c0 + r] -= sum_{c in [kb, ke)} L[r][c] X[c0 + c] for the rows r
// of super-block J (task = front, row tile of BM, K range).
template <typename R, int BM, int KC>
__global__ void __launch_bounds__(256) k_fwd_sb(const cx<R> *__restrict__ L, int64_t lstride,
                                                const FrontDev *__restrict__ F, const int4 *__restrict__ tasks,
                                                int sb, cx<R> *__restrict__ Y, const cx<R> *__restrict__ X,
                                                int64_t vstride, int nrhs, int nchunk,
                                                 const int *__restrict__ pmap) {
  constexpr int RW = BM / 8;
  const int4 t = tasks[blockIdx.x];
  const FrontDev f = F[t.x];
  const int p = pole_of(blockIdx.y / nchunk, pmap), ch = blockIdx.y % nchunk;
  const int64_t n = f.ld;   // column stride
  const int rlo = sb * kSB, rhi = min(f.k, rlo + kSB);
  const int i0 = rlo + t.y * BM;
  const cx<R> *A = L + p * lstride + f.lofs;
  const cx<R> *Xp = X + p * vstride;
  cx<R> *Yp = Y + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Ls[KC][BM];
  __shared__ cx<R> Xs[KC][32];
  cx<R> acc[RW];
#pragma unroll
  for (int q = 0; q < RW; q++) acc[q] = mk<R>(R(0), R(0));
  for (int c0 = t.z; c0 < t.w; c0 += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * BM; idx += 256) {
      int c = idx / BM, i = idx % BM;
      Ls[c][i] = (c0 + c < t.w && i0 + i < rhi) ? A[int64_t(c0 + c) * n + i0 + i] : mk<R>(R(0), R(0));
    }
    for (int c = warp; c < KC; c += 8)
      Xs[c][lane] = (ok && c0 + c < t.w) ? Xp[int64_t(f.c0 + c0 + c) * nrhs + rhs] : mk<R>(R(0), R(0));
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < KC; c++) {
      const cx<R> x = Xs[c][lane];
#pragma unroll
      for (int q = 0; q < RW; q++) cfma(acc[q], Ls[c][warp * RW + q], x);
    }
  }
  if (!ok) return;
#pragma unroll
  for (int q = 0; q < RW; q++) {
    const int i = i0 + warp * RW + q;
    if (i < rhi) atomic_add_cx(Yp + int64_t(f.c0 + i) * nrhs + rhs, mk<R>(-acc[q].x, -acc[q].y));
  }
}

// Backward: W[c0 + c] -= sum_{r in [kb, ke)} L[r][c] X[c0 + r] for the
// columns c of super-block J (task = front, column tile of BN, K range of rows).
template <typename R, int BN, int KC>
__global__ void __launch_bounds__(256) k_bwd_sb(const cx<R> *__restrict__ L, int64_t lstride,
                                                const FrontDev *__restrict__ F, const int4 *__restrict__ tasks,
                                                int sb, cx<R> *__restrict__ Y, const cx<R> *__restrict__ X,
                                                int64_t vstride, int nrhs, int nchunk,
                                                 const int *__restrict__ pmap) {
  constexpr int CW = BN / 8;
  const int4 t = tasks[blockIdx.x];
  const FrontDev f = F[t.x];
  const int p = pole_of(blockIdx.y / nchunk, pmap), ch = blockIdx.y % nchunk;
  const int64_t n = f.ld;   // column stride
  const int clo = sb * kSB, chi = min(f.k, clo + kSB);
  const int cb = clo + t.y * BN;
  const cx<R> *A = L + p * lstride + f.lofs;
  const cx<R> *Xp = X + p * vstride;
  cx<R> *Yp = Y + p * vstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < nrhs;
  __shared__ cx<R> Ls[KC][BN + 1];
  __shared__ cx<R> Xs[KC][32];
  cx<R> acc[CW];
#pragma unroll
  for (int q = 0; q < CW; q++) acc[q] = mk<R>(R(0), R(0));
  for (int i0 = t.z; i0 < t.w; i0 += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * BN; idx += 256) {
      int i = idx % KC, c = idx / KC;
      Ls[i][c] = (i0 + i < t.w && cb + c < chi) ? A[int64_t(cb + c) * n + i0 + i] : mk<R>(R(0), R(0));
    }
    for (int i = warp; i < KC; i += 8)
      Xs[i][lane] = (ok && i0 + i < t.w) ? Xp[int64_t(f.c0 + i0 + i) * nrhs + rhs] : mk<R>(R(0), R(0));
    __syncthreads();
#pragma unroll 4
    for (int i = 0; i < KC; i++) {
      const cx<R> x = Xs[i][lane];
#pragma unroll
      for (int q = 0; q < CW; q++) cfma(acc[q], Ls[i][warp * CW + q], x);
    }
  }
  if (!ok) return;
#pragma unroll
  for (int q = 0; q < CW; q++) {
    const int c = cb + warp * CW + q;
    if (c >= chi) break;
    atomic_add_cx(Yp + int64_t(f.c0 + c) * nrhs + rhs, mk<R>(-acc[q].x, -acc[q].y));
  }
}

template <typename R>
void SolvePlan<R>::forward_level(const LevelDev &lv, cudaStream_t s) {
  if (g_prof) g_prof->cur_level = lv.h;
  if constexpr (std::is_same<R, float>::value) {
    // explicit pivot-block inverses: two products per level
    if (g_prof) g_prof->begin(KC_FWD, s);
    launch_prod(PM_TRI_F, *this, lv, s);
    if (g_prof) g_prof->end(KC_FWD, s);
    if (g_prof) g_prof->begin(KC_FWD21, s);
    launch_prod(PM_FWD21, *this, lv, s);
    if (g_prof) g_prof->end(KC_FWD21, s);
  } else {
    const int nchunk = (nrhs + 31) / 32;
    const int per_sb = kSB / kNB;
    for (int step = 0; step < (int)lv.steps.size(); step++) {
      const int sb = step / per_sb;
      if (step % per_sb == 0 && sb > 0 && lv.sb[sb].n_fwd > 0) {
        dim3 g(lv.sb[sb].n_fwd, np * nchunk);
        if (g_prof) g_prof->begin(KC_FWD_SB, s);
        tem::count_launch();
        k_fwd_sb<R, SolveTile<R>::BM, SolveTile<R>::KC><<<g, 256, 0, s>>>(L, lstride, F, lv.sb[sb].fwd, sb, Y, X,
                                                                           vstride, nrhs, nchunk, pmap);
        if (g_prof) g_prof->end(KC_FWD_SB, s);
      }
      const StepDims &sd = lv.steps[step];
      dim3 g(sd.fwd_tiles, sd.nfronts, np * nchunk);
      if (g_prof) g_prof->begin(KC_FWD, s);
      tem::count_launch();
      k_fwd_l11<R, kNB, SolveTile<R>::RT><<<g, 256, 0, s>>>(L, lstride, Linv, istride, F, lv.fronts, step, Y, X,
                                                             vstride, nrhs, nchunk, pmap);
      if (g_prof) g_prof->end(KC_FWD, s);
    }
    if (lv.n_f21 > 0) {
      dim3 g(lv.n_f21, np * nchunk);
      if (g_prof) g_prof->begin(KC_FWD21, s);
      tem::count_launch();
      k_fwd_l21<R, SolveTile<R>::BM, SolveTile<R>::KC><<<g, 256, 0, s>>>(L, lstride, F, lv.f21_tasks, rows, Y,
                                                                          X, vstride, nrhs, nchunk, pmap);
      if (g_prof) g_prof->end(KC_FWD21, s);
    }
  }
}

template <typename R>
void SolvePlan<R>::backward_level(const LevelDev &lv, cudaStream_t s) {
  if (g_prof) g_prof->cur_level = lv.h;
  if constexpr (std::is_same<R, float>::value) {
    if (g_prof) g_prof->begin(KC_BWD_UPD, s);
    launch_prod(PM_BWD21, *this, lv, s);
    if (g_prof) g_prof->end(KC_BWD_UPD, s);
    if (g_prof) g_prof->begin(KC_BWD, s);
    launch_prod(PM_TRI_B, *this, lv, s);
    if (g_prof) g_prof->end(KC_BWD, s);
  } else {
    const int nchunk = (nrhs + 31) / 32;
    const int per_sb = kSB / kNB;
    if (lv.n_b21 > 0) {
      dim3 g(lv.n_b21, np * nchunk);
      if (g_prof) g_prof->begin(KC_BWD_UPD, s);
      tem::count_launch();
      k_bwd_l21<R, SolveTile<R>::BN, SolveTile<R>::KC><<<g, 256, 0, s>>>(L, lstride, F, lv.b21_tasks, rows, Y,
                                                                          X, vstride, nrhs, nchunk, pmap);
      if (g_prof) g_prof->end(KC_BWD_UPD, s);
    }
    for (int step = (int)lv.steps.size() - 1; step >= 0; step--) {
      const int sb = step / per_sb;
      if ((step == (int)lv.steps.size() - 1 || step % per_sb == per_sb - 1) && lv.sb[sb].n_bwd > 0) {
        dim3 g(lv.sb[sb].n_bwd, np * nchunk);
        if (g_prof) g_prof->begin(KC_BWD_SB, s);
        tem::count_launch();
        k_bwd_sb<R, SolveTile<R>::BN, SolveTile<R>::KC><<<g, 256, 0, s>>>(L, lstride, F, lv.sb[sb].bwd, sb, Y, X,
                                                                           vstride, nrhs, nchunk, pmap);
        if (g_prof) g_prof->end(KC_BWD_SB, s);
      }
      const StepDims &sd = lv.steps[step];
      dim3 g(sd.bwd_tiles, sd.nfronts, np * nchunk);
      if (g_prof) g_prof->begin(KC_BWD, s);
      tem::count_launch();
      k_bwd_l11<R, kNB, SolveTile<R>::CT><<<g, 256, 0, s>>>(L, lstride, Linv, istride, F, lv.fronts, step, Y, X,
                                                             vstride, nrhs, nchunk, pmap);
      if (g_prof) g_prof->end(KC_BWD, s);
    }
  }
}

template struct SolvePlan<float>;
template struct SolvePlan<double>;

}  // namespace tem
