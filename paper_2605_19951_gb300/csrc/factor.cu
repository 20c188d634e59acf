// Numeric multifrontal LDL^T of the shifted matrices A_i = K - xi_i M(sigma)
// (Algorithm 1: form A_i, factor), all poles batched in the grid's z dimension.
//
// Storage (per pole, pole stride lstride / ustride elements):
//   factor store: front f owns an n x k column-major block at lofs (column
//     stride ld = n rounded up to even, so columns start on 16-byte boundaries):
//     rows 0..k-1 = L11 (unit lower, D on the diagonal), rows k..n-1 = L21.
//   update arena: front f owns a b x b column-major block at uofs (ld b)
//     holding its Schur complement (lower triangle) until the parent has
//     absorbed it (extend-add).
// Per level of the assembly tree: zero, scatter the original entries,
// extend-add the children, then a blocked right-looking partial LDL^T:
// k_panel factors the NB x NB diagonal block and the panel rows below it,
// k_update applies the rank-NB update to the trailing lower triangle.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace tem {

__global__ void k_sigma(const double *__restrict__ logs, const int32_t *__restrict__ ptet,
                        int64_t P, double *__restrict__ sigma) {
  int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p < P) sigma[ptet[p]] = exp(logs[p]);
}

// Conductivity-weighted values: M_z = sum over element contributions
// sigma_t E_t[a][b], with `per` table entries per tetrahedron (36: the edge
// mass matrices M1_t; 16: the P1 stiffness of the nodal gradient space).
template <typename T>
__global__ void k_mvals(const int64_t *__restrict__ mc_ptr, const uint32_t *__restrict__ mc_idx,
                        const double *__restrict__ sigma, const double *__restrict__ me1, uint32_t per,
                        int64_t nnz, T *__restrict__ mval) {
  for (int64_t z = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; z < nnz;
       z += int64_t(gridDim.x) * blockDim.x) {
    double s = 0;
    for (int64_t q = mc_ptr[z]; q < mc_ptr[z + 1]; q++) {
      uint32_t idx = mc_idx[q];
      s += sigma[idx / per] * me1[idx];
    }
    mval[z] = T(s);
  }
}

// Mass values of the factored matrix of pole p in FP32 mode: the conductivity
// is floored at tau / (|xi_p| mu0 h_t^2) (tetfloor_t = 1 / (mu0 h_t^2)).
// Only the factor (the preconditioner of the refinement) sees the floor; the
// FP64 residual uses the true M.
__global__ void k_mvals_floor(const int64_t *__restrict__ mc_ptr, const uint32_t *__restrict__ mc_idx,
                              const double *__restrict__ sigma, const double *__restrict__ tetfloor,
                              const double *__restrict__ me1, const double2 *__restrict__ xi, double tau,
                              int64_t nnz, double *__restrict__ mval) {
  const int p = blockIdx.y;
  const double ax = tau / hypot(xi[p].x, xi[p].y);
  double *out = mval + p * nnz;
  for (int64_t z = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; z < nnz;
       z += int64_t(gridDim.x) * blockDim.x) {
    double s = 0;
    for (int64_t q = mc_ptr[z]; q < mc_ptr[z + 1]; q++) {
      uint32_t idx = mc_idx[q];
      uint32_t t = idx / 36;
      s += fmax(sigma[t], tetfloor[t] * ax) * me1[idx];
    }
    out[z] = s;
  }
}

template <typename R>
__global__ void k_assemble_orig(cx<R> *__restrict__ L, int64_t lstride, const double *__restrict__ kv,
                                const double *__restrict__ mv, int64_t mstride,
                                const int64_t *__restrict__ onz, const int64_t *__restrict__ odst,
                                int64_t cnt, const double2 *__restrict__ xi) {
  const int p = blockIdx.y;
  const double2 s = xi[p];
  cx<R> *Lp = L + p * lstride;
  mv += p * mstride;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x) {
    int64_t z = onz[e];
    double k = kv[z], m = mv[z];
    Lp[odst[e]] = mk<R>(R(k - s.x * m), R(-s.y * m));
  }
}

template <typename R>
__global__ void k_zero_u(cx<R> *__restrict__ U, int64_t ustride, const FrontDev *__restrict__ F,
                         const int32_t *__restrict__ lev) {
  const FrontDev f = F[lev[blockIdx.y]];
  const int64_t b = f.n - f.k;
  if (b == 0) return;
  cx<R> *u = U + blockIdx.z * ustride + f.uofs;
  const int64_t cnt = b * b;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x)
    u[e] = mk<R>(R(0), R(0));
}

// One task = one column j of a child's update block, added into the parent.
template <typename R>
__global__ void k_extend_add(cx<R> *__restrict__ L, int64_t lstride, cx<R> *__restrict__ U,
                             int64_t ustride, const FrontDev *__restrict__ F,
                             const int32_t *__restrict__ rel, const int32_t *__restrict__ ea_child,
                             const int32_t *__restrict__ ea_col) {
  const int64_t task = blockIdx.x;
  const int p = blockIdx.y;
  const FrontDev C = F[ea_child[task]];
  const FrontDev Pf = F[C.parent];
  const int32_t j = ea_col[task];
  const int32_t bc = C.n - C.k, bp = Pf.n - Pf.k;
  const cx<R> *uc = U + p * ustride + C.uofs + int64_t(j) * bc;
  const int32_t *rl = rel + C.rel_off;
  const int32_t rj = rl[j];
  // each parent entry receives at most one child entry per launch (one child slot), so the
  // atomic adds equal load, add, store without a round trip per entry; the relative map is
  // only read here
  if (rj < Pf.k) {
    cx<R> *dst = L + p * lstride + Pf.lofs + int64_t(rj) * Pf.ld;
    for (int32_t i = j + threadIdx.x; i < bc; i += blockDim.x) atomic_add_cx(dst + __ldg(rl + i), uc[i]);
  } else {
    cx<R> *dst = U + p * ustride + Pf.uofs + int64_t(rj - Pf.k) * bp;
    // rows below a column >= k lie in the update block
    for (int32_t i = j + threadIdx.x; i < bc; i += blockDim.x) atomic_add_cx(dst + (__ldg(rl + i) - Pf.k), uc[i]);
  }
}

template <typename R>
__device__ __forceinline__ R pivot_floor();
template <>
__device__ __forceinline__ float pivot_floor<float>() { return 1e-36f; }
template <>
__device__ __forceinline__ double pivot_floor<double>() { return 1e-300; }

// Panel step: factor the diagonal block of step `step` (redundantly in every
// CTA, from the untouched original) and compute L for RT rows below it.
// The factored diagonal block goes to dscr (copied into place by k_update,
// so no CTA here reads a block another CTA has already overwritten).
template <typename R, int NB, int RT>
__global__ void __launch_bounds__(RT) k_panel(cx<R> *__restrict__ L, int64_t lstride,
                                              const FrontDev *__restrict__ F,
                                              const int32_t *__restrict__ lev, int step,
                                              cx<R> *__restrict__ dscr, cx<R> *__restrict__ linv,
                                              int64_t istride, DevStatus *st) {
  const int fi = blockIdx.y;
  const FrontDev f = F[lev[fi]];
  const int p = blockIdx.z;
  const int j0 = step * NB;
  if (j0 >= f.k) return;
  const int nb = min(NB, f.k - j0);
  const int rbeg = j0 + nb;
  const int tile = blockIdx.x;
  if (tile > 0 && rbeg + tile * RT >= f.n) return;
  cx<R> *A = L + p * lstride + f.lofs;
  const int64_t n = f.n, ld = f.ld;
  __shared__ cx<R> Dg[NB][NB + 1];
  __shared__ cx<R> w[NB];
  __shared__ cx<R> inv[NB];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += RT) {
    int r = idx % NB, c = idx / NB;
    if (r < nb && c < nb && r >= c) Dg[r][c] = A[(j0 + c) * ld + j0 + r];
  }
  __syncthreads();
  for (int c = 0; c < nb; c++) {
    if (tid == 0) {
      cx<R> d = Dg[c][c];
      R a = cabs1(d);
      if (!(a > pivot_floor<R>()) || !isfinite(a)) {
        if (tile == 0 && atomicExch(&st->pivot_fail, 1) == 0) st->pivot_front = lev[fi];
        d = mk<R>(R(1), R(0));
      }
      if (tile == 0) {
        double ad = hypot(double(d.x), double(d.y));
        atomicMin(&st->min_pivot_bits, (unsigned long long)__double_as_longlong(ad));
      }
      inv[c] = crecip(d);
    }
    __syncthreads();
    const cx<R> ic = inv[c];
    for (int r = c + 1 + tid; r < nb; r += RT) {
      cx<R> wv = Dg[r][c];
      w[r] = wv;
      Dg[r][c] = wv * ic;
    }
    __syncthreads();
    const int m = nb - c - 1;
    for (int idx = tid; idx < m * m; idx += RT) {
      int r = c + 1 + idx % m, s = c + 1 + idx / m;
      if (s <= r) cfms(Dg[r][s], w[r], Dg[s][c]);
    }
    __syncthreads();
  }
  if (tile == 0) {
    cx<R> *ds = dscr + (int64_t(fi) * gridDim.z + p) * NB * NB;
    for (int idx = tid; idx < NB * NB; idx += RT) {
      int r = idx % NB, c = idx / NB;
      if (r < nb && c < nb && r >= c) ds[c * NB + r] = Dg[r][c];
    }
    // inverse of the unit lower block for the solves: column c by forward
    // substitution (thread c), zero padded to NB x NB, stored column-major
    __shared__ cx<R> Iv[NB][NB + 1];
    if (tid < NB) {
      const int c = tid;
      for (int r = 0; r < NB; r++) Iv[c][r] = mk<R>(R(0), R(0));
      if (c < nb) {
        Iv[c][c] = mk<R>(R(1), R(0));
        for (int r = c + 1; r < nb; r++) {
          cx<R> acc = mk<R>(R(0), R(0));
          for (int q = c; q < r; q++) cfma(acc, Dg[r][q], Iv[c][q]);
          Iv[c][r] = mk<R>(-acc.x, -acc.y);
        }
      }
    }
    __syncthreads();
    cx<R> *iv = linv + p * istride + (f.inv_off + step) * (NB * NB);
    for (int idx = tid; idx < NB * NB; idx += RT) iv[idx] = Iv[idx / NB][idx % NB];
  }
  const int64_t r = rbeg + int64_t(tile) * RT + tid;
  if (r < n) {
    cx<R> wr[NB];
#pragma unroll
    for (int c = 0; c < NB; c++)
      if (c < nb) wr[c] = A[(j0 + c) * ld + r];
#pragma unroll
    for (int c = 0; c < NB; c++) {
      if (c < nb) {
#pragma unroll
        for (int c2 = 0; c2 < c; c2++) cfms(wr[c], wr[c2], Dg[c][c2]);
      }
    }
#pragma unroll
    for (int c = 0; c < NB; c++)
      if (c < nb) A[(j0 + c) * ld + r] = wr[c] * inv[c];
  }
}

// Trailing update of step `step`: F[r][s] -= sum_c L[r][c] D_c L[s][c] over
// the panel columns, for r >= s in the trailing part; tiles of TM x TM in the
// lower triangle, 16 x 16 threads with (TM/16)^2 outputs each.  CTA 0 of
// each front first copies the factored diagonal block into place.  With
// blk > 0 only the columns of the step's block of blk pivots are updated (the
// rest of the trailing part gets the block's rank-blk update on the tensor
// cores once the block is factored).
template <typename R, int NB, int TM>
__global__ void __launch_bounds__(256) k_update(cx<R> *__restrict__ L, int64_t lstride,
                                                cx<R> *__restrict__ U, int64_t ustride,
                                                const FrontDev *__restrict__ F,
                                                const int32_t *__restrict__ lev, int step,
                                                const cx<R> *__restrict__ dscr, int blk) {
  constexpr int PT = TM / 16;
  const int fi = blockIdx.y;
  const FrontDev f = F[lev[fi]];
  const int p = blockIdx.z;
  const int j0 = step * NB;
  if (j0 >= f.k) return;
  const int nb = min(NB, f.k - j0);
  const int64_t n = f.n, ld = f.ld;
  cx<R> *A = L + p * lstride + f.lofs;
  const int tid = threadIdx.x;
  if (blockIdx.x == 0) {
    const cx<R> *ds = dscr + (int64_t(fi) * gridDim.z + p) * NB * NB;
    for (int idx = tid; idx < NB * NB; idx += 256) {
      int r = idx % NB, c = idx / NB;
      if (r < nb && c < nb && r >= c) A[(j0 + c) * ld + j0 + r] = ds[c * NB + r];
    }
  }
  const int64_t pbeg = j0 + nb;
  const int64_t tn = n - pbeg;
  if (tn <= 0) return;
  const int64_t T = (tn + TM - 1) / TM;
  const int64_t q = blockIdx.x;
  const int64_t s_end = blk > 0 ? min(int64_t(f.k), (int64_t(j0) / blk + 1) * blk) : n;
  int64_t ti, tj;
  if (blk > 0) {
    // tiles (ti >= tj) of the first TJ tile columns, column by column
    const int64_t TJ = s_end > pbeg ? (s_end - pbeg + TM - 1) / TM : 0;
    int64_t qq = q;
    tj = 0;
    while (tj < TJ && qq >= T - tj) {
      qq -= T - tj;
      tj++;
    }
    if (tj >= TJ) return;
    ti = tj + qq;
  } else {
    if (q >= T * (T + 1) / 2) return;
    ti = int64_t((sqrt(8.0 * double(q) + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= q) ti++;
    while (ti * (ti + 1) / 2 > q) ti--;
    tj = q - ti * (ti + 1) / 2;
  }
  const int64_t r0 = pbeg + ti * TM, s0 = pbeg + tj * TM;
  __shared__ cx<R> As[NB][TM];
  __shared__ cx<R> Bs[NB][TM];
  __shared__ cx<R> Dd[NB];
  if (tid < nb) {
    // the pivot: diagonal of the factored block (scratch copy, always valid)
    const cx<R> *ds = dscr + (int64_t(fi) * gridDim.z + p) * NB * NB;
    Dd[tid] = ds[tid * NB + tid];
  }
  __syncthreads();
  for (int idx = tid; idx < NB * TM; idx += 256) {
    int c = idx / TM, i = idx % TM;
    cx<R> a = mk<R>(R(0), R(0)), b = mk<R>(R(0), R(0));
    if (c < nb) {
      int64_t r = r0 + i, s = s0 + i;
      if (r < n) a = A[(j0 + c) * ld + r];
      if (s < n) b = A[(j0 + c) * ld + s] * Dd[c];
    }
    As[c][i] = a;
    Bs[c][i] = b;
  }
  __syncthreads();
  const int tx = tid % 16, ty = tid / 16;
  cx<R> acc[PT][PT];
#pragma unroll
  for (int i = 0; i < PT; i++)
#pragma unroll
    for (int j = 0; j < PT; j++) acc[i][j] = mk<R>(R(0), R(0));
  for (int c = 0; c < nb; c++) {
    cx<R> a[PT], b[PT];
#pragma unroll
    for (int i = 0; i < PT; i++) a[i] = As[c][tx + 16 * i];
#pragma unroll
    for (int j = 0; j < PT; j++) b[j] = Bs[c][ty + 16 * j];
#pragma unroll
    for (int i = 0; i < PT; i++)
#pragma unroll
      for (int j = 0; j < PT; j++) cfma(acc[i][j], a[i], b[j]);
  }
  const int64_t k = f.k, b = n - k;
#pragma unroll
  for (int j = 0; j < PT; j++) {
    const int64_t s = s0 + ty + 16 * j;
    if (s >= s_end) continue;
    // column s lives in the factor block (s < k) or in the update block
    cx<R> *col = (s < k) ? (A + s * ld) : (U + p * ustride + f.uofs + (s - k) * b);
    const int64_t roff = (s < k) ? 0 : k;
#pragma unroll
    for (int i = 0; i < PT; i++) {
      const int64_t r = r0 + tx + 16 * i;
      // one tile per entry in a launch: an atomic add of -acc equals load, subtract, store
      // and leaves the read to the L2 instead of a round trip per entry
      if (r < n && r >= s) atomic_add_cx(col + (r - roff), mk<R>(-acc[i][j].x, -acc[i][j].y));
    }
  }
}

// Row-major copy of one kKB block of pivot columns for the tensor-core
// trailing update: for the front of task (f, prow, t0, kb), rows t0..n-1 of
// columns j0 = t0 - kb .. t0 - 1 go to rows prow + r of Pc (row pitch kKB,
// columns kb..kKB-1 zero).  A CTA transposes 32 rows through shared memory.
__global__ void __launch_bounds__(256) k_panel_copy(const c64 *__restrict__ L, int64_t lstride,
                                                    const FrontDev *__restrict__ F, const int4 *__restrict__ tasks,
                                                    c64 *__restrict__ Pc, int64_t pstride) {
  const int4 tk = tasks[blockIdx.y];
  const FrontDev f = F[tk.x];
  const int p = blockIdx.z;
  const int64_t t0 = tk.z, kb = tk.w, j0 = t0 - kb;
  const int64_t r0 = t0 + int64_t(blockIdx.x) * 32;
  if (r0 >= f.n) return;
  __shared__ c64 tile[kKB][33];
  const c64 *A = L + p * lstride + f.lofs;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  for (int c = wq; c < kKB; c += 8) {
    const int64_t r = r0 + lane;
    tile[c][lane] = (c < kb && r < f.n) ? A[(j0 + c) * f.ld + r] : mk<float>(0.f, 0.f);
  }
  __syncthreads();
  c64 *out = Pc + p * pstride + (int64_t(tk.y) + r0) * kKB;
  for (int idx = tid; idx < 32 * kKB; idx += 256) {
    const int rr = idx / kKB, c = idx % kKB;
    if (r0 + rr < f.n) out[int64_t(rr) * kKB + c] = tile[c][rr];
  }
}

// ---------------------------------------------------------------------------
// launch wrappers

void launch_sigma(const double *logs, const int32_t *ptet, int64_t P, double *sigma, cudaStream_t s) {
  if (P == 0) return;
  tem::count_launch();
  k_sigma<<<div_up(P, 256), 256, 0, s>>>(logs, ptet, P, sigma);
}

void launch_mvals(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                  const double *me1, int per, int64_t nnz, double *mval, cudaStream_t s) {
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(div_up(nnz, 256), 152 * 16));
  tem::count_launch();
  k_mvals<double><<<blocks, 256, 0, s>>>(mc_ptr, mc_idx, sigma, me1, uint32_t(per), nnz, mval);
}

void launch_mvals(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                  const double *me1, int per, int64_t nnz, float *mval, cudaStream_t s) {
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(div_up(nnz, 256), 152 * 16));
  tem::count_launch();
  k_mvals<float><<<blocks, 256, 0, s>>>(mc_ptr, mc_idx, sigma, me1, uint32_t(per), nnz, mval);
}

void launch_mvals_floor(const int64_t *mc_ptr, const uint32_t *mc_idx, const double *sigma,
                        const double *tetfloor, const double *me1, const double2 *xi, double tau, int m,
                        int64_t nnz, double *mval, cudaStream_t s) {
  dim3 g((unsigned)std::min<int64_t>(div_up(nnz, 256), 1024), m);
  tem::count_launch();
  k_mvals_floor<<<g, 256, 0, s>>>(mc_ptr, mc_idx, sigma, tetfloor, me1, xi, tau, nnz, mval);
}

template <typename R>
void FactorPlan<R>::level(int h, const LevelDev &lv, cudaStream_t s) {
  const int m = this->m;
  if (g_prof) g_prof->cur_level = lv.h;
  // 1. zero this level's factor blocks and update blocks
  if (lv.lend > lv.lbeg)
    for (int p = 0; p < m; p++)
      cudaMemsetAsync(L + p * lstride + lv.lbeg, 0, (lv.lend - lv.lbeg) * sizeof(cx<R>), s);
  if (lv.nf > 0) {
    dim3 g(64, lv.nf, m);
    tem::count_launch();
    k_zero_u<R><<<g, 256, 0, s>>>(U, ustride, F, lv.fronts);
  }
  // 2. original entries of A_i
  const int64_t cnt = lv.oend - lv.obeg;
  if (cnt > 0) {
    dim3 g((unsigned)std::min<int64_t>(div_up(cnt, 256), 4096), m);
    tem::count_launch();
    k_assemble_orig<R><<<g, 256, 0, s>>>(L, lstride, kval, mval, mstride, orig_nz + lv.obeg,
                                         orig_dst + lv.obeg, cnt, xi);
  }
  // 3. extend-add, one child slot at a time (no two tasks of a launch hit
  //    the same parent entry)
  for (int sl = 0; sl < 4; sl++) {
    const int64_t nt = lv.ea_end[sl] - lv.ea_beg[sl];
    if (nt <= 0) continue;
    dim3 g((unsigned)nt, m);
    if (g_prof) g_prof->begin(KC_EXTEND_ADD, s);
    tem::count_launch();
    k_extend_add<R><<<g, 128, 0, s>>>(L, lstride, U, ustride, F, rel, ea_child + lv.ea_beg[sl],
                                       ea_col + lv.ea_beg[sl]);
    if (g_prof) g_prof->end(KC_EXTEND_ADD, s);
  }
  // 4. blocked partial LDL^T.  With tc_update (FP32) the pivots go in blocks of
  //    kKB: each 32-wide panel step updates only the rest of its block, and
  //    after the block's last step the rest of the trailing part gets the
  //    block's rank-kKB update on the tensor cores (from a row-major copy of
  //    the block's rows below it).
  constexpr int kPer = kKB / kNB;
  const bool tc = tc_update && std::is_same<R, float>::value && !lv.upd.empty();
  const int nsteps = (int)lv.steps.size();
  for (int step = 0; step < nsteps; step++) {
    const StepDims &sd = lv.steps[step];
    dim3 gp(sd.panel_tiles, sd.nfronts, m);
    if (g_prof) g_prof->begin(KC_PANEL, s);
    tem::count_launch();
    k_panel<R, kNB, kPanelRT><<<gp, kPanelRT, 0, s>>>(L, lstride, F, lv.fronts, step, dscr, linv, istride,
                                                      status);
    if (g_prof) g_prof->end(KC_PANEL, s);
    dim3 gu(tc ? sd.update_tiles_blk : sd.update_tiles, sd.nfronts, m);
    if (g_prof) g_prof->begin(KC_UPDATE, s);
    tem::count_launch();
    k_update<R, kNB, UpdateTile<R>::TM><<<gu, 256, 0, s>>>(L, lstride, U, ustride, F, lv.fronts, step,
                                                            dscr, tc ? kKB : 0);
    if (g_prof) g_prof->end(KC_UPDATE, s);
    if constexpr (std::is_same<R, float>::value) {
      if (tc && ((step + 1) % kPer == 0 || step + 1 == nsteps)) {
        const UpdBlock &ub = lv.upd[step / kPer];
        if (ub.ncopy > 0) {
          dim3 gc(ub.copy_tiles, ub.ncopy, m);
          if (g_prof) g_prof->begin(KC_UPDATE_TC, s);
          tem::count_launch();
          k_panel_copy<<<gc, 256, 0, s>>>(L, lstride, F, ub.copies, Pc, pstride);
          launch_tc_update(*this, ub, s);
          if (g_prof) g_prof->end(KC_UPDATE_TC, s);
        }
      }
    }
  }
}

template struct FactorPlan<float>;
template struct FactorPlan<double>;

}  // namespace tem
