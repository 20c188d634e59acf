// Vector kernels around the solves: right-hand-side staging and iterative
// refinement (FP64 residual r = b - (K - xi M) x), residue sums through the
// observation operator (Section 2.3, Section 3), the element-local mass-derivative
// products of J v and J^T w (Section 3.1), sparse matrix-vector products of the
// regulariser root, and the device-scalar LSQR steps (Section 3.3).
#include <algorithm>

#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace tem {

// ---- right-hand sides and refinement ---------------------------------------

// Column maxima of max(|re|, |im|) per (pole, rhs): 8 row groups x 32 RHS
// lanes per block, shared-memory reduction over the groups, one atomic per
// block and column.
__global__ void k_colmax(const c128 *__restrict__ b, int64_t bstride, double *colmax, int64_t N,
                         int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const c128 *bp = b + p * bstride;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  __shared__ double red[8][32];
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int rhs = c0 + lane;
    double mx = 0.0;
    if (rhs < nrhs)
      for (int64_t r = blockIdx.x * int64_t(8) + grp; r < N; r += int64_t(gridDim.x) * 8) {
        const c128 v = bp[r * nrhs + rhs];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
      }
    red[grp][lane] = mx;
    __syncthreads();
    if (grp == 0 && rhs < nrhs) {
      for (int g = 1; g < 8; g++) mx = fmax(mx, red[g][lane]);
      if (mx > 0)
        atomicMax((unsigned long long *)&colmax[p * nrhs + rhs], (unsigned long long)__double_as_longlong(mx));
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void k_rhs_to_work(const c128 *__restrict__ b, int64_t bstride, cx<R> *__restrict__ Y,
                              const double *__restrict__ colmax, int64_t N, int nrhs,
                              const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const c128 *bp = b + p * bstride;
  cx<R> *yp = Y + p * N * nrhs;
  const int64_t cnt = N * nrhs;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x) {
    c128 v = bp[e];
    double s = 1.0;
    if (colmax) {
      double c = colmax[p * nrhs + e % nrhs];
      s = c > 0 ? 1.0 / c : 1.0;
    }
    yp[e] = mk<R>(R(v.x * s), R(v.y * s));
  }
}

__global__ void k_zero_colmax(double *colmax, int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.x, pmap);
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) colmax[p * nrhs + r] = 0.0;
}

template <typename R>
void launch_rhs_to_work(const c128 *b, int64_t bstride, cx<R> *Y, double *colmax, int np, const int *pmap,
                        int64_t N, int nrhs, bool scale, cudaStream_t s) {
  dim3 g((unsigned)std::min<int64_t>(div_up(N * nrhs, 256), 2048), np);
  if (scale) {
    tem::count_launch();
    k_zero_colmax<<<np, 64, 0, s>>>(colmax, nrhs, pmap);
    dim3 gc((unsigned)std::min<int64_t>(div_up(N, 8), 512), np);
    tem::count_launch();
    k_colmax<<<gc, 256, 0, s>>>(b, bstride, colmax, N, nrhs, pmap);
  }
  tem::count_launch();
  k_rhs_to_work<R><<<g, 256, 0, s>>>(b, bstride, Y, scale ? colmax : nullptr, N, nrhs, pmap);
}

template <typename R>
__global__ void k_accumulate(const cx<R> *__restrict__ X, const double *__restrict__ colmax,
                             c128 *__restrict__ x, int64_t N, int nrhs, int add,
                             const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const cx<R> *Xp = X + p * N * nrhs;
  c128 *xp = x + p * N * nrhs;
  const int64_t cnt = N * nrhs;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x) {
    double s = 1.0;
    if (colmax) {
      double c = colmax[p * nrhs + e % nrhs];
      s = c > 0 ? c : 1.0;
    }
    cx<R> v = Xp[e];
    c128 o = add ? xp[e] : mk<double>(0.0, 0.0);
    xp[e] = mk<double>(o.x + s * double(v.x), o.y + s * double(v.y));
  }
}

template <typename R>
void launch_accumulate(const cx<R> *X, const double *colmax, c128 *x, int np, const int *pmap, int64_t N,
                       int nrhs, bool add, cudaStream_t s) {
  dim3 g((unsigned)std::min<int64_t>(div_up(N * nrhs, 256), 2048), np);
  tem::count_launch();
  k_accumulate<R><<<g, 256, 0, s>>>(X, colmax, x, N, nrhs, add ? 1 : 0, pmap);
}

// Per pole: max over masked rows and all RHS of |colmax * X| (the correction
// just added) and of |x| (the refined solution), as double bits.
template <typename R>
__global__ void k_progress(const cx<R> *__restrict__ X, const double *__restrict__ colmax,
                           const c128 *__restrict__ x, const uint8_t *__restrict__ mask, double *num,
                           double *den, int64_t N, int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const cx<R> *Xp = X + p * N * nrhs;
  const c128 *xp = x + p * N * nrhs;
  double a = 0.0, b = 0.0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < N * nrhs;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (!mask[e / nrhs]) continue;
    const double c = colmax ? colmax[p * nrhs + e % nrhs] : 1.0;
    const cx<R> d = Xp[e];
    const c128 v = xp[e];
    a = fmax(a, c * fmax(fabs(double(d.x)), fabs(double(d.y))));
    b = fmax(b, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (a > 0) atomicMax((unsigned long long *)&num[p], (unsigned long long)__double_as_longlong(a));
    if (b > 0) atomicMax((unsigned long long *)&den[p], (unsigned long long)__double_as_longlong(b));
  }
}

template <typename R>
void launch_progress(const cx<R> *X, const double *colmax, const c128 *x, const uint8_t *mask, double *num,
                     double *den, int np, const int *pmap, int64_t N, int nrhs, cudaStream_t s) {
  dim3 g((unsigned)std::min<int64_t>(div_up(N * nrhs, 256), 1024), np);
  tem::count_launch();
  k_progress<R><<<g, 256, 0, s>>>(X, colmax, x, mask, num, den, N, nrhs, pmap);
}

// r = b - (K - xi_p M) x for every pole; one warp per row, lanes over RHS.
__global__ void k_residual(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ kv, const double *__restrict__ mv,
                           const double2 *__restrict__ xi, const c128 *__restrict__ b,
                           int64_t bstride, const c128 *__restrict__ x, c128 *__restrict__ r,
                           int64_t N, int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const int lane = threadIdx.x & 31;
  const int64_t row = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= N) return;
  const double2 s = xi[p];
  const c128 *xp = x + p * N * nrhs;
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int rhs = c0 + lane;
    if (rhs >= nrhs) break;
    c128 acc = b[p * bstride + row * nrhs + rhs];
    for (int64_t z = rp[row]; z < rp[row + 1]; z++) {
      const double k = kv[z], m = mv[z];
      const c128 a = mk<double>(k - s.x * m, -s.y * m);
      cfms(acc, a, xp[int64_t(ci[z]) * nrhs + rhs]);
    }
    r[p * N * nrhs + row * nrhs + rhs] = acc;
  }
}

void launch_residual(const int64_t *rp, const int32_t *ci, const double *kv, const double *mv,
                     const double2 *xi, const c128 *b, int64_t bstride, const c128 *x, c128 *r,
                     int np, const int *pmap, int64_t N, int nrhs, cudaStream_t s) {
  dim3 g(div_up(N, 8), np);
  tem::count_launch();
  k_residual<<<g, 256, 0, s>>>(rp, ci, kv, mv, xi, b, bstride, x, r, N, nrhs, pmap);
}

__global__ void k_real_to_c128(const double *__restrict__ f, c128 *__restrict__ b, int64_t cnt) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x)
    b[e] = mk<double>(f[e], 0.0);
}

void launch_real_to_c128(const double *f, c128 *b, int64_t count, cudaStream_t s) {
  tem::count_launch();
  k_real_to_c128<<<(unsigned)std::min<int64_t>(div_up(count, 256), 4096), 256, 0, s>>>(f, b, count);
}

// ---- observation and residue sums ------------------------------------------

constexpr int kMaxPoles = 32;

// an entry of y in FP64: complex FP64, or a double-float pair (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ c128 as_c128(c128 v) { return v; }
__device__ __forceinline__ c128 as_c128(float4 v) {
  return mk<double>(double(v.x) + double(v.y), double(v.z) + double(v.w));
}

// d[x][r][j] = 2 Re sum_p alpha[p][j] (Q y_p)[r][x] for the ntx transmitters
// (y rows hold nrhs >= ntx right-hand sides; the rest are padding)
template <typename T>
__global__ void k_residue(const int64_t *__restrict__ q_rp, const int32_t *__restrict__ q_ci,
                          const double *__restrict__ q_val, const double2 *__restrict__ alpha,
                          const T *__restrict__ y, double *__restrict__ d, int m, int64_t N,
                          int nrhs, int ntx, int n_rx, int K) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= int64_t(n_rx) * ntx) return;
  const int x = int(t % ntx), r = int(t / ntx);
  c128 yq[kMaxPoles];
  for (int p = 0; p < m; p++) {
    c128 acc = mk<double>(0.0, 0.0);
    const T *yp = y + p * N * nrhs;
    for (int64_t z = q_rp[r]; z < q_rp[r + 1]; z++) {
      const c128 v = as_c128(yp[int64_t(q_ci[z]) * nrhs + x]);
      acc.x += q_val[z] * v.x;
      acc.y += q_val[z] * v.y;
    }
    yq[p] = acc;
  }
  for (int j = 0; j < K; j++) {
    double s = 0;
    for (int p = 0; p < m; p++) {
      const double2 a = alpha[p * K + j];
      s += a.x * yq[p].x - a.y * yq[p].y;
    }
    d[(int64_t(x) * n_rx + r) * K + j] = 2.0 * s;
  }
}

void launch_residue(const int64_t *q_rp, const int32_t *q_ci, const double *q_val,
                    const double2 *alpha, const c128 *y, double *d, int m, int64_t N, int nrhs,
                    int ntx, int n_rx, int K, cudaStream_t s) {
  const int64_t cnt = int64_t(n_rx) * ntx;
  tem::count_launch();
  k_residue<c128><<<div_up(cnt, 128), 128, 0, s>>>(q_rp, q_ci, q_val, alpha, y, d, m, N, nrhs, ntx, n_rx, K);
}

void launch_residue(const int64_t *q_rp, const int32_t *q_ci, const double *q_val,
                    const double2 *alpha, const float4 *y, double *d, int m, int64_t N, int nrhs,
                    int ntx, int n_rx, int K, cudaStream_t s) {
  const int64_t cnt = int64_t(n_rx) * ntx;
  tem::count_launch();
  k_residue<float4><<<div_up(cnt, 128), 128, 0, s>>>(q_rp, q_ci, q_val, alpha, y, d, m, N, nrhs, ntx, n_rx, K);
}

// rhs_p[qdof][x] = sum_{r} Qt[qdof][r] * sum_j alpha[p][j] w[x][r][j], x < ntx
// (the padding right-hand sides x >= ntx stay zero)
// an FP64 complex value stored as is, or as the double-float pairs the FP32 refinement takes
__device__ __forceinline__ void store_cx(c128 *dst, c128 v) { *dst = v; }
__device__ __forceinline__ void store_cx(float4 *dst, c128 v) {
  const dfl a = split(v.x), b = split(v.y);
  *dst = make_float4(a.hi, a.lo, b.hi, b.lo);
}

template <typename T>
__global__ void k_qt_rhs(const int32_t *__restrict__ qt_dof, const int64_t *__restrict__ qt_rp,
                         const int32_t *__restrict__ qt_ci, const double *__restrict__ qt_val,
                         int n_qdof, const double2 *__restrict__ alpha, const double *__restrict__ w,
                         T *__restrict__ rhs, int64_t N, int nrhs, int ntx, int n_rx, int K) {
  const int p = blockIdx.y;
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (t >= int64_t(n_qdof) * ntx) return;
  const int x = int(t % ntx), q = int(t / ntx);
  c128 acc = mk<double>(0.0, 0.0);
  for (int64_t z = qt_rp[q]; z < qt_rp[q + 1]; z++) {
    const int r = qt_ci[z];
    const double *wr = w + (int64_t(x) * n_rx + r) * K;
    double sr = 0, si = 0;
    for (int j = 0; j < K; j++) {
      const double2 a = alpha[p * K + j];
      sr += a.x * wr[j];
      si += a.y * wr[j];
    }
    acc.x += qt_val[z] * sr;
    acc.y += qt_val[z] * si;
  }
  store_cx(rhs + p * N * nrhs + int64_t(qt_dof[q]) * nrhs + x, acc);
}

template <typename T>
void qt_rhs(const int32_t *qt_dof, const int64_t *qt_rp, const int32_t *qt_ci, const double *qt_val, int n_qdof,
            const double2 *alpha, const double *w, T *rhs, int m, int64_t N, int nrhs, int ntx, int n_rx, int K,
            cudaStream_t s) {
  cudaMemsetAsync(rhs, 0, sizeof(T) * m * N * nrhs, s);
  const int64_t cnt = int64_t(n_qdof) * ntx;
  if (cnt == 0) return;
  dim3 g(div_up(cnt, 128), m);
  tem::count_launch();
  k_qt_rhs<T><<<g, 128, 0, s>>>(qt_dof, qt_rp, qt_ci, qt_val, n_qdof, alpha, w, rhs, N, nrhs, ntx, n_rx, K);
}
void launch_qt_rhs(const int32_t *qt_dof, const int64_t *qt_rp, const int32_t *qt_ci,
                   const double *qt_val, int n_qdof, const double2 *alpha, const double *w, c128 *rhs,
                   int m, int64_t N, int nrhs, int ntx, int n_rx, int K, cudaStream_t s) {
  qt_rhs(qt_dof, qt_rp, qt_ci, qt_val, n_qdof, alpha, w, rhs, m, N, nrhs, ntx, n_rx, K, s);
}
void launch_qt_rhs(const int32_t *qt_dof, const int64_t *qt_rp, const int32_t *qt_ci,
                   const double *qt_val, int n_qdof, const double2 *alpha, const double *w, float4 *rhs,
                   int m, int64_t N, int nrhs, int ntx, int n_rx, int K, cudaStream_t s) {
  qt_rhs(qt_dof, qt_rp, qt_ci, qt_val, n_qdof, alpha, w, rhs, m, N, nrhs, ntx, n_rx, K, s);
}

// ---- mass-derivative products ------------------------------------------------

// h_p[d][x] = xi_p sum over the tets t at unknown d (local edge a) of
//             v_t sigma_t sum_b M1_t[a][b] g_p[tdof_t[b]][x]
// T is the arithmetic type of the per-unknown sums.  Both modes use double:
// the primary field cancels strongly in these sums, and FP32 sums put J v
// off by ~1e-5 relative.
template <typename T>
__global__ void k_dm_apply(const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_tet,
                           const int8_t *__restrict__ inc_loc, const int32_t *__restrict__ tdof,
                           const int32_t *__restrict__ pidx, const double *__restrict__ v,
                           const double *__restrict__ sigma, const double *__restrict__ me1,
                           const double2 *__restrict__ xi, const c128 *__restrict__ g,
                           c128 *__restrict__ h, int64_t N, int nrhs) {
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t d = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (d >= N) return;
  const c128 *gp = g + p * N * nrhs;
  const double2 s = xi[p];
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int x = c0 + lane;
    if (x >= nrhs) break;
    T ax = 0, ay = 0;
    for (int64_t q = inc_ptr[d]; q < inc_ptr[d + 1]; q++) {
      const int32_t t = inc_tet[q];
      const int32_t pt = pidx[t];
      if (pt < 0) continue;
      const T coef = T(v[pt] * sigma[t]);
      if (coef == T(0)) continue;
      const int a = inc_loc[q];
      const double *Me = me1 + int64_t(t) * 36 + a * 6;
      T sx = 0, sy = 0;
      for (int b = 0; b < 6; b++) {
        const int32_t db = tdof[int64_t(t) * 6 + b];
        if (db < 0) continue;
        const c128 gv = gp[int64_t(db) * nrhs + x];
        const T mb = T(Me[b]);
        sx += mb * T(gv.x);
        sy += mb * T(gv.y);
      }
      ax += coef * sx;
      ay += coef * sy;
    }
    const double acx = double(ax), acy = double(ay);
    h[p * N * nrhs + d * nrhs + x] = mk<double>(s.x * acx - s.y * acy, s.x * acy + s.y * acx);
  }
}

// Refined-FP32 mode: the J v right-hand sides in double-float pairs, from the
// forward solutions as pairs (gdf) and vs[t] = v_t sigma_t as pairs (zero on
// cells that are not parameters): per unknown one Dot2 sum over its
// tetrahedra and their six local unknowns, then times xi_p in FP64.
__global__ void k_vsig_df(const int32_t *__restrict__ ptet, int64_t P, const double *__restrict__ v,
                          const double *__restrict__ sigma, float2 *__restrict__ vs) {
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < P; p += int64_t(gridDim.x) * blockDim.x) {
    const int32_t t = ptet[p];
    const dfl d = split(v[p] * sigma[t]);
    vs[t] = make_float2(d.hi, d.lo);
  }
}

__global__ void k_dm_apply_df(const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_tet,
                              const int8_t *__restrict__ inc_loc, const int32_t *__restrict__ tdof,
                              const float2 *__restrict__ vs, const float2 *__restrict__ me1df,
                              const double2 *__restrict__ xi, const float4 *__restrict__ g, float4 *__restrict__ h,
                              int64_t N, int nrhs) {
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t d = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (d >= N) return;
  const float4 *gp = g + p * N * nrhs;
  const dfl sr = split(xi[p].x), si = split(xi[p].y);
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int x = c0 + lane;
    if (x >= nrhs) break;
    Dot2 ar, ai;
    for (int64_t q = inc_ptr[d]; q < inc_ptr[d + 1]; q++) {
      const int32_t t = inc_tet[q];
      const float2 c2 = vs[t];
      if (c2.x == 0.f) continue;
      const dfl coef = {c2.x, c2.y};
      const float2 *Me = me1df + int64_t(t) * 36 + inc_loc[q] * 6;
      for (int b = 0; b < 6; b++) {
        const int32_t db = tdof[int64_t(t) * 6 + b];
        if (db < 0) continue;
        const float2 m2 = Me[b];
        const dfl cm = df_mul(coef, {m2.x, m2.y});
        const float4 gv = gp[int64_t(db) * nrhs + x];
        ar.add(cm, {gv.x, gv.y});
        ai.add(cm, {gv.z, gv.w});
      }
    }
    // h = xi (ar + i ai), kept as pairs: the refinement takes its right-hand side in this form
    const dfl acx = ar.value(), acy = ai.value();
    const dfl hr = df_add(df_mul(sr, acx), df_neg(df_mul(si, acy)));
    const dfl hi = df_add(df_mul(sr, acy), df_mul(si, acx));
    h[p * N * nrhs + d * nrhs + x] = make_float4(hr.hi, hr.lo, hi.hi, hi.lo);
  }
}

void launch_dm_apply_df(const int64_t *inc_ptr, const int32_t *inc_tet, const int8_t *inc_loc, const int32_t *tdof,
                        const int32_t *ptet, int64_t P, const double *v, const double *sigma, float2 *vs, int64_t nt,
                        const float2 *me1df, const double2 *xi, const float4 *gdf, float4 *h, int m, int64_t N,
                        int nrhs, cudaStream_t s) {
  cudaMemsetAsync(vs, 0, sizeof(float2) * nt, s);
  if (P > 0) {
    tem::count_launch();
    k_vsig_df<<<(unsigned)std::min<int64_t>(div_up(P, 256), 4096), 256, 0, s>>>(ptet, P, v, sigma, vs);
  }
  dim3 gr(div_up(N, 8), m);
  tem::count_launch();
  k_dm_apply_df<<<gr, 256, 0, s>>>(inc_ptr, inc_tet, inc_loc, tdof, vs, me1df, xi, gdf, h, N, nrhs);
}

void launch_dm_apply(const int64_t *inc_ptr, const int32_t *inc_tet, const int8_t *inc_loc,
                     const int32_t *tdof, const int32_t *pidx, const double *v, const double *sigma,
                     const double *me1, const double2 *xi, const c128 *g, c128 *h, int m, int64_t N,
                     int nrhs, cudaStream_t s) {
  dim3 gr(div_up(N, 8), m);
  tem::count_launch();
  k_dm_apply<double><<<gr, 256, 0, s>>>(inc_ptr, inc_tet, inc_loc, tdof, pidx, v, sigma, me1, xi, g, h, N, nrhs);
}

// grad[pt] = 2 sigma_t Re sum_i xi_i sum_x (P_t z_ix)^T M1_t (P_t g_ix); one warp per cell
// (FP64 mode: T = double).
template <typename T>
__global__ void k_bilinear(const int32_t *__restrict__ ptet, int64_t P, const int32_t *__restrict__ tdof,
                           const double *__restrict__ sigma, const double *__restrict__ me1,
                           const double2 *__restrict__ xi, const c128 *__restrict__ g,
                           const c128 *__restrict__ z, double *__restrict__ grad, int m, int64_t N,
                           int nrhs) {
  const int lane = threadIdx.x & 31;
  const int64_t pt = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pt >= P) return;
  const int32_t t = ptet[pt];
  int32_t td[6];
  for (int a = 0; a < 6; a++) td[a] = tdof[int64_t(t) * 6 + a];
  const double *Me = me1 + int64_t(t) * 36;
  double total = 0;
  for (int p = 0; p < m; p++) {
    const c128 *gp = g + p * N * nrhs;
    const c128 *zp = z + p * N * nrhs;
    c128 acc = mk<double>(0.0, 0.0);
    for (int x = lane; x < nrhs; x += 32) {
      cx<T> gl[6], zl[6];
      for (int a = 0; a < 6; a++) {
        const c128 gv = td[a] >= 0 ? gp[int64_t(td[a]) * nrhs + x] : mk<double>(0.0, 0.0);
        const c128 zv = td[a] >= 0 ? zp[int64_t(td[a]) * nrhs + x] : mk<double>(0.0, 0.0);
        gl[a] = mk<T>(T(gv.x), T(gv.y));
        zl[a] = mk<T>(T(zv.x), T(zv.y));
      }
      cx<T> sum = mk<T>(T(0), T(0));
      for (int a = 0; a < 6; a++) {
        cx<T> mg = mk<T>(T(0), T(0));
        for (int b = 0; b < 6; b++) {
          const T mab = T(Me[a * 6 + b]);
          mg.x += mab * gl[b].x;
          mg.y += mab * gl[b].y;
        }
        cfma(sum, zl[a], mg);
      }
      acc.x += double(sum.x);
      acc.y += double(sum.y);
    }
    const double2 s = xi[p];
    total += s.x * acc.x - s.y * acc.y;
  }
  for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(0xffffffffu, total, o);
  if (lane == 0) grad[pt] = 2.0 * sigma[t] * total;
}

// Refined-FP32 mode: the same cell sums in double-float arithmetic on the FP32
// pipes, one warp per (cell, pole): part[p][pt] = Re xi_p sum_x (P z_px)^T M1_t (P g_px),
// with g, z the refined solutions as pairs [m][N][nrhs] (re.hi, re.lo, im.hi,
// im.lo) and M1 as pairs, accumulated with Dot2.  The sums over poles cancel
// (residue-like), so FP32 cell sums (relative 1e-7 each) would leave J^T w near
// 1e-6; pairs leave it near 1e-12.
__global__ void k_bilinear_df(const int32_t *__restrict__ ptet, int64_t P, const int32_t *__restrict__ tdof,
                              const float2 *__restrict__ me1df, const double2 *__restrict__ xi,
                              const float4 *__restrict__ g, const float4 *__restrict__ z, double *__restrict__ part,
                              int64_t N, int nrhs) {
  const int p = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int64_t pt = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (pt >= P) return;
  const int32_t t = ptet[pt];
  int32_t td[6];
  for (int a = 0; a < 6; a++) td[a] = tdof[int64_t(t) * 6 + a];
  const float2 *Me = me1df + int64_t(t) * 36;
  const float4 *gp = g + p * N * nrhs;
  const float4 *zp = z + p * N * nrhs;
  // sums over the right-hand sides in double-float pairs (FP64 runs at 1/64 of the FP32 rate here)
  dfl ar = {0.f, 0.f}, ai = {0.f, 0.f};
  for (int x = lane; x < nrhs; x += 32) {
    float4 gl[6];
    for (int b = 0; b < 6; b++) gl[b] = td[b] >= 0 ? gp[int64_t(td[b]) * nrhs + x] : make_float4(0.f, 0.f, 0.f, 0.f);
    Dot2 sr, si;
    for (int a = 0; a < 6; a++) {
      if (td[a] < 0) continue;
      Dot2 mr, mi;
      for (int b = 0; b < 6; b++) {
        const float2 m2 = Me[a * 6 + b];
        const dfl mab = {m2.x, m2.y};
        mr.add(mab, {gl[b].x, gl[b].y});
        mi.add(mab, {gl[b].z, gl[b].w});
      }
      const dfl Mr = mr.value(), Mi = mi.value();
      const float4 zv = zp[int64_t(td[a]) * nrhs + x];
      const dfl zr = {zv.x, zv.y}, zi = {zv.z, zv.w};
      sr.add(zr, Mr);
      sr.add(df_neg(zi), Mi);
      si.add(zr, Mi);
      si.add(zi, Mr);
    }
    ar = df_add(ar, sr.value());
    ai = df_add(ai, si.value());
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar = df_add(ar, {__shfl_down_sync(0xffffffffu, ar.hi, o), __shfl_down_sync(0xffffffffu, ar.lo, o)});
    ai = df_add(ai, {__shfl_down_sync(0xffffffffu, ai.hi, o), __shfl_down_sync(0xffffffffu, ai.lo, o)});
  }
  if (lane == 0) {
    const double2 s = xi[p];
    part[p * P + pt] = s.x * df_to_double(ar) - s.y * df_to_double(ai);
  }
}

// grad[pt] = 2 sigma_t sum_p part[p][pt]  (poles summed in a fixed order)
__global__ void k_bilinear_sum(const int32_t *__restrict__ ptet, int64_t P, const double *__restrict__ sigma,
                               const double *__restrict__ part, double *__restrict__ grad, int m) {
  for (int64_t pt = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; pt < P; pt += int64_t(gridDim.x) * blockDim.x) {
    double s = 0;
    for (int p = 0; p < m; p++) s += part[p * P + pt];
    grad[pt] = 2.0 * sigma[ptet[pt]] * s;
  }
}

void launch_bilinear(const int32_t *ptet, int64_t P, const int32_t *tdof, const double *sigma,
                     const double *me1, const double2 *xi, const c128 *g, const c128 *z, double *grad,
                     int m, int64_t N, int nrhs, cudaStream_t s) {
  if (P == 0) return;
  tem::count_launch();
  k_bilinear<double><<<div_up(P, 8), 256, 0, s>>>(ptet, P, tdof, sigma, me1, xi, g, z, grad, m, N, nrhs);
}

void launch_bilinear_df(const int32_t *ptet, int64_t P, const int32_t *tdof, const double *sigma,
                        const float2 *me1df, const double2 *xi, const float4 *gdf, const float4 *zdf, double *grad,
                        int m, int64_t N, int nrhs, double *part, cudaStream_t s) {
  if (P == 0) return;
  dim3 gr(div_up(P, 8), m);
  tem::count_launch();
  k_bilinear_df<<<gr, 256, 0, s>>>(ptet, P, tdof, me1df, xi, gdf, zdf, part, N, nrhs);
  tem::count_launch();
  k_bilinear_sum<<<(unsigned)std::min<int64_t>(div_up(P, 256), 4096), 256, 0, s>>>(ptet, P, sigma, part, grad, m);
}

__global__ void k_csr_mv(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                         const double *__restrict__ val, const double *__restrict__ x,
                         double *__restrict__ y, int64_t rows, double alpha, double beta) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < rows;
       r += int64_t(gridDim.x) * blockDim.x) {
    double s = 0;
    for (int64_t z = rp[r]; z < rp[r + 1]; z++) s += val[z] * x[ci[z]];
    y[r] = alpha * s + (beta == 0.0 ? 0.0 : beta * y[r]);
  }
}

void launch_csr_mv(const int64_t *rp, const int32_t *ci, const double *val, const double *x, double *y,
                   int64_t rows, double alpha, double beta, cudaStream_t s) {
  if (rows == 0) return;
  tem::count_launch();
  k_csr_mv<<<(unsigned)std::min<int64_t>(div_up(rows, 256), 4096), 256, 0, s>>>(rp, ci, val, x, y, rows,
                                                                                alpha, beta);
}

// ---- LSQR (all scalars on the device) ----------------------------------------

__global__ void k_sumsq(const double *__restrict__ x, int64_t n, double *out) {
  double s = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    s += x[e] * x[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

void launch_sumsq(const double *x, int64_t n, double *out, cudaStream_t s) {
  if (n == 0) return;
  tem::count_launch();
  k_sumsq<<<(unsigned)std::min<int64_t>(div_up(n, 256), 1024), 256, 0, s>>>(x, n, out);
}

// LSQR element-wise steps; op selects the formula, scalars come from sc.
//   0: a = a / sqrt(sumsq)          (normalise; beta <- norm)
//   1: a = a / sqrt(sumsq)          (normalise; alpha <- norm)
//   2: a = b * c - alpha * a         (u1 <- W_d (J v) - alpha u1)
//   3: a = b - beta * a              (v <- (A^T u) - beta v)
//   4: x(a) += phi/rho * w(b); w(b) = v(c) - theta/rho * w(b)
//   5: a = b * c                     (element-wise product)
//   6: a = -(b - c) * wd             (u1 <- -W_d (d - d_obs))
//   7: a = b - alpha * a             (u2 <- sqrt(lam) W v - alpha u2)
__global__ void k_lsqr(int op, LsqrScalars *sc, double *__restrict__ a, const double *__restrict__ b,
                       const double *__restrict__ c, const double *__restrict__ wd, int64_t n) {
  const int64_t i0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t st = int64_t(gridDim.x) * blockDim.x;
  if (op == 0 || op == 1) {
    const double nrm = sqrt(sc->sumsq);
    const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
    for (int64_t i = i0; i < n; i += st) a[i] *= inv;
  } else if (op == 2) {
    const double al = sc->alpha;
    for (int64_t i = i0; i < n; i += st) a[i] = b[i] * c[i] - al * a[i];
  } else if (op == 3) {
    const double be = sc->beta;
    for (int64_t i = i0; i < n; i += st) a[i] = b[i] - be * a[i];
  } else if (op == 4) {
    const double f1 = sc->phi / sc->rho, f2 = sc->theta / sc->rho;
    double *w = const_cast<double *>(b);
    for (int64_t i = i0; i < n; i += st) {
      const double wi = w[i];
      a[i] += f1 * wi;
      w[i] = c[i] - f2 * wi;
    }
  } else if (op == 5) {
    for (int64_t i = i0; i < n; i += st) a[i] = b[i] * c[i];
  } else if (op == 6) {
    for (int64_t i = i0; i < n; i += st) a[i] = -(b[i] - c[i]) * wd[i];
  } else if (op == 7) {
    const double al = sc->alpha;
    for (int64_t i = i0; i < n; i += st) a[i] = b[i] - al * a[i];
  }
}

// Scalar bookkeeping: which = 0 -> beta = sqrt(sumsq); 1 -> alpha = sqrt(sumsq);
// 2 -> start (phibar = beta, rhobar = alpha); 3 -> Givens step of one iteration.
__global__ void k_lsqr_scalars(LsqrScalars *sc, int which) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (which == 0) {
    sc->beta = sqrt(sc->sumsq);
  } else if (which == 1) {
    sc->alpha = sqrt(sc->sumsq);
  } else if (which == 2) {
    sc->phibar = sc->beta;
    sc->rhobar = sc->alpha;
  } else {
    const double rho = hypot(sc->rhobar, sc->beta);
    const double c = rho > 0 ? sc->rhobar / rho : 1.0;
    const double s = rho > 0 ? sc->beta / rho : 0.0;
    sc->rho = rho > 0 ? rho : 1.0;
    sc->c = c;
    sc->sn = s;
    sc->theta = s * sc->alpha;
    sc->rhobar = -c * sc->alpha;
    sc->phi = c * sc->phibar;
    sc->phibar = s * sc->phibar;
  }
  sc->sumsq = 0.0;
}

void launch_lsqr_kernel(int op, LsqrScalars *sc, double *a, const double *b, const double *c,
                        const double *wd, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  tem::count_launch();
  k_lsqr<<<(unsigned)std::min<int64_t>(div_up(n, 256), 2048), 256, 0, s>>>(op, sc, a, b, c, wd, n);
}

void launch_lsqr_scalars(LsqrScalars *sc, int which, cudaStream_t s) {
  tem::count_launch();
  k_lsqr_scalars<<<1, 32, 0, s>>>(sc, which);
}

template void launch_rhs_to_work<float>(const c128 *, int64_t, c64 *, double *, int, const int *, int64_t, int,
                                        bool, cudaStream_t);
template void launch_rhs_to_work<double>(const c128 *, int64_t, c128 *, double *, int, const int *, int64_t,
                                         int, bool, cudaStream_t);
template void launch_accumulate<float>(const c64 *, const double *, c128 *, int, const int *, int64_t, int,
                                       bool, cudaStream_t);
template void launch_accumulate<double>(const c128 *, const double *, c128 *, int, const int *, int64_t, int,
                                        bool, cudaStream_t);
template void launch_progress<float>(const c64 *, const double *, const c128 *, const uint8_t *, double *,
                                     double *, int, const int *, int64_t, int, cudaStream_t);

// Status words before a factorisation: no pivot failure, no timeout, smallest pivot +huge.
__global__ void k_status_init(DevStatus *st) {
  st->pivot_fail = 0;
  st->pivot_front = -1;
  st->tc_timeout = 0;
  st->min_pivot_bits = (unsigned long long)__double_as_longlong(1e308);
}

void launch_status_init(DevStatus *st, cudaStream_t s) {
  tem::count_launch();
  k_status_init<<<1, 1, 0, s>>>(st);
}

// ---- Gauss-Newton bookkeeping (Section 3.3) ----------------------------------

// t = wd (d - d_obs), t2 = wd^2 (d - d_obs)
__global__ void k_gn_res(const double *__restrict__ d, const double *__restrict__ d_obs,
                         const double *__restrict__ wd, double *__restrict__ t, double *__restrict__ t2, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double r = wd[i] * (d[i] - d_obs[i]);
    t[i] = r;
    t2[i] = wd[i] * r;
  }
}

// *out += sum x y
__global__ void k_dot(const double *__restrict__ x, const double *__restrict__ y, int64_t n, double *out) {
  double acc = 0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    acc += x[i] * y[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < int(blockDim.x >> 5); w++) t += red[w];
    atomicAdd(out, t);
  }
}

// out = m + eta dm
__global__ void k_axpy(const double *__restrict__ m, const double *__restrict__ dm, double eta,
                       double *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = m[i] + eta * dm[i];
}

void launch_gn_res(const double *d, const double *d_obs, const double *wd, double *t, double *t2, int64_t n,
                   cudaStream_t s) {
  if (n <= 0) return;
  tem::count_launch();
  k_gn_res<<<(unsigned)std::min<int64_t>(div_up(n, 256), 4096), 256, 0, s>>>(d, d_obs, wd, t, t2, n);
}

void launch_dot(const double *x, const double *y, int64_t n, double *out, cudaStream_t s) {
  if (n <= 0) return;
  tem::count_launch();
  k_dot<<<(unsigned)std::min<int64_t>(div_up(n, 256), 1024), 256, 0, s>>>(x, y, n, out);
}

void launch_axpy(const double *m, const double *dm, double eta, double *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  tem::count_launch();
  k_axpy<<<(unsigned)std::min<int64_t>(div_up(n, 256), 4096), 256, 0, s>>>(m, dm, eta, out, n);
}

}  // namespace tem
