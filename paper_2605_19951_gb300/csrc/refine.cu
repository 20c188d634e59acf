// Iterative refinement of the FP32 solves (x += P^-1 (b - A x), Algorithm 1
// with a reduced-precision factor) without the FP64 pipes.
//
// The residual r = b - (K - xi M) x needs about twice FP32's precision; on
// this GPU the FP64 pipe is slow (a 10.7 M-nonzero A times 320 right-hand
// sides is 13.6 G FP64 FMAs per residual), so the refinement keeps b and the
// iterate x as double-float pairs (hi + lo, 48-bit significand) and evaluates
// the residual on the FP32 pipes with error-free transformations: Knuth's
// TwoSum, the FMA form of Dekker's TwoProduct, and the compensated dot
// product of Ogita, Rump and Oishi (Dot2, 2005), which returns a sum as if
// accumulated in twice the working precision.  FP64 is used only to split b
// into pairs once per solve and to add the pairs of x back into FP64 once at
// the end.  K x and M x are accumulated separately (the pair-valued K and M
// are pole independent) and combined per row: r = b - K x + xi (M x).
#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace tem {


// pairs of a real FP64 array (K or M values)
__global__ void k_split_real(const double *__restrict__ v, float2 *__restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const dfl d = split(v[e]);
    out[e] = make_float2(d.hi, d.lo);
  }
}

// pairs of a complex FP64 array: (re.hi, re.lo, im.hi, im.lo)
__global__ void k_split_cx(const c128 *__restrict__ v, float4 *__restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const c128 z = v[e];
    const dfl a = split(z.x), b = split(z.y);
    out[e] = make_float4(a.hi, a.lo, b.hi, b.lo);
  }
}

// x = hi + lo in FP64
__global__ void k_join_cx(const float4 *__restrict__ v, c128 *__restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const float4 z = v[e];
    out[e] = mk<double>(double(z.x) + double(z.y), double(z.z) + double(z.w));
  }
}

// r = b - K x + xi (M x) for every mapped pole; one warp per row, lanes over
// right-hand sides; r rounded to FP32 (it only feeds the FP32 correction).
// A block walks kResRows consecutive rows (its eight warps on interleaved
// rows), so the x rows that neighbouring rows share are reused from L1.
constexpr int kResRows = 128;
__global__ void __launch_bounds__(256) k_residual_df(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                     const float2 *__restrict__ kdf, const float2 *__restrict__ mdf,
                                                     const double2 *__restrict__ xi, const float4 *__restrict__ bdf,
                                                     int64_t bstride, const float4 *__restrict__ xdf,
                                                     c64 *__restrict__ r, int64_t N, int nrhs,
                                                     const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const int lane = threadIdx.x & 31;
  const dfl xr = split(xi[p].x), xq = split(xi[p].y);
  const float4 *xp = xdf + p * N * nrhs;
  const int64_t rbeg = blockIdx.x * int64_t(kResRows), rend = rbeg + kResRows < N ? rbeg + kResRows : N;
  for (int64_t row = rbeg + (threadIdx.x >> 5); row < rend; row += blockDim.x >> 5) {
    const int64_t z0 = rp[row], z1 = rp[row + 1];
    for (int c0 = 0; c0 < nrhs; c0 += 32) {
      const int rhs = c0 + lane;
      if (rhs >= nrhs) break;
      Dot2 kr, ki, mr, mi;
      for (int64_t z = z0; z < z1; z++) {
        const float2 kv = kdf[z], mv = mdf[z];
        const float4 v = xp[int64_t(ci[z]) * nrhs + rhs];
        const dfl k = {kv.x, kv.y}, mm = {mv.x, mv.y};
        const dfl vr = {v.x, v.y}, vi = {v.z, v.w};
        kr.add(k, vr);
        ki.add(k, vi);
        mr.add(mm, vr);
        mi.add(mm, vi);
      }
      const dfl Kr = kr.value(), Ki = ki.value(), Mr = mr.value(), Mi = mi.value();
      // xi (M x) = (xr Mr - xq Mi) + i (xr Mi + xq Mr)
      const dfl sr = df_add(df_mul(xr, Mr), df_neg(df_mul(xq, Mi)));
      const dfl si = df_add(df_mul(xr, Mi), df_mul(xq, Mr));
      const float4 b = bdf[p * bstride + row * nrhs + rhs];
      const dfl rr = df_add(df_add({b.x, b.y}, df_neg(Kr)), sr);
      const dfl ri = df_add(df_add({b.z, b.w}, df_neg(Ki)), si);
      r[p * N * nrhs + row * nrhs + rhs] = mk<float>(__fadd_rn(rr.hi, rr.lo), __fadd_rn(ri.hi, ri.lo));
    }
  }
}

// Column maxima (per pole and right-hand side) of max(|re|, |im|) of a
// complex FP32 array, or of the hi parts of pairs; colmax zeroed first.
template <typename T>
__device__ __forceinline__ float absmax_of(T v);
template <>
__device__ __forceinline__ float absmax_of<c64>(c64 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
template <>
__device__ __forceinline__ float absmax_of<float4>(float4 v) { return fmaxf(fabsf(v.x), fabsf(v.z)); }

template <typename T>
__global__ void k_colmax_f(const T *__restrict__ v, int64_t vstride, float *colmax, int64_t N, int nrhs,
                           const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const T *vp = v + p * vstride;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  __shared__ float red[8][32];
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int rhs = c0 + lane;
    float mx = 0.f;
    if (rhs < nrhs)
      for (int64_t r = blockIdx.x * int64_t(8) + grp; r < N; r += int64_t(gridDim.x) * 8)
        mx = fmaxf(mx, absmax_of<T>(vp[r * nrhs + rhs]));
    red[grp][lane] = mx;
    __syncthreads();
    if (grp == 0 && rhs < nrhs) {
      for (int g = 1; g < 8; g++) mx = fmaxf(mx, red[g][lane]);
      if (mx > 0) atomicMax(reinterpret_cast<unsigned *>(&colmax[p * nrhs + rhs]), __float_as_uint(mx));
    }
    __syncthreads();
  }
}

__global__ void k_zero_colmax_f(float *colmax, int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.x, pmap);
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) colmax[p * nrhs + r] = 0.f;
}

// Y = v / colmax (FP32), v complex FP32 (the residual) or the hi parts of b's pairs
template <typename T>
__device__ __forceinline__ c64 as_c64(T v);
template <>
__device__ __forceinline__ c64 as_c64<c64>(c64 v) { return v; }
template <>
__device__ __forceinline__ c64 as_c64<float4>(float4 v) { return mk<float>(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w)); }

template <typename T>
__global__ void k_scale_to_work(const T *__restrict__ v, int64_t vstride, c64 *__restrict__ Y,
                                const float *__restrict__ colmax, int64_t N, int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const T *vp = v + p * vstride;
  c64 *yp = Y + p * N * nrhs;
  const int64_t cnt = N * nrhs;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt; e += int64_t(gridDim.x) * blockDim.x) {
    const float c = colmax[p * nrhs + e % nrhs];
    const float s = c > 0.f ? 1.f / c : 1.f;
    const c64 z = as_c64<T>(vp[e]);
    yp[e] = mk<float>(z.x * s, z.y * s);
  }
}

// x (+)= colmax X as pairs: c X is formed exactly (TwoProduct) and added.
// With the nodal part (Xn != nullptr) the gradient-space correction of the
// same step is added too: x += -(psi[hi] - psi[lo]) / xi_p, psi = colmax_n Xn.
__global__ void k_accumulate_df(const c64 *__restrict__ X, const float *__restrict__ colmax, float4 *__restrict__ x,
                                int64_t N, int nrhs, int add, const int *__restrict__ pmap, NodalPart nd) {
  const int p = pole_of(blockIdx.y, pmap);
  const c64 *Xp = X + p * N * nrhs;
  float4 *xp = x + p * N * nrhs;
  const int64_t cnt = N * nrhs;
  const float2 w = nd.Xn ? nd.ninv_xi[p] : make_float2(0.f, 0.f);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt; e += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(e % nrhs);
    const float cm = colmax[p * nrhs + j];
    const float c = cm > 0.f ? cm : 1.f;
    const c64 v = Xp[e];
    const float pr = __fmul_rn(c, v.x), pi = __fmul_rn(c, v.y);
    dfl ar = {pr, __fmaf_rn(c, v.x, -pr)}, ai = {pi, __fmaf_rn(c, v.y, -pi)};
    if (add) {
      const float4 o = xp[e];
      ar = df_add({o.x, o.y}, ar);
      ai = df_add({o.z, o.w}, ai);
    }
    if (nd.Xn) {
      const int64_t d = e / nrhs, col = int64_t(p) * nrhs + j;
      const int lo = nd.e_lo[d], hi = nd.e_hi[d];
      c64 g = mk<float>(0.f, 0.f);
      if (hi >= 0) g = nd.Xn[int64_t(hi) * nd.ncol + col];
      if (lo >= 0) {
        const c64 l = nd.Xn[int64_t(lo) * nd.ncol + col];
        g.x -= l.x;
        g.y -= l.y;
      }
      const float cn = nd.colmax_n[col];
      const float sc = cn > 0.f ? cn : 1.f;
      g.x *= sc;
      g.y *= sc;
      ar = df_add(ar, {g.x * w.x - g.y * w.y, 0.f});
      ai = df_add(ai, {g.x * w.y + g.y * w.x, 0.f});
    }
    xp[e] = make_float4(ar.hi, ar.lo, ai.hi, ai.lo);
  }
}

// Refinement progress of each mapped pole over the masked unknowns:
// num[p] = max |colmax X|, den[p] = max |x| (double bits, max-accumulated).
__global__ void k_progress_df(const c64 *__restrict__ X, const float *__restrict__ colmax,
                              const float4 *__restrict__ x, const uint8_t *__restrict__ mask, double *num,
                              double *den, int64_t N, int nrhs, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const c64 *Xp = X + p * N * nrhs;
  const float4 *xp = x + p * N * nrhs;
  float a = 0.f, b = 0.f;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < N * nrhs;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (!mask[e / nrhs]) continue;
    const float c = colmax[p * nrhs + e % nrhs];
    const c64 d = Xp[e];
    const float4 v = xp[e];
    a = fmaxf(a, c * fmaxf(fabsf(d.x), fabsf(d.y)));
    b = fmaxf(b, fmaxf(fabsf(v.x), fabsf(v.z)));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmaxf(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (a > 0) atomicMax((unsigned long long *)&num[p], (unsigned long long)__double_as_longlong(double(a)));
    if (b > 0) atomicMax((unsigned long long *)&den[p], (unsigned long long)__double_as_longlong(double(b)));
  }
}

// ---- gradient-space (nodal) correction of the refinement -------------------
//
// The floored factor leaves the gradient fields of the floored (air) cells
// uncorrected: P_i^-1 A_i has eigenvalues sigma / s ~ 0 on them.  Each step
// therefore also solves the residual equation on the gradient space
// {G psi}: with K G = 0, G^T A_i G = -xi_i G^T M(sigma) G = -xi_i L_sigma, so
//   psi = L_sigma^-1 G^T r,   x += -G psi / xi_i,   r -= M(sigma) G psi
// (the residual update needs no K: (K - xi M) G psi / (-xi) = M G psi), one
// pole-independent Laplacian for all poles and right-hand sides.

// Yn[a][p nrhs + j] = (G^T r_p)[a][j] = sum over the edges at node a of +-r_p[e][j]
// (one warp per node, lanes over right-hand sides); r complex FP32 [m][N][nrhs].
__global__ void k_nodal_rhs(const int64_t *__restrict__ g_ptr, const int32_t *__restrict__ g_edge,
                            const int8_t *__restrict__ g_sign, const c64 *__restrict__ r, c64 *__restrict__ Yn,
                            int64_t Nn, int64_t N, int nrhs, int ncol, const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const int lane = threadIdx.x & 31;
  const int64_t a = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (a >= Nn) return;
  const c64 *rp = r + p * N * nrhs;
  const int64_t q0 = g_ptr[a], q1 = g_ptr[a + 1];
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int j = c0 + lane;
    if (j >= nrhs) break;
    float sr = 0.f, si = 0.f;
    for (int64_t q = q0; q < q1; q++) {
      const c64 v = rp[int64_t(g_edge[q]) * nrhs + j];
      const float sg = float(g_sign[q]);
      sr = fmaf(sg, v.x, sr);
      si = fmaf(sg, v.y, si);
    }
    Yn[a * ncol + int64_t(p) * nrhs + j] = mk<float>(sr, si);
  }
}

// With psi = colmax_n * Xn (the scaled nodal solution), for every edge unknown d:
//   r_p[d][j] -= (C psi)[d],  C = M(sigma) G (sparse rows c_rp / c_ci / c_val, FP32);
// the matching x update is added by k_accumulate_df after the edge sweeps.
// One warp per edge unknown, lanes over right-hand sides.
__global__ void k_nodal_apply(const int64_t *__restrict__ c_rp, const int32_t *__restrict__ c_ci,
                              const float *__restrict__ c_val, const c64 *__restrict__ Xn,
                              const float *__restrict__ colmax_n, c64 *__restrict__ r, int64_t N, int nrhs, int ncol,
                              const int *__restrict__ pmap) {
  const int p = pole_of(blockIdx.y, pmap);
  const int lane = threadIdx.x & 31;
  const int64_t d = blockIdx.x * int64_t(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (d >= N) return;
  const int64_t z0 = c_rp[d], z1 = c_rp[d + 1];
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int j = c0 + lane;
    if (j >= nrhs) break;
    const int64_t col = int64_t(p) * nrhs + j;
    const float cm = colmax_n[col];
    const float sc = cm > 0.f ? cm : 1.f;
    float ar = 0.f, ai = 0.f;
    for (int64_t q = z0; q < z1; q++) {
      const float cv = c_val[q];
      const c64 v = Xn[int64_t(c_ci[q]) * ncol + col];
      ar = fmaf(cv, v.x, ar);
      ai = fmaf(cv, v.y, ai);
    }
    const int64_t e = p * N * nrhs + d * nrhs + j;
    c64 rv = r[e];
    rv.x = fmaf(-sc, ar, rv.x);
    rv.y = fmaf(-sc, ai, rv.y);
    r[e] = rv;
  }
}

// ---------------------------------------------------------------------------

namespace {
unsigned grid_for(int64_t n, int64_t cap = 4096) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(div_up(n, 256), cap)); }
}  // namespace

void launch_split_real(const double *v, float2 *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  tem::count_launch();
  k_split_real<<<grid_for(n), 256, 0, s>>>(v, out, n);
}

void launch_split_cx(const c128 *v, float4 *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  tem::count_launch();
  k_split_cx<<<grid_for(n), 256, 0, s>>>(v, out, n);
}

void launch_join_cx(const float4 *v, c128 *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  tem::count_launch();
  k_join_cx<<<grid_for(n), 256, 0, s>>>(v, out, n);
}

void launch_residual_df(const int64_t *rp, const int32_t *ci, const float2 *kdf, const float2 *mdf,
                        const double2 *xi, const float4 *bdf, int64_t bstride, const float4 *xdf, c64 *r, int np,
                        const int *pmap, int64_t N, int nrhs, cudaStream_t s) {
  dim3 g(div_up(N, kResRows), np);
  tem::count_launch();
  k_residual_df<<<g, 256, 0, s>>>(rp, ci, kdf, mdf, xi, bdf, bstride, xdf, r, N, nrhs, pmap);
}

template <typename T>
void launch_scale_to_work(const T *v, int64_t vstride, c64 *Y, float *colmax, int np, const int *pmap, int64_t N,
                          int nrhs, cudaStream_t s) {
  tem::count_launch();
  k_zero_colmax_f<<<np, 64, 0, s>>>(colmax, nrhs, pmap);
  dim3 gc((unsigned)std::min<int64_t>(div_up(N, 8), 512), np);
  tem::count_launch();
  k_colmax_f<T><<<gc, 256, 0, s>>>(v, vstride, colmax, N, nrhs, pmap);
  dim3 g(grid_for(N * nrhs, 2048), np);
  tem::count_launch();
  k_scale_to_work<T><<<g, 256, 0, s>>>(v, vstride, Y, colmax, N, nrhs, pmap);
}
template void launch_scale_to_work<c64>(const c64 *, int64_t, c64 *, float *, int, const int *, int64_t, int,
                                        cudaStream_t);
template void launch_scale_to_work<float4>(const float4 *, int64_t, c64 *, float *, int, const int *, int64_t, int,
                                           cudaStream_t);

void launch_accumulate_df(const c64 *X, const float *colmax, float4 *x, int np, const int *pmap, int64_t N, int nrhs,
                          bool add, cudaStream_t s, const NodalPart &nd) {
  dim3 g(grid_for(N * nrhs, 2048), np);
  tem::count_launch();
  k_accumulate_df<<<g, 256, 0, s>>>(X, colmax, x, N, nrhs, add ? 1 : 0, pmap, nd);
}

void launch_progress_df(const c64 *X, const float *colmax, const float4 *x, const uint8_t *mask, double *num,
                        double *den, int np, const int *pmap, int64_t N, int nrhs, cudaStream_t s) {
  dim3 g(grid_for(N * nrhs, 1024), np);
  tem::count_launch();
  k_progress_df<<<g, 256, 0, s>>>(X, colmax, x, mask, num, den, N, nrhs, pmap);
}

void launch_nodal_rhs(const int64_t *g_ptr, const int32_t *g_edge, const int8_t *g_sign, const c64 *r, c64 *Yn,
                      int64_t Nn, int np, const int *pmap, int m, int64_t N, int nrhs, cudaStream_t s) {
  const int ncol = m * nrhs;
  if (pmap) cudaMemsetAsync(Yn, 0, sizeof(c64) * Nn * ncol, s);   // poles not refining: zero columns
  dim3 g((unsigned)div_up(Nn, 8), np);
  tem::count_launch();
  k_nodal_rhs<<<g, 256, 0, s>>>(g_ptr, g_edge, g_sign, r, Yn, Nn, N, nrhs, ncol, pmap);
}

void launch_nodal_apply(const int64_t *c_rp, const int32_t *c_ci, const float *c_val, const c64 *Xn,
                        const float *colmax_n, c64 *r, int np, const int *pmap, int m, int64_t N, int nrhs,
                        cudaStream_t s) {
  dim3 g((unsigned)div_up(N, 8), np);
  tem::count_launch();
  k_nodal_apply<<<g, 256, 0, s>>>(c_rp, c_ci, c_val, Xn, colmax_n, r, N, nrhs, m * nrhs, pmap);
}

}  // namespace tem
