// Explicit inverses of the pivot blocks for the FP32 solves.
//
// After a level of the factorisation, each front's unit-lower pivot block
// L11 is replaced in place by T11 = L11^-1, so that every step of the solves
// is a product (dense, tensor-core friendly) instead of a substitution.  The
// inverse is built by merging diagonal blocks pairwise,
//   inv([[A, 0], [B, C]]) = [[A^-1, 0], [-C^-1 B A^-1, C^-1]],
// starting from the 32 x 32 block inverses the panel kernel already forms
// (stage 0 copies them into place) and doubling the block size per stage:
// G1 forms Y = B A^-1 in a scratch buffer, G2 overwrites B with -C^-1 Y.
// Blocks that are merged are never read again by another pair of the same
// stage, so each stage is two launches over all fronts of the level.  The
// diagonal, which still holds D during the merges (read as 1 by the
// products), is finally moved to dinv = D^-1 and set to 1.  Last, T11 and
// L21 are copied row-major (rows contiguous) for the tensor-core forward
// products, which read them along rows.
#include "common.cuh"
#include "kernels.h"

namespace tem {

namespace {
constexpr int TM = 64;   // output tile
constexpr int KC = 16;   // inner chunk

// 64 x 64 output tile of a complex product with operands given by loaders;
// 256 threads as 16 x 16, 4 x 4 outputs each (rows tx + 16 ii, cols ty + 16 jj).
template <class ALoad, class BLoad>
__device__ __forceinline__ void tile_product(int kbeg, int kend, ALoad aop, BLoad bop, c64 (&acc)[4][4]) {
  __shared__ c64 As[KC][TM + 1];
  __shared__ c64 Bs[KC][TM + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = mk<float>(0.f, 0.f);
  for (int k0 = kbeg; k0 < kend; k0 += KC) {
    __syncthreads();
    for (int idx = tid; idx < KC * TM; idx += 256) {
      const int i = idx % TM, kk = idx / TM;          // A: rows contiguous in memory
      As[kk][i] = (k0 + kk < kend) ? aop(i, k0 + kk) : mk<float>(0.f, 0.f);
      const int kb = idx % KC, j = idx / KC;          // B: inner index contiguous in memory
      Bs[kb][j] = (k0 + kb < kend) ? bop(k0 + kb, j) : mk<float>(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; kk++) {
      c64 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) cfma(acc[i][j], a[i], b[j]);
    }
  }
}
}  // namespace

// Stage 0: the strictly lower part of each 32 x 32 diagonal-block inverse.
__global__ void k_inv_diag(c64 *__restrict__ L, int64_t lstride, const c64 *__restrict__ linv, int64_t istride,
                           const FrontDev *__restrict__ F, const int2 *__restrict__ tasks) {
  const int2 t = tasks[blockIdx.x];
  const int p = blockIdx.y;
  const FrontDev f = F[t.x];
  const int j0 = t.y * kNB, nb = min(kNB, f.k - j0);
  c64 *A = L + p * lstride + f.lofs;
  const c64 *iv = linv + p * istride + (f.inv_off + t.y) * (kNB * kNB);
  for (int idx = threadIdx.x; idx < kNB * kNB; idx += blockDim.x) {
    const int r = idx % kNB, c = idx / kNB;
    if (r > c && r < nb) A[int64_t(j0 + c) * f.ld + j0 + r] = iv[c * kNB + r];
  }
}

// G1: Y = B A^-1 (B = rows of C x columns of A, A^-1 unit lower in place).
__global__ void __launch_bounds__(256) k_inv_g1(const c64 *__restrict__ L, int64_t lstride,
                                                const FrontDev *__restrict__ F, const InvTask *__restrict__ tasks,
                                                c64 *__restrict__ Y, int64_t ystride) {
  const InvTask t = tasks[blockIdx.x];
  const int p = blockIdx.y;
  const FrontDev f = F[t.front];
  const int64_t n = f.ld;   // column stride
  const c64 *Lp = L + p * lstride + f.lofs;
  const int a0 = t.a0, s = t.s, sc = t.sc;
  const int i0 = TM * t.ti, j0 = TM * t.tj;
  auto aop = [&](int i, int c) -> c64 {        // B[i][c]
    return (i0 + i < sc) ? Lp[int64_t(a0 + c) * n + a0 + s + i0 + i] : mk<float>(0.f, 0.f);
  };
  auto bop = [&](int c, int j) -> c64 {        // A^-1[c][j]
    const int jj = j0 + j;
    if (jj >= s || c < jj) return mk<float>(0.f, 0.f);
    if (c == jj) return mk<float>(1.f, 0.f);
    return Lp[int64_t(a0 + jj) * n + a0 + c];
  };
  c64 acc[4][4];
  tile_product(j0, s, aop, bop, acc);
  c64 *y = Y + p * ystride + t.ybase;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int jj = 0; jj < 4; jj++) {
    const int j = j0 + ty + 16 * jj;
    if (j >= s) continue;
#pragma unroll
    for (int ii = 0; ii < 4; ii++) {
      const int i = i0 + tx + 16 * ii;
      if (i < sc) y[int64_t(j) * sc + i] = acc[ii][jj];
    }
  }
}

// G2: B <- -C^-1 Y (C^-1 unit lower in place).
__global__ void __launch_bounds__(256) k_inv_g2(c64 *__restrict__ L, int64_t lstride, const FrontDev *__restrict__ F,
                                                const InvTask *__restrict__ tasks, const c64 *__restrict__ Y,
                                                int64_t ystride) {
  const InvTask t = tasks[blockIdx.x];
  const int p = blockIdx.y;
  const FrontDev f = F[t.front];
  const int64_t n = f.ld;   // column stride
  c64 *Lp = L + p * lstride + f.lofs;
  const int a0 = t.a0, s = t.s, sc = t.sc;
  const int i0 = TM * t.ti, j0 = TM * t.tj;
  const int c1 = a0 + s;
  const c64 *y = Y + p * ystride + t.ybase;
  auto aop = [&](int i, int c) -> c64 {        // C^-1[i][c]
    const int ii = i0 + i;
    if (ii >= sc || c > ii) return mk<float>(0.f, 0.f);
    if (c == ii) return mk<float>(1.f, 0.f);
    return Lp[int64_t(c1 + c) * n + c1 + ii];
  };
  auto bop = [&](int c, int j) -> c64 {        // Y[c][j]
    return (j0 + j < s) ? y[int64_t(j0 + j) * sc + c] : mk<float>(0.f, 0.f);
  };
  c64 acc[4][4];
  tile_product(0, min(sc, i0 + TM), aop, bop, acc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int jj = 0; jj < 4; jj++) {
    const int j = j0 + ty + 16 * jj;
    if (j >= s) continue;
#pragma unroll
    for (int ii = 0; ii < 4; ii++) {
      const int i = i0 + tx + 16 * ii;
      if (i < sc) Lp[int64_t(a0 + j) * n + c1 + i] = mk<float>(-acc[ii][jj].x, -acc[ii][jj].y);
    }
  }
}

// D -> dinv = D^-1 and a unit diagonal.
__global__ void k_inv_finish(c64 *__restrict__ L, int64_t lstride, const FrontDev *__restrict__ F,
                             const int32_t *__restrict__ lev, c64 *__restrict__ dinv, int64_t N) {
  const FrontDev f = F[lev[blockIdx.x]];
  const int p = blockIdx.y;
  c64 *Lp = L + p * lstride + f.lofs;
  for (int c = threadIdx.x; c < f.k; c += blockDim.x) {
    const int64_t at = int64_t(c) * f.ld + c;
    dinv[p * N + f.c0 + c] = crecip(Lp[at]);
    Lp[at] = mk<float>(1.f, 0.f);
  }
}

// Row-major copies of a level's pivot-block inverses and update rows:
// T11R[i][c] = T11[i][c] (zero for c > i) and L21T[i][c] = L21[i][c], rows of
// ld2 = k rounded up to even entries; 32 x 32 tiles through shared memory.
// Task: (front, 0 = T11 / 1 = L21, 32-row block).
__global__ void __launch_bounds__(256) k_row_copy(const c64 *__restrict__ L, int64_t lstride, c64 *__restrict__ T11R,
                                                  int64_t tstride, c64 *__restrict__ L21T, int64_t rstride,
                                                  const FrontDev *__restrict__ F, const int64_t *__restrict__ t11r_ofs,
                                                  const int64_t *__restrict__ l21t_ofs, const int4 *__restrict__ tasks) {
  const int4 t = tasks[blockIdx.x];
  const int p = blockIdx.y;
  const FrontDev f = F[t.x];
  const int k = f.k, ld2 = k + (k & 1);
  const bool l21 = t.y != 0;
  const int nrows = l21 ? f.n - k : k, row0 = l21 ? k : 0;
  const c64 *src = L + p * lstride + f.lofs;
  c64 *dst = l21 ? L21T + p * rstride + l21t_ofs[t.x] : T11R + p * tstride + t11r_ofs[t.x];
  __shared__ c64 tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = 32 * t.z + tx;
  for (int cb = 0; cb < ld2; cb += 32) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int c = cb + ty + 8 * q;
      const bool ok = c < k && i < nrows && (l21 || c <= i);
      tile[ty + 8 * q][tx] = ok ? src[int64_t(c) * f.ld + row0 + i] : mk<float>(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int r = 32 * t.z + ty + 8 * q, c = cb + tx;
      if (r < nrows && c < ld2) dst[int64_t(r) * ld2 + c] = tile[tx][ty + 8 * q];
    }
    __syncthreads();
  }
}

template <>
void FactorPlan<float>::invert_level(const LevelDev &lv, cudaStream_t s) {
  if (lv.nf == 0) return;
  if (g_prof) g_prof->begin(KC_INVERT, s);
  if (lv.n_inv_diag > 0) {
    tem::count_launch();
    k_inv_diag<<<dim3(lv.n_inv_diag, m), 256, 0, s>>>(L, lstride, linv, istride, F, lv.inv_diag);
  }
  for (const LevelDev::InvStage &st : lv.inv) {
    if (st.n == 0) continue;
    tem::count_launch();
    k_inv_g1<<<dim3(st.n, m), 256, 0, s>>>(L, lstride, F, st.tasks, yscr, yscr_stride);
    tem::count_launch();
    k_inv_g2<<<dim3(st.n, m), 256, 0, s>>>(L, lstride, F, st.tasks, yscr, yscr_stride);
  }
  tem::count_launch();
  k_inv_finish<<<dim3(lv.nf, m), 256, 0, s>>>(L, lstride, F, lv.fronts, dinv, N);
  if (lv.n_rcopy > 0 && T11R) {
    tem::count_launch();
    k_row_copy<<<dim3(lv.n_rcopy, m), 256, 0, s>>>(L, lstride, T11R, t11r_stride, L21T, l21t_stride, F, t11r_ofs,
                                                   l21t_ofs, lv.rcopy);
  }
  if (g_prof) g_prof->end(KC_INVERT, s);
}

template <>
void FactorPlan<double>::invert_level(const LevelDev &, cudaStream_t) {}

}  // namespace tem
