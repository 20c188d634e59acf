// Update-row products of the FP32 solves on the fifth-generation tensor
// cores (tcgen05.mma kind::tf32, accumulators in TMEM).
//
// A complex product C = L X is one real GEMM: the rows of L are viewed as
// interleaved (re, im) real rows, the 32 complex right-hand sides as 64 real
// columns, so P = L_real X_real holds P[2i+a][2j+b] = sum L_a(i,.) X_b(.,j)
// and re C(i,j) = P[2i][2j] - P[2i+1][2j+1], im C(i,j) = P[2i][2j+1] +
// P[2i+1][2j].  Every operand is split into TF32 hi + lo parts and three
// MMAs (hi.hi + hi.lo + lo.hi) give FP32 accuracy: a single TF32 pass is not
// accurate enough for the refinement to converge.
//
// One CTA computes a 128 x 64 real tile (64 complex rows x 32 RHS) with a
// warp-specialised pipeline: warps 0-3 load K chunks from global memory,
// split them and stage them in a ring of NSTAGE shared-memory buffers
// (K-major, no swizzle) and signal "full"; warp 4 issues the MMAs of a full
// stage and commits them to the stage's "empty" barrier, which frees it for
// the producers.  After the last chunk warps 0-3 read the accumulators from
// TMEM (warp w owns lanes 32w..32w+31) and write the complex results.
// Every wait is bounded; a wait that gives up raises the CTA's abort flag
// and the status word, and all warps wind down to the TMEM release.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace tem {

namespace {
constexpr int TBM = 128;     // real rows per CTA (64 complex)
constexpr int TBN = 64;      // real columns (32 complex RHS)
constexpr int TKC = 16;      // K per stage (2 MMA k-steps of 8)
constexpr int NSTAGE = 3;
constexpr int NPROD = 128;   // producer / epilogue threads (warps 0-3)
constexpr uint32_t kWaitIter = 1u << 26;

struct Stage {
  float A[2][TBM * TKC];   // hi, lo
  float B[2][TBN * TKC];   // hi, lo
};
struct TcShared {
  Stage st[NSTAGE];
  uint64_t full[NSTAGE], empty[NSTAGE], done;
  uint32_t tmem;
  int abort;
};
constexpr size_t kTcSmem = sizeof(TcShared);

// float offset of element (row r, k c) of a K-major no-swizzle tile with `rows` rows
__device__ __forceinline__ int kmaj_off(int r, int c, int rows) {
  return (c >> 3) * (rows * 8) + (r >> 3) * 64 + ((c & 7) >> 2) * 32 + (r & 7) * 4 + (c & 3);
}

// Split four consecutive-k values of one row and store them as 16-byte
// vectors (a core-matrix row holds exactly 4 consecutive k).
__device__ __forceinline__ void put4(float *hi, float *lo, int off, float a, float b, float c, float d) {
  const float4 h = make_float4(tc::to_tf32(a), tc::to_tf32(b), tc::to_tf32(c), tc::to_tf32(d));
  *reinterpret_cast<float4 *>(hi + off) = h;
  *reinterpret_cast<float4 *>(lo + off) =
      make_float4(tc::to_tf32(a - h.x), tc::to_tf32(b - h.y), tc::to_tf32(c - h.z), tc::to_tf32(d - h.w));
}

// B operand (64 real columns = 32 complex RHS) of a chunk: thread t stages
// column nn = t % 64 for the 8 consecutive k = 8 (t / 64) + 0..7.
template <class RowPtr>
__device__ __forceinline__ void stage_b(Stage &s, const float *X, int k0, int kmax, int nrhs, int ch, int ncols,
                                        RowPtr row_of, int tid) {
  const int nn = tid & 63, cb = (tid >> 6) * 8;
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int c = k0 + cb + j;
    v[j] = (c < kmax && (nn >> 1) < ncols) ? X[2 * (int64_t(row_of(c)) * nrhs + ch * 32) + nn] : 0.f;
  }
  put4(s.B[0], s.B[1], kmaj_off(nn, cb, TBN), v[0], v[1], v[2], v[3]);
  put4(s.B[0], s.B[1], kmaj_off(nn, cb + 4, TBN), v[4], v[5], v[6], v[7]);
}

// Forward operand geometry: A = L21 rows i0..i0+63 (real rows 2i+a), K =
// pivot columns; B = X pivot rows.
struct FwdOps {
  const float *A;   // float view of L21 (column c at 2 (c n + i0))
  const float *X;
  int64_t n;
  int i0, b, k, c0, nrhs, ch, ncols;
  __device__ int kdim() const { return k; }
  __device__ void stage(Stage &s, int k0, int tid) const {
    // thread t owns real row r = t for all TKC k of the chunk
    const int r = tid;
    const bool rok = i0 + (r >> 1) < b;
    float v[TKC];
#pragma unroll
    for (int c = 0; c < TKC; c++)
      v[c] = (rok && k0 + c < k) ? A[2 * (int64_t(k0 + c) * n + i0) + r] : 0.f;
#pragma unroll
    for (int g = 0; g < TKC; g += 4) put4(s.A[0], s.A[1], kmaj_off(r, g, TBM), v[g], v[g + 1], v[g + 2], v[g + 3]);
    const int cbase = c0;
    stage_b(s, X, k0, k, nrhs, ch, ncols, [cbase](int c) { return cbase + c; }, tid);
  }
};

// Backward operand geometry: A = L21 columns cb..cb+63 transposed (real
// rows 2c+a), K = update rows; B = X at the update rows.
struct BwdOps {
  const float *L;   // float view of the front block (column c at 2 c n)
  const float *X;
  const int32_t *urow;
  int64_t n;
  int cb, b, k, nrhs, ch, ncols;
  __device__ int kdim() const { return b; }
  __device__ void stage(Stage &s, int k0, int tid) const {
    // thread t owns real row r = t = 2c + a for all TKC update rows of the chunk
    const int r = tid, c = cb + (r >> 1), a = r & 1;
    const bool cok = c < k;
    const float *col = L + 2 * (int64_t(c) * n + k) + a;
    float v[TKC];
#pragma unroll
    for (int i = 0; i < TKC; i++) v[i] = (cok && k0 + i < b) ? col[2 * (k0 + i)] : 0.f;
#pragma unroll
    for (int g = 0; g < TKC; g += 4) put4(s.A[0], s.A[1], kmaj_off(r, g, TBM), v[g], v[g + 1], v[g + 2], v[g + 3]);
    const int32_t *ur = urow;
    stage_b(s, X, k0, b, nrhs, ch, ncols, [ur](int i) { return ur[i]; }, tid);
  }
};

// Runs the pipeline; returns true (on the producer threads) when the
// accumulator in TMEM holds the whole product.
template <class Ops>
__device__ bool run_pipeline(TcShared &sh, const Ops &ops, DevStatus *st) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunks = (ops.kdim() + TKC - 1) / TKC;
  if (warp < 4) {
    for (int c = 0; c < nchunks; c++) {
      const int s = c % NSTAGE, round = c / NSTAGE;
      if (round > 0 && !tc::mbar_wait_or_abort(&sh.empty[s], (round - 1) & 1, kWaitIter, &sh.abort)) {
        sh.abort = 1;
        atomicExch(&st->tc_timeout, 1);
        break;
      }
      ops.stage(sh.st[s], c * TKC, tid);
      tc::fence_async_smem();
      tc::mbar_arrive(&sh.full[s]);
    }
  } else if (lane == 0) {
    const uint32_t idesc = tc::idesc_tf32(TBM, TBN);
    for (int c = 0; c < nchunks; c++) {
      const int s = c % NSTAGE, round = c / NSTAGE;
      if (!tc::mbar_wait_or_abort(&sh.full[s], round & 1, kWaitIter, &sh.abort)) {
        sh.abort = 1;
        atomicExch(&st->tc_timeout, 1);
        break;
      }
      tc::fence_after();
      Stage &S = sh.st[s];
#pragma unroll
      for (int ks = 0; ks < TKC / 8; ks++) {
        const uint64_t ah = tc::desc_kmajor(tc::smem_addr(&S.A[0][ks * TBM * 8]), 128, 256);
        const uint64_t al = tc::desc_kmajor(tc::smem_addr(&S.A[1][ks * TBM * 8]), 128, 256);
        const uint64_t bh = tc::desc_kmajor(tc::smem_addr(&S.B[0][ks * TBN * 8]), 128, 256);
        const uint64_t bl = tc::desc_kmajor(tc::smem_addr(&S.B[1][ks * TBN * 8]), 128, 256);
        tc::mma_tf32(sh.tmem, ah, bh, idesc, !(c == 0 && ks == 0));
        tc::mma_tf32(sh.tmem, ah, bl, idesc, true);
        tc::mma_tf32(sh.tmem, al, bh, idesc, true);
      }
      tc::commit(&sh.empty[s]);
    }
    tc::commit(&sh.done);   // arrives when every MMA issued above has completed
  }
  if (warp >= 4) return false;
  if (nchunks == 0) return false;
  const bool ok = tc::mbar_wait_or_abort(&sh.done, 0, kWaitIter, &sh.abort) && !sh.abort;
  if (!ok) atomicExch(&st->tc_timeout, 1);
  tc::fence_after();
  return ok;
}

__device__ __forceinline__ void setup(TcShared &sh) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 4) tc::tmem_alloc(&sh.tmem, TBN);
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; s++) {
      tc::mbar_init(&sh.full[s], NPROD);
      tc::mbar_init(&sh.empty[s], 1);
    }
    tc::mbar_init(&sh.done, 1);
    sh.abort = 0;
    tc::fence_async_smem();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

__device__ __forceinline__ void teardown(TcShared &sh) {
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if ((threadIdx.x >> 5) == 4) tc::tmem_dealloc(sh.tmem, TBN);
}

// The even lane of each (re, im) row pair gets the complex results of RHS j:
// cre[j], cim[j] (j < 32).  Executed by whole warps 0-3.
__device__ __forceinline__ void read_complex(uint32_t tmem, int warp, float *cre, float *cim) {
#pragma unroll
  for (int cb = 0; cb < TBN; cb += 16) {
    float v[16];
    tc::tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + cb, v);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const float p0 = v[2 * q], p1 = v[2 * q + 1];            // P[r][2j], P[r][2j+1]
      const float o0 = __shfl_xor_sync(0xffffffffu, p0, 1);     // partner row (im of L)
      const float o1 = __shfl_xor_sync(0xffffffffu, p1, 1);
      const int j = cb / 2 + q;
      cre[j] = p0 - o1;
      cim[j] = p1 + o0;
    }
  }
}
}  // namespace

// Forward: Y[rows_i] -= sum_c L21[i][c] X[c0 + c] for 64 update rows i.
__global__ void __launch_bounds__(160) k_fwd_l21_tc(const c64 *__restrict__ L, int64_t lstride,
                                                    const FrontDev *__restrict__ F,
                                                    const int2 *__restrict__ tasks,
                                                    const int32_t *__restrict__ rows, c64 *__restrict__ Y,
                                                    const c64 *__restrict__ X, int64_t vstride, int nrhs,
                                                    int nchunk, const int *__restrict__ pmap,
                                                    DevStatus *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TcShared &sh = *reinterpret_cast<TcShared *>(smem_raw);
  const int2 t = tasks[blockIdx.x];
  const FrontDev f = F[t.x];
  const int p = pole_of(blockIdx.y / nchunk, pmap), ch = blockIdx.y % nchunk;
  FwdOps ops;
  ops.A = reinterpret_cast<const float *>(L + p * lstride + f.lofs + f.k);
  ops.X = reinterpret_cast<const float *>(X + p * vstride);
  ops.n = f.n;
  ops.i0 = t.y * (TBM / 2);
  ops.b = f.n - f.k;
  ops.k = f.k;
  ops.c0 = f.c0;
  ops.nrhs = nrhs;
  ops.ch = ch;
  ops.ncols = min(32, nrhs - ch * 32);
  setup(sh);
  const bool ok = run_pipeline(sh, ops, st);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (ok) {
    float cre[32], cim[32];
    read_complex(sh.tmem, warp, cre, cim);
    const int r = warp * 32 + lane;
    const int i = ops.i0 + (r >> 1);
    if ((r & 1) == 0 && i < ops.b) {
      const int32_t g = rows[f.rows_off + i];
      c64 *y = Y + p * vstride + int64_t(g) * nrhs + ch * 32;
      for (int j = 0; j < ops.ncols; j++) atomic_add_cx(y + j, mk<float>(-cre[j], -cim[j]));
    }
  }
  teardown(sh);
}

// Backward: W[c0 + c] = X[c0 + c] / D_c - sum_i L21[i][c] X[rows_i] for 64 pivot columns c.
__global__ void __launch_bounds__(160) k_bwd_l21_tc(const c64 *__restrict__ L, int64_t lstride,
                                                    const FrontDev *__restrict__ F,
                                                    const int2 *__restrict__ tasks,
                                                    const int32_t *__restrict__ rows, c64 *__restrict__ Y,
                                                    const c64 *__restrict__ X, int64_t vstride, int nrhs,
                                                    int nchunk, const int *__restrict__ pmap,
                                                    DevStatus *st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TcShared &sh = *reinterpret_cast<TcShared *>(smem_raw);
  const int2 t = tasks[blockIdx.x];
  const FrontDev f = F[t.x];
  const int p = pole_of(blockIdx.y / nchunk, pmap), ch = blockIdx.y % nchunk;
  const c64 *Lp = L + p * lstride + f.lofs;
  BwdOps ops;
  ops.L = reinterpret_cast<const float *>(Lp);
  ops.X = reinterpret_cast<const float *>(X + p * vstride);
  ops.urow = rows + f.rows_off;
  ops.n = f.n;
  ops.cb = t.y * (TBM / 2);
  ops.b = f.n - f.k;
  ops.k = f.k;
  ops.nrhs = nrhs;
  ops.ch = ch;
  ops.ncols = min(32, nrhs - ch * 32);
  setup(sh);
  const bool ok = run_pipeline(sh, ops, st);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp < 4 && (ok || ops.b == 0) && !sh.abort) {
    float cre[32], cim[32];
    if (ops.b > 0) {
      read_complex(sh.tmem, warp, cre, cim);
    } else {
#pragma unroll
      for (int j = 0; j < 32; j++) cre[j] = cim[j] = 0.f;
    }
    const int r = warp * 32 + lane;
    const int c = ops.cb + (r >> 1);
    if ((r & 1) == 0 && c < f.k) {
      const c64 dinv = crecip(Lp[int64_t(c) * f.n + c]);
      const int64_t at = p * vstride + int64_t(f.c0 + c) * nrhs + ch * 32;
      for (int j = 0; j < ops.ncols; j++) Y[at + j] = X[at + j] * dinv - mk<float>(cre[j], cim[j]);
    }
  }
  teardown(sh);
}

namespace {
void set_smem_once() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_fwd_l21_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
  cudaFuncSetAttribute(k_bwd_l21_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
  done = true;
}
}  // namespace

void launch_fwd_l21_tc(const SolvePlan<float> &P, const LevelDev &lv, DevStatus *st, cudaStream_t s) {
  set_smem_once();
  const int nchunk = (P.nrhs + 31) / 32;
  dim3 g(lv.n_f21tc, P.np * nchunk);
  tem::count_launch();
  k_fwd_l21_tc<<<g, 160, kTcSmem, s>>>(P.L, P.lstride, P.F, lv.f21tc_tasks, P.rows, P.Y, P.X, P.vstride, P.nrhs,
                                        nchunk, P.pmap, st);
}

void launch_bwd_l21_tc(const SolvePlan<float> &P, const LevelDev &lv, DevStatus *st, cudaStream_t s) {
  set_smem_once();
  const int nchunk = (P.nrhs + 31) / 32;
  dim3 g(lv.n_b21tc, P.np * nchunk);
  tem::count_launch();
  k_bwd_l21_tc<<<g, 160, kTcSmem, s>>>(P.L, P.lstride, P.F, lv.b21tc_tasks, P.rows, P.Y, P.X, P.vstride, P.nrhs,
                                        nchunk, P.pmap, st);
}

}  // namespace tem
