// Front products of the FP32 solves (Algorithm 1: solve with the cached
// factors).  With the pivot blocks stored as their explicit inverses
// T11 = L11^-1, every step of both sweeps is a product of a factor block with
// the 32 right-hand sides of one pole (modes in kernels.h):
//   forward, per level:  TRI_F (X_piv = T11 Y_piv), FWD21 (Y_upd -= L21 X_piv)
//   backward, per level: BWD21 (Y_piv = D^-1 X_piv - L21^T X_upd), TRI_B (X_piv = T11^T Y_piv)
//
// Tensor-core kernel (k_tc_kint): one persistent CTA per SM slot (two per
// SM) walks a static list of (tile, pole, RHS chunk) items; each item is 128
// output indices (TMEM lanes) x 32 right-hand sides, streamed over its inner
// dimension in chunks of 16 complex values.  Both operands are split into
// TF32 hi + lo parts and three MMAs (hi.hi + hi.lo + lo.hi, kind::tf32, FP32
// accumulation) give FP32 accuracy; the factor's hi part is the raw FP32
// value itself (the tensor core truncates its inputs to TF32), so only lo is
// formed.  Roles:
//   warp 9    (loader) issues the TMA loads of each chunk (the factor box
//              from the front's tensor map, the B rows from the vector's map)
//              into a ring of slots once the MMAs have freed the slot;
//   warps 0-3  (producers) form the factor's lo part (into TMEM, thread =
//              lane) and the B operand's hi / lo parts (shared memory);
//   warp 8     issues the MMAs (factor hi from the slot, lo from TMEM, B
//              from shared memory) into one of two TMEM accumulators;
//   warps 4-7  (epilogue) read the accumulator of the previous item and
//              store / atomically subtract while the next item accumulates.
// Every wait is bounded: a wait that gives up raises the CTA's abort flag and
// the status word, all roles wind down, the MMA issuer drains its
// outstanding MMAs, in-flight loads land and the TMEM is released.
//
// The SIMT kernel (k_prod_simt) computes the same products on the FP32 pipes.
#include <atomic>
#include <cstring>
#include <cuda.h>   // CUtensorMap and the encoder's signature (called through the runtime's entry point)

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace tem {

namespace {
constexpr int NTHR = 320;     // 4 producer + 4 epilogue warps, MMA issuer (warp 8), TMA loader (warp 9)
constexpr uint32_t kWaitIter = 1u << 26;
constexpr unsigned kFull = 0xffffffffu;

// modes whose factor operand is read along its columns in the column-major
// store (the SIMT kernel; the tensor-core kernel reads the row-major copies
// for the other two)
__host__ __device__ constexpr bool row_major(int mode) { return mode == PM_BWD21 || mode == PM_TRI_B; }
// the SIMT kernel gathers BWD21's B rows itself; the tensor-core kernel reads them pre-gathered
__host__ __device__ constexpr bool gathered_b(int mode) { return mode == PM_BWD21; }

struct ProdArgs {
  const c64 *L;
  int64_t lstride;
  const TcTask *tasks;
  int ntask;         // tensor-core tiles (128 wide)
  int ntask_simt;    // SIMT tiles (64 wide)
  const int32_t *rows;
  const c64 *B;      // source of the B rows
  c64 *out;          // destination
  const c64 *xaux;   // BWD21: X (the D^-1 X term)
  const c64 *dinv;   // BWD21: [pole][N]
  const CUtensorMap *tmaps;
  const CUtensorMap *bmap;   // B rows by TMA
  int64_t N;
  int64_t vstride;   // pole stride of the outputs (and of B, except BWD21 on the tensor cores)
  int nrhs, nchunk, np;
  const int *pmap;
  DevStatus *st;
  uint32_t wait_iter;   // limits of the pipeline waits (polls, ns); the drains after an abort keep the defaults
  uint64_t wait_ns;
  // PM_UPD (trailing update of the factorisation): fronts, factor store and update arena
  const FrontDev *F;
  c64 *Lw;
  c64 *Uw;
  int64_t ustride;
};

// An item: task of pole p, RHS chunk ch (items are numbered per CTA).
struct Item {
  TcTask t;
  int p, ch, nch;
  bool valid;
};

// Item j of this CTA.  Items are the (task, pole, RHS chunk) triples; a
// level's tasks are stored in decreasing length, and the CTAs take the items
// in snake order (round j: position j G + b, or j G + G - 1 - b on odd
// rounds), which balances items of very different lengths over the grid.
__device__ __forceinline__ Item load_item(const ProdArgs &a, int j) {
  Item it;
  const int64_t G = gridDim.x, per = int64_t(a.np) * a.nchunk;
  const int64_t pos = int64_t(j) * G + ((j & 1) ? G - 1 - blockIdx.x : blockIdx.x);
  it.valid = pos < int64_t(a.ntask) * per;
  int q = 0, ti = 0;
  if (it.valid) {
    const int64_t r = pos / per;
    q = int(pos - r * per);
    ti = int(r);
  }
  if (!it.valid) {
    it.nch = 0;
    it.p = it.ch = 0;
    it.t = TcTask{0, 0, 0, 0, 0, 0, 0, 0, 0};
    return it;
  }
  const int ps = q / a.nchunk;
  it.ch = q - ps * a.nchunk;
  it.p = pole_of(ps, a.pmap);
  const int4 *src = reinterpret_cast<const int4 *>(a.tasks + ti);
  const int4 w0 = __ldg(src), w1 = __ldg(src + 1);
  it.t.map = w0.x;
  it.t.x0 = w0.y;
  it.t.y0 = w0.z;
  it.t.kdim = w0.w;
  it.t.mrows = w1.x;
  it.t.bbase = w1.y;
  it.t.obase = w1.z;
  it.t.mfirst = int16_t(w1.w & 0xffff);
  it.t.kfirst = int16_t(uint32_t(w1.w) >> 16);
  it.nch = 0;
  return it;
}

// float offset of element (row r, k c) of a K-major no-swizzle tile with `rows` rows
__device__ __forceinline__ int kmaj_off(int r, int c, int rows) {
  return (c >> 3) * (rows * 8) + (r >> 3) * 64 + ((c & 7) >> 2) * 32 + (r & 7) * 4 + (c & 3);
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away
// from zero, on the integer pipe: adding half a TF32 unit to the magnitude
// bits carries into bit 13 exactly when the dropped 13 bits are >= half
// (IEEE-754 binary32 layout; a carry out of the mantissa moves to the next
// binade).  Finite inputs.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

__device__ __forceinline__ void split4(float *hi, float *lo, int off, const float *v) {
  const float4 h = make_float4(tf32_rna(v[0]), tf32_rna(v[1]), tf32_rna(v[2]), tf32_rna(v[3]));
  *reinterpret_cast<float4 *>(hi + off) = h;
  *reinterpret_cast<float4 *>(lo + off) = make_float4(tf32_rna(v[0] - h.x), tf32_rna(v[1] - h.y),
                                                      tf32_rna(v[2] - h.z), tf32_rna(v[3] - h.w));
}
}  // namespace

// ---------------------------------------------------------------------------
// Tensor-core products with the inner dimension interleaved.  The operand
// is read along contiguous runs: BWD21 and TRI_B along a column of the
// column-major store (their output index is the pivot column), TRI_F and
// FWD21 along a row of the row-major copies of T11 and L21 (their output
// index is the row).  One output index is one TMEM lane and its run of
// complex inner indices i gives real inner indices (i, re) and (i, im), so
// the raw TMA box of 128 runs x 16 complex values (128-byte rows, 128-byte
// swizzle) is already a K-major operand.  The tensor core reads it directly
// as the TF32 hi part (it truncates FP32 inputs to TF32, so hi = the raw
// value and lo = x - trunc(x) exactly); the producers compute only lo (into
// TMEM) and the B operand X^ of the real embedding:
//   X^[(i, 0)][(j, re)] = Re X(i,j),  X^[(i, 1)][(j, re)] = -Im X(i,j),
//   X^[(i, 0)][(j, im)] = Im X(i,j),  X^[(i, 1)][(j, im)] =  Re X(i,j),
// so that lane c of the accumulator holds (re, im) of sum_i A(i,c) X(i,j)
// for the 32 right-hand sides j, without a lane-pair combine.

namespace {
constexpr int KI_K = 16;         // complex inner indices per chunk (32 real, four MMA k-steps)
constexpr int KI_SLOTS = 3;
constexpr uint32_t KI_TMEM = 256;
constexpr uint32_t KI_COL_LO = 128;   // lo stages after the two 64-column accumulators

struct KiSlot {
  float A[128 * 32];          // raw A box: 128 columns x 32 floats, 128-byte swizzle (16 KB)
  float Xr[KI_K * 64];        // raw B rows: 16 rows x 64 floats (4 KB)
  float Bh[64 * 32];          // X^ hi, K-major core matrices (8 KB)
  float Bl[64 * 32];          // X^ lo
};
struct KiShared {
  KiSlot sl[KI_SLOTS];
  uint64_t rawfull[KI_SLOTS], full[KI_SLOTS], freeb[KI_SLOTS], accf[2], acce[2], fin;
  int kval[KI_SLOTS], kfst[KI_SLOTS];
  uint32_t tmem;
  int abort;
};
constexpr size_t kKiSmem = sizeof(KiShared) + 1024;

// A pipeline wait; one that gives up raises the CTA's abort flag and the
// status word.  Every role then stops issuing; the loader waits for its TMA
// loads in flight and the MMA issuer for its MMAs (with the default limits)
// before the CTA frees its TMEM and exits.
__device__ __forceinline__ bool ki_wait(const ProdArgs &a, KiShared &sh, uint64_t *bar, uint32_t parity) {
  if (tc::mbar_wait_or_abort(bar, parity, a.wait_iter, &sh.abort, a.wait_ns)) return true;
  sh.abort = 1;
  atomicExch(&a.st->tc_timeout, 1);
  return false;
}

// Every role loads the descriptor of its next item at the start of the
// current one and takes the chunk count only when the item begins, so the
// load latency overlaps the current item's work.
__device__ __forceinline__ Item ki_item(const ProdArgs &a, int j) { return load_item(a, j); }
__device__ __forceinline__ Item ki_begin(const Item &nxt) {
  Item it = nxt;
  it.nch = (it.t.kdim + KI_K - 1) / KI_K;
  return it;
}

// Rows of the row-gather map (pole p's block of X) that feed inner indices
// k0 + 4q .. k0 + 4q + 3 of a BWD21 item: X row rows[bbase + kk]; indices
// outside [kfirst, kdim) repeat a valid row (the producers zero them).
__device__ __forceinline__ int4 ki_gather_rows(const ProdArgs &a, const Item &it, int k0, int q) {
  const TcTask &t = it.t;
  if (t.kdim <= int(t.kfirst)) return make_int4(0, 0, 0, 0);   // no update rows: no chunks, nothing loaded
  const int base = it.p * int(a.N);   // m * N < 2^31 (checked when the map is built)
  int r[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const int kk = min(max(k0 + 4 * q + e, int(t.kfirst)), t.kdim - 1);
    r[e] = base + __ldg(a.rows + t.bbase + kk);
  }
  return make_int4(r[0], r[1], r[2], r[3]);
}

// Loader (warp 9, a warp of its own so that its waits never hold up the MMA
// issue): the TMA loads of every chunk, in order, into slot gc % KI_SLOTS as
// soon as the MMAs of the slot's previous chunk are done.  Lane 0 loads the
// factor box and (except for BWD21) the 16 contiguous B rows; for BWD21 lanes
// 0-3 each gather four B rows of X, whose indices they fetch one chunk ahead.
template <int MODE>
__device__ void ki_loader(const ProdArgs &a, KiShared &sh, int lane) {
  constexpr bool kGather = MODE == PM_BWD21;
  int gc = 0;
  bool ok = true;
  Item nxt = ki_item(a, 0);
  int4 rnext = make_int4(0, 0, 0, 0);
  if (kGather && lane < 4 && nxt.valid) rnext = ki_gather_rows(a, nxt, 0, lane);
#pragma unroll 1
  for (int j = 0; ok; j++) {
    if (!nxt.valid) break;
    const Item it = ki_begin(nxt);
    nxt = ki_item(a, j + 1);
    const TcTask &t = it.t;
#pragma unroll 1
    for (int c = 0; c < it.nch; c++, gc++) {
      const int slot = gc % KI_SLOTS;
      const int4 rows = rnext;
      if (kGather && lane < 4) {
        if (c + 1 < it.nch) rnext = ki_gather_rows(a, it, (c + 1) * KI_K, lane);
        else if (nxt.valid) rnext = ki_gather_rows(a, nxt, 0, lane);
      }
      bool free = true;
      if (gc >= KI_SLOTS) {
        if (lane == 0) free = ki_wait(a, sh, &sh.freeb[slot], ((gc / KI_SLOTS) - 1) & 1);
        free = __shfl_sync(kFull, free, 0);
      }
      if (!free) {
        ok = false;
        break;
      }
      const int k0 = c * KI_K;
      if (lane == 0) {
        sh.kval[slot] = min(KI_K, t.kdim - k0);
        sh.kfst[slot] = max(0, int(t.kfirst) - k0);
        tc::mbar_arrive_expect_tx(&sh.rawfull[slot], (128 * 32 + KI_K * 64) * 4);
        if (MODE == PM_UPD) {
          // A: rows of the panel copy; B: columns j0 + k0 .. of the factor store, rows s0 .. s0 + 31
          tc::tma_load_3d(sh.sl[slot].A, a.bmap, 2 * k0, t.x0 + t.y0, it.p, &sh.rawfull[slot]);
          tc::tma_load_3d(sh.sl[slot].Xr, a.tmaps + t.map, 2 * t.bbase, t.obase + k0, it.p, &sh.rawfull[slot]);
        } else {
          tc::tma_load_3d(sh.sl[slot].A, a.tmaps + t.map, t.x0 + 2 * k0, t.y0, it.p, &sh.rawfull[slot]);
          if (!kGather) tc::tma_load_3d(sh.sl[slot].Xr, a.bmap, 64 * it.ch, t.bbase + k0, it.p, &sh.rawfull[slot]);
        }
      }
      if (kGather) {
        __syncwarp();   // the slot's byte count is posted before its row gathers are issued
        if (lane < 4) tc::tma_gather4(sh.sl[slot].Xr + lane * 4 * 64, a.bmap, 64 * it.ch, rows, &sh.rawfull[slot]);
      }
    }
  }
  // after an abort: let the loads still in flight land before the CTA exits
  if (!ok && lane == 0)
    for (int q = max(0, gc - KI_SLOTS); q < gc; q++) tc::mbar_wait(&sh.rawfull[q % KI_SLOTS], (q / KI_SLOTS) & 1, kWaitIter);
}

template <int MODE>
__device__ void ki_producer(const ProdArgs &a, KiShared &sh, int tid) {
  const int w = tid >> 5, l = tid & 31;
  int g = 0;
  bool ok = true;
  Item nxt = ki_item(a, 0);
#pragma unroll 1
  for (int j = 0; ok; j++) {
    if (!nxt.valid) break;
    const Item it = ki_begin(nxt);
    nxt = ki_item(a, j + 1);
    // PM_UPD: the B operand is D_c L[s][c]; D_c sits on the diagonal of the factor block
    const c64 *dg = nullptr;
    int64_t dstep = 0;
    if (MODE == PM_UPD && it.nch > 0) {
      const FrontDev f = a.F[it.t.map];
      dstep = int64_t(f.ld) + 1;
      dg = a.L + int64_t(it.p) * a.lstride + f.lofs + int64_t(it.t.obase) * dstep;
    }
#pragma unroll 1
    for (int c = 0; c < it.nch; c++, g++) {
      const int slot = g % KI_SLOTS;
      ok = ki_wait(a, sh, &sh.rawfull[slot], (g / KI_SLOTS) & 1);
      if (!__all_sync(kFull, ok)) {
        ok = false;
        break;
      }
      KiSlot &S = sh.sl[slot];
      // lo of factor column tid: its 32 floats, 16-byte chunks swizzled by tid & 7
      {
        float v[32];
        const float4 *row = reinterpret_cast<const float4 *>(S.A + tid * 32);
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const float4 x = row[q ^ (tid & 7)];
          v[4 * q] = x.x;
          v[4 * q + 1] = x.y;
          v[4 * q + 2] = x.z;
          v[4 * q + 3] = x.w;
        }
#pragma unroll
        for (int q = 0; q < 32; q++) {
          const float h = __uint_as_float(__float_as_uint(v[q]) & 0xffffe000u);   // what the MMA reads of v
          v[q] = tf32_rna(__fsub_rn(v[q], h));
        }
        tc::tmem_st32(sh.tmem + (uint32_t(w * 32) << 16) + KI_COL_LO + 32 * slot, v);
      }
      // X^ row n = l and n = 32 + l (right-hand side n / 2, re row if n even):
      // inner indices 8w..8w+7 = complex rows i = 4w..4w+3
      {
        const int kv = sh.kval[slot], kf = sh.kfst[slot];
        c64 dq[4];
        if (MODE == PM_UPD) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int i = 4 * w + q;
            dq[q] = i < kv ? dg[int64_t(c * KI_K + i) * dstep] : mk<float>(0.f, 0.f);
          }
        }
#pragma unroll
        for (int half = 0; half < 2; half++) {
          const int n = 32 * half + l, jr = n >> 1;
          float r[8];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int i = 4 * w + q;
            const float2 x = *reinterpret_cast<const float2 *>(S.Xr + i * 64 + 2 * jr);
            const bool in = i < kv && i >= kf;
            float re = in ? x.x : 0.f, im = in ? x.y : 0.f;
            if (MODE == PM_UPD) {
              const c64 dx = dq[q] * mk<float>(re, im);
              re = dx.x;
              im = dx.y;
            }
            r[2 * q] = (n & 1) ? im : re;
            r[2 * q + 1] = (n & 1) ? re : -im;
          }
          split4(S.Bh, S.Bl, kmaj_off(n, 8 * w, 64), r);
          split4(S.Bh, S.Bl, kmaj_off(n, 8 * w + 4, 64), r + 4);
        }
      }
      tc::tmem_st_wait();
      tc::fence_async_smem();
      tc::fence_before();
      tc::mbar_arrive(&sh.full[slot]);
      if (__any_sync(kFull, *reinterpret_cast<volatile int *>(&sh.abort) != 0)) {
        ok = false;
        break;
      }
    }
  }
}

__device__ void ki_mma(const ProdArgs &a, KiShared &sh) {
  const uint32_t idesc = tc::idesc_tf32(128, 64);
  int g = 0;
  bool ok = true;
  Item nxt = ki_item(a, 0);
#pragma unroll 1
  for (int j = 0; ok; j++) {
    if (!nxt.valid) break;
    const Item it = ki_begin(nxt);
    nxt = ki_item(a, j + 1);
    const int buf = j & 1, use = j >> 1;
    if (use > 0 && !ki_wait(a, sh, &sh.acce[buf], (use - 1) & 1)) break;
    tc::fence_after();
    const uint32_t d = sh.tmem + 64 * buf;
#pragma unroll 1
    for (int c = 0; c < it.nch; c++, g++) {
      const int slot = g % KI_SLOTS;
      if (!ki_wait(a, sh, &sh.full[slot], (g / KI_SLOTS) & 1)) {
        ok = false;
        break;
      }
      tc::fence_after();
      const KiSlot &S = sh.sl[slot];
#pragma unroll
      for (int ks = 0; ks < 4; ks++) {
        const uint64_t ah = tc::desc_kmajor_sw128(tc::smem_addr(S.A) + 32 * ks, 1024);
        const uint32_t al = sh.tmem + KI_COL_LO + 32 * slot + 8 * ks;
        const uint64_t bh = tc::desc_kmajor(tc::smem_addr(&S.Bh[ks * 64 * 8]), 128, 256);
        const uint64_t bl = tc::desc_kmajor(tc::smem_addr(&S.Bl[ks * 64 * 8]), 128, 256);
        tc::mma_tf32(d, ah, bh, idesc, c > 0 || ks > 0);
        tc::mma_tf32(d, ah, bl, idesc, true);
        tc::mma_tf32_ts(d, al, bh, idesc, true);
      }
      tc::commit(&sh.freeb[slot]);   // the slot (and its lo stage) is free once these MMAs are done
    }
    if (!ok) break;
    tc::commit(&sh.accf[buf]);
  }
  tc::commit(&sh.fin);
  if (!tc::mbar_wait(&sh.fin, 0, kWaitIter)) atomicExch(&a.st->tc_timeout, 1);
}

// lane e = pivot column m of the tile: (re, im) of the 32 right-hand sides
template <int MODE>
__device__ void ki_epilogue(const ProdArgs &a, KiShared &sh, int e) {
  const int we = e >> 5;
  Item nxt = ki_item(a, 0);
#pragma unroll 1
  for (int j = 0;; j++) {
    if (!nxt.valid) break;
    const Item it = ki_begin(nxt);
    nxt = ki_item(a, j + 1);
    const int buf = j & 1, use = j >> 1;
    const bool ok = ki_wait(a, sh, &sh.accf[buf], use & 1);
    if (!__all_sync(kFull, ok)) break;
    tc::fence_after();
    if constexpr (MODE == PM_UPD) {
      // F[r][s] -= acc for the tile's columns s >= t0 with r >= s, r = row m of the tile (lane),
      // as an atomic add of -acc: every entry is updated by exactly one item of a launch, so
      // the result is the same as load, subtract, store (o + (-v) == o - v), but nothing waits
      // for the load (the L2 does the update), which a read-modify-write per column did at
      // one memory latency per batch.  The accumulator is read in two halves of 16 columns.
      const int m = e;
      const FrontDev f = a.F[it.t.map];
      const int64_t r = int64_t(it.t.y0) + m, k = f.k, n = f.n;
      c64 *lp = a.Lw + int64_t(it.p) * a.lstride + f.lofs;
      c64 *up = a.Uw + int64_t(it.p) * a.ustride + f.uofs;
      const int q0 = int(it.t.mfirst);
      const bool row_ok = m < it.t.mrows;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        float v[32];
        if (it.nch > 0) {
          tc::tmem_ld16(sh.tmem + (uint32_t(we * 32) << 16) + 64 * buf + 32 * h, v);
          tc::tmem_ld16(sh.tmem + (uint32_t(we * 32) << 16) + 64 * buf + 32 * h + 16, v + 16);
        } else {
#pragma unroll
          for (int q = 0; q < 32; q++) v[q] = 0.f;
        }
        if (!row_ok) continue;
#pragma unroll
        for (int x = 0; x < 16; x++) {
          const int q = 16 * h + x;
          const int64_t sc = int64_t(it.t.bbase) + q;
          if (q < q0 || sc >= n || sc > r) continue;
          c64 *dst = sc < k ? lp + sc * f.ld + r : up + (sc - k) * (n - k) + (r - k);
          atomicAdd(reinterpret_cast<float2 *>(dst), make_float2(-v[2 * x], -v[2 * x + 1]));
        }
      }
      tc::fence_before();
      tc::mbar_arrive(&sh.acce[buf]);
      continue;
    }
    float v[64];
    if (it.nch > 0) {
      tc::tmem_ld64(sh.tmem + (uint32_t(we * 32) << 16) + 64 * buf, v);
    } else {
#pragma unroll
      for (int q = 0; q < 64; q++) v[q] = 0.f;
    }
    tc::fence_before();
    tc::mbar_arrive(&sh.acce[buf]);
    const int m = e;
    if (m >= it.t.mrows) continue;

    const int ncols = min(32, a.nrhs - it.ch * 32);
    const int64_t pv = int64_t(it.p) * a.vstride + it.ch * 32;
    const int64_t row = MODE == PM_FWD21 ? int64_t(__ldg(a.rows + it.t.obase + m)) : int64_t(it.t.obase) + m;
    // rows start on 16-byte boundaries (even nrhs): two right-hand sides per access
    float4 *y = reinterpret_cast<float4 *>(a.out + pv + row * a.nrhs);
    if (MODE == PM_FWD21) {
#pragma unroll
      for (int q = 0; q < 16; q++)
        if (2 * q < ncols) atomicAdd(y + q, make_float4(-v[4 * q], -v[4 * q + 1], -v[4 * q + 2], -v[4 * q + 3]));
    } else if (MODE == PM_BWD21) {
      const c64 di = a.dinv[int64_t(it.p) * a.N + row];
      const float4 *x = reinterpret_cast<const float4 *>(a.xaux + pv + row * a.nrhs);
#pragma unroll
      for (int q = 0; q < 16; q++)
        if (2 * q < ncols) {
          const float4 xv = x[q];
          const c64 d0 = di * mk<float>(xv.x, xv.y), d1 = di * mk<float>(xv.z, xv.w);
          y[q] = make_float4(d0.x - v[4 * q], d0.y - v[4 * q + 1], d1.x - v[4 * q + 2], d1.y - v[4 * q + 3]);
        }
    } else {
#pragma unroll
      for (int q = 0; q < 16; q++)
        if (2 * q < ncols) y[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
}
}  // namespace

template <int MODE>
__global__ void __launch_bounds__(NTHR, 2) k_tc_kint(const ProdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  KiShared &sh = *reinterpret_cast<KiShared *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 8) tc::tmem_alloc(&sh.tmem, KI_TMEM);
  if (tid == 0) {
    for (int s = 0; s < KI_SLOTS; s++) {
      tc::mbar_init(&sh.rawfull[s], 1);
      tc::mbar_init(&sh.full[s], 128);
      tc::mbar_init(&sh.freeb[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      tc::mbar_init(&sh.accf[b], 1);
      tc::mbar_init(&sh.acce[b], 128);
    }
    tc::mbar_init(&sh.fin, 1);
    sh.abort = 0;
    tc::fence_async_smem();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp < 4) ki_producer<MODE>(a, sh, tid);
  else if (warp < 8) ki_epilogue<MODE>(a, sh, tid - 128);
  else if (warp == 8 && (tid & 31) == 0) ki_mma(a, sh);
  else if (warp == 9) ki_loader<MODE>(a, sh, tid & 31);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 8) tc::tmem_dealloc(sh.tmem, KI_TMEM);
}

// ---------------------------------------------------------------------------
// SIMT version: one CTA per item, 256 threads, lane = right-hand side,
// warp w owns complex rows 8w..8w+7 of the 64-row tile.

template <int MODE>
__global__ void __launch_bounds__(256) k_prod_simt(const ProdArgs a, const SimtTask *__restrict__ tasks) {
  constexpr int KC = 32;
  const int ti = blockIdx.x;
  const int ps = blockIdx.y / a.nchunk, ch = blockIdx.y % a.nchunk;
  const int p = pole_of(ps, a.pmap);
  const SimtTask t = tasks[ti];
  const c64 *Lp = a.L + int64_t(p) * a.lstride + t.aoff;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rhs = ch * 32 + lane;
  const bool ok = rhs < a.nrhs;
  const int64_t pv = int64_t(p) * a.vstride;
  __shared__ c64 As[KC][65];
  __shared__ c64 Bs[KC][32];
  c64 acc[8];
#pragma unroll
  for (int q = 0; q < 8; q++) acc[q] = mk<float>(0.f, 0.f);
  for (int k0 = 0; k0 < t.kdim; k0 += KC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < KC * 64; idx += 256) {
      int m, kk;
      if (!row_major(MODE)) {
        m = idx % 64;
        kk = idx / 64;
      } else {
        kk = idx % KC;
        m = idx / KC;
      }
      const bool v = m < t.mrows && k0 + kk < t.kdim;
      const int64_t off = row_major(MODE) ? int64_t(m) * t.lda + k0 + kk : int64_t(k0 + kk) * t.lda + m;
      As[kk][m] = v ? Lp[off] : mk<float>(0.f, 0.f);
    }
    for (int kk = warp; kk < KC; kk += 8) {
      const int k = k0 + kk;
      c64 bv = mk<float>(0.f, 0.f);
      if (ok && k < t.kdim && k >= t.kfirst) {
        const int64_t row = gathered_b(MODE) ? int64_t(a.rows[t.bbase + k]) : int64_t(t.bbase) + k;
        bv = a.B[pv + row * a.nrhs + rhs];
      }
      Bs[kk][lane] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; kk++) {
      const c64 bv = Bs[kk][lane];
#pragma unroll
      for (int q = 0; q < 8; q++) cfma(acc[q], As[kk][warp * 8 + q], bv);
    }
  }
  if (!ok) return;
#pragma unroll
  for (int q = 0; q < 8; q++) {
    const int m = warp * 8 + q;
    if (m >= t.mrows) break;
    if (m < t.mfirst) continue;
    if (MODE == PM_FWD21) {
      const int64_t g = a.rows[t.obase + m];
      atomic_add_cx(a.out + pv + g * a.nrhs + rhs, mk<float>(-acc[q].x, -acc[q].y));
    } else if (MODE == PM_BWD21) {
      const int64_t row = int64_t(t.obase) + m;
      const int64_t at = pv + row * a.nrhs + rhs;
      a.out[at] = a.dinv[int64_t(p) * a.N + row] * a.xaux[at] - acc[q];
    } else {
      a.out[pv + (int64_t(t.obase) + m) * a.nrhs + rhs] = acc[q];
    }
  }
}

namespace {
int g_tc_occupancy = 0;
uint32_t g_wait_iter = kWaitIter;   // pipeline-wait limits (tests of the timeout status shorten them)
uint64_t g_wait_ns = 1000000000ull;
std::atomic<int64_t> g_tc_launches{0}, g_simt_launches{0}, g_upd_launches{0};

template <int MODE>
void run_mode(const ProdArgs &a, const SimtTask *simt, bool use_tc, cudaStream_t s) {
  if (use_tc) {
    static int grid_max = 0;
    if (grid_max == 0) {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaFuncSetAttribute(k_tc_kint<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kKiSmem));
      // all of the unified L1 / shared storage as shared memory
      cudaFuncSetAttribute(k_tc_kint<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      // Two CTAs per SM: 256 of the 512 TMEM columns, under half of the shared
      // memory and 2 x 320 x 96 registers each.  (The occupancy calculator
      // reports one for this 9-warp block; two are resident, as measured by
      // counting CTAs per SM.)
      static_assert(2 * (kKiSmem + 1024) <= 228 * 1024, "two CTAs per SM must fit in shared memory");
      g_tc_occupancy = 2;
      grid_max = 2 * (sms > 0 ? sms : 1);
    }
    const int64_t total = int64_t(a.ntask) * a.np * a.nchunk;
    const int grid = int(total < grid_max ? total : grid_max);
    tem::count_launch();
    (MODE == PM_UPD ? g_upd_launches : g_tc_launches).fetch_add(1, std::memory_order_relaxed);
    k_tc_kint<MODE><<<grid, NTHR, kKiSmem, s>>>(a);
  } else if constexpr (MODE != PM_UPD) {
    dim3 g(a.ntask_simt, a.np * a.nchunk);
    tem::count_launch();
    g_simt_launches.fetch_add(1, std::memory_order_relaxed);
    k_prod_simt<MODE><<<g, 256, 0, s>>>(a, simt);
  }
}
}  // namespace

int tc_ctas_per_sm() { return g_tc_occupancy; }
void set_tc_wait_limit(uint32_t polls, uint64_t ns) {
  g_wait_iter = polls;
  g_wait_ns = ns;
}
int64_t prod_launches(bool tensor_cores) { return (tensor_cores ? g_tc_launches : g_simt_launches).load(); }
int64_t update_launches() { return g_upd_launches.load(); }

void launch_tc_update(const FactorPlan<float> &P, const UpdBlock &ub, cudaStream_t s) {
  if (ub.ntask == 0 || P.m == 0) return;
  ProdArgs a;
  memset(&a, 0, sizeof(a));
  a.L = P.L;
  a.lstride = P.lstride;
  a.tasks = ub.tasks;
  a.ntask = ub.ntask;
  a.nrhs = 32;
  a.nchunk = 1;
  a.np = P.m;
  a.pmap = nullptr;
  a.st = P.status;
  a.wait_iter = g_wait_iter;
  a.wait_ns = g_wait_ns;
  a.tmaps = static_cast<const CUtensorMap *>(P.cmaps);   // B: per front, its column-major block
  a.bmap = static_cast<const CUtensorMap *>(P.pcmap);    // A: the panel copy
  a.F = P.F;
  a.Lw = P.L;
  a.Uw = P.U;
  a.ustride = P.ustride;
  run_mode<PM_UPD>(a, nullptr, true, s);
}

void launch_prod(int mode, const SolvePlan<float> &P, const LevelDev &lv, cudaStream_t s) {
  // The tensor-core kernel loads B rows by TMA, which needs 16-byte rows (an
  // even number of right-hand sides); otherwise the SIMT kernels run.  (It is
  // also faster than the SIMT kernel on levels of small fronts, where most of
  // a 128-lane tile is idle.)
  const bool use_tc = P.use_tc && P.vmaps != nullptr;
  if ((use_tc ? lv.n_prod[mode] : lv.n_prod_simt[mode]) == 0 || P.np == 0) return;
  ProdArgs a;
  a.L = P.L;
  a.lstride = P.lstride;
  a.tasks = lv.prod[mode];
  a.ntask = lv.n_prod[mode];
  a.ntask_simt = lv.n_prod_simt[mode];
  a.rows = P.rows;
  a.N = P.N;
  a.vstride = P.vstride;
  a.nrhs = P.nrhs;
  a.nchunk = (P.nrhs + 31) / 32;
  a.np = P.np;
  a.pmap = P.pmap;
  a.st = P.status;
  a.wait_iter = g_wait_iter;
  a.wait_ns = g_wait_ns;
  a.dinv = P.dinv;
  a.tmaps = static_cast<const CUtensorMap *>(P.tmaps);
  const CUtensorMap *vm = static_cast<const CUtensorMap *>(P.vmaps);   // [0] Y, [1] X (nullptr: odd nrhs)
  a.bmap = nullptr;
  a.xaux = nullptr;
  switch (mode) {
    case PM_TRI_F:
      a.bmap = vm ? vm : nullptr;
      a.B = P.Y;
      a.out = P.X;
      run_mode<PM_TRI_F>(a, lv.prod_simt[mode], use_tc, s);
      break;
    case PM_FWD21:
      a.bmap = vm ? vm + 1 : nullptr;
      a.B = P.X;
      a.out = P.Y;
      run_mode<PM_FWD21>(a, lv.prod_simt[mode], use_tc, s);
      break;
    case PM_BWD21:
      a.B = P.X;
      a.out = P.Y;
      a.xaux = P.X;
      // the tensor-core kernel loads the update rows of X by TMA row gathers
      a.bmap = vm ? vm + 2 : nullptr;
      run_mode<PM_BWD21>(a, lv.prod_simt[mode], use_tc, s);
      break;
    default:
      a.bmap = vm ? vm : nullptr;
      a.B = P.Y;
      a.out = P.X;
      run_mode<PM_TRI_B>(a, lv.prod_simt[mode], use_tc, s);
      break;
  }
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
}  // namespace

// Per front, four maps, each 3-D over floats (two per complex entry) with
// 128 runs x 16 complex values per box and the 128-byte swizzle; entries
// outside the dims read as zero:
//   TRI_F: rows of the row-major T11 copy (run = row, k entries, k rows),
//   FWD21: rows of the row-major L21 copy (b rows of k entries),
//   BWD21: columns of the column-major store (rows 0..n-1 of each of the k columns),
//   TRI_B: columns of the column-major store restricted to the pivot rows 0..k-1.
std::string build_tensor_maps(const std::vector<FrontGeom> &fronts, const FactorViews &v, int m, void **out) {
  *out = nullptr;
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return "cuTensorMapEncodeTiled is not available from the driver";
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  std::vector<CUtensorMap> maps(4 * fronts.size());
  memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
  for (size_t i = 0; i < fronts.size(); i++) {
    const FrontGeom &f = fronts[i];
    const int b = f.n - f.k;
    if (f.k <= 0) continue;
    for (int kind = 0; kind < 4; kind++) {
      const c64 *base;
      cuuint64_t runlen, runs, stride, pstride;
      if (kind == PM_TRI_F) {
        base = v.T11R + f.t11r_ofs, runlen = f.k, runs = f.k, stride = f.ld2, pstride = v.t11r_stride;
      } else if (kind == PM_FWD21) {
        if (b <= 0) continue;
        base = v.L21T + f.l21t_ofs, runlen = f.k, runs = b, stride = f.ld2, pstride = v.l21t_stride;
      } else {
        base = v.L + f.lofs, runlen = kind == PM_TRI_B ? f.k : f.n, runs = f.k, stride = f.ld, pstride = v.lstride;
      }
      const cuuint64_t dims[3] = {2 * runlen, runs, cuuint64_t(m)};
      const cuuint64_t strides[2] = {stride * sizeof(c64), pstride * sizeof(c64)};
      const cuuint32_t box[3] = {32u, 128u, 1u};
      const cuuint32_t estr[3] = {1, 1, 1};
      const CUresult r = encode(&maps[4 * i + kind], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<c64 *>(base),
                                dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed for front " + std::to_string(i);
    }
  }
  void *d = nullptr;
  if (cudaMalloc(&d, maps.size() * sizeof(CUtensorMap) + 64) != cudaSuccess) return "cudaMalloc of tensor maps failed";
  if (cudaMemcpy(d, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return "copy of tensor maps failed";
  }
  *out = d;
  return "";
}

// Maps over the two solve vectors Y, X ([pole][N][nrhs] complex) viewed as
// floats: rows of 2 nrhs floats, R rows, m poles; a box is 16 rows x 32
// right-hand sides.  Needs an even nrhs (16-byte row stride); *out = nullptr
// otherwise (the kernels then copy B rows with cp.async).
std::string build_vector_maps(const std::vector<VecBuf> &bufs, int gather, int nrhs, int m, void **out) {
  *out = nullptr;
  if (nrhs & 1) return "";
  EncodeTiledFn encode = nullptr;
  {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return "cuTensorMapEncodeTiled is not available from the driver";
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  std::vector<CUtensorMap> maps(bufs.size() + 1);
  for (size_t i = 0; i < bufs.size(); i++) {
    const int64_t rows = bufs[i].rows > 0 ? bufs[i].rows : 1;
    const cuuint64_t dims[3] = {cuuint64_t(2) * nrhs, cuuint64_t(rows), cuuint64_t(m)};
    const cuuint64_t strides[2] = {cuuint64_t(nrhs) * sizeof(c64), cuuint64_t(rows) * nrhs * sizeof(c64)};
    const cuuint32_t box[3] = {64u, 16u, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<c64 *>(bufs[i].base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return "cuTensorMapEncodeTiled failed for a solve vector";
  }
  {
    const VecBuf &g = bufs.at(gather);
    const int64_t rows = (g.rows > 0 ? g.rows : 1) * m;
    if (rows >= (int64_t(1) << 31)) return "too many vector rows for the row-gather map";
    const cuuint64_t dims[2] = {cuuint64_t(2) * nrhs, cuuint64_t(rows)};
    const cuuint64_t strides[1] = {cuuint64_t(nrhs) * sizeof(c64)};
    const cuuint32_t box[2] = {64u, 1u};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&maps[bufs.size()], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<c64 *>(g.base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return "cuTensorMapEncodeTiled failed for the row-gather map";
  }
  void *d = nullptr;
  const size_t bytes = maps.size() * sizeof(CUtensorMap);
  if (cudaMalloc(&d, bytes) != cudaSuccess) return "cudaMalloc of tensor maps failed";
  if (cudaMemcpy(d, maps.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return "copy of tensor maps failed";
  }
  *out = d;
  return "";
}

// Maps of the tensor-core trailing update: per front, 3-D over its column-major
// factor block (floats along a column: 2 n; columns: k; poles), boxes of 64
// floats (32 complex rows) x 16 columns, no swizzle (the B rows of a chunk);
// and one 3-D map over the panel copy (floats along a row: 2 kKB; rows; poles),
// boxes of 32 floats x 128 rows with the 128-byte swizzle (the A operand, like
// the solves' row-major copies).  Entries outside the dims read as zero.
std::string build_update_maps(const std::vector<FrontGeom> &fronts, const c64 *L, int64_t lstride, const c64 *Pc,
                              int64_t prows, int m, void **cmaps, void **pcmap) {
  *cmaps = *pcmap = nullptr;
  EncodeTiledFn encode = nullptr;
  {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return "cuTensorMapEncodeTiled is not available from the driver";
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  std::vector<CUtensorMap> maps(std::max<size_t>(1, fronts.size()));
  memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
  for (size_t i = 0; i < fronts.size(); i++) {
    const FrontGeom &f = fronts[i];
    if (f.k <= 0) continue;
    const cuuint64_t dims[3] = {cuuint64_t(2) * f.n, cuuint64_t(f.k), cuuint64_t(m)};
    const cuuint64_t strides[2] = {cuuint64_t(f.ld) * sizeof(c64), cuuint64_t(lstride) * sizeof(c64)};
    const cuuint32_t box[3] = {64u, 16u, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<c64 *>(L + f.lofs), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return "cuTensorMapEncodeTiled failed for the column map of front " + std::to_string(i);
  }
  CUtensorMap pm;
  {
    const cuuint64_t dims[3] = {cuuint64_t(2) * kKB, cuuint64_t(std::max<int64_t>(1, prows)), cuuint64_t(m)};
    const cuuint64_t strides[2] = {cuuint64_t(kKB) * sizeof(c64),
                                   cuuint64_t(std::max<int64_t>(1, prows)) * kKB * sizeof(c64)};
    const cuuint32_t box[3] = {32u, 128u, 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&pm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<c64 *>(Pc), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return "cuTensorMapEncodeTiled failed for the panel-copy map";
  }
  void *d = nullptr, *e = nullptr;
  if (cudaMalloc(&d, maps.size() * sizeof(CUtensorMap)) != cudaSuccess) return "cudaMalloc of tensor maps failed";
  if (cudaMalloc(&e, sizeof(CUtensorMap)) != cudaSuccess) {
    cudaFree(d);
    return "cudaMalloc of tensor maps failed";
  }
  if (cudaMemcpy(d, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(e, &pm, sizeof(CUtensorMap), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    cudaFree(e);
    return "copy of tensor maps failed";
  }
  *cmaps = d;
  *pcmap = e;
  return "";
}

}  // namespace tem
