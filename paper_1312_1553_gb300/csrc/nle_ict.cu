// Device IC(lfil, tau_IC) factor (Section 2: the incomplete Cholesky factor
// L of Phat_0 = (L L^T)^{-1}).
//
// The same left-looking column algorithm, with the same operation order, as
// the host factor (ic_factor_host), so that the pattern and every value of L
// are bit-identical to it:
//   w = lower part of column j of A, each value added once to 0.0, and
//   ||A(:,j)||_2 = sqrt of the squares of row j of A summed in ascending
//   column order;
//   for every k < j with L(j,k) != 0, in ascending k: w[i] -= L(i,k) L(j,k)
//   for every row i >= j of column k (one rounding for the product, one for
//   the difference);
//   L(j,j) = sqrt(w[j]) (w[j] <= 0: not SPD); L(i,j) = w[i] / L(j,j) for
//   the other rows, dropped when |L(i,j)| < tau ||A(:,j)||_2; of the rest the
//   lfil largest |L(i,j)| are kept (ties: smaller row first), sorted by row.
// Products, sums, the division and the square root are the correctly
// rounded intrinsics, so no contraction or reassociation can change a value.
//
// Scheduling.  One warp computes one column at a time; column j goes to
// warp j mod (warps per CTA) of CTA (j / warps per CTA) mod gridDim, so a
// warp takes its columns in ascending order.  Which k < j have L(j,k) != 0
// is decided while column j runs: L(j,k) can only be nonzero when A(j,k) !=
// 0 or when some k' < k has L(j,k') != 0 and L(k,k') != 0 (the update of
// column k by column k' is the only way a fill entry appears in row j).  So
// the warp keeps a set of candidate columns (the lower part of row j of A,
// then the rows between k' and j of every column k' found to have L(j,k') !=
// 0), takes them in ascending order, waits for each candidate column to be
// finished and reads its pattern.  Every wait is on a smaller column, every
// warp takes its columns in ascending order and all warps are resident
// (cooperative launch), so the smallest unfinished column can always
// proceed and every wait ends; each wait is also bounded in time.  A
// finished column is also copied into a per-CTA shared-memory mirror, where
// the later columns of its own block of 32 (in natural order: the next
// columns of the same grid line) find it without a trip through L2.
//
// Output: column j is written to a record of lfil + 1 slots (diagonal
// first, then the kept rows ascending) and its entry count.  Slots start as
// sentinels (row -1, value NaN; count -1) and each is written once, so a
// reader that sees a count c >= 1 and c valid slots has the whole column: no
// flag, fence or acquire is needed.
#include <cuda_runtime.h>

#include <cstdint>

#include "nle_ict.h"

namespace nle {
namespace {

constexpr int kWarps = ICT_WARPS;
constexpr int kSpa = 256;   // slots of a warp's sparse accumulator (power of two)
constexpr int kCand = 256;  // slots of a warp's candidate set (power of two)
constexpr int kKeep = 128;  // entries of a column that survive the drop test
constexpr int kEmpty = -1;

__device__ __forceinline__ int ld_rlx(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_rlx(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx(int *p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rlx(double *p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned slot_of(int key, int mask) { return ((unsigned)key * 2654435761u) >> 8 & mask; }

struct WarpMem {
  int spa_key[kSpa];
  double spa_val[kSpa];
  int cand[kCand];
  int keep_row[kKeep];
  double keep_val[kKeep];
};

// First error wins; every warp leaves at its next check.
__device__ void ict_fail(IctError *err, int code, int64_t col) {
  if (atomicCAS(&err->code, 0, code) == 0) err->col = col;
}

// Slot of `key` in an open-addressing table, inserting it when absent.
// Returns the slot, or -1 when the table is full.  *fresh tells whether the
// key was inserted by this call.  Concurrent callers insert distinct keys.
template <int N>
__device__ __forceinline__ int find_or_insert(int *keys, int key, bool *fresh) {
  unsigned s = slot_of(key, N - 1);
  for (int probe = 0; probe < N; probe++, s = (s + 1) & (N - 1)) {
    int cur = *(volatile int *)&keys[s];
    if (cur == key) {
      *fresh = false;
      return (int)s;
    }
    if (cur == kEmpty) {
      cur = atomicCAS(&keys[s], kEmpty, key);
      if (cur == kEmpty) {
        *fresh = true;
        return (int)s;
      }
      if (cur == key) {
        *fresh = false;
        return (int)s;
      }
    }
  }
  return -1;
}

template <int N>
__device__ __forceinline__ int find_slot(const int *keys, int key) {
  unsigned s = slot_of(key, N - 1);
  for (int probe = 0; probe < N; probe++, s = (s + 1) & (N - 1)) {
    const int cur = keys[s];
    if (cur == key) return (int)s;
    if (cur == kEmpty) return -1;
  }
  return -1;
}

// Records of the CTA's current columns (one per warp) in shared memory, so
// that a column waiting for a column of its own block (the previous columns
// of a grid line, in natural order) sees it without a trip through L2.  A
// slot holds the column named by its tag; the writer sets the tag to
// kBusy, fills the slot and then sets the tag to the column (a sequence
// lock: a reader that finds the same tag before and after reading has a
// consistent copy).  Tags only grow, so a tag above the column a reader
// wants means that column is finished and its global record complete.
struct Mirror {
  int tag[kWarps];
  int cnt[kWarps];
  int row[kWarps][32];
  double val[kWarps][32];
};
constexpr int kBusy = -2;

// Bounded wait, called after every unsuccessful poll: the first one starts
// the clock; every `every` polls lane 0 checks the error word and the time
// and the warp follows its decision.  True: leave the kernel.
__device__ __forceinline__ bool wait_expired(int polls, int every, long long &t0, long long spin_ns, IctError *err,
                                             int64_t j, int lane) {
  if (t0 < 0) {
    t0 = now_ns();
    return false;
  }
  if (polls % every != 0) return false;
  int leave = 0;
  if (lane == 0) {
    if (ld_rlx(&err->code) != 0) leave = 1;
    else if (now_ns() - t0 > spin_ns) {
      ict_fail(err, ICT_ERR_TIMEOUT, j);
      leave = 1;
    }
  }
  return __shfl_sync(0xffffffffu, leave, 0) != 0;
}

__device__ __forceinline__ int vld(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ double vld(const double *p) { return *(const volatile double *)p; }
__device__ __forceinline__ void vst(int *p, int v) { *(volatile int *)p = v; }
__device__ __forceinline__ void vst(double *p, double v) { *(volatile double *)p = v; }

__global__ void __launch_bounds__(32 * ICT_WARPS, 1)
    k_ict(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ va,
          int lfil, double tau, int *cnt, int *crow, double *cval, IctError *err, long long spin_ns) {
  extern __shared__ __align__(16) unsigned char ict_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpMem &M = reinterpret_cast<WarpMem *>(ict_smem)[warp];
  Mirror &MR = *reinterpret_cast<Mirror *>(ict_smem + sizeof(WarpMem) * kWarps);
  const int RS = lfil + 1;
  const int64_t stride = (int64_t)gridDim.x * kWarps;
  if (threadIdx.x < kWarps) MR.tag[threadIdx.x] = -1;
  __syncthreads();
  for (int64_t j = (int64_t)blockIdx.x * kWarps + warp; j < n; j += stride) {
    if (__shfl_sync(0xffffffffu, lane == 0 ? ld_rlx(&err->code) : 0, 0) != 0) return;
    for (int s = lane; s < kSpa; s += 32) M.spa_key[s] = kEmpty;
    for (int s = lane; s < kCand; s += 32) M.cand[s] = kEmpty;
    __syncwarp();
    // row j of A: ||A(:,j)||^2 in ascending column order, w for i >= j,
    // candidates for i < j
    const int64_t a0 = rp[j], a1 = rp[j + 1];
    double nrm2 = 0.0;
    bool over = false;
    for (int64_t e0 = a0; e0 < a1; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool have = e < a1;
      const int i = have ? ci[e] : 0;
      const double a = have ? va[e] : 0.0;
      const int m = a1 - e0 < 32 ? (int)(a1 - e0) : 32;
      for (int t = 0; t < m; t++) {
        const double at = __shfl_sync(0xffffffffu, a, t);
        nrm2 = __dadd_rn(nrm2, __dmul_rn(at, at));
      }
      if (have) {
        bool fresh;
        if (i >= j) {
          const int s = find_or_insert<kSpa>(M.spa_key, i, &fresh);
          if (s < 0) over = true;
          else M.spa_val[s] = __dadd_rn(0.0, a);
        } else if (find_or_insert<kCand>(M.cand, i, &fresh) < 0) {
          over = true;
        }
      }
    }
    if (__any_sync(0xffffffffu, over)) {
      if (lane == 0) ict_fail(err, ICT_ERR_CAPACITY, j);
      return;
    }
    __syncwarp();
    const double thr = __dmul_rn(tau, __dsqrt_rn(nrm2));
    // candidate columns in ascending order
    int last = -1;
    for (;;) {
      // every candidate added later is larger than the one being taken, so
      // "the smallest candidate above the last one taken" walks them in order
      int mine = INT32_MAX;
      for (int s = lane; s < kCand; s += 32) {
        const int c = M.cand[s];
        if (c > last && c < mine) mine = c;
      }
      const int k = (int)__reduce_min_sync(0xffffffffu, (unsigned)mine);
      if (k == INT32_MAX) break;
      last = k;
      // wait until column k is complete: from the CTA's mirror when k is a
      // column of this block, else (or once the mirror has moved on) from
      // its global record
      int c = 0, r = -1;
      double v = 0.0;
      bool got = false;
      long long t0 = -1;
      int polls = 0;
      if ((k >> 5) == (int)(j >> 5)) {
        const int wk = k & 31;
        for (;;) {
          const int t1 = __shfl_sync(0xffffffffu, lane == 0 ? vld(&MR.tag[wk]) : 0, 0);
          if (t1 == k) {
            c = vld(&MR.cnt[wk]);
            if (lane < c) {
              r = vld(&MR.row[wk][lane]);
              v = vld(&MR.val[wk][lane]);
            }
            __threadfence_block();
            const int t2 = __shfl_sync(0xffffffffu, lane == 0 ? vld(&MR.tag[wk]) : 0, 0);
            if (t2 == k) {
              got = true;
              break;
            }
          } else if (t1 > k) {
            break;
          }
          if (wait_expired(++polls, 256, t0, spin_ns, err, j, lane)) return;
        }
      }
      if (!got) {
        const int64_t base = (int64_t)k * RS;
        for (;;) {
          c = lane == 0 ? ld_rlx(cnt + k) : 0;
          if (lane < RS) {
            r = ld_rlx(crow + base + lane);
            v = ld_rlx(cval + base + lane);
          }
          c = __shfl_sync(0xffffffffu, c, 0);
          // a written slot: not the all-ones fill (tested on the bits: a
          // floating-point test in this spin would occupy the FP64 pipe the
          // finishing columns need)
          const bool ok = lane >= c || (r >= 0 && __double_as_longlong(v) != -1LL);
          if (c >= 1 && __all_sync(0xffffffffu, ok)) break;
          if (wait_expired(++polls, 16, t0, spin_ns, err, j, lane)) return;
        }
      }
      // is row j in column k?  (slot 0 is the diagonal, rows ascending)
      const unsigned hit = __ballot_sync(0xffffffffu, lane < c && r == j);
      if (!hit) continue;
      const int e0 = __ffs(hit) - 1;
      const double ljk = __shfl_sync(0xffffffffu, v, e0);
      bool bad = false;
      if (lane < c && lane >= e0) {  // rows >= j: update w
        bool fresh;
        const int s = find_or_insert<kSpa>(M.spa_key, r, &fresh);
        if (s < 0) bad = true;
        else M.spa_val[s] = __dsub_rn(fresh ? 0.0 : M.spa_val[s], __dmul_rn(v, ljk));
      } else if (lane >= 1 && lane < e0) {  // rows between k and j: candidates
        bool fresh;
        if (find_or_insert<kCand>(M.cand, r, &fresh) < 0) bad = true;
      }
      if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) ict_fail(err, ICT_ERR_CAPACITY, j);
        return;
      }
      __syncwarp();
    }
    // pivot
    const int sj = find_slot<kSpa>(M.spa_key, (int)j);
    const double d = sj >= 0 ? M.spa_val[sj] : 0.0;
    if (!(d > 0.0)) {
      if (lane == 0) ict_fail(err, ICT_ERR_NOT_SPD, j);
      return;
    }
    const double ljj = __dsqrt_rn(d);
    // the off-diagonal entries, compacted, then divided (one division per
    // entry) and tested against the drop threshold
    int nent = 0;
    for (int s0 = 0; s0 < kSpa; s0 += 32) {
      const int i = M.spa_key[s0 + lane];
      const bool occ = i >= 0 && i != (int)j;
      const unsigned b = __ballot_sync(0xffffffffu, occ);
      const int pos = nent + __popc(b & ((1u << lane) - 1));
      if (occ && pos < kKeep) {
        M.keep_row[pos] = i;
        M.keep_val[pos] = M.spa_val[s0 + lane];
      }
      nent += __popc(b);
    }
    if (nent > kKeep) {
      if (lane == 0) ict_fail(err, ICT_ERR_CAPACITY, j);
      return;
    }
    __syncwarp();
    int krow[kKeep / 32];
    double kval[kKeep / 32];
    bool kk[kKeep / 32];
    int nkeep = 0;
#pragma unroll
    for (int q = 0; q < kKeep / 32; q++) {
      const int x = lane + 32 * q;
      kk[q] = false;
      krow[q] = -1;
      kval[q] = 0.0;
      if (q * 32 < nent) {
        if (x < nent) {
          krow[q] = M.keep_row[x];
          kval[q] = __ddiv_rn(M.keep_val[x], ljj);
          kk[q] = !(fabs(kval[q]) < thr);
        }
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kKeep / 32; q++) {
      const unsigned b = __ballot_sync(0xffffffffu, kk[q]);
      if (kk[q]) {
        const int pos = nkeep + __popc(b & ((1u << lane) - 1));
        M.keep_row[pos] = krow[q];
        M.keep_val[pos] = kval[q];
      }
      nkeep += __popc(b);
    }
    __syncwarp();
    // the lfil largest |L(i,j)| (ties: smaller row), then ascending rows:
    // entry x is kept when fewer than lfil entries precede it in that order,
    // and lands after every kept entry of a smaller row
#pragma unroll
    for (int q = 0; q < kKeep / 32; q++) {
      const int x = lane + 32 * q;
      kk[q] = false;
      if (x < nkeep) {
        krow[q] = M.keep_row[x];
        kval[q] = M.keep_val[x];
        const double ax = fabs(kval[q]);
        int rank = 0;
        if (nkeep > lfil)
          for (int y = 0; y < nkeep; y++) {
            const double ay = fabs(M.keep_val[y]);
            rank += (ay > ax || (ay == ax && M.keep_row[y] < krow[q])) ? 1 : 0;
          }
        kk[q] = rank < lfil;
      }
    }
    __syncwarp();
    // publish the kept rows' flags through keep_row (negative = dropped)
#pragma unroll
    for (int q = 0; q < kKeep / 32; q++) {
      const int x = lane + 32 * q;
      if (x < nkeep && !kk[q]) M.keep_row[x] = -1 - M.keep_row[x];
    }
    __syncwarp();
    // write column j: the mirror slot (sequence lock) and the global record
    if (lane == 0) vst(&MR.tag[warp], kBusy);
    __threadfence_block();
    __syncwarp();
    int nout = 0;
#pragma unroll
    for (int q = 0; q < kKeep / 32; q++) {
      const int x = lane + 32 * q;
      if (x < nkeep && kk[q]) {
        int pos = 0;
        for (int y = 0; y < nkeep; y++) {
          const int ry = M.keep_row[y];
          pos += (ry >= 0 && ry < krow[q]) ? 1 : 0;
        }
        vst(&MR.row[warp][1 + pos], krow[q]);
        vst(&MR.val[warp][1 + pos], kval[q]);
        st_rlx(crow + (int64_t)j * RS + 1 + pos, krow[q]);
        st_rlx(cval + (int64_t)j * RS + 1 + pos, kval[q]);
      }
      nout += __popc(__ballot_sync(0xffffffffu, x < nkeep && kk[q]));
    }
    if (lane == 0) {
      vst(&MR.row[warp][0], (int)j);
      vst(&MR.val[warp][0], ljj);
      vst(&MR.cnt[warp], 1 + nout);
      st_rlx(crow + (int64_t)j * RS, (int)j);
      st_rlx(cval + (int64_t)j * RS, ljj);
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) {
      vst(&MR.tag[warp], (int)j);
      st_rlx(cnt + j, 1 + nout);
    }
  }
}

}  // namespace

int ict_smem_bytes() { return (int)(sizeof(WarpMem) * kWarps + sizeof(Mirror)); }

cudaError_t ict_launch(int grid, int64_t n, const int64_t *rp, const int32_t *ci, const double *va, int lfil,
                       double tau, int *cnt, int *crow, double *cval, IctError *err, long long spin_ns,
                       cudaStream_t stream) {
  const int smem = ict_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_ict, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  void *args[] = {&n, &rp, &ci, &va, &lfil, &tau, &cnt, &crow, &cval, &err, &spin_ns};
  return cudaLaunchCooperativeKernel((const void *)k_ict, dim3(grid), dim3(32 * kWarps), args, smem, stream);
}

int ict_max_grid(int nsm) {
  int per = 0;
  cudaFuncSetAttribute(k_ict, cudaFuncAttributeMaxDynamicSharedMemorySize, ict_smem_bytes());
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ict, 32 * kWarps, ict_smem_bytes()) != cudaSuccess)
    return 0;
  return per * nsm;
}

}  // namespace nle
