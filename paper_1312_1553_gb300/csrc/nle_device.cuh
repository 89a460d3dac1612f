// Device primitives of the persistent solver kernels: vector loads, bounded
// grid barrier, deterministic block/grid reductions, SELL SpMV and the
// sync-free triangular solves.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "nle_internal.h"

namespace nle {

// ---------------------------------------------------------------------------
// precision traits: VW rows per thread so that one row group is 16 bytes
// ---------------------------------------------------------------------------
template <typename T>
struct VT;
template <>
struct VT<float> {
  static constexpr int W = 4;
};
template <>
struct VT<double> {
  static constexpr int W = 2;
};

// Coherent (L2) vector loads of W consecutive elements of a vector that is
// written inside the kernel; read-only loads (__ldg) for the matrices.
__device__ __forceinline__ void ldc(const float *p, float (&o)[4]) {
  float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
  o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
__device__ __forceinline__ void ldc(const double *p, double (&o)[2]) {
  double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  o[0] = v.x, o[1] = v.y;
}
__device__ __forceinline__ void ldc(const double *p, double (&o)[4]) {
  double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
  double2 b = __ldcg(reinterpret_cast<const double2 *>(p + 2));
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}
__device__ __forceinline__ void stv(float *p, const float (&o)[4]) {
  __stcg(reinterpret_cast<float4 *>(p), make_float4(o[0], o[1], o[2], o[3]));
}
__device__ __forceinline__ void stv(double *p, const double (&o)[2]) {
  __stcg(reinterpret_cast<double2 *>(p), make_double2(o[0], o[1]));
}
__device__ __forceinline__ void stv(double *p, const double (&o)[4]) {
  __stcg(reinterpret_cast<double2 *>(p), make_double2(o[0], o[1]));
  __stcg(reinterpret_cast<double2 *>(p + 2), make_double2(o[2], o[3]));
}
__device__ __forceinline__ void ldr(const float *p, float (&o)[4]) {
  float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
__device__ __forceinline__ void ldr(const double *p, double (&o)[2]) {
  double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  o[0] = v.x, o[1] = v.y;
}
__device__ __forceinline__ void ldr(const double *p, double (&o)[4]) {
  double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  double2 b = __ldg(reinterpret_cast<const double2 *>(p + 2));
  o[0] = a.x, o[1] = a.y, o[2] = b.x, o[3] = b.y;
}
__device__ __forceinline__ void ldr(const int32_t *p, int (&o)[4]) {
  int4 v = __ldg(reinterpret_cast<const int4 *>(p));
  o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
}
__device__ __forceinline__ void ldr(const int32_t *p, int (&o)[2]) {
  int2 v = __ldg(reinterpret_cast<const int2 *>(p));
  o[0] = v.x, o[1] = v.y;
}

// Read-only loads issued exactly where they are written: the descriptor
// loads of the chain schedule are meant to be in flight while the warp works
// on the previous task, and a plain read-only load may be sunk by the
// compiler down to its first use, which puts its latency back on the
// dependency chain.  (The level schedule keeps plain read-only loads: with
// its rows per warp step a compile-time constant they measured faster.)
__device__ __forceinline__ int ld_pinned(const int32_t *p) {
  int v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_pinned(const float *p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_pinned(const double *p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// ---------------------------------------------------------------------------
// memory-model helpers (PTX): relaxed gpu-scope loads/stores bypass L1 and
// observe other SMs' stores; acquire/release for the grid barrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ld_relaxed(const float *p) {
  float v;
  asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_relaxed(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(float *p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(double *p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_int(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Not-yet-computed marker of the triangular solves: a NaN payload that GPU
// arithmetic never produces (it returns the canonical NaN 0x7fffffff).
__device__ __forceinline__ bool is_sent(float v) { return __float_as_uint(v) == 0xFFC0BAD1u; }
__device__ __forceinline__ bool is_sent(double v) {
  return __double_as_longlong(v) == (long long)0xFFF8BAD1BAD1BAD1ull;
}
template <typename T>
__device__ __forceinline__ T sentinel();
template <>
__device__ __forceinline__ float sentinel<float>() {
  return __uint_as_float(0xFFC0BAD1u);
}
template <>
__device__ __forceinline__ double sentinel<double>() {
  return __longlong_as_double((long long)0xFFF8BAD1BAD1BAD1ull);
}

__device__ __forceinline__ void record_error(State *st, int code, int where) {
  if (atomicCAS(&st->err, 0, code) == 0) st->err_where = where;
}

// ---------------------------------------------------------------------------
// CTA group working on one problem: blocks [s_gbase, s_gbase + s_gsize).
// A single-problem launch uses the whole grid; the batched kernel runs
// several problems at once, one group of CTAs each.  Thread ownership,
// barriers, reductions and triangular-solve slabs are group-relative.
// ---------------------------------------------------------------------------
__shared__ int s_gbase;
__shared__ int s_gsize;
__device__ __forceinline__ int grank() { return (int)blockIdx.x - s_gbase; }
__device__ __forceinline__ bool lead_cta() { return (int)blockIdx.x == s_gbase; }

// ---------------------------------------------------------------------------
// per-CTA shared state
// ---------------------------------------------------------------------------
struct Shared {
  double red[NWARP][RED_MAX];  // warp partial sums of the current pass
  double sc[RED_MAX];          // grid-reduced scalars of the last pass
  double a[KMAX], b[KMAX], ab[KMAX];
  double sg[KMAX];             // S^T g
  double alpha[KMAX];          // s_s^T r_s (chronological)
  double gsr[KMAX][KMAX];      // s_s^T r_t
  double gqs[MMAX][KMAX];      // q_c^T s_t
  double zq[MMAX];             // Q^T c (Algorithm 3.1, last two steps)
  double qv[MMAX];             // Q^T v of the current projection
  double cadj[MMAX];           // adjoint: v_i^T gbar
  int order[KMAX];             // chronological -> physical pair slot
  int ok;                      // error word broadcast after each barrier
  long long tlast;             // phase timer (CTA 0, thread 0)
  long long tacc[8];
};

struct Ctl {
  unsigned epoch;  // barriers passed by this CTA (thread 0 only)
  int rbuf;        // reduction buffer parity
  long long spin_ns;
  int twarps;      // warps of this CTA that take part in the triangular solves
  int poll_ns;     // pause between two polls of a triangular-solve wait
};

// Phase timers: CTA 0 / thread 0 charges the time since the last mark to
// `phase` (called right after a barrier, so the time covers the whole grid).
enum { PH_SPMV = 0, PH_UPDATE = 1, PH_FWD = 2, PH_BWD = 3, PH_DOTS = 4, PH_DIR = 5, PH_OUTER = 6, PH_OTHER = 7 };
__device__ __forceinline__ void tmark(Shared &sh, int phase) {
  if (lead_cta() && threadIdx.x == 0) {
    const long long t = gtimer();
    sh.tacc[phase] += t - sh.tlast;
    sh.tlast = t;
  }
}

// Grid-wide barrier for a cooperative launch.  Monotone counter: barrier
// number e completes when the counter reaches e * gridDim.x.  Every wait is
// bounded: after spin_ns without progress, or when another CTA already
// recorded an error, the CTA records NLE_ERR_TIMEOUT (first error wins) and
// leaves the barrier.  Returns false when the solver must stop.
__device__ __forceinline__ bool grid_sync(State *st, Shared &sh, Ctl &ctl, int where) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl.epoch++;
    const unsigned target = ctl.epoch * (unsigned)s_gsize;
    __threadfence();
    red_release_add(&st->bar, 1u);
    long long t0 = 0;
    int spins = 0;
    while (ld_acquire(&st->bar) < target) {
      if (++spins >= 32) {
        spins = 0;
        if (ld_relaxed_int(&st->err) != 0) break;
        const long long now = gtimer();
        if (t0 == 0)
          t0 = now;
        else if (now - t0 > ctl.spin_ns) {
          record_error(st, 8 /*NLE_ERR_TIMEOUT*/, where);
          break;
        }
      }
    }
    __threadfence();
    sh.ok = (ld_relaxed_int(&st->err) == 0);
  }
  __syncthreads();
  return sh.ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic reductions.  Every warp of every CTA calls red_put for the
// same slots in the same order; red_flush writes the CTA's sums; after a
// grid barrier red_collect sums the CTAs' partials in CTA order, so every
// CTA obtains bit-identical scalars and takes the same control decisions.
__device__ __forceinline__ void red_put(Shared &sh, int slot, double v) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5][slot] = v;
}

template <typename T>
__device__ __forceinline__ void red_flush(const Dev<T> &D, Shared &sh, Ctl &ctl, int nslots) {
  __syncthreads();
  double *part = D.part + (size_t)ctl.rbuf * RED_MAX * s_gsize;
  for (int s = threadIdx.x; s < nslots; s += TPB) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < NWARP; w++) v += sh.red[w][s];
    part[(size_t)s * s_gsize + grank()] = v;
  }
}

template <typename T>
__device__ __forceinline__ void red_collect(const Dev<T> &D, Shared &sh, Ctl &ctl, int nslots) {
  const double *part = D.part + (size_t)ctl.rbuf * RED_MAX * s_gsize;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = warp; s < nslots; s += NWARP) {
    double v = 0.0;
    for (int b = lane; b < s_gsize; b += 32) v += __ldcg(part + (size_t)s * s_gsize + b);
    v = warp_sum(v);
    if (lane == 0) sh.sc[s] = v;
  }
  ctl.rbuf ^= 1;
  __syncthreads();
}

// flush + barrier + collect
template <typename T>
__device__ __forceinline__ bool reduce_all(const Dev<T> &D, Shared &sh, Ctl &ctl, int nslots, int where) {
  red_flush(D, sh, ctl, nslots);
  if (!grid_sync(D.st, sh, ctl, where)) return false;
  red_collect(D, sh, ctl, nslots);
  return true;
}

// ---------------------------------------------------------------------------
// row ownership: thread t owns row groups ("chunks") t, t+TT, t+2TT, ...;
// chunk c holds rows c*W .. c*W+W-1.  Backward sweeps use the mirrored
// numbering nchunks-1-(t + i TT).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t gtid() { return (int64_t)grank() * TPB + threadIdx.x; }
__device__ __forceinline__ int64_t gthreads() { return (int64_t)s_gsize * TPB; }

// y[v] = sum_e val * x[col] for the W rows of one chunk of a SELL matrix.
template <int W, typename TV, typename TX, typename TA>
__device__ __forceinline__ void sell_rows(const Sell<TV> &M, const TX *__restrict__ x, int64_t chunk,
                                          TA (&acc)[W]) {
  constexpr int H = 32 * W;
  const int64_t slice = chunk >> 5;
  const int lanepos = (int)(chunk & 31);
  const int64_t base = __ldg(M.sptr + slice);
  const int width = (int)((__ldg(M.sptr + slice + 1) - base) / H);
#pragma unroll
  for (int v = 0; v < W; v++) acc[v] = TA(0);
  const int64_t off0 = base + (int64_t)lanepos * W;
  int e = 0;
  for (; e + 2 <= width; e += 2) {
    int c0[W], c1[W];
    TV a0[W], a1[W];
    ldr(M.col + off0 + (int64_t)e * H, c0);
    ldr(M.col + off0 + (int64_t)(e + 1) * H, c1);
    ldr(M.val + off0 + (int64_t)e * H, a0);
    ldr(M.val + off0 + (int64_t)(e + 1) * H, a1);
    TX x0[W], x1[W];
#pragma unroll
    for (int v = 0; v < W; v++) {
      x0[v] = __ldcg(x + c0[v]);
      x1[v] = __ldcg(x + c1[v]);
    }
#pragma unroll
    for (int v = 0; v < W; v++) {
      acc[v] += TA(a0[v]) * TA(x0[v]);
      acc[v] += TA(a1[v]) * TA(x1[v]);
    }
  }
  if (e < width) {
    int c0[W];
    TV a0[W];
    ldr(M.col + off0 + (int64_t)e * H, c0);
    ldr(M.val + off0 + (int64_t)e * H, a0);
#pragma unroll
    for (int v = 0; v < W; v++) acc[v] += TA(a0[v]) * TA(__ldcg(x + c0[v]));
  }
}

// Sync-free triangular solve, one slab of rows per CTA.
//
// The unknowns are labelled slab-major, level-minor: CTA c owns positions
// [c*bsize, (c+1)*bsize), which are a contiguous range of the natural row
// order sorted by the level of each row in L.  A dependency inside the slab
// is read from the CTA's shared-memory copy of the slab's results; one in
// another slab (lower slabs for L, higher for L^T) is polled in global memory
// with relaxed loads.  Results start as a NaN payload that GPU arithmetic
// never produces and are published both to shared and to global memory; the
// value is its own ready flag.
//
// Each slab stores its rows in ELL form (width = the slab's longest row,
// rounded up to 8), so the address of a row's entries follows from the row
// index without a dependent load.  A warp takes R consecutive rows at a time
// (R = 4, or 2 for factors with wide rows; a compile-time constant of each
// instance), 32 / R lanes per row, TRSV_EPL entries per lane in flight,
// and fetches the
// next group's entries, right-hand sides (from shared memory) and pivots
// (reciprocals computed on the host, so no division and no load sits on the
// dependency chain) before the current group waits.
// The wait is warp-uniform: the warp re-polls the entries still missing
// until every lane holds its values (a vote), then reduces with shuffles; a
// per-lane wait followed by the warp's reconvergence measured about 1.5x
// slower per dependency hop.  The rows of a group are done in rounds
// separated by __syncwarp (round[r] precomputed), so a lane never waits for
// a lane of its own warp.  The rows of one round publish together, so a
// round waits for the inputs of all of them; every wait ends when each
// round's inputs come from strictly earlier levels (or, in the slab order of
// the natural ordering, from earlier positions of the same slab or from
// lower slabs only).  Natural order: round[r] = longest dependency chain to
// r inside its group.  Slabs whose dependencies can point to later slabs
// (the multicolour ordering): one level per round.  Every wait is also
// bounded in time; every warp and CTA is resident (cooperative launch).
template <typename T>
struct TriEll {
  const int64_t *off;    // per slab: first entry
  const int32_t *width;  // per slab: entries per row (multiple of 8)
  const int32_t *col;    // -1 = padding
  const T *val;
  const T *rdiag;         // npad: reciprocal pivots 1 / L_rr
  const uint16_t *round;  // npad: round of the row inside its group of rows (bits 0-3), the
                          // group's last round (4-7) and overflow steps (8-15, 255: to width)
  int rows;               // rows a warp takes at a time: 4 (8 lanes per row) or 2 (16 lanes)
};

template <typename T>
struct TriPre {
  int c[TRSV_EPL];  // columns of the lane's first entries (-1: none)
  T a[TRSV_EPL];
  T rhs, rdg;  // right-hand side and 1 / pivot (lane g == 0 of each row)
  int rnd;
};

template <bool LOWER, int R, typename T, typename RHS>
__device__ __forceinline__ void trsv_fetch(const TriEll<T> &M, int64_t b0, int64_t base, int wd, int64_t ngrp,
                                           int64_t it, int q, int g, RHS &rhs_of, TriPre<T> &P) {
  constexpr int lanes = 32 / R;
  const int64_t gi = LOWER ? it : ngrp - 1 - it;
  const int64_t r = b0 + (int64_t)R * gi + q;
  const int64_t e = base + (r - b0) * wd + g;
#pragma unroll
  for (int k = 0; k < TRSV_EPL; k++) {
    P.c[k] = -1;
    P.a[k] = T(0);
    if (g + k * lanes < wd) {
      P.c[k] = __ldg(M.col + e + k * lanes);
      P.a[k] = __ldg(M.val + e + k * lanes);
    }
  }
  P.rnd = __ldg(M.round + r);
  P.rhs = T(0);
  P.rdg = T(1);
  if (g == 0) {
    P.rhs = rhs_of(r);
    P.rdg = __ldg(M.rdiag + r);
  }
}

// Where a triangular solve reads its dependencies: its CTA's slab [b0, b1)
// of the output x is copied in shared memory (stage); a dependency in
// another slab is read from global memory.
template <typename T>
struct TriSrc {
  const T *x;
  const volatile T *stage;
  int64_t b0, b1;
};

// Current value of dependency c (the not-yet-computed marker if it is not
// ready).
template <typename T>
__device__ __forceinline__ T trsv_peek(const TriSrc<T> &S, int c) {
  if (c >= S.b0 && c < S.b1) return S.stage[c - S.b0];
  return ld_relaxed(S.x + c);
}

// Warp-uniform wait: returns once every lane of the warp holds values (not
// the marker) for its N entries c[k] (c < 0: no entry).  The clock is read
// only after 2^20 rounds of polling; past spin_ns the wait records
// NLE_ERR_TIMEOUT and substitutes 0 so that dependants still finish.
template <int N, typename T>
__device__ __forceinline__ void trsv_wait(const TriSrc<T> &S, const int *c, T *v, State *st, long long spin_ns,
                                          int poll_ns = 0) {
  auto ready = [&]() {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < N; k++) ok = ok && !(c[k] >= 0 && is_sent(v[k]));
    return ok;
  };
  bool ok = ready();
  if (__all_sync(0xffffffffu, ok)) return;
  long long t0 = 0;
  for (int it = 0;; it++) {
#pragma unroll
    for (int k = 0; k < N; k++)
      if (c[k] >= 0 && is_sent(v[k])) v[k] = trsv_peek(S, c[k]);
    ok = ready();
    if (__all_sync(0xffffffffu, ok)) return;
    if (poll_ns > 0) __nanosleep(poll_ns);
    if (it >= (1 << 20)) {
      if (it == (1 << 20)) t0 = clock64();
      const bool late = clock64() - t0 > spin_ns * 21 / 10;  // cycles at about 2.1 GHz
      if (__any_sync(0xffffffffu, late)) {
        if (!ok) record_error(st, 8 /*NLE_ERR_TIMEOUT*/, 102);
#pragma unroll
        for (int k = 0; k < N; k++)
          if (c[k] >= 0 && is_sent(v[k])) v[k] = T(0);
        return;
      }
    }
  }
}

template <bool LOWER, int R, typename T, typename RHS>
__device__ __noinline__ void trsv_block_r(const TriEll<T> &M, T *x, int64_t npad, int64_t bsize, int twarps,
                                          long long spin_ns, int poll_ns, State *st, T *stage_mem, RHS rhs_of) {
  const int64_t b0 = (int64_t)grank() * bsize;
  const int64_t b1 = min(npad, b0 + bsize);
  const int64_t nb = b1 > b0 ? b1 - b0 : 0;
  volatile T *stage = stage_mem;
  const T sent = sentinel<T>();
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) stage[i] = sent;
  __syncthreads();
  const TriSrc<T> S{x, stage, b0, b1};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int lanes = 32 / R;            // lanes per row (R = 4 or 2; bsize is a multiple of 4)
  const int64_t ngrp = nb / R;
  int64_t it = warp;
  if (warp < twarps && it < ngrp) {
    const int q = lane / lanes, g = lane % lanes;
    const int64_t base = __ldg(M.off + grank());
    const int wd = __ldg(M.width + grank());
    // one group: its rounds, each a warp-uniform wait, the reduction and the
    // publication of the round's rows
    auto process = [&](const TriPre<T> &cur, int64_t itc) {
      const int64_t gi = LOWER ? itc : ngrp - 1 - itc;
      const int64_t r = b0 + (int64_t)R * gi + q;
      const int rounds = 1 + ((cur.rnd >> 4) & 15);  // the same in every lane of the group
      const int steps = cur.rnd >> 8;                 // overflow steps, likewise
      const int kend = steps == 255 ? wd : min(wd, TRSV_EPL * lanes + steps * lanes);
      for (int rd = 0; rd < rounds; rd++) {
        const bool active = ((cur.rnd & 15) == rd);
        int c[TRSV_EPL];
        T v[TRSV_EPL];
#pragma unroll
        for (int k = 0; k < TRSV_EPL; k++) {
          c[k] = active ? cur.c[k] : -1;
          v[k] = T(0);
          if (c[k] >= 0) v[k] = trsv_peek(S, c[k]);
        }
        trsv_wait<TRSV_EPL, T>(S, c, v, st, spin_ns, poll_ns);
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < TRSV_EPL; k++)
          if (c[k] >= 0) acc += cur.a[k] * v[k];
        // entries beyond the first TRSV_EPL * lanes of a row, one per lane
        // and step, up to the group's longest row (not the slab's width);
        // every lane takes the same number of steps
        const int64_t e = base + (r - b0) * wd;
        for (int k0 = TRSV_EPL * lanes; k0 < kend; k0 += lanes) {
          const int k = k0 + g;
          int ce[1] = {(active && k < kend) ? __ldg(M.col + e + k) : -1};
          T ve[1] = {T(0)};
          if (ce[0] >= 0) ve[0] = trsv_peek(S, ce[0]);
          trsv_wait<1, T>(S, ce, ve, st, spin_ns, poll_ns);
          if (ce[0] >= 0) acc += __ldg(M.val + e + k) * ve[0];
        }
#pragma unroll
        for (int o = lanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (active && g == 0) {
          const T val = (cur.rhs - acc) * cur.rdg;
          stage[r - b0] = val;
          st_relaxed(x + r, val);
        }
        if (rounds > 1) __syncwarp();
      }
    };
    // two descriptor sets used in turn: the next group's entries load while
    // this one waits, and no register copy waits for those loads
    TriPre<T> p0, p1;
    trsv_fetch<LOWER, R, T>(M, b0, base, wd, ngrp, it, q, g, rhs_of, p0);
    for (;;) {
      const int64_t it1 = it + twarps;
      if (it1 < ngrp) trsv_fetch<LOWER, R, T>(M, b0, base, wd, ngrp, it1, q, g, rhs_of, p1);
      process(p0, it);
      if (it1 >= ngrp) break;
      const int64_t it2 = it1 + twarps;
      if (it2 < ngrp) trsv_fetch<LOWER, R, T>(M, b0, base, wd, ngrp, it2, q, g, rhs_of, p0);
      process(p1, it1);
      if (it2 >= ngrp) break;
      it = it2;
    }
  }
  __syncthreads();
}

// The level schedule with the rows per warp step of the factor's layout
// (4, or 2 for factors with wide rows), each a compile-time instance.  The
// instances are called, not inlined: inside the persistent solver kernels
// the inlined solves raised register spills and measured 4-10 % slower per
// whole solve (the call happens once per triangular solve).
template <bool LOWER, typename T, typename RHS>
__device__ __forceinline__ void trsv_block(const TriEll<T> &M, T *x, int64_t npad, int64_t bsize, int twarps,
                                           long long spin_ns, int poll_ns, State *st, T *stage_mem, RHS rhs_of) {
  if (M.rows == 2)
    trsv_block_r<LOWER, 2, T>(M, x, npad, bsize, twarps, spin_ns, poll_ns, st, stage_mem, rhs_of);
  else
    trsv_block_r<LOWER, 4, T>(M, x, npad, bsize, twarps, spin_ns, poll_ns, st, stage_mem, rhs_of);
}

// Chain schedule of the sync-free triangular solve, one slab per CTA.
//
// The slab's rows (the factored matrix's own order) are cut into tasks of at
// most TRSV_ROWS consecutive rows in processing order (ascending for L,
// descending for L^T), and every warp owns a list of tasks, built on the
// host: runs of tasks whose first row depends on the previous task's last
// row ("strands", the lines of a grid in natural order) stay on one warp.
// A task is solved with TRSV_LANES lanes per row: the entries pointing to
// rows outside the task and outside the previous task's last row are
// "external" and gathered as in trsv_block (shared-memory copy inside the
// slab, relaxed global loads outside it, the value being its own ready
// flag, bounded warp-uniform wait); the entries pointing to earlier rows of
// the same task or to the previous task's last row are stored with column
// -2 - d (d = distance back in processing order) and resolved in registers,
// so a dependency chain along a strand costs one shuffle per row instead
// of a trip through memory:
//   v_a = rhs_a - sum_external L_ac x_c - L_{a,prev} x_prev,
//   x_s = v_s / L_ss and v_a -= L_as x_s for a > s, s = 0, 1, ...
// The next task's entries are fetched, and its external values loaded,
// before the current task waits, which hides the latency of the loads from
// other slabs behind the current task.  Every wait ends: the host deals the
// strands to the warps in a topological order of the strand graph of each
// slab and every dependency points to a lower slab (L) or a higher one
// (L^T), so the earliest unfinished task always has its inputs; all CTAs
// are resident (cooperative launch) and every wait is also bounded in time.
template <typename T>
struct TriChain {
  const int64_t *off;    // per slab: first entry
  const int32_t *width;  // per slab: entries per row (multiple of 8)
  const int32_t *col;    // -1 = padding, -2 - d = register-resolved entry
  const T *val;
  const T *rdiag;
  const int32_t *wptr;   // per slab: NWARP + 1 offsets into task
  const int2 *task;      // {first row processed, rows | sequential << 3}
};

template <typename T>
struct ChainPre {
  int c[TRSV_EPL];
  T a[TRSV_EPL];
  T v[TRSV_EPL];  // values of the external entries (loaded ahead; marker if not ready)
  T rhs, rdg;
  int r0, meta;
};

template <bool LOWER, typename T, typename RHS>
__device__ __forceinline__ void chain_fetch(const TriChain<T> &M, const TriSrc<T> &S, int64_t b0, int64_t base, int wd,
                                            int ti, int q, int g, RHS &rhs_of, ChainPre<T> &P) {
  const int2 tk = make_int2(ld_pinned(&M.task[ti].x), ld_pinned(&M.task[ti].y));
  P.r0 = tk.x;
  P.meta = tk.y;
  const bool active = q < (tk.y & 7);
  const int64_t r = LOWER ? (int64_t)tk.x + q : (int64_t)tk.x - q;
  const int64_t e = base + (r - b0) * wd + g;
#pragma unroll
  for (int k = 0; k < TRSV_EPL; k++) {
    P.c[k] = -1;
    P.a[k] = T(0);
    if (active && g + k * TRSV_LANES < wd) {
      P.c[k] = ld_pinned(M.col + e + k * TRSV_LANES);
      P.a[k] = ld_pinned(M.val + e + k * TRSV_LANES);
    }
  }
#pragma unroll
  for (int k = 0; k < TRSV_EPL; k++) P.v[k] = (P.c[k] >= 0) ? trsv_peek(S, P.c[k]) : T(0);
  P.rhs = T(0);
  P.rdg = T(1);
  if (active) {
    P.rhs = rhs_of(r);
    P.rdg = ld_pinned(M.rdiag + r);
  }
}

template <bool LOWER, typename T, typename RHS>
__device__ __forceinline__ void trsv_chain(const TriChain<T> &M, T *x, int64_t npad, int64_t bsize, long long spin_ns,
                                           int poll_ns, State *st, T *stage_mem, RHS rhs_of) {
  const int64_t b0 = (int64_t)grank() * bsize;
  const int64_t b1 = min(npad, b0 + bsize);
  const int64_t nb = b1 > b0 ? b1 - b0 : 0;
  volatile T *stage = stage_mem;
  const T sent = sentinel<T>();
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) stage[i] = sent;
  __syncthreads();
  const TriSrc<T> S{x, stage, b0, b1};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // a CTA past the last slab has no rows (and no task offsets)
  const int t0 = nb > 0 ? __ldg(M.wptr + grank() * (NWARP + 1) + warp) : 0;
  const int t1 = nb > 0 ? __ldg(M.wptr + grank() * (NWARP + 1) + warp + 1) : 0;
  if (t0 < t1) {
    const int q = lane / TRSV_LANES, g = lane % TRSV_LANES;
    const int64_t base = __ldg(M.off + grank());
    const int wd = __ldg(M.width + grank());
    T xprev = T(0);
    auto process = [&](ChainPre<T> &cur) {
      const int cnt = cur.meta & 7;
      const int64_t r = LOWER ? (int64_t)cur.r0 + q : (int64_t)cur.r0 - q;
      const bool active = q < cnt;
      trsv_wait<TRSV_EPL, T>(S, cur.c, cur.v, st, spin_ns, poll_ns);
      T acc = T(0), cf[TRSV_ROWS];
#pragma unroll
      for (int d = 0; d < TRSV_ROWS; d++) cf[d] = T(0);
#pragma unroll
      for (int k = 0; k < TRSV_EPL; k++) {
        if (cur.c[k] >= 0) acc += cur.a[k] * cur.v[k];
#pragma unroll
        for (int d = 0; d < TRSV_ROWS; d++)
          if (cur.c[k] == -3 - d) cf[d] += cur.a[k];
      }
      // external entries beyond the first 16 of a row (same trip count in
      // every lane)
      const int64_t e = base + (r - b0) * wd;
      for (int k = g + 16; k < wd; k += TRSV_LANES) {
        int ce[1] = {active ? __ldg(M.col + e + k) : -1};
        T ve[1] = {T(0)};
        if (ce[0] >= 0) ve[0] = trsv_peek(S, ce[0]);
        trsv_wait<1, T>(S, ce, ve, st, spin_ns, poll_ns);
        if (ce[0] >= 0) acc += __ldg(M.val + e + k) * ve[0];
      }
#pragma unroll
      for (int o = TRSV_LANES / 2; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
#pragma unroll
        for (int d = 0; d < TRSV_ROWS; d++) cf[d] += __shfl_xor_sync(0xffffffffu, cf[d], o);
      }
      // cf[d]: coefficient of the row d + 1 positions back; row q reaches the
      // previous task's last row at distance q + 1 and row s of this task at
      // distance q - s
      T v = cur.rhs - acc;
      T kp = T(0);
#pragma unroll
      for (int d = 0; d < TRSV_ROWS; d++)
        if (d == q) kp = cf[d];
      if (kp != T(0)) v -= kp * xprev;
      if (cur.meta & 8) {
#pragma unroll
        for (int s = 0; s + 1 < TRSV_ROWS; s++) {
          if (s + 1 >= cnt) break;
          const T xs = __shfl_sync(0xffffffffu, v * cur.rdg, s * TRSV_LANES);
          T ks = T(0);
#pragma unroll
          for (int d = 0; d < TRSV_ROWS; d++)
            if (d == q - s - 1) ks = cf[d];
          v -= ks * xs;
        }
      }
      const T val = v * cur.rdg;
      if (active && g == 0) {
        stage[r - b0] = val;
        st_relaxed(x + r, val);
      }
      xprev = __shfl_sync(0xffffffffu, val, (cnt - 1) * TRSV_LANES);
    };
    ChainPre<T> p0, p1;
    int ti = t0;
    chain_fetch<LOWER, T>(M, S, b0, base, wd, ti, q, g, rhs_of, p0);
    for (;;) {
      if (ti + 1 < t1) chain_fetch<LOWER, T>(M, S, b0, base, wd, ti + 1, q, g, rhs_of, p1);
      process(p0);
      if (ti + 1 >= t1) break;
      if (ti + 2 < t1) chain_fetch<LOWER, T>(M, S, b0, base, wd, ti + 2, q, g, rhs_of, p0);
      process(p1);
      if (ti + 2 >= t1) break;
      ti += 2;
    }
  }
  __syncthreads();
}

}  // namespace nle
