// Persistent cooperative kernels of the DACG-Newton eigensolver.
//
// One launch runs a whole phase on the device: DACG for eigenpair j
// (Section 4.1), the Newton iteration for eigenpair j with every inner PCG
// solve (Section 4.3, Algorithm 3.2), or one of the building blocks exposed
// for verification.  Passes over the vectors are separated by a bounded grid
// barrier; scalars are reduced deterministically so that every CTA takes the
// same control decisions without a host round trip.
//
// Algorithm 3.1 is applied in Gram form: with G_SR[s][t] = s_s^T r_t and
// G_QS[c][t] = q_c^T s_t (computed once per Newton step from the stored,
// rounded vectors), the two loops of Algorithm 3.1 reduce to k x k
// recurrences on scalars,
//   a_s = (s_s^T g - sum_{t>s} a_t G_SR[s][t]) / alpha_s,   w = g - R a,
//   c0  = Phat_0 w = L^{-T} L^{-1} w,
//   b_s = (r_s^T c0 - sum_{t<s} (a_t+b_t) G_SR[t][s]) / alpha_s,
//   z   = Q^T c0 - G_QS (a+b),   c = c0 - S (a+b) - Q z,
// which is algebraically identical to the paper's loop (same a_s, b_s, z)
// but needs one pass over S and R per dot-product group instead of 2k.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "nle_device.cuh"

namespace nle {

// ---------------------------------------------------------------------------
// small helpers over the chunks owned by a thread
// ---------------------------------------------------------------------------
// out[i][v] += sgn * sum_c coef[c] * X_c[row]   (X column c at X + c*ld),
// four columns per step for memory-level parallelism.
template <typename T, int RPC>
__device__ __forceinline__ void comb_add(const T *X, int64_t ld, int ncol, const double *coef, const int *slot,
                                         const Dev<T> &D, T (&out)[RPC][VT<T>::W], double sgn) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  int c = 0;
  for (; c + 4 <= ncol; c += 4) {
    const T *col[4];
    T cf[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      col[u] = X + (int64_t)(slot ? slot[c + u] : c + u) * ld;
      cf[u] = T(sgn * coef[c + u]);
    }
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        T q[4][W];
#pragma unroll
        for (int u = 0; u < 4; u++) ldc(col[u] + ch * W, q[u]);
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
          for (int v = 0; v < W; v++) out[i][v] += cf[u] * q[u][v];
      }
    }
  }
  for (; c < ncol; c++) {
    const T cf = T(sgn * coef[c]);
    const T *cl = X + (int64_t)(slot ? slot[c] : c) * ld;
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        T q[W];
        ldc(cl + ch * W, q);
#pragma unroll
        for (int v = 0; v < W; v++) out[i][v] += cf * q[v];
      }
    }
  }
}

// slot0 + c: sum over owned rows of X_c[row] * val[i][v], for each column c.
// Four columns per step so that 4*RPC independent loads are in flight.
template <typename T, int RPC>
__device__ __forceinline__ void dots_put(Shared &sh, int slot0, const T *X, int64_t ld, int ncol, const int *slot,
                                         const Dev<T> &D, const T (&val)[RPC][VT<T>::W], bool reverse) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  int c = 0;
  for (; c + 4 <= ncol; c += 4) {
    const T *col[4];
#pragma unroll
    for (int u = 0; u < 4; u++) col[u] = X + (int64_t)(slot ? slot[c + u] : c + u) * ld;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t k = tid + i * TT;
      const int64_t ch = reverse ? D.nchunks - 1 - k : k;
      if (k < D.nchunks) {
        T q[4][W];
#pragma unroll
        for (int u = 0; u < 4; u++) ldc(col[u] + ch * W, q[u]);
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
          for (int v = 0; v < W; v++) acc[u] += double(q[u][v]) * double(val[i][v]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) red_put(sh, slot0 + c + u, acc[u]);
  }
  for (; c < ncol; c++) {
    const T *cl = X + (int64_t)(slot ? slot[c] : c) * ld;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t k = tid + i * TT;
      const int64_t ch = reverse ? D.nchunks - 1 - k : k;
      if (k < D.nchunks) {
        T q[W];
        ldc(cl + ch * W, q);
#pragma unroll
        for (int v = 0; v < W; v++) acc += double(q[v]) * double(val[i][v]);
      }
    }
    red_put(sh, slot0 + c, acc);
  }
}

template <typename T, int RPC>
__device__ __forceinline__ double self_dot(const T (&a)[RPC][VT<T>::W], const T (&b)[RPC][VT<T>::W]) {
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < RPC; i++)
#pragma unroll
    for (int v = 0; v < VT<T>::W; v++) acc += double(a[i][v]) * double(b[i][v]);
  return acc;
}

// ---------------------------------------------------------------------------
// Gram form of Algorithm 3.1: scalar recurrences (one thread, every CTA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void coef_a(Shared &sh, int k) {
  if (threadIdx.x == 0) {
    for (int s = k - 1; s >= 0; s--) {
      double t = sh.sg[s];
      for (int u = s + 1; u < k; u++) t -= sh.a[u] * sh.gsr[s][u];
      sh.a[s] = t / sh.alpha[s];
    }
  }
  __syncthreads();
}

// rc[t] = r_t^T c0 (chronological), qc[c] = q_c^T c0
__device__ __forceinline__ void coef_b(Shared &sh, int k, int m, const double *rc, const double *qc) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < k; s++) {
      double t = rc[s];
      for (int u = 0; u < s; u++) t -= sh.ab[u] * sh.gsr[u][s];
      sh.b[s] = t / sh.alpha[s];
      sh.ab[s] = sh.a[s] + sh.b[s];
    }
    for (int c = 0; c < m; c++) {
      double t = qc[c];
      for (int u = 0; u < k; u++) t -= sh.ab[u] * sh.gqs[c][u];
      sh.zq[c] = t;
    }
  }
  __syncthreads();
}

// Gram matrices of the stored pairs: gsr[s][t] = s_s^T r_t, gqs[c][t] = q_c^T s_t.
template <typename T, int RPC>
__device__ bool gram(const Dev<T> &D, Shared &sh, Ctl &ctl, int m, int k) {
  constexpr int W = VT<T>::W;
  if (k == 0) return true;
  const int64_t tid = gtid(), TT = gthreads();
  const int per_s = k + m;  // slots per pair
  const int smax = RED_MAX / per_s;
  for (int s0 = 0; s0 < k; s0 += smax) {
    const int s1 = min(k, s0 + smax);
    for (int s = s0; s < s1; s++) {
      T sv[RPC][W];
      const T *scol = D.S + (int64_t)sh.order[s] * D.npad;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks)
          ldc(scol + ch * W, sv[i]);
        else
#pragma unroll
          for (int v = 0; v < W; v++) sv[i][v] = T(0);
      }
      dots_put<T, RPC>(sh, (s - s0) * per_s, D.R, D.npad, k, sh.order, D, sv, false);
      dots_put<T, RPC>(sh, (s - s0) * per_s + k, D.Q, D.npad, m, nullptr, D, sv, false);
    }
    if (!reduce_all(D, sh, ctl, (s1 - s0) * per_s, 10)) return false;
    if (threadIdx.x == 0)
      for (int s = s0; s < s1; s++) {
        for (int t = 0; t < k; t++) sh.gsr[s][t] = sh.sc[(s - s0) * per_s + t];
        for (int c = 0; c < m; c++) sh.gqs[c][s] = sh.sc[(s - s0) * per_s + k + c];
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int s = 0; s < k; s++) sh.alpha[s] = sh.gsr[s][s];
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// preconditioner tail: forward solve on w = g - R a, backward solve, the dot
// products of Algorithm 3.1's forward loop and Gram-Schmidt, and the output
// pass out = c0 - S(a+b) - Q z (+ beta * out, beta = gamma'/gamma_old when
// use_beta).  On entry z/c0 hold the not-yet-computed marker and the solve
// queues are reset.  *gamma_new receives gamma' = g^T c.
//
// The triangular solves (trsv_block) work slab by slab, one slab per CTA,
// with ctl.twarps warps of the CTA taking the slab's rows in order.  Dynamic
// shared memory holds two slab-sized buffers: A receives the forward results
// z of the slab, B first holds the forward right-hand side w and then the
// backward results; no right-hand side is fetched from global memory on the
// dependency chain.
// ---------------------------------------------------------------------------
extern __shared__ __align__(16) unsigned char nle_dyn_smem[];  // two slabs of the triangular solves

// Schedule of the triangular solves compiled into this translation unit
// (the build compiles every (precision, rows-per-thread) pair once per
// schedule, so each kernel holds one solve only and keeps its registers);
// the kernels carry it as a template argument so that the two builds'
// kernels have distinct names.
#ifndef NLE_CHAIN_TU
#define NLE_CHAIN_TU 0
#endif
constexpr bool kChainTU = NLE_CHAIN_TU != 0;

template <typename T>
__device__ __forceinline__ void trsv_forward(const Dev<T> &D, Shared &sh, const Ctl &ctl, int k) {
  const TriEll<T> L{D.Loff, D.Lw, D.Lcol, D.Lval, D.rdiag, D.Lround, D.trows};
  T *bufA = reinterpret_cast<T *>(nle_dyn_smem);
  T *bufB = bufA + D.bsize;
  const int64_t b0 = (int64_t)grank() * D.bsize;
  const int64_t nb = max((int64_t)0, min(D.npad, b0 + D.bsize) - b0);
  // w = g - R a for the slab's rows (trsv_block's first barrier orders these
  // stores before any use)
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
    T w = __ldcg(D.g + b0 + i);
    for (int t = 0; t < k; t++) w -= T(sh.a[t]) * __ldcg(D.R + (int64_t)sh.order[t] * D.npad + b0 + i);
    bufB[i] = w;
  }
  if constexpr (kChainTU) {
    const TriChain<T> C{D.Loff, D.Lw, D.Lcol, D.Lval, D.rdiag, D.Lwp, D.Ltask};
    trsv_chain<true, T>(C, D.z, D.npad, D.bsize, ctl.spin_ns, ctl.poll_ns, D.st, bufA,
                        [&](int64_t r) { return bufB[r - b0]; });
  } else {
    trsv_block<true, T>(L, D.z, D.npad, D.bsize, ctl.twarps, ctl.spin_ns, ctl.poll_ns, D.st, bufA,
                        [&](int64_t r) { return bufB[r - b0]; });
  }
}

// The right-hand side of the backward solve is the forward result of the
// CTA's own slab (buffer A), complete after trsv_forward's closing
// __syncthreads, so no grid barrier separates the two solves.
template <typename T>
__device__ __forceinline__ void trsv_backward(const Dev<T> &D, const Ctl &ctl) {
  const TriEll<T> U{D.Uoff, D.Uw, D.Ucol, D.Uval, D.rdiag, D.Uround, D.trows};
  const T *bufA = reinterpret_cast<const T *>(nle_dyn_smem);
  T *bufB = reinterpret_cast<T *>(nle_dyn_smem) + D.bsize;
  const int64_t b0 = (int64_t)grank() * D.bsize;
  if constexpr (kChainTU) {
    const TriChain<T> C{D.Uoff, D.Uw, D.Ucol, D.Uval, D.rdiag, D.Uwp, D.Utask};
    trsv_chain<false, T>(C, D.c0, D.npad, D.bsize, ctl.spin_ns, ctl.poll_ns, D.st, bufB,
                         [&](int64_t r) { return bufA[r - b0]; });
  } else {
    trsv_block<false, T>(U, D.c0, D.npad, D.bsize, ctl.twarps, ctl.spin_ns, ctl.poll_ns, D.st, bufB,
                         [&](int64_t r) { return bufA[r - b0]; });
  }
}

template <typename T>
__device__ __forceinline__ void reset_queues(const Dev<T> &D) {
  if (lead_cta() && threadIdx.x == 0) {
    D.st->qf = 0u;
    D.st->qb = 0u;
  }
}

template <typename T, int RPC>
__device__ bool precond_tail(const Dev<T> &D, Shared &sh, Ctl &ctl, int m, int k, T *out, double gamma_old,
                             bool use_beta, double *gamma_new) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  trsv_forward<T>(D, sh, ctl, k);
  tmark(sh, PH_FWD);
  trsv_backward<T>(D, ctl);
  if (!grid_sync(D.st, sh, ctl, 21)) return false;
  tmark(sh, PH_BWD);
  // dot products of c0: slots [0,k) r_t^T c0 ; k: g^T c0 ; [k+1, k+1+m) q_c^T c0
  T cv[RPC][W];
  {
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        T gg[W];
        ldc(D.c0 + ch * W, cv[i]);
        ldc(D.g + ch * W, gg);
#pragma unroll
        for (int v = 0; v < W; v++) acc += double(gg[v]) * double(cv[i][v]);
      } else {
#pragma unroll
        for (int v = 0; v < W; v++) cv[i][v] = T(0);
      }
    }
    red_put(sh, k, acc);
    dots_put<T, RPC>(sh, 0, D.R, D.npad, k, sh.order, D, cv, false);
    dots_put<T, RPC>(sh, k + 1, D.Q, D.npad, m, nullptr, D, cv, false);
  }
  if (!reduce_all(D, sh, ctl, k + 1 + m, 22)) return false;
  tmark(sh, PH_DOTS);
  const double gc0 = sh.sc[k];
  coef_b(sh, k, m, sh.sc, sh.sc + k + 1);
  // gamma' = g^T c = g^T c0 - (S^T g)(a+b)   (g is orthogonal to Q)
  double gnew = gc0;
  for (int s = 0; s < k; s++) gnew -= sh.sg[s] * sh.ab[s];
  *gamma_new = gnew;
  const double beta = use_beta ? gnew / gamma_old : 0.0;
  // output pass: out = c0 - S ab - Q z + beta*out
  {
    if (k > 0) comb_add<T, RPC>(D.S, D.npad, k, sh.ab, sh.order, D, cv, -1.0);
    if (m > 0) comb_add<T, RPC>(D.Q, D.npad, m, sh.zq, nullptr, D, cv, -1.0);
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        if (use_beta) {
          T po[W];
          ldc(out + ch * W, po);
#pragma unroll
          for (int v = 0; v < W; v++) cv[i][v] += T(beta) * po[v];
        }
        stv(out + ch * W, cv[i]);
      }
    }
  }
  const bool ok = grid_sync(D.st, sh, ctl, 23);
  tmark(sh, PH_DIR);
  return ok;
}

// ---------------------------------------------------------------------------
// PCG on the correction equation (Section 4.3): J s = -r, s perp Q, with
// J = (I-QQ^T)(A - theta I)(I-QQ^T) and P_k by Algorithm 3.1.
// Inputs in device memory: rT (r in working precision), Q (m columns), the
// k stored pairs (sh.order, S, R) and their Gram matrices (sh.gsr, sh.gqs,
// sh.alpha).  Output: s.  The residual g is kept orthogonal to Q by
// g <- g - alpha (y - Q (Q^T y)), which equals the update followed by the
// projection of g when g is orthogonal to Q.
// ---------------------------------------------------------------------------
struct PcgOut {
  int its;
  int exit;
  double rs;  // r^T s at exit (= alpha of the new pair)
  double g0, gn, eres;
};

template <typename T, int RPC>
__device__ bool pcg_solve(const Dev<T> &D, const Opts &O, Shared &sh, Ctl &ctl, int m, int k, double theta,
                          int max_pcg, PcgOut &res) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  const T Tsent = sentinel<T>();
  T gv[RPC][W];
  // --- initial residual g = -(I - QQ^T) r, s = 0
  {
    T rv[RPC][W];
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks)
        ldc(D.rT + ch * W, rv[i]);
      else
#pragma unroll
        for (int v = 0; v < W; v++) rv[i][v] = T(0);
    }
    dots_put<T, RPC>(sh, 0, D.Q, D.npad, m, nullptr, D, rv, false);
    if (!reduce_all(D, sh, ctl, m, 30)) return false;
    for (int c = threadIdx.x; c < m; c += TPB) sh.qv[c] = -sh.sc[c];
    __syncthreads();
    comb_add<T, RPC>(D.Q, D.npad, m, sh.qv, nullptr, D, rv, 1.0);  // rv = r - Q Q^T r
    T sent[W], zero[W];
#pragma unroll
    for (int v = 0; v < W; v++) sent[v] = Tsent, zero[v] = T(0);
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
#pragma unroll
      for (int v = 0; v < W; v++) gv[i][v] = -rv[i][v];
      if (ch < D.nchunks) {
        stv(D.g + ch * W, gv[i]);
        stv(D.s + ch * W, zero);
        stv(D.z + ch * W, sent);
        stv(D.c0 + ch * W, sent);
      }
    }
    reset_queues(D);
    red_put(sh, 0, self_dot<T, RPC>(gv, gv));
    dots_put<T, RPC>(sh, 1, D.S, D.npad, k, sh.order, D, gv, false);
    if (!reduce_all(D, sh, ctl, 1 + k, 31)) return false;
    tmark(sh, PH_UPDATE);
  }
  const double g0 = sqrt(sh.sc[0]);
  if (threadIdx.x == 0)
    for (int s = 0; s < k; s++) sh.sg[s] = sh.sc[1 + s];
  __syncthreads();
  coef_a(sh, k);
  double gamma;
  if (!precond_tail<T, RPC>(D, sh, ctl, m, k, D.p, 0.0, false, &gamma)) return false;

  res.g0 = g0;
  res.gn = g0;
  res.eres = 0.0;
  res.rs = 0.0;
  res.exit = 1;  // NLE_EXIT_MAXIT
  res.its = 0;
  double gprev = g0, eprev = 0.0;
  for (int l = 0; l < max_pcg; l++) {
    // --- pass A: y = (A - theta I) p, delta = p^T y, Q^T y
    T yv[RPC][W];
    {
      double pty = 0.0;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          T acc[W], pp[W];
          sell_rows<W, T, T, T>(D.A, D.p, ch, acc);
          ldc(D.p + ch * W, pp);
#pragma unroll
          for (int v = 0; v < W; v++) {
            yv[i][v] = acc[v] - T(theta) * pp[v];
            pty += double(pp[v]) * double(yv[i][v]);
          }
          stv(D.y + ch * W, yv[i]);
        } else {
#pragma unroll
          for (int v = 0; v < W; v++) yv[i][v] = T(0);
        }
      }
      red_put(sh, 0, pty);
      dots_put<T, RPC>(sh, 1, D.Q, D.npad, m, nullptr, D, yv, false);
      if (!reduce_all(D, sh, ctl, 1 + m, 32)) return false;
      tmark(sh, PH_SPMV);
    }
    const double delta = sh.sc[0];
    if (!(delta > 0.0)) {
      res.exit = 4;  // NLE_EXIT_BREAKDOWN
      res.its = l;
      break;
    }
    res.its = l + 1;
    const double alpha = gamma / delta;
    // --- pass B: s += alpha p; g -= alpha (y - Q Q^T y); exit scalars; S^T g
    {
      for (int c = threadIdx.x; c < m; c += TPB) sh.qv[c] = -sh.sc[1 + c];
      __syncthreads();
      comb_add<T, RPC>(D.Q, D.npad, m, sh.qv, nullptr, D, yv, 1.0);  // yv = (I - QQ^T) y
      double rs = 0.0, sg = 0.0, ss = 0.0;
      T sent[W];
#pragma unroll
      for (int v = 0; v < W; v++) sent[v] = Tsent;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          T pp[W], sv[W], rr[W];
          ldc(D.p + ch * W, pp);
          ldc(D.s + ch * W, sv);
          ldc(D.g + ch * W, gv[i]);
          ldc(D.rT + ch * W, rr);
#pragma unroll
          for (int v = 0; v < W; v++) {
            sv[v] += T(alpha) * pp[v];
            gv[i][v] -= T(alpha) * yv[i][v];
            rs += double(rr[v]) * double(sv[v]);
            sg += double(sv[v]) * double(gv[i][v]);
            ss += double(sv[v]) * double(sv[v]);
          }
          stv(D.s + ch * W, sv);
          stv(D.g + ch * W, gv[i]);
          stv(D.z + ch * W, sent);
          stv(D.c0 + ch * W, sent);
        } else {
#pragma unroll
          for (int v = 0; v < W; v++) gv[i][v] = T(0);
        }
      }
      reset_queues(D);
      red_put(sh, 0, self_dot<T, RPC>(gv, gv));
      red_put(sh, 1, rs);
      red_put(sh, 2, sg);
      red_put(sh, 3, ss);
      dots_put<T, RPC>(sh, 4, D.S, D.npad, k, sh.order, D, gv, false);
      if (!reduce_all(D, sh, ctl, 4 + k, 33)) return false;
      tmark(sh, PH_UPDATE);
    }
    const double gn = sqrt(sh.sc[0]);
    const double rs = sh.sc[1], sg = sh.sc[2], ss = sh.sc[3];
    // Exit (iii), eq. "residual", without a product with A.  With x = u + s,
    // s orthogonal to Q (u is a column of Q), (A - theta I) u = r and
    // J s = -r - g, and neglecting v_i^T (A - theta I) s for the converged
    // v_i: ||A x - theta x||^2 = ||g||^2 + (r^T s)^2,
    // x^T (A - theta I) x = r^T s - s^T g, so rho - theta =
    // (r^T s - s^T g) / (1 + ||s||^2) and ||A x - rho x||^2 =
    // ||A x - theta x||^2 - (rho - theta)^2 (1 + ||s||^2).
    const double x2 = 1.0 + ss;
    const double dth = (rs - sg) / x2;
    const double e2 = gn * gn + rs * rs - dth * dth * x2;
    const double eres = sqrt(fmax(e2, 0.0) / x2);
    const double rho = theta + dth;
    res.gn = gn;
    res.eres = eres;
    res.rs = rs;
    if (gn <= O.tau_pcg * g0) {
      res.exit = 0;
      break;
    }
    if (O.exit_eigres && eres < O.tol * rho) {
      res.exit = 2;
      break;
    }
    if (O.exit_stag && l >= 1 && eres / eprev > gn / gprev) {
      res.exit = 3;
      break;
    }
    if (l + 1 == max_pcg) {
      res.exit = 1;
      break;
    }
    if (threadIdx.x == 0)
      for (int s = 0; s < k; s++) sh.sg[s] = sh.sc[4 + s];
    __syncthreads();
    coef_a(sh, k);
    double gnew;
    if (!precond_tail<T, RPC>(D, sh, ctl, m, k, D.p, gamma, true, &gnew)) return false;
    gamma = gnew;
    gprev = gn;
    eprev = eres;
  }
  return true;
}

// ---------------------------------------------------------------------------
// FP64 pieces of the outer step
// ---------------------------------------------------------------------------

// Au = A u (FP64), returns u^T A u and u^T u in sh.sc[0..1].  u = Qt column j.
template <typename T, int RPC>
__device__ bool fp64_rayleigh(const Dev<T> &D, Shared &sh, Ctl &ctl, const double *u) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  double uau = 0.0, uu = 0.0;
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks) {
      double acc[W], uv[W];
      sell_rows<W, double, double, double>(D.A64, u, ch, acc);
      ldc(u + ch * W, uv);
#pragma unroll
      for (int v = 0; v < W; v++) {
        uau += uv[v] * acc[v];
        uu += uv[v] * uv[v];
      }
      stv(D.Au + ch * W, acc);
    }
  }
  red_put(sh, 0, uau);
  red_put(sh, 1, uu);
  return reduce_all(D, sh, ctl, 2, 40);
}

// r = A u - theta u (FP64, and its working-precision copy rT), ||r||^2 in
// sh.sc[0]; shadows Q[:, j] = u.  With stage >= 0 (full BFGS update) the staged pair's second vector, which
// holds r_k, becomes w = r_k - r_{k+1} and sc[1] = s^T w.
template <typename T, int RPC>
__device__ bool fp64_residual(const Dev<T> &D, Shared &sh, Ctl &ctl, const double *u, double theta, int j,
                              int stage = -1) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  double rr = 0.0, sw = 0.0;
  T *uq = D.Q + (int64_t)j * D.npad;
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks) {
      double au[W], uv[W], rv[W];
      ldc(D.Au + ch * W, au);
      ldc(u + ch * W, uv);
      T rt[W], ut[W];
#pragma unroll
      for (int v = 0; v < W; v++) {
        rv[v] = au[v] - theta * uv[v];
        rr += rv[v] * rv[v];
        rt[v] = T(rv[v]);
        ut[v] = T(uv[v]);
      }
      stv(D.r + ch * W, rv);
      stv(D.rT + ch * W, rt);
      stv(uq + ch * W, ut);
      if (stage >= 0) {
        T sv[W], wv[W];
        ldc(D.S + (int64_t)stage * D.npad + ch * W, sv);
        ldc(D.R + (int64_t)stage * D.npad + ch * W, wv);
#pragma unroll
        for (int v = 0; v < W; v++) {
          wv[v] = T(double(wv[v]) - rv[v]);
          sw += double(sv[v]) * double(wv[v]);
        }
        stv(D.R + (int64_t)stage * D.npad + ch * W, wv);
      }
    }
  }
  red_put(sh, 0, rr);
  if (stage >= 0) red_put(sh, 1, sw);
  return reduce_all(D, sh, ctl, stage >= 0 ? 2 : 1, 41);
}

template <typename T>
__device__ void load_state(const Dev<T> &D, Shared &sh, Ctl &ctl, const Opts &O, int gbase = 0, int gsize = -1) {
  if (threadIdx.x == 0) {
    s_gbase = gbase;
    s_gsize = gsize > 0 ? gsize : (int)gridDim.x;
  }
  ctl.epoch = 0;
  ctl.rbuf = 0;
  ctl.spin_ns = O.spin_ns;
  ctl.twarps = max(1, min(NWARP, O.trsv_warps));
  ctl.poll_ns = O.poll_ns;
  if (threadIdx.x == 0) {
    sh.ok = 1;
    for (int s = 0; s < KMAX; s++) sh.order[s] = s;
    for (int q = 0; q < 8; q++) sh.tacc[q] = 0;
    sh.tlast = gtimer();
  }
  __syncthreads();
}

// add this launch's phase times to the state (CTA 0)
__device__ __forceinline__ void flush_timers(State *st, Shared &sh) {
  if (lead_cta() && threadIdx.x == 0)
    for (int q = 0; q < 8; q++) st->tphase[q] += sh.tacc[q];
}

// ---------------------------------------------------------------------------
// Kernel: Newton iteration for eigenpair j (Algorithm 3.2, inner loop)
// ---------------------------------------------------------------------------
template <typename T, int RPC>
__device__ bool newton_body(const Dev<T> &D, const Opts &O, Shared &sh, Ctl &ctl, int j) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  const int m = j + 1;
  double *u = D.Qt + (int64_t)j * D.npad;
  int k = 0;  // pairs reset for every eigenpair
  int spare = O.kmax;  // full update: physical slot staging the newest pair
  if (threadIdx.x == 0)
    for (int s = 0; s < KMAX; s++) sh.order[s] = s;
  __syncthreads();
  long long mvp = 0, pcg_total = 0, sum_m = 0, sum_k = 0;
  int pcg_sum = 0;
  int exits[5] = {0, 0, 0, 0, 0};

  if (!fp64_rayleigh<T, RPC>(D, sh, ctl, u)) return false;
  mvp++;
  double theta = sh.sc[0] / sh.sc[1];
  if (!fp64_residual<T, RPC>(D, sh, ctl, u, theta, j)) return false;
  double rnorm = sqrt(sh.sc[0]);
  tmark(sh, PH_OUTER);
  int it = 0;
  while (rnorm > O.tol * theta && it < O.max_newton) {
    if (!gram<T, RPC>(D, sh, ctl, m, k)) return false;
    tmark(sh, PH_OTHER);
    PcgOut po;
    if (!pcg_solve<T, RPC>(D, O, sh, ctl, m, k, theta, O.max_pcg, po)) return false;
    mvp += po.its;
    pcg_total += po.its;
    pcg_sum += po.its;
    sum_m += (long long)po.its * m;
    sum_k += (long long)po.its * k;
    exits[po.exit]++;
    // simplified update: store the pair (s_k, r_k) when alpha = s^T r_k < 0
    // (Theorem 3.2) in the ring of k_max slots.  Full update: copy (s_k, r_k)
    // into the spare slot; it becomes (s_k, r_k - r_{k+1}) with the next
    // residual and joins the ring if s^T w < 0.
    int slot = -1, stage = -1;
    if (O.kmax > 0 && O.bfgs_full) {
      stage = spare;
    } else if (O.kmax > 0 && po.rs < 0.0) {
      if (k < O.kmax) {
        slot = k;
        if (threadIdx.x == 0) sh.order[k] = k;
        k++;
      } else {
        if (threadIdx.x == 0) {
          slot = sh.order[0];
          for (int s = 0; s + 1 < k; s++) sh.order[s] = sh.order[s + 1];
          sh.order[k - 1] = slot;
        }
        __syncthreads();
        slot = sh.order[k - 1];
      }
    }
    __syncthreads();
    const int wslot = slot >= 0 ? slot : stage;
    // N1: t = u + s (FP64); copy the pair; ||t||^2, Qt^T t
    double tv[RPC][W];
    {
      double tt = 0.0;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          double uv[W];
          T sv[W];
          ldc(u + ch * W, uv);
          ldc(D.s + ch * W, sv);
#pragma unroll
          for (int v = 0; v < W; v++) {
            tv[i][v] = uv[v] + double(sv[v]);
            tt += tv[i][v] * tv[i][v];
          }
          if (wslot >= 0) {
            T rt[W];
            ldc(D.rT + ch * W, rt);
            stv(D.S + (int64_t)wslot * D.npad + ch * W, sv);
            stv(D.R + (int64_t)wslot * D.npad + ch * W, rt);
          }
        } else {
#pragma unroll
          for (int v = 0; v < W; v++) tv[i][v] = 0.0;
        }
      }
      red_put(sh, 0, tt);
      for (int c = 0; c < j; c++) {
        const double *qc = D.Qt + (int64_t)c * D.npad;
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < RPC; i++) {
          const int64_t ch = tid + i * TT;
          if (ch < D.nchunks) {
            double q[W];
            ldc(qc + ch * W, q);
#pragma unroll
            for (int v = 0; v < W; v++) acc += q[v] * tv[i][v];
          }
        }
        red_put(sh, 1 + c, acc);
      }
      if (!reduce_all(D, sh, ctl, 1 + j, 42)) return false;
    }
    // N2: u = (t - Qt (Qt^T t)) / ||.||  (re-orthogonalisation against the
    // converged eigenvectors, then normalisation)
    {
      double nq = 0.0;
      for (int c = 0; c < j; c++) nq += sh.sc[1 + c] * sh.sc[1 + c];
      const double inv = 1.0 / sqrt(sh.sc[0] - nq);
      for (int c = 0; c < j; c++) {
        const double *qc = D.Qt + (int64_t)c * D.npad;
        const double cf = sh.sc[1 + c];
#pragma unroll
        for (int i = 0; i < RPC; i++) {
          const int64_t ch = tid + i * TT;
          if (ch < D.nchunks) {
            double q[W];
            ldc(qc + ch * W, q);
#pragma unroll
            for (int v = 0; v < W; v++) tv[i][v] -= cf * q[v];
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
#pragma unroll
          for (int v = 0; v < W; v++) tv[i][v] *= inv;
          stv(u + ch * W, tv[i]);
        }
      }
      if (!grid_sync(D.st, sh, ctl, 43)) return false;
    }
    if (!fp64_rayleigh<T, RPC>(D, sh, ctl, u)) return false;
    mvp++;
    theta = sh.sc[0] / sh.sc[1];
    if (!fp64_residual<T, RPC>(D, sh, ctl, u, theta, j, stage)) return false;
    rnorm = sqrt(sh.sc[0]);
    if (stage >= 0 && sh.sc[1] < 0.0) {
      // the staged pair joins the ring; the slot it replaces (or the lowest
      // free one) becomes the spare
      if (k < O.kmax) {
        if (threadIdx.x == 0) sh.order[k] = stage;
        k++;
        __syncthreads();
        for (spare = 0;; spare++) {
          bool used = false;
          for (int s = 0; s < k; s++) used = used || sh.order[s] == spare;
          if (!used) break;
        }
      } else {
        const int evicted = sh.order[0];
        __syncthreads();
        if (threadIdx.x == 0) {
          for (int s = 0; s + 1 < k; s++) sh.order[s] = sh.order[s + 1];
          sh.order[k - 1] = stage;
        }
        spare = evicted;
      }
      __syncthreads();
    }
    tmark(sh, PH_OUTER);
    it++;
  }
  flush_timers(D.st, sh);
  if (lead_cta() && threadIdx.x == 0) {
    State *st = D.st;
    st->theta = theta;
    st->rnorm = rnorm;
    st->lambda[j] = theta;
    st->res[j] = rnorm / theta;
    st->outer_its[j] = it;
    st->pcg_its[j] = pcg_sum;
    st->conv[j] = (rnorm <= O.tol * theta) ? 1 : 0;
    st->mvp_newton += mvp;
    st->pcg_total += pcg_total;
    st->pcg_sum_m += sum_m;
    st->pcg_sum_k += sum_k;
    for (int e = 0; e < 5; e++) st->exits[e] += exits[e];
  }
  return true;
}

template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_newton(Dev<T> D, Opts O) {
  __shared__ Shared sh;
  Ctl ctl;
  load_state(D, sh, ctl, O);
  newton_body<T, RPC>(D, O, sh, ctl, D.st->j);
}

// ---------------------------------------------------------------------------
// Kernel: DACG for eigenpair j (Section 4.1): preconditioned nonlinear CG on
// the Rayleigh quotient in the complement of the converged eigenvectors.
// On entry x holds the start vector; on exit Qt[:, j] holds u_0 (FP64).
// ---------------------------------------------------------------------------
template <typename T, int RPC>
__device__ bool dacg_body(const Dev<T> &D, const Opts &O, Shared &sh, Ctl &ctl, int j) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  const int mq = j;  // converged eigenvectors (shadow columns of Q)
  const T Tsent = sentinel<T>();
  long long mvp = 0;
  T xv[RPC][W];
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks)
      ldc((D.X0 ? D.X0 + (int64_t)j * D.npad : D.x) + ch * W, xv[i]);
    else
#pragma unroll
      for (int v = 0; v < W; v++) xv[i][v] = T(0);
  }
  // x0 projected on the complement of Q~ twice (classical Gram-Schmidt)
  for (int rep = 0; rep < 2 && mq > 0; rep++) {
    dots_put<T, RPC>(sh, 0, D.Q, D.npad, mq, nullptr, D, xv, false);
    if (!reduce_all(D, sh, ctl, mq, 50)) return false;
    for (int c = threadIdx.x; c < mq; c += TPB) sh.qv[c] = -sh.sc[c];
    __syncthreads();
    comb_add<T, RPC>(D.Q, D.npad, mq, sh.qv, nullptr, D, xv, 1.0);
  }
  red_put(sh, 0, self_dot<T, RPC>(xv, xv));
  if (!reduce_all(D, sh, ctl, 1, 51)) return false;
  {
    const T inv = T(1.0 / sqrt(sh.sc[0]));
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
#pragma unroll
      for (int v = 0; v < W; v++) xv[i][v] *= inv;
      if (ch < D.nchunks) stv(D.x + ch * W, xv[i]);
    }
  }
  if (!grid_sync(D.st, sh, ctl, 52)) return false;
  // Ax
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks) {
      T acc[W];
      sell_rows<W, T, T, T>(D.A, D.x, ch, acc);
      stv(D.Ax + ch * W, acc);
    }
  }
  mvp++;
  if (!grid_sync(D.st, sh, ctl, 53)) return false;

  double nx = 1.0, gg_prev = 0.0;
  int its = 0;
  for (int it = 0; it < O.max_dacg; it++) {
    // P1: normalise x, Ax by the last norm; q = x^T A x, f = x^T x
    T av[RPC][W];
    {
      const T inv = T(1.0 / nx);
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          ldc(D.x + ch * W, xv[i]);
          ldc(D.Ax + ch * W, av[i]);
          if (nx != 1.0) {
#pragma unroll
            for (int v = 0; v < W; v++) xv[i][v] *= inv, av[i][v] *= inv;
            stv(D.x + ch * W, xv[i]);
            stv(D.Ax + ch * W, av[i]);
          }
        } else {
#pragma unroll
          for (int v = 0; v < W; v++) xv[i][v] = T(0), av[i][v] = T(0);
        }
      }
      red_put(sh, 0, self_dot<T, RPC>(xv, av));
      red_put(sh, 1, self_dot<T, RPC>(xv, xv));
      if (!reduce_all(D, sh, ctl, 2, 54)) return false;
      nx = 1.0;  // x and Ax now hold the normalised iterate
    }
    const double q = sh.sc[0], f = sh.sc[1];
    // P2: g = A x - q x, ||g||; reset the solve outputs
    T gv[RPC][W];
    {
      T sent[W];
#pragma unroll
      for (int v = 0; v < W; v++) sent[v] = Tsent;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
#pragma unroll
        for (int v = 0; v < W; v++) gv[i][v] = av[i][v] - T(q) * xv[i][v];
        if (ch < D.nchunks) {
          stv(D.g + ch * W, gv[i]);
          stv(D.z + ch * W, sent);
          stv(D.c0 + ch * W, sent);
        }
      }
      reset_queues(D);
      red_put(sh, 0, self_dot<T, RPC>(gv, gv));
      if (!reduce_all(D, sh, ctl, 1, 55)) return false;
      tmark(sh, PH_UPDATE);
    }
    if (sqrt(sh.sc[0]) <= O.tau_dacg * q) break;
    // P3-P5: gt = (I - Q~Q~^T) Phat_0 g,  p = -gt + beta p
    double gg;
    {
      // Phat_0 g via the preconditioner tail with no pairs, writing into Ap as
      // scratch: Ap = c0 - Q z, then p = -Ap + beta p below.
      if (!precond_tail<T, RPC>(D, sh, ctl, mq, 0, D.Ap, 0.0, false, &gg)) return false;
      const double beta = (it == 0) ? 0.0 : gg / gg_prev;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          T gt[W], pp[W];
          ldc(D.Ap + ch * W, gt);
          if (it > 0) {
            ldc(D.p + ch * W, pp);
#pragma unroll
            for (int v = 0; v < W; v++) pp[v] = -gt[v] + T(beta) * pp[v];
          } else {
#pragma unroll
            for (int v = 0; v < W; v++) pp[v] = -gt[v];
          }
          stv(D.p + ch * W, pp);
        }
      }
      if (!grid_sync(D.st, sh, ctl, 56)) return false;
      tmark(sh, PH_DIR);
    }
    // P6: Ap = A p; line-search scalars
    {
      double a = 0.0, b = 0.0, d = 0.0, e = 0.0;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          T acc[W], pp[W];
          sell_rows<W, T, T, T>(D.A, D.p, ch, acc);
          ldc(D.p + ch * W, pp);
#pragma unroll
          for (int v = 0; v < W; v++) {
            a += double(pp[v]) * double(acc[v]);
            b += double(xv[i][v]) * double(acc[v]);
            d += double(pp[v]) * double(pp[v]);
            e += double(xv[i][v]) * double(pp[v]);
          }
          stv(D.Ap + ch * W, acc);
        }
      }
      mvp++;
      red_put(sh, 0, a);
      red_put(sh, 1, b);
      red_put(sh, 2, d);
      red_put(sh, 3, e);
      if (!reduce_all(D, sh, ctl, 4, 57)) return false;
      tmark(sh, PH_SPMV);
    }
    double al;
    {
      const double a = sh.sc[0], b = sh.sc[1], c = q, d = sh.sc[2], e = sh.sc[3];
      const double A2 = a * e - b * d, B2 = a * f - c * d, C2 = b * f - c * e;
      if (A2 == 0.0) {
        al = (B2 != 0.0) ? -C2 / B2 : 0.0;
      } else {
        const double disc = fmax(B2 * B2 - 4.0 * A2 * C2, 0.0);
        const double t = -0.5 * (B2 + copysign(sqrt(disc), B2));
        const double r1 = t / A2;
        al = r1;
        if (t != 0.0) {
          const double r2 = C2 / t;
          const double q1 = (c + 2 * r1 * b + r1 * r1 * a) / (f + 2 * r1 * e + r1 * r1 * d);
          const double q2 = (c + 2 * r2 * b + r2 * r2 * a) / (f + 2 * r2 * e + r2 * r2 * d);
          if (q2 < q1) al = r2;
        }
      }
    }
    // P7: x += al p, Ax += al Ap, ||x||
    {
      double xx = 0.0;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          T pp[W], ap[W];
          ldc(D.p + ch * W, pp);
          ldc(D.Ap + ch * W, ap);
#pragma unroll
          for (int v = 0; v < W; v++) {
            xv[i][v] += T(al) * pp[v];
            av[i][v] += T(al) * ap[v];
            xx += double(xv[i][v]) * double(xv[i][v]);
          }
          stv(D.x + ch * W, xv[i]);
          stv(D.Ax + ch * W, av[i]);
        }
      }
      red_put(sh, 0, xx);
      if (!reduce_all(D, sh, ctl, 1, 58)) return false;
      nx = sqrt(sh.sc[0]);
      tmark(sh, PH_UPDATE);
    }
    its = it + 1;
    if (O.recompute > 0 && its % O.recompute == 0) {
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          T acc[W];
          sell_rows<W, T, T, T>(D.A, D.x, ch, acc);
          stv(D.Ax + ch * W, acc);
        }
      }
      mvp++;
      if (!grid_sync(D.st, sh, ctl, 59)) return false;
    }
    gg_prev = gg;
  }
  // u_0 = x / ||x|| in FP64 into Qt[:, j]
  {
    double *u = D.Qt + (int64_t)j * D.npad;
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        T xx[W];
        ldc(D.x + ch * W, xx);
        double uv[W];
#pragma unroll
        for (int v = 0; v < W; v++) uv[v] = double(xx[v]) / nx;
        stv(u + ch * W, uv);
      }
    }
  }
  flush_timers(D.st, sh);
  if (lead_cta() && threadIdx.x == 0) {
    D.st->dacg_its[j] = its;
    D.st->mvp_dacg += mvp;
    D.st->dacg_total += its;
    D.st->dacg_sum_m += (long long)its * mq;
  }
  return true;
}

template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_dacg(Dev<T> D, Opts O) {
  __shared__ Shared sh;
  Ctl ctl;
  load_state(D, sh, ctl, O);
  dacg_body<T, RPC>(D, O, sh, ctl, D.st->j);
}

// ---------------------------------------------------------------------------
// Kernels exposing single building blocks (verification entry points)
// ---------------------------------------------------------------------------

// y = (A - theta I) x  (x in D.p, y in D.y)
template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_shifted(Dev<T> D, double theta) {
  constexpr int W = VT<T>::W;
  if (threadIdx.x == 0) {
    s_gbase = 0;
    s_gsize = (int)gridDim.x;
  }
  __syncthreads();
  const int64_t tid = gtid(), TT = gthreads();
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks) {
      T acc[W], pp[W];
      sell_rows<W, T, T, T>(D.A, D.p, ch, acc);
      ldc(D.p + ch * W, pp);
#pragma unroll
      for (int v = 0; v < W; v++) acc[v] -= T(theta) * pp[v];
      stv(D.y + ch * W, acc);
    }
  }
}

// c = P_k g by Algorithm 3.1 (g in D.g, output in D.y); m columns of Q, k pairs
// in slots 0..k-1 (chronological).
template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_prec(Dev<T> D, Opts O, int m, int k) {
  constexpr int W = VT<T>::W;
  __shared__ Shared sh;
  Ctl ctl;
  load_state(D, sh, ctl, O);
  if (threadIdx.x == 0)
    for (int s = 0; s < KMAX; s++) sh.order[s] = s;
  __syncthreads();
  if (!gram<T, RPC>(D, sh, ctl, m, k)) return;
  const int64_t tid = gtid(), TT = gthreads();
  const T Tsent = sentinel<T>();
  T gv[RPC][W];
  T sent[W];
#pragma unroll
  for (int v = 0; v < W; v++) sent[v] = Tsent;
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks) {
      ldc(D.g + ch * W, gv[i]);
      stv(D.z + ch * W, sent);
      stv(D.c0 + ch * W, sent);
    } else {
#pragma unroll
      for (int v = 0; v < W; v++) gv[i][v] = T(0);
    }
  }
  reset_queues(D);
  dots_put<T, RPC>(sh, 0, D.S, D.npad, k, sh.order, D, gv, false);
  if (!reduce_all(D, sh, ctl, k, 60)) return;
  if (threadIdx.x == 0)
    for (int s = 0; s < k; s++) sh.sg[s] = sh.sc[s];
  __syncthreads();
  coef_a(sh, k);
  double gamma;
  precond_tail<T, RPC>(D, sh, ctl, m, k, D.y, 0.0, false, &gamma);
}

// One inner solve: theta given, r in rT, Q with m columns, k pairs in slots 0..k-1.
template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_pcg(Dev<T> D, Opts O, int m, int k, double theta, int max_pcg) {
  __shared__ Shared sh;
  Ctl ctl;
  load_state(D, sh, ctl, O);
  if (threadIdx.x == 0)
    for (int s = 0; s < KMAX; s++) sh.order[s] = s;
  __syncthreads();
  if (!gram<T, RPC>(D, sh, ctl, m, k)) return;
  PcgOut po;
  if (!pcg_solve<T, RPC>(D, O, sh, ctl, m, k, theta, max_pcg, po)) return;
  if (lead_cta() && threadIdx.x == 0) {
    D.st->last_its = po.its;
    D.st->last_exit = po.exit;
    D.st->last_g0 = po.g0;
    D.st->last_gn = po.gn;
    D.st->last_eres = po.eres;
  }
}

// ---------------------------------------------------------------------------
// Kernel: adjoint solve for eigenvector j (not in the paper).
// On entry b64 holds gbar_j (device order, FP64, already multiplied by the
// sign of the output eigenvector); Qt holds v_1..v_p (FP64) and Q their
// working-precision shadows; st->lambda the eigenvalues.  Computes
//   c_i = v_i^T gbar,   b = gbar - V c,
//   y perp V solving (I-VV^T)(A - lambda_j I)(I-VV^T) y = b,
//   xi = -sum_{i != j} v_i c_i / (lambda_i - lambda_j) - y   (written to t),
// the solve by iterative refinement: FP64 residual rho = b - (I-VV^T)(A -
// lambda_j I) y with the FP64 matrix, correction by the inner projected PCG
// of the correction equation (Q = V, IC preconditioner, shift lambda_j) in the
// working precision, until ||rho|| <= tol ||b||.
// ---------------------------------------------------------------------------
template <typename T, int RPC>
__device__ bool fp64_project_dots(const Dev<T> &D, Shared &sh, Ctl &ctl, int p, const double (&v)[RPC][VT<T>::W],
                                  int where) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  int c = 0;
  for (; c < p; c++) {
    const double *qc = D.Qt + (int64_t)c * D.npad;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        double q[W];
        ldc(qc + ch * W, q);
#pragma unroll
        for (int u = 0; u < W; u++) acc += q[u] * v[i][u];
      }
    }
    red_put(sh, c, acc);
  }
  return reduce_all(D, sh, ctl, p, where);
}

template <typename T, int RPC>
__device__ void fp64_comb_add(const Dev<T> &D, int p, const double *coef, double sgn, double (&v)[RPC][VT<T>::W]) {
  constexpr int W = VT<T>::W;
  const int64_t tid = gtid(), TT = gthreads();
  for (int c = 0; c < p; c++) {
    const double *qc = D.Qt + (int64_t)c * D.npad;
    const double cf = sgn * coef[c];
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        double q[W];
        ldc(qc + ch * W, q);
#pragma unroll
        for (int u = 0; u < W; u++) v[i][u] += cf * q[u];
      }
    }
  }
}

template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_adjoint(Dev<T> D, Opts O, int j, int p, double tol, int max_refine) {
  constexpr int W = VT<T>::W;
  __shared__ Shared sh;
  Ctl ctl;
  load_state(D, sh, ctl, O);
  const int64_t tid = gtid(), TT = gthreads();
  const double lam = D.st->lambda[j];
  double v[RPC][W];
  // 1-2: c = V^T gbar, b = gbar - V c, y = 0
#pragma unroll
  for (int i = 0; i < RPC; i++) {
    const int64_t ch = tid + i * TT;
    if (ch < D.nchunks)
      ldc(D.b64 + ch * W, v[i]);
    else
#pragma unroll
      for (int u = 0; u < W; u++) v[i][u] = 0.0;
  }
  if (!fp64_project_dots<T, RPC>(D, sh, ctl, p, v, 70)) return;
  for (int c = threadIdx.x; c < p; c += TPB) sh.cadj[c] = sh.sc[c];
  __syncthreads();
  fp64_comb_add<T, RPC>(D, p, sh.cadj, -1.0, v);
  {
    double bb = 0.0;
    const double zero[W] = {};
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        stv(D.b64 + ch * W, v[i]);
        double zz[W];
#pragma unroll
        for (int u = 0; u < W; u++) zz[u] = zero[u];
        stv(D.y64 + ch * W, zz);
#pragma unroll
        for (int u = 0; u < W; u++) bb += v[i][u] * v[i][u];
      }
    }
    red_put(sh, 0, bb);
    if (!reduce_all(D, sh, ctl, 1, 71)) return;
  }
  const double bn = sqrt(sh.sc[0]);
  int refine = 0, inner = 0;
  double res = 0.0;
  for (int it = 0; bn > 0.0 && it < max_refine; it++) {
    // a: w = (A - lambda I) y in FP64, V^T w
    double w[RPC][W];
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        double acc[W], yy[W];
        sell_rows<W, double, double, double>(D.A64, D.y64, ch, acc);
        ldc(D.y64 + ch * W, yy);
#pragma unroll
        for (int u = 0; u < W; u++) w[i][u] = acc[u] - lam * yy[u];
      } else {
#pragma unroll
        for (int u = 0; u < W; u++) w[i][u] = 0.0;
      }
    }
    if (!fp64_project_dots<T, RPC>(D, sh, ctl, p, w, 72)) return;
    for (int c = threadIdx.x; c < p; c += TPB) sh.qv[c] = sh.sc[c];
    __syncthreads();
    fp64_comb_add<T, RPC>(D, p, sh.qv, -1.0, w);  // w = (I - VV^T)(A - lambda I) y
    // b: rho = b - w, ||rho||, rT = -rho
    {
      double rr = 0.0;
#pragma unroll
      for (int i = 0; i < RPC; i++) {
        const int64_t ch = tid + i * TT;
        if (ch < D.nchunks) {
          double bv[W];
          T rt[W];
          ldc(D.b64 + ch * W, bv);
#pragma unroll
          for (int u = 0; u < W; u++) {
            const double rho = bv[u] - w[i][u];
            rr += rho * rho;
            rt[u] = T(-rho);
          }
          stv(D.rT + ch * W, rt);
        }
      }
      red_put(sh, 0, rr);
      if (!reduce_all(D, sh, ctl, 1, 73)) return;
    }
    res = sqrt(sh.sc[0]) / bn;
    if (res <= tol) break;
    // d: correction by the inner projected PCG (J s = rho)
    PcgOut po;
    if (!pcg_solve<T, RPC>(D, O, sh, ctl, p, 0, lam, O.max_pcg, po)) return;
    inner += po.its;
    refine++;
    // e: y += s, then y -= V V^T y
    double yv[RPC][W];
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        T sv[W];
        ldc(D.y64 + ch * W, yv[i]);
        ldc(D.s + ch * W, sv);
#pragma unroll
        for (int u = 0; u < W; u++) yv[i][u] += double(sv[u]);
      } else {
#pragma unroll
        for (int u = 0; u < W; u++) yv[i][u] = 0.0;
      }
    }
    if (!fp64_project_dots<T, RPC>(D, sh, ctl, p, yv, 74)) return;
    for (int c = threadIdx.x; c < p; c += TPB) sh.qv[c] = sh.sc[c];
    __syncthreads();
    fp64_comb_add<T, RPC>(D, p, sh.qv, -1.0, yv);
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) stv(D.y64 + ch * W, yv[i]);
    }
    if (!grid_sync(D.st, sh, ctl, 75)) return;
  }
  // xi = -y - sum_{i != j} v_i c_i / (lambda_i - lambda_j)
  if (threadIdx.x == 0)
    for (int c = 0; c < p; c++) sh.qv[c] = (c == j) ? 0.0 : sh.cadj[c] / (D.st->lambda[c] - lam);
  __syncthreads();
  {
    double xi[RPC][W];
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) {
        ldc(D.y64 + ch * W, xi[i]);
#pragma unroll
        for (int u = 0; u < W; u++) xi[i][u] = -xi[i][u];
      } else {
#pragma unroll
        for (int u = 0; u < W; u++) xi[i][u] = 0.0;
      }
    }
    fp64_comb_add<T, RPC>(D, p, sh.qv, -1.0, xi);
#pragma unroll
    for (int i = 0; i < RPC; i++) {
      const int64_t ch = tid + i * TT;
      if (ch < D.nchunks) stv(D.t + ch * W, xi[i]);
    }
  }
  if (lead_cta() && threadIdx.x == 0) {
    D.st->adj_refine = refine;
    D.st->adj_inner = inner;
    D.st->adj_res = res;
  }
}

// ---------------------------------------------------------------------------
// Kernel: batched solve.  Groups of B.G consecutive CTAs take problems from a
// device work queue (largest first); a group runs the whole of Algorithm 3.2
// for its problem (DACG and Newton for every eigenpair) with group-relative
// barriers and reductions, then takes the next problem.  A problem whose
// layout was built for g < G CTAs runs on the first g CTAs of the group.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ bool group_sync(const Batch<T> &B, int group, unsigned &gepoch, Shared &sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    gepoch++;
    const unsigned target = gepoch * (unsigned)B.G;
    __threadfence();
    red_release_add(&B.gbar[group], 1u);
    long long t0 = 0;
    int spins = 0;
    int ok = 1;
    while (ld_acquire(&B.gbar[group]) < target) {
      if (++spins >= 64) {
        spins = 0;
        __nanosleep(256);
        if (ld_relaxed_int(&B.gerr[group]) != 0) {
          ok = 0;
          break;
        }
        const long long now = gtimer();
        if (t0 == 0)
          t0 = now;
        else if (now - t0 > B.group_spin_ns) {
          atomicExch(&B.gerr[group], 8 /*NLE_ERR_TIMEOUT*/);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    sh.ok = ok && ld_relaxed_int(&B.gerr[group]) == 0;
  }
  __syncthreads();
  return sh.ok != 0;
}

template <typename T, int RPC, int CH>
__global__ void __launch_bounds__(TPB, 1) k_batch(Batch<T> B, Opts O) {
  __shared__ Shared sh;
  __shared__ __align__(16) unsigned char sD_raw[sizeof(Dev<T>)];  // problem descriptor
  Dev<T> &sD = *reinterpret_cast<Dev<T> *>(sD_raw);
  __shared__ int s_idx;
  const int group = (int)blockIdx.x / B.G, rank = (int)blockIdx.x % B.G;
  unsigned gepoch = 0;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      const unsigned idx = atomicAdd(B.queue, 1u);
      atomicExch(&B.gslot[group], (int)idx);
    }
    if (!group_sync(B, group, gepoch, sh)) return;
    if (threadIdx.x == 0) s_idx = ld_relaxed_int(&B.gslot[group]);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= B.count) return;
    if (threadIdx.x == 0) sD = B.devs[B.order[idx]];
    __syncthreads();
    const int gi = sD.grid;
    if (rank < gi) {
      Ctl ctl;
      load_state(sD, sh, ctl, O, group * B.G, gi);
      for (int j = 0; j < B.p; j++) {
        if (!dacg_body<T, RPC>(sD, O, sh, ctl, j)) break;
        if (!grid_sync(sD.st, sh, ctl, 80)) break;
        if (!newton_body<T, RPC>(sD, O, sh, ctl, j)) break;
        if (!grid_sync(sD.st, sh, ctl, 81)) break;
      }
    }
    // every CTA of the group is done with this problem before the slot moves on
    if (!group_sync(B, group, gepoch, sh)) return;
  }
}

// ---------------------------------------------------------------------------
// host-side launch table.  This file is compiled once per (precision, RPC)
// pair (NLE_T, NLE_RPC, NLE_TAG defined by the build) so that the
// instantiations compile in parallel.
// ---------------------------------------------------------------------------
#if defined(NLE_T) && defined(NLE_RPC) && defined(NLE_TAG)
#define NLE_CAT2(a, b) a##b
#define NLE_CAT(a, b) NLE_CAT2(a, b)
void *NLE_CAT(kernel_ptr_, NLE_TAG)(int id) {
  switch (id) {
    case 0: return (void *)k_newton<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
    case 1: return (void *)k_dacg<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
    case 2: return (void *)k_shifted<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
    case 3: return (void *)k_prec<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
    case 4: return (void *)k_pcg<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
    case 5: return (void *)k_adjoint<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
    case 6: return (void *)k_batch<NLE_T, NLE_RPC, NLE_CHAIN_TU>;
  }
  return nullptr;
}
#endif

}  // namespace nle
