// C ABI of the nle library (include/nle.h): handle management, device
// memory, cooperative launches of the persistent kernels and the small
// relabelling kernels around them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/nle.h"
#include "nle_device.cuh"
#include "nle_ict.h"
#include "nle_internal.h"
#include "nle_setup.h"

namespace nle {
// one translation unit of nle_kernels.cu per (precision, rows-per-thread,
// triangular-solve schedule)
#define NLE_KTAB(tag) void *kernel_ptr_##tag(int);
NLE_KTAB(f1) NLE_KTAB(f2) NLE_KTAB(f4) NLE_KTAB(f8) NLE_KTAB(d1) NLE_KTAB(d2) NLE_KTAB(d4) NLE_KTAB(d8)
NLE_KTAB(f1c) NLE_KTAB(f2c) NLE_KTAB(f4c) NLE_KTAB(f8c) NLE_KTAB(d1c) NLE_KTAB(d2c) NLE_KTAB(d4c) NLE_KTAB(d8c)
#undef NLE_KTAB
enum KernelId { K_NEWTON = 0, K_DACG = 1, K_SHIFTED = 2, K_PREC = 3, K_PCG = 4, K_ADJOINT = 5, K_BATCH = 6 };
template <typename T>
void *kernel_ptr(int id, int rpc, int chain);
template <>
void *kernel_ptr<float>(int id, int rpc, int chain) {
  switch (rpc * 2 + (chain ? 1 : 0)) {
    case 2: return kernel_ptr_f1(id);
    case 3: return kernel_ptr_f1c(id);
    case 4: return kernel_ptr_f2(id);
    case 5: return kernel_ptr_f2c(id);
    case 8: return kernel_ptr_f4(id);
    case 9: return kernel_ptr_f4c(id);
    case 16: return kernel_ptr_f8(id);
    case 17: return kernel_ptr_f8c(id);
  }
  return nullptr;
}
template <>
void *kernel_ptr<double>(int id, int rpc, int chain) {
  switch (rpc * 2 + (chain ? 1 : 0)) {
    case 2: return kernel_ptr_d1(id);
    case 3: return kernel_ptr_d1c(id);
    case 4: return kernel_ptr_d2(id);
    case 5: return kernel_ptr_d2c(id);
    case 8: return kernel_ptr_d4(id);
    case 9: return kernel_ptr_d4c(id);
    case 16: return kernel_ptr_d8(id);
    case 17: return kernel_ptr_d8c(id);
  }
  return nullptr;
}

// ---------------------------------------------------------------------------
// relabelling kernels
// ---------------------------------------------------------------------------
// dst[i] = T(src[perm[i]]) for i < n, 0 for n <= i < npad
template <typename T>
__global__ void k_gather(T *dst, const double *src, const int32_t *perm, int64_t n, int64_t npad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (i < n) ? T(src[perm[i]]) : T(0);
}
// dst[o] = double(src[iperm[o]]) for o < n
template <typename T>
__global__ void k_scatter(double *dst, const T *src, const int32_t *iperm, int64_t n) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x)
    dst[o] = double(src[iperm[o]]);
}
// V[j*n + o] = sgn_j * Qt[j*npad + iperm[o]], sgn_j making the entry of
// largest modulus positive (lowest natural index on ties).  One block per j.
__global__ void k_output_vectors(double *V, const double *Qt, const int32_t *iperm, int64_t n, int64_t npad,
                                 State *st) {
  const int j = blockIdx.x;
  const double *q = Qt + (int64_t)j * npad;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t o = threadIdx.x; o < n; o += blockDim.x) {
    const double a = fabs(q[iperm[o]]);
    if (a > best) best = a, bi = o;
  }
  __shared__ double sb[1024];
  __shared__ int64_t si[1024];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double b2 = sb[threadIdx.x + s];
      const int64_t i2 = si[threadIdx.x + s];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) sb[threadIdx.x] = b2, si[threadIdx.x] = i2;
    }
    __syncthreads();
  }
  const double sgn = (q[iperm[si[0]]] < 0.0) ? -1.0 : 1.0;
  if (threadIdx.x == 0) st->sign[j] = sgn;
  for (int64_t o = threadIdx.x; o < n; o += blockDim.x) V[(int64_t)j * n + o] = sgn * q[iperm[o]];
}
// dst[i] = sign_j * src[perm[i]] (FP64, device order), 0 on padding
__global__ void k_gather_signed(double *dst, const double *src, const int32_t *perm, int64_t n, int64_t npad,
                                const State *st, int j) {
  const double sg = st->sign[j];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (i < n) ? sg * src[perm[i]] : 0.0;
}
// grad[e] += sum_j gl[j] v_j[a] v_j[b] for every stored entry e = (a, b)
__global__ void k_grad_lambda(double *grad, const int32_t *erow, const int32_t *ecol, int64_t nnz,
                              const int32_t *iperm, const double *Qt, int64_t npad, int p, const double *gl) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = iperm[erow[e]], b = iperm[ecol[e]];
    double acc = 0.0;
    for (int j = 0; j < p; j++) acc += gl[j] * Qt[(int64_t)j * npad + a] * Qt[(int64_t)j * npad + b];
    grad[e] += acc;
  }
}
// grad[e] += xi[a] v_j[b]
__global__ void k_grad_vec(double *grad, const int32_t *erow, const int32_t *ecol, int64_t nnz, const int32_t *iperm,
                           const double *xi, const double *vj) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    grad[e] += xi[iperm[erow[e]]] * vj[iperm[ecol[e]]];
}
__global__ void k_set_j(State *st, int j) {
  st->j = j;
  st->bar = 0u;
}
// fixed pseudo-random start vector when the caller passes none
__global__ void k_default_start(double *x, int64_t n, int j) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)(j + 1) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = double(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

}  // namespace nle

using namespace nle;

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
namespace {

struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  ~DBuf() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename X>
  X *as() const {
    return reinterpret_cast<X *>(p);
  }
};

struct Status {
  nle_status code;
  std::string msg;
};

}  // namespace

struct nle_ctx {
  int device = 0;
  int nsm = 0;
  cudaStream_t stream = nullptr;
  nle_options opt{};
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  bool factored = false;
  Factor F;
  std::vector<int32_t> perm, iperm;
  int vw = 4;
  int64_t npad = 0, nchunks = 0;
  int grid = 0, rpc = 0;
  int64_t bsize = 0;
  int ldq = 0;
  // device memory
  DBuf d_perm, d_iperm;
  DBuf A_sptr, A_col, A_val, A64_val, d_diag;
  DBuf L_off, L_w, L_col, L_val, L_round, U_off, U_w, U_col, U_val, U_round;
  DBuf L_wp, L_task, U_wp, U_task;  // chain schedule: per-warp task lists
  int chain = 0;                     // schedule of the triangular solves in use (1 = chain)
  int trows = TRSV_ROWS;             // level schedule: rows a warp takes at a time (4 or 2)
  double tune_ms[3] = {0.0, 0.0, 0.0};  // measured application time: level (4 rows), chain, level (2 rows)
  int64_t nstrands = 0;
  int ic_on_device = 0;                         // the factor in use was computed on the device
  double ic_ms[3] = {0.0, 0.0, 0.0};            // factor (wall), its kernel (device), whole set-up (wall)
  DBuf vecs;   // working-precision vectors
  DBuf vec64;  // Au, r, t
  DBuf dQ, dQt, dS, dR;
  DBuf part, state;
  DBuf scratch;  // 2 * n doubles for host transfers
  DBuf d_erow, d_ecol, d_grad;  // natural-order entries (adjoint)
  DBuf dX0;                      // start vectors for the batched kernel (p columns, device order)
  std::vector<double> pinned_dummy;
  bool solved = false;
  int last_p = 0;
  std::vector<double> lambda;
  std::string err;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float last_batch_ms = 0.f;  // device time of the last nle_batch_solve led by this handle
  nle_stats last_stats{};     // statistics of the last solve (single or batched)
  bool has_stats = false;
};

static thread_local std::string g_create_error;

namespace nle {
// message for nle_last_error(NULL) from calls that take no handle
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace nle

static nle_status fail(nle_t h, nle_status code, const std::string &msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return code;
}

#define NLE_CUDA(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      return fail(h, e_ == cudaErrorMemoryAllocation ? NLE_ERR_OOM : NLE_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    }                                                                                      \
  } while (0)

// Allocation, zeroing and uploads are ordered on the stream the kernels
// run on (a non-blocking stream does not wait for the legacy default
// stream).  A copy from pageable host memory returns once the data is
// staged, so the host vector may be released right after the call.
static cudaError_t dalloc(DBuf &b, size_t bytes, cudaStream_t stream) {
  b.reset();
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) {
    b.bytes = bytes;
    e = cudaMemsetAsync(b.p, 0, bytes, stream);
  }
  return e;
}

template <typename X>
static cudaError_t upload(DBuf &b, const std::vector<X> &v, cudaStream_t stream) {
  cudaError_t e = dalloc(b, v.size() * sizeof(X), stream);
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, stream);
  return e;
}

static bool mixed(nle_t h) { return h->opt.precision == NLE_MIXED; }

template <typename T>
static Dev<T> make_dev(nle_t h) {
  Dev<T> D;
  D.n = h->n;
  D.npad = h->npad;
  D.nchunks = h->nchunks;
  D.ldq = h->ldq;
  D.bsize = h->bsize;
  D.grid = h->grid;
  const int64_t ns = h->npad / (32 * h->vw);
  D.A = {ns, h->A_sptr.as<int64_t>(), h->A_col.as<int32_t>(), h->A_val.as<T>()};
  D.A64 = {ns, h->A_sptr.as<int64_t>(), h->A_col.as<int32_t>(), h->A64_val.as<double>()};
  D.Loff = h->L_off.as<int64_t>();
  D.Lw = h->L_w.as<int32_t>();
  D.Lcol = h->L_col.as<int32_t>();
  D.Lval = h->L_val.as<T>();
  D.Lround = h->L_round.as<uint16_t>();
  D.Uoff = h->U_off.as<int64_t>();
  D.Uw = h->U_w.as<int32_t>();
  D.Ucol = h->U_col.as<int32_t>();
  D.Uval = h->U_val.as<T>();
  D.Uround = h->U_round.as<uint16_t>();
  D.rdiag = h->d_diag.as<T>();
  D.chain = h->chain;
  D.trows = h->trows;
  D.Lwp = h->L_wp.as<int32_t>();
  D.Uwp = h->U_wp.as<int32_t>();
  D.Ltask = h->L_task.as<int2>();
  D.Utask = h->U_task.as<int2>();
  const int64_t np = h->npad, ext = h->npad + 32 * h->vw;
  T *v = h->vecs.as<T>();
  D.p = v + 0 * np;
  D.y = v + 1 * np;
  D.s = v + 2 * np;
  D.g = v + 3 * np;
  D.rT = v + 4 * np;
  D.x = v + 5 * np;
  D.Ax = v + 6 * np;
  D.Ap = v + 7 * np;
  D.z = v + 8 * np;
  D.c0 = v + 8 * np + ext;
  double *w = h->vec64.as<double>();
  D.Au = w;
  D.r = w + np;
  D.t = w + 2 * np;
  D.y64 = w + 3 * np;
  D.b64 = w + 4 * np;
  D.u = nullptr;
  D.Q = h->dQ.as<T>();
  D.Qt = h->dQt.as<double>();
  D.S = h->dS.as<T>();
  D.R = h->dR.as<T>();
  D.part = h->part.as<double>();
  D.st = h->state.as<State>();
  return D;
}

static Opts make_opts(nle_t h, double tol, int max_newton, int max_pcg) {
  Opts O;
  O.tol = tol;
  O.tau_pcg = h->opt.tau_pcg;
  O.tau_dacg = h->opt.tau_dacg;
  O.max_newton = max_newton;
  O.max_pcg = max_pcg;
  O.max_dacg = h->opt.max_dacg;
  O.kmax = h->opt.k_max;
  O.exit_eigres = h->opt.exit_eigres;
  O.exit_stag = h->opt.exit_stagnation;
  O.recompute = h->opt.dacg_recompute;
  O.spin_ns = (long long)(h->opt.spin_timeout_s * 1e9);
  O.trsv_warps = h->opt.trsv_warps;
  O.poll_ns = std::max(0, std::min(10000, h->opt.trsv_poll_ns));
  O.bfgs_full = h->opt.bfgs_update == NLE_BFGS_FULL ? 1 : 0;
  return O;
}

// Cooperative launch of kernel `id` (persistent, gridDim = h->grid).
template <typename T>
static nle_status launch(nle_t h, int id, void **args) {
  void *fn = kernel_ptr<T>(id, h->rpc, h->chain);
  if (!fn) return fail(h, NLE_ERR_ARG, "no kernel instance for this size");
  // dynamic shared memory: two slab-sized buffers of the triangular solves
  const size_t dyn = 2 * (size_t)h->bsize * (mixed(h) ? 4 : 8);
  NLE_CUDA(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int nb = 0;
  NLE_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, TPB, dyn));
  if (nb < 1 || h->grid > nb * h->nsm) return fail(h, NLE_ERR_CUDA, "persistent grid does not fit on the device");
  // reset the grid-barrier counter
  State *st = h->state.as<State>();
  NLE_CUDA(h, cudaMemsetAsync(&st->bar, 0, sizeof(unsigned), h->stream));
  NLE_CUDA(h, cudaLaunchCooperativeKernel(fn, dim3(h->grid), dim3(TPB), args, dyn, h->stream));
  return NLE_OK;
}

static nle_status check_state_error(nle_t h) {
  State st;
  NLE_CUDA(h, cudaMemcpyAsync(&st.err, &h->state.as<State>()->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  if (st.err != 0) {
    char buf[128];
    snprintf(buf, sizeof buf, "device wait ran out (code %d at site %d)", st.err, st.err_where);
    // clear it so the handle stays usable
    NLE_CUDA(h, cudaMemsetAsync(&h->state.as<State>()->err, 0, 2 * sizeof(int), h->stream));
    NLE_CUDA(h, cudaStreamSynchronize(h->stream));
    return fail(h, (nle_status)st.err, buf);
  }
  return NLE_OK;
}

// Make sure Q / Qt have room for m columns.
static nle_status ensure_q(nle_t h, int m) {
  if (m <= h->ldq) return NLE_OK;
  const size_t tsz = mixed(h) ? 4 : 8;
  NLE_CUDA(h, dalloc(h->dQ, (size_t)h->npad * m * tsz, h->stream));
  NLE_CUDA(h, dalloc(h->dQt, (size_t)h->npad * m * 8, h->stream));
  h->ldq = m;
  return NLE_OK;
}

// Copy p vectors of length n (natural order, FP64, host or device) into a
// device array of working-precision columns (device order) at dst + c*npad.
template <typename T>
static nle_status put_vectors(nle_t h, const double *src, int count, T *dst, int on_device) {
  const int64_t n = h->n;
  for (int c = 0; c < count; c++) {
    const double *s = src + (int64_t)c * n;
    if (!on_device) {
      NLE_CUDA(h, cudaMemcpyAsync(h->scratch.p, s, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      s = h->scratch.as<double>();
    }
    k_gather<T><<<1024, 256, 0, h->stream>>>(dst + (int64_t)c * h->npad, s, h->d_perm.as<int32_t>(), n, h->npad);
    NLE_CUDA(h, cudaGetLastError());
  }
  return NLE_OK;
}

template <typename T>
static nle_status get_vector(nle_t h, const T *src, double *dst, int on_device) {
  double *d = on_device ? dst : h->scratch.as<double>();
  k_scatter<T><<<1024, 256, 0, h->stream>>>(d, src, h->d_iperm.as<int32_t>(), h->n);
  NLE_CUDA(h, cudaGetLastError());
  if (!on_device) NLE_CUDA(h, cudaMemcpyAsync(dst, d, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return NLE_OK;
}

// Device layout of a factored handle: the relabelling, A in SELL (working
// precision and FP64), the triangular factors in the layout of the chosen
// schedule (chain = 1: the factored matrix's own order with per-warp task
// lists; 0: slab-major level-minor order with level rounds), uploaded on the
// handle's stream.  rp/ci/va: the matrix that was factored.
template <typename TV>
static nle_status upload_layout(nle_t h, const Permuted &P, bool level_rounds, int chain) {
  const int H = 32 * h->vw;
  SellSet<TV> S;
  build_sell<TV>(P, H, h->bsize, level_rounds, h->trows, S);
  NLE_CUDA(h, upload(h->A_sptr, S.A.sptr, h->stream));
  NLE_CUDA(h, upload(h->A_col, S.A.col, h->stream));
  NLE_CUDA(h, upload(h->A_val, S.A.val, h->stream));
  NLE_CUDA(h, upload(h->A64_val, S.A64.val, h->stream));
  NLE_CUDA(h, upload(h->d_diag, S.diag, h->stream));
  if (chain) {
    const int nw = std::max(1, std::min(NWARP, h->opt.trsv_warps));
    ChainHost<TV> CL, CU;
    build_chain<TV>(P, h->bsize, true, nw, CL);
    build_chain<TV>(P, h->bsize, false, nw, CU);
    h->nstrands = CL.nstrands;
    S.L = std::move(CL.ell);
    S.U = std::move(CU.ell);
    NLE_CUDA(h, upload(h->L_wp, CL.wptr, h->stream));
    NLE_CUDA(h, upload(h->L_task, CL.task, h->stream));
    NLE_CUDA(h, upload(h->U_wp, CU.wptr, h->stream));
    NLE_CUDA(h, upload(h->U_task, CU.task, h->stream));
    S.L.round.assign(1, 0);
    S.U.round.assign(1, 0);
  }
  NLE_CUDA(h, upload(h->L_off, S.L.off, h->stream));
  NLE_CUDA(h, upload(h->L_w, S.L.width, h->stream));
  NLE_CUDA(h, upload(h->L_col, S.L.col, h->stream));
  NLE_CUDA(h, upload(h->L_val, S.L.val, h->stream));
  NLE_CUDA(h, upload(h->L_round, S.L.round, h->stream));
  NLE_CUDA(h, upload(h->U_off, S.U.off, h->stream));
  NLE_CUDA(h, upload(h->U_w, S.U.width, h->stream));
  NLE_CUDA(h, upload(h->U_col, S.U.col, h->stream));
  NLE_CUDA(h, upload(h->U_val, S.U.val, h->stream));
  NLE_CUDA(h, upload(h->U_round, S.U.round, h->stream));
  // the host vectors above are released on return: copies from pageable
  // memory are staged before cudaMemcpyAsync returns
  return NLE_OK;
}

static nle_status build_layout(nle_t h, const std::vector<int32_t> &P0, const int64_t *rp, const int32_t *ci,
                               const double *va, int chain, int trows = TRSV_ROWS) {
  h->trows = chain ? TRSV_ROWS : trows;
  if (chain) {
    h->perm.resize(h->n);
    h->iperm.resize(h->n);
    for (int64_t i = 0; i < h->n; i++) h->perm[i] = h->iperm[i] = (int32_t)i;
  } else {
    // with a multicolour ordering the slabs still follow the caller's row
    // order (P0[k] = caller's row of row k of P A P^T), which keeps each
    // slab's rows and their neighbours together
    slab_level_order(h->F, h->bsize, P0.empty() ? nullptr : P0.data(), h->perm, h->iperm);
  }
  Permuted P;
  permute(h->n, rp, ci, va, h->F, h->perm, h->iperm, h->npad, P);
  if (!P0.empty()) {
    // device position -> row of the caller's numbering, through P A P^T
    for (int64_t p = 0; p < h->n; p++) h->perm[p] = P0[h->perm[p]];
    for (int64_t p = 0; p < h->n; p++) h->iperm[h->perm[p]] = (int32_t)p;
  }
  nle_status s = mixed(h) ? upload_layout<float>(h, P, !P0.empty(), chain)
                          : upload_layout<double>(h, P, !P0.empty(), chain);
  if (s != NLE_OK) return s;
  NLE_CUDA(h, upload(h->d_perm, h->perm, h->stream));
  NLE_CUDA(h, upload(h->d_iperm, h->iperm, h->stream));
  h->chain = chain;
  return NLE_OK;
}

// Device time of one application of (L L^T)^{-1} (k = 0 pairs, no
// projection) with the handle's current layout: the median of three
// launches after one warm-up, on the handle's stream.
template <typename T>
static nle_status time_precond_t(nle_t h, double *ms) {
  Dev<T> D = make_dev<T>(h);
  k_default_start<<<1024, 256, 0, h->stream>>>(h->scratch.as<double>(), h->n, 0);
  NLE_CUDA(h, cudaGetLastError());
  k_gather<T><<<1024, 256, 0, h->stream>>>(D.g, h->scratch.as<double>(), h->d_perm.as<int32_t>(), h->n, h->npad);
  NLE_CUDA(h, cudaGetLastError());
  Opts O = make_opts(h, 1e-8, 1, 1);
  // the timing runs are the library's own: their waits are bounded by at
  // least 2 s whatever the caller's limit for its solves
  O.spin_ns = std::max(O.spin_ns, 2000000000LL);
  NLE_CUDA(h, cudaMemsetAsync(h->state.p, 0, sizeof(State), h->stream));
  int m = 0, k = 0;
  void *args[] = {&D, &O, &m, &k};
  float t[4];
  for (int it = 0; it < 4; it++) {
    NLE_CUDA(h, cudaEventRecord(h->ev[0], h->stream));
    nle_status s = launch<T>(h, K_PREC, args);
    if (s != NLE_OK) return s;
    NLE_CUDA(h, cudaEventRecord(h->ev[1], h->stream));
    NLE_CUDA(h, cudaEventSynchronize(h->ev[1]));
    NLE_CUDA(h, cudaEventElapsedTime(&t[it], h->ev[0], h->ev[1]));
  }
  nle_status s = check_state_error(h);
  if (s != NLE_OK) return s;
  std::sort(t + 1, t + 4);
  *ms = t[2];
  return NLE_OK;
}

static nle_status time_precond(nle_t h, double *ms) {
  return mixed(h) ? time_precond_t<float>(h, ms) : time_precond_t<double>(h, ms);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void nle_default_options(nle_options *o) {
  if (!o) return;
  o->k_max = 5;
  o->tau_pcg = 1e-2;
  o->tau_dacg = 1e-2;
  o->max_dacg = 5000;
  o->precision = NLE_FP64;
  o->exit_eigres = 1;
  o->exit_stagnation = 1;
  o->dacg_recompute = 50;
  o->spin_timeout_s = 2.0;
  o->grid_ctas = 0;
  o->trsv_warps = 16;
  o->ordering = NLE_ORDER_NATURAL;
  o->bfgs_update = NLE_BFGS_SIMPLIFIED;
  o->trsv_schedule = NLE_SCHED_AUTO;
  o->trsv_poll_ns = 0;
  o->trsv_rows = 0;
  o->ic_device = NLE_IC_AUTO;
}

const char *nle_last_error(nle_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void nle_destroy(nle_t h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

nle_status nle_create(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col, const double *val,
                      int on_device, void *stream, const nle_options *opt, nle_t *out) {
  if (!out) return fail(nullptr, NLE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 2 || nnz < n || !rowptr || !col || !val) return fail(nullptr, NLE_ERR_ARG, "need n >= 2, nnz >= n and non-NULL CSR arrays");
  if (n >= (int64_t)1 << 30) return fail(nullptr, NLE_ERR_ARG, "n too large");
  std::unique_ptr<nle_ctx> h(new nle_ctx);
  if (opt)
    h->opt = *opt;
  else
    nle_default_options(&h->opt);
  if (h->opt.k_max < 0 || h->opt.k_max > NLE_MAX_KMAX) return fail(nullptr, NLE_ERR_ARG, "k_max out of range");
  if (h->opt.precision != NLE_FP64 && h->opt.precision != NLE_MIXED) return fail(nullptr, NLE_ERR_ARG, "bad precision");
  if (!(h->opt.spin_timeout_s > 0)) return fail(nullptr, NLE_ERR_ARG, "spin_timeout_s must be positive");
  if (h->opt.trsv_warps < 1 || h->opt.trsv_warps > NWARP) return fail(nullptr, NLE_ERR_ARG, "trsv_warps out of range");
  if (h->opt.ordering < NLE_ORDER_NATURAL || h->opt.ordering > NLE_ORDER_MULTICOLOR2)
    return fail(nullptr, NLE_ERR_ARG, "unknown ordering");
  if (h->opt.trsv_schedule < NLE_SCHED_AUTO || h->opt.trsv_schedule > NLE_SCHED_CHAIN)
    return fail(nullptr, NLE_ERR_ARG, "unknown trsv_schedule");
  if (h->opt.trsv_rows != 0 && h->opt.trsv_rows != 2 && h->opt.trsv_rows != 4)
    return fail(nullptr, NLE_ERR_ARG, "trsv_rows must be 0 (tuned), 2 or 4");
  if (h->opt.ic_device < NLE_IC_AUTO || h->opt.ic_device > NLE_IC_DEVICE)
    return fail(nullptr, NLE_ERR_ARG, "ic_device must be NLE_IC_AUTO, NLE_IC_HOST or NLE_IC_DEVICE");
  if (h->opt.bfgs_update != NLE_BFGS_SIMPLIFIED && h->opt.bfgs_update != NLE_BFGS_FULL)
    return fail(nullptr, NLE_ERR_ARG, "unknown bfgs_update");
  if (h->opt.bfgs_update == NLE_BFGS_FULL && h->opt.k_max > NLE_MAX_KMAX - 1)
    return fail(nullptr, NLE_ERR_ARG, "the full BFGS update keeps one slot for the newest pair: k_max <= NLE_MAX_KMAX - 1");
  h->n = n;
  h->nnz = nnz;
  h->rowptr.resize(n + 1);
  h->col.resize(nnz);
  h->val.resize(nnz);
  if (on_device) {
    // read on the caller's stream, after the work that produced the arrays
    cudaStream_t cs = (cudaStream_t)stream;
    if (cudaMemcpyAsync(h->rowptr.data(), rowptr, (n + 1) * 8, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaMemcpyAsync(h->col.data(), col, nnz * 4, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaMemcpyAsync(h->val.data(), val, nnz * 8, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
      return fail(nullptr, NLE_ERR_CUDA, "copy of the CSR arrays failed");
  } else {
    memcpy(h->rowptr.data(), rowptr, (n + 1) * 8);
    memcpy(h->col.data(), col, nnz * 4);
    memcpy(h->val.data(), val, nnz * 8);
  }
  // host-side validation first: it needs no device
  std::string msg;
  const int rc = validate_csr(n, nnz, h->rowptr.data(), h->col.data(), h->val.data(), msg);
  if (rc == 2) return fail(nullptr, NLE_ERR_CSR, msg);
  if (rc == 3) return fail(nullptr, NLE_ERR_NOT_SPD, msg);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(nullptr, NLE_ERR_NO_DEVICE, "no CUDA device");
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
  h->stream = (cudaStream_t)stream;
  h->vw = (h->opt.precision == NLE_MIXED) ? 4 : 2;
  for (auto &e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(nullptr, NLE_ERR_CUDA, "cudaEventCreate failed");
  *out = h.release();
  return NLE_OK;
}

nle_status nle_multicolor_order(int64_t n, const int64_t *rowptr, const int32_t *col, int distance, int32_t *perm,
                                int32_t *ncolors) {
  if (n < 1 || !rowptr || !col || !perm || !ncolors || (distance != 1 && distance != 2)) {
    g_create_error = "nle_multicolor_order: need n >= 1, non-NULL arrays and distance 1 or 2";
    return NLE_ERR_ARG;
  }
  if (rowptr[0] != 0) {
    g_create_error = "nle_multicolor_order: rowptr[0] != 0";
    return NLE_ERR_CSR;
  }
  for (int64_t i = 0; i < n; i++) {
    if (rowptr[i + 1] < rowptr[i]) {
      g_create_error = "nle_multicolor_order: rowptr decreases at row " + std::to_string(i);
      return NLE_ERR_CSR;
    }
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
      if (col[e] < 0 || col[e] >= n) {
        g_create_error = "nle_multicolor_order: column out of range in row " + std::to_string(i);
        return NLE_ERR_CSR;
      }
  }
  std::vector<int32_t> P;
  *ncolors = multicolor_order(n, rowptr, col, distance, P);
  memcpy(perm, P.data(), n * sizeof(int32_t));
  return NLE_OK;
}

// IC(lfil, tau_IC) on the device (csrc/nle_ict.cu): the columns of
// ic_factor_host, bit for bit.  NLE_ERR_NOT_SPD sets *bad; a column that
// outgrows the kernel's per-warp tables sets *capacity and returns
// NLE_ERR_ARG.
static nle_status ic_factor_device(nle_t h, const int64_t *rp, const int32_t *ci, const double *va, int lfil,
                                   double tau, Factor &F, int64_t *bad, bool *capacity, double *kernel_ms) {
  const int64_t n = h->n, nnz = rp[n];
  const int RS = lfil + 1;
  cudaStream_t st = h->stream;
  DBuf drp, dci, dva, dcnt, drow, dval, derr;
  NLE_CUDA(h, dalloc(drp, (size_t)(n + 1) * 8, st));
  NLE_CUDA(h, dalloc(dci, (size_t)nnz * 4, st));
  NLE_CUDA(h, dalloc(dva, (size_t)nnz * 8, st));
  NLE_CUDA(h, cudaMemcpyAsync(drp.p, rp, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st));
  NLE_CUDA(h, cudaMemcpyAsync(dci.p, ci, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
  NLE_CUDA(h, cudaMemcpyAsync(dva.p, va, (size_t)nnz * 8, cudaMemcpyHostToDevice, st));
  NLE_CUDA(h, dalloc(dcnt, (size_t)n * 4, st));
  NLE_CUDA(h, dalloc(drow, (size_t)n * RS * 4, st));
  NLE_CUDA(h, dalloc(dval, (size_t)n * RS * 8, st));
  NLE_CUDA(h, dalloc(derr, sizeof(IctError), st));
  NLE_CUDA(h, cudaMemsetAsync(dcnt.p, 0xFF, (size_t)n * 4, st));
  NLE_CUDA(h, cudaMemsetAsync(drow.p, 0xFF, (size_t)n * RS * 4, st));
  NLE_CUDA(h, cudaMemsetAsync(dval.p, 0xFF, (size_t)n * RS * 8, st));
  int grid = ict_max_grid(h->nsm);
  if (grid < 1) return fail(h, NLE_ERR_CUDA, "device IC factor: kernel does not fit on an SM");
  grid = (int)std::min<int64_t>(grid, (n + ICT_WARPS - 1) / ICT_WARPS);
  const long long spin_ns = (long long)(h->opt.spin_timeout_s * 1e9);
  NLE_CUDA(h, cudaEventRecord(h->ev[0], st));
  NLE_CUDA(h, ict_launch(grid, n, drp.as<int64_t>(), dci.as<int32_t>(), dva.as<double>(), lfil, tau,
                         dcnt.as<int>(), drow.as<int>(), dval.as<double>(), derr.as<IctError>(), spin_ns, st));
  NLE_CUDA(h, cudaEventRecord(h->ev[1], st));
  IctError e{};
  std::vector<int> cnt(n), row((size_t)n * RS);
  std::vector<double> val((size_t)n * RS);
  NLE_CUDA(h, cudaMemcpyAsync(&e, derr.p, sizeof(e), cudaMemcpyDeviceToHost, st));
  NLE_CUDA(h, cudaMemcpyAsync(cnt.data(), dcnt.p, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
  NLE_CUDA(h, cudaMemcpyAsync(row.data(), drow.p, (size_t)n * RS * 4, cudaMemcpyDeviceToHost, st));
  NLE_CUDA(h, cudaMemcpyAsync(val.data(), dval.p, (size_t)n * RS * 8, cudaMemcpyDeviceToHost, st));
  NLE_CUDA(h, cudaStreamSynchronize(st));
  float ms = 0.f;
  NLE_CUDA(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
  *kernel_ms = ms;
  if (e.code == ICT_ERR_NOT_SPD) {
    *bad = e.col;
    return NLE_ERR_NOT_SPD;
  }
  if (e.code == ICT_ERR_CAPACITY) {
    *capacity = true;
    return fail(h, NLE_ERR_ARG, "device IC factor: column " + std::to_string(e.col) +
                                    " needs more entries than the kernel's per-warp tables hold");
  }
  if (e.code == ICT_ERR_TIMEOUT)
    return fail(h, NLE_ERR_TIMEOUT, "device IC factor: a wait timed out at column " + std::to_string(e.col));
  if (e.code != ICT_OK) return fail(h, NLE_ERR_CUDA, "device IC factor: error " + std::to_string(e.code));
  std::vector<int64_t> cs(n + 1, 0);
  for (int64_t j = 0; j < n; j++) {
    if (cnt[j] < 1 || cnt[j] > RS)
      return fail(h, NLE_ERR_CUDA, "device IC factor: column " + std::to_string(j) + " was not written");
    cs[j + 1] = cs[j] + cnt[j];
  }
  std::vector<int32_t> rows(cs[n]);
  std::vector<double> vals(cs[n]);
  for (int64_t j = 0; j < n; j++)
    for (int t = 0; t < cnt[j]; t++) {
      rows[cs[j] + t] = row[(size_t)j * RS + t];
      vals[cs[j] + t] = val[(size_t)j * RS + t];
    }
  factor_from_columns(n, std::move(cs), std::move(rows), std::move(vals), F);
  return NLE_OK;
}

nle_status nle_factor_ic(nle_t h, int lfil, double tau_ic) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (lfil < 0 || !(tau_ic >= 0.0)) return fail(h, NLE_ERR_ARG, "need lfil >= 0 and tau_ic >= 0");
  cudaSetDevice(h->device);
  h->factored = false;
  h->solved = false;
  int64_t bad = -1;
  // the matrix factored: A itself, or P A P^T for a multicolour ordering
  const int64_t *rp = h->rowptr.data();
  const int32_t *ci = h->col.data();
  const double *va = h->val.data();
  std::vector<int32_t> P0;
  std::vector<int64_t> brp;
  std::vector<int32_t> bci;
  std::vector<double> bva;
  if (h->opt.ordering != NLE_ORDER_NATURAL) {
    multicolor_order(h->n, rp, ci, h->opt.ordering, P0);
    permute_csr(h->n, rp, ci, va, P0, brp, bci, bva);
    rp = brp.data();
    ci = bci.data();
    va = bva.data();
  }
  // the numeric factor: on the device (NLE_IC_DEVICE, or NLE_IC_AUTO when
  // lfil fits the kernel's column records) or on the host; both give the
  // same factor bit for bit
  using clk = std::chrono::steady_clock;
  const auto t_setup = clk::now();
  Factor F;
  int icdev = h->opt.ic_device;
  if (icdev == NLE_IC_DEVICE && lfil > ICT_LFIL_MAX)
    return fail(h, NLE_ERR_ARG, "the device IC factor needs lfil <= " + std::to_string(ICT_LFIL_MAX));
  const bool on_dev = icdev == NLE_IC_DEVICE || (icdev == NLE_IC_AUTO && lfil <= ICT_LFIL_MAX);
  h->ic_on_device = 0;
  h->ic_ms[0] = h->ic_ms[1] = h->ic_ms[2] = 0.0;
  bool host = !on_dev;
  if (on_dev) {
    bool capacity = false;
    const nle_status ds = ic_factor_device(h, rp, ci, va, lfil, tau_ic, F, &bad, &capacity, &h->ic_ms[1]);
    if (ds == NLE_ERR_NOT_SPD) return fail(h, ds, "non-positive pivot in IC column " + std::to_string(bad));
    if (ds == NLE_OK) h->ic_on_device = 1;
    else if (capacity && icdev == NLE_IC_AUTO) host = true;  // same factor, computed on the host
    else return ds;
  }
  if (host && ic_factor_host(h->n, rp, ci, va, lfil, tau_ic, F, &bad) != 0)
    return fail(h, NLE_ERR_NOT_SPD, "non-positive pivot in IC column " + std::to_string(bad));
  h->ic_ms[0] = std::chrono::duration<double, std::milli>(clk::now() - t_setup).count();
  h->F = std::move(F);
  const int H = 32 * h->vw;
  h->npad = ((h->n + H - 1) / H) * H;
  h->nchunks = h->npad / h->vw;
  // persistent grid: one CTA per SM, fewer for small problems
  int grid = h->opt.grid_ctas > 0 ? h->opt.grid_ctas : h->nsm;
  const int64_t need = (h->nchunks + TPB - 1) / TPB;
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, need));
  int rpc = 0;
  for (int r : {1, 2, 4, 8})
    if ((int64_t)r * grid * TPB >= h->nchunks) {
      rpc = r;
      break;
    }
  if (!rpc) return fail(h, NLE_ERR_ARG, "n too large for one persistent grid");
  h->grid = grid;
  h->rpc = rpc;
  // one slab of rows per CTA in the triangular solves (a multiple of TRSV_ROWS rows,
  // staged in shared memory)
  h->bsize = ((h->npad + TRSV_ROWS * grid - 1) / (TRSV_ROWS * grid)) * TRSV_ROWS;
  if (2 * h->bsize * (int64_t)(mixed(h) ? 4 : 8) > 192 * 1024)
    return fail(h, NLE_ERR_ARG, "n too large for the shared-memory slab of one persistent grid");
  const size_t tsz = mixed(h) ? 4 : 8;
  const int64_t ext = h->npad + 32 * h->vw;
  NLE_CUDA(h, dalloc(h->vecs, (size_t)(8 * h->npad + 2 * ext) * tsz, h->stream));
  NLE_CUDA(h, dalloc(h->vec64, (size_t)5 * h->npad * 8, h->stream));
  NLE_CUDA(h, dalloc(h->dS, (size_t)h->npad * KMAX * tsz, h->stream));
  NLE_CUDA(h, dalloc(h->dR, (size_t)h->npad * KMAX * tsz, h->stream));
  NLE_CUDA(h, dalloc(h->part, (size_t)2 * RED_MAX * h->grid * 8, h->stream));
  NLE_CUDA(h, dalloc(h->state, sizeof(State), h->stream));
  NLE_CUDA(h, dalloc(h->scratch, (size_t)2 * h->n * 8, h->stream));
  h->ldq = 0;
  nle_status s = ensure_q(h, 8);
  if (s != NLE_OK) return s;
  // schedule of the triangular solves: the chain schedule needs the factored
  // matrix's own row order (natural ordering); the level schedule takes 4
  // rows per warp step (8 lanes and 16 entries of a row in flight) or 2 (16
  // lanes, 32 entries: factors with wide rows).  NLE_SCHED_AUTO times one
  // preconditioner application with each candidate (level with 4 rows,
  // chain, level with 2 rows) and keeps the fastest; an explicit
  // trsv_rows fixes the rows of the level schedule.
  const bool chain_ok = P0.empty();
  int sched = h->opt.trsv_schedule;
  if (sched == NLE_SCHED_CHAIN && !chain_ok)
    return fail(h, NLE_ERR_ARG, "the chain schedule needs the natural ordering");
  h->tune_ms[0] = h->tune_ms[1] = h->tune_ms[2] = 0.0;
  const int rows_opt = h->opt.trsv_rows;
  if (sched == NLE_SCHED_AUTO) {
    struct Cand {
      int chain, rows, slot;
    };
    std::vector<Cand> cands;
    if (rows_opt == 0 || rows_opt == 4) cands.push_back({0, 4, 0});
    if (chain_ok) cands.push_back({1, TRSV_ROWS, 1});
    if (rows_opt == 0 || rows_opt == 2) cands.push_back({0, 2, 2});
    int best = -1;
    for (size_t c = 0; c < cands.size(); c++) {
      if ((s = build_layout(h, P0, rp, ci, va, cands[c].chain, cands[c].rows)) != NLE_OK) return s;
      if ((s = time_precond(h, &h->tune_ms[cands[c].slot])) != NLE_OK) return s;
      if (best < 0 || h->tune_ms[cands[c].slot] < h->tune_ms[cands[best].slot]) best = (int)c;
    }
    // the last candidate's layout is in place; rebuild the fastest one
    if (best != (int)cands.size() - 1 &&
        (s = build_layout(h, P0, rp, ci, va, cands[best].chain, cands[best].rows)) != NLE_OK)
      return s;
  } else {
    if ((s = build_layout(h, P0, rp, ci, va, sched == NLE_SCHED_CHAIN ? 1 : 0, rows_opt == 2 ? 2 : 4)) != NLE_OK)
      return s;
  }
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->ic_ms[2] = std::chrono::duration<double, std::milli>(clk::now() - t_setup).count();
  h->factored = true;
  return NLE_OK;
}

nle_status nle_get_factor(nle_t h, int64_t *nnzL, int64_t *Lrowptr, int32_t *Lcol, double *Lval, int32_t *levL,
                          int32_t *levU, int64_t *nlevL, int64_t *nlevU) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (!h->factored) return fail(h, NLE_ERR_STATE, "nle_factor_ic has not been called");
  const Factor &F = h->F;
  if (nnzL) *nnzL = (int64_t)F.Lcol.size();
  if (Lrowptr) memcpy(Lrowptr, F.Lrowptr.data(), (h->n + 1) * 8);
  if (Lcol) memcpy(Lcol, F.Lcol.data(), F.Lcol.size() * 4);
  if (Lval) memcpy(Lval, F.Lval.data(), F.Lval.size() * 8);
  if (levL) memcpy(levL, F.levL.data(), h->n * 4);
  if (levU) memcpy(levU, F.levU.data(), h->n * 4);
  if (nlevL) *nlevL = F.nlevL;
  if (nlevU) *nlevU = F.nlevU;
  return NLE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
// Per-solve statistics from the device state of one problem.
static void fill_stats(const State &st, int p, double ms_dacg, double ms_newton, int64_t launches, double ms_batch,
                       nle_stats *stats) {
  memset(stats, 0, sizeof(*stats));
  stats->p = p;
  bool asc = true;
  for (int j = 0; j < p; j++) {
    stats->dacg_its[j] = st.dacg_its[j];
    stats->outer_its[j] = st.outer_its[j];
    stats->pcg_its[j] = st.pcg_its[j];
    stats->converged[j] = st.conv[j];
    stats->final_res[j] = st.res[j];
    if (j > 0 && !(st.lambda[j] > st.lambda[j - 1])) asc = false;
  }
  stats->mvp_dacg = st.mvp_dacg;
  stats->mvp_newton = st.mvp_newton;
  for (int e = 0; e < 5; e++) stats->exit_count[e] = st.exits[e];
  stats->ms_dacg = ms_dacg;
  stats->ms_newton = ms_newton;
  stats->pcg_iterations = st.pcg_total;
  stats->pcg_sum_m = st.pcg_sum_m;
  stats->pcg_sum_k = st.pcg_sum_k;
  stats->dacg_iterations = st.dacg_total;
  stats->dacg_sum_m = st.dacg_sum_m;
  stats->kernel_launches = launches;
  for (int q = 0; q < 8; q++) stats->ms_phase[q] = st.tphase[q] * 1e-6;
  stats->ascending = asc ? 1 : 0;
  stats->ms_batch = ms_batch;
}

// schedule of the handle's triangular solves and the autotuner's timings
static void schedule_stats(nle_t h, nle_stats *stats) {
  stats->trsv_schedule = h->chain ? NLE_SCHED_CHAIN : NLE_SCHED_LEVEL;
  stats->trsv_rows = h->trows;
  stats->tune_ms_level = h->tune_ms[0];
  stats->tune_ms_chain = h->tune_ms[1];
  stats->tune_ms_level2 = h->tune_ms[2];
  stats->strands = h->chain ? h->nstrands : 0;
  stats->ic_on_device = h->ic_on_device;
  stats->ms_ic_factor = h->ic_ms[0];
  stats->ms_ic_kernel = h->ic_ms[1];
  stats->ms_ic_setup = h->ic_ms[2];
}

template <typename T>
static nle_status solve_impl(nle_t h, int p, double tol, int max_newton, int max_pcg, const double *X0,
                             double *lambda, double *V, nle_stats *stats, int on_dev) {
  nle_status s = ensure_q(h, p);
  if (s != NLE_OK) return s;
  Dev<T> D = make_dev<T>(h);
  Opts O = make_opts(h, tol, max_newton, max_pcg);
  NLE_CUDA(h, cudaMemsetAsync(h->state.p, 0, sizeof(State), h->stream));
  double ms_dacg = 0.0, ms_newton = 0.0;
  int64_t launches = 0;
  for (int j = 0; j < p; j++) {
    launches += X0 ? 4 : 5;
    k_set_j<<<1, 1, 0, h->stream>>>(D.st, j);
    NLE_CUDA(h, cudaGetLastError());
    if (X0) {
      s = put_vectors<T>(h, X0 + (int64_t)j * h->n, 1, D.x, on_dev);
      if (s != NLE_OK) return s;
    } else {
      k_default_start<<<1024, 256, 0, h->stream>>>(h->scratch.as<double>(), h->n, j);
      s = put_vectors<T>(h, h->scratch.as<double>(), 1, D.x, 1);
      if (s != NLE_OK) return s;
    }
    void *args[] = {&D, &O};
    NLE_CUDA(h, cudaEventRecord(h->ev[0], h->stream));
    s = launch<T>(h, K_DACG, args);
    if (s != NLE_OK) return s;
    NLE_CUDA(h, cudaEventRecord(h->ev[1], h->stream));
    s = launch<T>(h, K_NEWTON, args);
    if (s != NLE_OK) return s;
    NLE_CUDA(h, cudaEventRecord(h->ev[2], h->stream));
    NLE_CUDA(h, cudaEventSynchronize(h->ev[2]));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
    cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
    ms_dacg += a;
    ms_newton += b;
    s = check_state_error(h);
    if (s != NLE_OK) return s;
  }
  // outputs
  State st;
  NLE_CUDA(h, cudaMemcpyAsync(&st, h->state.p, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
  double *vout = on_dev ? V : nullptr;
  DBuf tmp;
  if (!on_dev) {
    NLE_CUDA(h, dalloc(tmp, (size_t)p * h->n * 8, h->stream));
    vout = tmp.as<double>();
  }
  k_output_vectors<<<p, 1024, 0, h->stream>>>(vout, D.Qt, h->d_iperm.as<int32_t>(), h->n, h->npad, D.st);
  launches++;
  NLE_CUDA(h, cudaGetLastError());
  if (!on_dev) NLE_CUDA(h, cudaMemcpyAsync(V, vout, (size_t)p * h->n * 8, cudaMemcpyDeviceToHost, h->stream));
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  if (on_dev) {
    NLE_CUDA(h, cudaMemcpyAsync(lambda, st.lambda, p * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  } else
    memcpy(lambda, st.lambda, p * sizeof(double));
  h->lambda.assign(st.lambda, st.lambda + p);
  h->solved = true;
  h->last_p = p;
  bool allconv = true;
  for (int j = 0; j < p; j++) allconv = allconv && st.conv[j];
  fill_stats(st, p, ms_dacg, ms_newton, launches, 0.0, &h->last_stats);
  schedule_stats(h, &h->last_stats);
  h->has_stats = true;
  if (stats) *stats = h->last_stats;
  if (!allconv) return fail(h, NLE_ERR_NOCONV, "some eigenpairs reached max_newton");
  return NLE_OK;
}

extern "C" nle_status nle_get_stats(nle_t h, nle_stats *stats) {
  if (!h || !stats) return fail(h, NLE_ERR_ARG, "NULL argument");
  if (!h->has_stats && !h->factored) return fail(h, NLE_ERR_STATE, "neither a factor nor a solve on this handle");
  nle_stats out{};
  if (h->has_stats) out = h->last_stats;
  if (h->factored) schedule_stats(h, &out);
  *stats = out;
  return NLE_OK;
}

extern "C" nle_status nle_solve(nle_t h, int p, double tol, int max_newton, int max_pcg, const double *X0,
                                double *lambda, double *V, nle_stats *stats, int buffers_on_device) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (!h->factored) return fail(h, NLE_ERR_STATE, "nle_factor_ic has not been called");
  if (p < 1 || p >= h->n || p > NLE_MAX_P || !(tol > 0) || max_newton < 0 || max_pcg < 1 || !lambda || !V)
    return fail(h, NLE_ERR_ARG, "bad nle_solve arguments");
  cudaSetDevice(h->device);
  return mixed(h) ? solve_impl<float>(h, p, tol, max_newton, max_pcg, X0, lambda, V, stats, buffers_on_device)
                  : solve_impl<double>(h, p, tol, max_newton, max_pcg, X0, lambda, V, stats, buffers_on_device);
}

// ---------------------------------------------------------------------------
// building blocks
// ---------------------------------------------------------------------------
template <typename T>
static nle_status shifted_impl(nle_t h, double theta, const double *x, double *y, int on_dev) {
  Dev<T> D = make_dev<T>(h);
  nle_status s = put_vectors<T>(h, x, 1, D.p, on_dev);
  if (s != NLE_OK) return s;
  void *fn = kernel_ptr<T>(K_SHIFTED, h->rpc, h->chain);
  void *args[] = {&D, &theta};
  NLE_CUDA(h, cudaLaunchKernel(fn, dim3(h->grid), dim3(TPB), args, 0, h->stream));
  s = get_vector<T>(h, D.y, y, on_dev);
  if (s != NLE_OK) return s;
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  return NLE_OK;
}

extern "C" nle_status nle_apply_shifted(nle_t h, double theta, const double *x, double *y, int buffers_on_device) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (!h->factored) return fail(h, NLE_ERR_STATE, "nle_factor_ic has not been called");
  if (!x || !y) return fail(h, NLE_ERR_ARG, "NULL vector");
  cudaSetDevice(h->device);
  return mixed(h) ? shifted_impl<float>(h, theta, x, y, buffers_on_device)
                  : shifted_impl<double>(h, theta, x, y, buffers_on_device);
}

template <typename T>
static nle_status prec_impl(nle_t h, int k, const double *S, const double *R, int m, const double *Q, const double *g,
                            double *c, int on_dev) {
  nle_status s = ensure_q(h, std::max(m, 1));
  if (s != NLE_OK) return s;
  Dev<T> D = make_dev<T>(h);
  if (k > 0) {
    if ((s = put_vectors<T>(h, S, k, D.S, on_dev)) != NLE_OK) return s;
    if ((s = put_vectors<T>(h, R, k, D.R, on_dev)) != NLE_OK) return s;
  }
  if (m > 0 && (s = put_vectors<T>(h, Q, m, D.Q, on_dev)) != NLE_OK) return s;
  if ((s = put_vectors<T>(h, g, 1, D.g, on_dev)) != NLE_OK) return s;
  Opts O = make_opts(h, 1e-8, 1, 1);
  NLE_CUDA(h, cudaMemsetAsync(h->state.p, 0, sizeof(State), h->stream));
  void *args[] = {&D, &O, &m, &k};
  if ((s = launch<T>(h, K_PREC, args)) != NLE_OK) return s;
  if ((s = check_state_error(h)) != NLE_OK) return s;
  if ((s = get_vector<T>(h, D.y, c, on_dev)) != NLE_OK) return s;
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  return NLE_OK;
}

extern "C" nle_status nle_apply_prec(nle_t h, int k, const double *S, const double *R, int m, const double *Q,
                                     const double *g, double *c, int buffers_on_device) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (!h->factored) return fail(h, NLE_ERR_STATE, "nle_factor_ic has not been called");
  if (k < 0 || k > NLE_MAX_KMAX || m < 0 || m > NLE_MAX_P || !g || !c || (k > 0 && (!S || !R)) || (m > 0 && !Q))
    return fail(h, NLE_ERR_ARG, "bad nle_apply_prec arguments");
  cudaSetDevice(h->device);
  h->solved = false;  // overwrites the stored eigenvectors
  return mixed(h) ? prec_impl<float>(h, k, S, R, m, Q, g, c, buffers_on_device)
                  : prec_impl<double>(h, k, S, R, m, Q, g, c, buffers_on_device);
}

template <typename T>
static nle_status pcg_impl(nle_t h, double theta, double tol, int max_pcg, const double *r, int m, const double *Q,
                           int k, const double *S, const double *R, double *sout, nle_pcg_info *info, int on_dev) {
  nle_status s = ensure_q(h, m);
  if (s != NLE_OK) return s;
  Dev<T> D = make_dev<T>(h);
  if (k > 0) {
    if ((s = put_vectors<T>(h, S, k, D.S, on_dev)) != NLE_OK) return s;
    if ((s = put_vectors<T>(h, R, k, D.R, on_dev)) != NLE_OK) return s;
  }
  if ((s = put_vectors<T>(h, Q, m, D.Q, on_dev)) != NLE_OK) return s;
  if ((s = put_vectors<T>(h, r, 1, D.rT, on_dev)) != NLE_OK) return s;
  Opts O = make_opts(h, tol, 1, max_pcg);
  NLE_CUDA(h, cudaMemsetAsync(h->state.p, 0, sizeof(State), h->stream));
  void *args[] = {&D, &O, &m, &k, &theta, &max_pcg};
  if ((s = launch<T>(h, K_PCG, args)) != NLE_OK) return s;
  if ((s = check_state_error(h)) != NLE_OK) return s;
  if ((s = get_vector<T>(h, D.s, sout, on_dev)) != NLE_OK) return s;
  State st;
  NLE_CUDA(h, cudaMemcpyAsync(&st, h->state.p, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  if (info) {
    info->its = st.last_its;
    info->exit = st.last_exit;
    info->gnorm0 = st.last_g0;
    info->gnorm = st.last_gn;
    info->eigres = st.last_eres;
  }
  return NLE_OK;
}

extern "C" nle_status nle_pcg(nle_t h, double theta, double tol, int max_pcg, const double *r, int m, const double *Q,
                              int k, const double *S, const double *R, double *s, nle_pcg_info *info,
                              int buffers_on_device) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (!h->factored) return fail(h, NLE_ERR_STATE, "nle_factor_ic has not been called");
  if (m < 1 || m > NLE_MAX_P || k < 0 || k > NLE_MAX_KMAX || max_pcg < 1 || !r || !Q || !s ||
      (k > 0 && (!S || !R)))
    return fail(h, NLE_ERR_ARG, "bad nle_pcg arguments");
  cudaSetDevice(h->device);
  h->solved = false;  // overwrites the stored eigenvectors
  return mixed(h) ? pcg_impl<float>(h, theta, tol, max_pcg, r, m, Q, k, S, R, s, info, buffers_on_device)
                  : pcg_impl<double>(h, theta, tol, max_pcg, r, m, Q, k, S, R, s, info, buffers_on_device);
}

template <typename T>
static nle_status backward_impl(nle_t h, const double *gl, const double *gV, double *grad_val, int on_dev) {
  const int p = h->last_p;
  const int64_t n = h->n, nnz = h->nnz;
  for (int i = 0; i < p; i++)
    for (int j = i + 1; j < p; j++)
      if (std::fabs(h->lambda[i] - h->lambda[j]) <= 1e-12 * std::fabs(h->lambda[j]))
        return fail(h, NLE_ERR_ARG, "repeated eigenvalue: the eigenvector adjoint is undefined");
  if (!h->d_erow.p) {
    std::vector<int32_t> er(nnz);
    for (int64_t i = 0; i < n; i++)
      for (int64_t e = h->rowptr[i]; e < h->rowptr[i + 1]; e++) er[e] = (int32_t)i;
    NLE_CUDA(h, upload(h->d_erow, er, h->stream));
    NLE_CUDA(h, upload(h->d_ecol, h->col, h->stream));
  }
  double *grad = grad_val;
  if (!on_dev) {
    NLE_CUDA(h, dalloc(h->d_grad, (size_t)nnz * 8, h->stream));
    NLE_CUDA(h, cudaMemcpyAsync(h->d_grad.p, grad_val, nnz * 8, cudaMemcpyHostToDevice, h->stream));
    grad = h->d_grad.as<double>();
  }
  Dev<T> D = make_dev<T>(h);
  const int32_t *erow = h->d_erow.as<int32_t>(), *ecol = h->d_ecol.as<int32_t>();
  const int32_t *iperm = h->d_iperm.as<int32_t>(), *perm = h->d_perm.as<int32_t>();
  if (gl) {
    const double *gld = gl;
    if (!on_dev) {
      NLE_CUDA(h, cudaMemcpyAsync(h->scratch.p, gl, p * 8, cudaMemcpyHostToDevice, h->stream));
      gld = h->scratch.as<double>();
    }
    k_grad_lambda<<<1024, 256, 0, h->stream>>>(grad, erow, ecol, nnz, iperm, D.Qt, h->npad, p, gld);
    NLE_CUDA(h, cudaGetLastError());
  }
  if (gV) {
    // inner solves: exits (iii)/(iv) off, relative tolerance per correction
    Opts O = make_opts(h, 1e-8, 1, 2000);
    O.tau_pcg = mixed(h) ? 1e-3 : 1e-6;
    O.exit_eigres = 0;
    O.exit_stag = 0;
    double tol = 1e-10;
    int max_refine = 40;
    for (int j = 0; j < p; j++) {
      const double *src = gV + (int64_t)j * n;
      if (!on_dev) {
        NLE_CUDA(h, cudaMemcpyAsync(h->scratch.p, src, n * 8, cudaMemcpyHostToDevice, h->stream));
        src = h->scratch.as<double>();
      }
      k_gather_signed<<<1024, 256, 0, h->stream>>>(D.b64, src, perm, n, h->npad, D.st, j);
      NLE_CUDA(h, cudaGetLastError());
      int jj = j, pp = p;
      void *args[] = {&D, &O, &jj, &pp, &tol, &max_refine};
      nle_status s = launch<T>(h, K_ADJOINT, args);
      if (s != NLE_OK) return s;
      if ((s = check_state_error(h)) != NLE_OK) return s;
      k_grad_vec<<<1024, 256, 0, h->stream>>>(grad, erow, ecol, nnz, iperm, D.t, D.Qt + (int64_t)j * h->npad);
      NLE_CUDA(h, cudaGetLastError());
    }
  }
  if (!on_dev) NLE_CUDA(h, cudaMemcpyAsync(grad_val, grad, nnz * 8, cudaMemcpyDeviceToHost, h->stream));
  NLE_CUDA(h, cudaStreamSynchronize(h->stream));
  return NLE_OK;
}

extern "C" nle_status nle_backward(nle_t h, const double *gbar_lambda, const double *gbar_V, double *grad_val,
                                   int buffers_on_device) {
  if (!h) return fail(nullptr, NLE_ERR_ARG, "NULL handle");
  if (!h->solved) return fail(h, NLE_ERR_STATE, "nle_solve has not completed");
  if (!grad_val) return fail(h, NLE_ERR_ARG, "grad_val is NULL");
  cudaSetDevice(h->device);
  return mixed(h) ? backward_impl<float>(h, gbar_lambda, gbar_V, grad_val, buffers_on_device)
                  : backward_impl<double>(h, gbar_lambda, gbar_V, grad_val, buffers_on_device);
}

template <typename T>
static nle_status batch_impl(int count, nle_t *hs, int p, double tol, int max_newton, int max_pcg,
                             const double *const *X0s, double *const *lambdas, double *const *Vs,
                             nle_status *per_problem) {
  nle_t h0 = hs[0];
  // CTAs per group: 4, or 8 when some handle was factored for more than 4
  int G = 4;
  for (int b = 0; b < count; b++)
    if (hs[b]->grid > 4) G = 8;
  int rpc = 1;
  size_t dyn = 0;
  std::vector<Dev<T>> devs(count);
  std::vector<int> order(count);
  for (int b = 0; b < count; b++) {
    nle_t h = hs[b];
    nle_status s = ensure_q(h, p);
    if (s != NLE_OK) return s;
    const size_t tsz = sizeof(T);
    if (h->dX0.bytes < (size_t)p * h->npad * tsz) NLE_CUDA(h0, dalloc(h->dX0, (size_t)p * h->npad * tsz, h->stream));
    Dev<T> D = make_dev<T>(h);
    T *x0 = h->dX0.as<T>();
    for (int j = 0; j < p; j++) {
      if (X0s && X0s[b]) {
        s = put_vectors<T>(h, X0s[b] + (int64_t)j * h->n, 1, x0 + (int64_t)j * h->npad, 1);
      } else {
        k_default_start<<<1024, 256, 0, h->stream>>>(h->scratch.as<double>(), h->n, j);
        s = put_vectors<T>(h, h->scratch.as<double>(), 1, x0 + (int64_t)j * h->npad, 1);
      }
      if (s != NLE_OK) return s;
    }
    D.X0 = x0;
    devs[b] = D;
    NLE_CUDA(h0, cudaMemsetAsync(h->state.p, 0, sizeof(State), h->stream));
    NLE_CUDA(h0, cudaStreamSynchronize(h->stream));
    while ((int64_t)rpc * h->grid * TPB < h->nchunks) rpc *= 2;
    dyn = std::max(dyn, 2 * (size_t)h->bsize * sizeof(T));
    order[b] = b;
  }
  if (rpc > 8) return fail(h0, NLE_ERR_ARG, "a problem is too large for its CTA group");
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->n > hs[b]->n; });
  const int ngroups = std::max(1, h0->nsm / G);
  DBuf d_devs, d_order, d_ctl;
  NLE_CUDA(h0, upload(d_devs, devs, h0->stream));
  NLE_CUDA(h0, upload(d_order, order, h0->stream));
  NLE_CUDA(h0, dalloc(d_ctl, (size_t)(1 + 3 * ngroups) * sizeof(int), h0->stream));
  Batch<T> B;
  B.devs = d_devs.as<Dev<T>>();
  B.order = d_order.as<int>();
  B.count = count;
  B.G = G;
  B.p = p;
  B.queue = d_ctl.as<unsigned>();
  B.gbar = d_ctl.as<unsigned>() + 1;
  B.gslot = d_ctl.as<int>() + 1 + ngroups;
  B.gerr = d_ctl.as<int>() + 1 + 2 * ngroups;
  // CTAs of a group that a small problem leaves idle wait in the group
  // barrier for that whole problem: their limit is the handle's wait limit
  // scaled by the grid barriers of a whole solve (every eigenpair, both
  // phases), at least the barrier limit itself
  B.group_spin_ns = (long long)(h0->opt.spin_timeout_s * 1e9 * 64.0 * p);
  Opts O = make_opts(h0, tol, max_newton, max_pcg);
  void *fn = kernel_ptr<T>(K_BATCH, rpc, h0->chain);
  if (!fn) return fail(h0, NLE_ERR_ARG, "no kernel instance for this size");
  NLE_CUDA(h0, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int nb = 0;
  NLE_CUDA(h0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, TPB, dyn));
  if (nb < 1) return fail(h0, NLE_ERR_CUDA, "batched kernel does not fit on an SM");
  void *args[] = {&B, &O};
  NLE_CUDA(h0, cudaEventRecord(h0->ev[0], h0->stream));
  NLE_CUDA(h0, cudaLaunchCooperativeKernel(fn, dim3(ngroups * G), dim3(TPB), args, dyn, h0->stream));
  NLE_CUDA(h0, cudaEventRecord(h0->ev[1], h0->stream));
  NLE_CUDA(h0, cudaStreamSynchronize(h0->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h0->ev[0], h0->ev[1]);
  h0->last_batch_ms = ms;
  std::vector<int> gerr(ngroups);
  NLE_CUDA(h0, cudaMemcpy(gerr.data(), B.gerr, ngroups * sizeof(int), cudaMemcpyDeviceToHost));
  int group_err = 0;
  for (int e : gerr) group_err = group_err ? group_err : e;
  nle_status worst = NLE_OK;
  for (int b = 0; b < count; b++) {
    nle_t h = hs[b];
    State st;
    NLE_CUDA(h0, cudaMemcpy(&st, h->state.p, sizeof(State), cudaMemcpyDeviceToHost));
    nle_status s = NLE_OK;
    if (st.err != 0 || group_err != 0) {
      s = (nle_status)(st.err ? st.err : group_err);
    } else {
      k_output_vectors<<<p, 1024, 0, h0->stream>>>(Vs[b], devs[b].Qt, h->d_iperm.as<int32_t>(), h->n, h->npad,
                                                  devs[b].st);
      NLE_CUDA(h0, cudaGetLastError());
      NLE_CUDA(h0, cudaMemcpyAsync(lambdas[b], &h->state.as<State>()->lambda[0], p * sizeof(double),
                                   cudaMemcpyDeviceToDevice, h0->stream));
      for (int j = 0; j < p; j++)
        if (!st.conv[j]) s = NLE_ERR_NOCONV;
      h->lambda.assign(st.lambda, st.lambda + p);
      h->last_p = p;
      h->solved = true;
    }
    fill_stats(st, p, 0.0, 0.0, 0, ms, &h->last_stats);
    schedule_stats(h, &h->last_stats);
    h->has_stats = true;
    if (per_problem) per_problem[b] = s;
    if (s != NLE_OK && (worst == NLE_OK || worst == NLE_ERR_NOCONV)) worst = s;
  }
  NLE_CUDA(h0, cudaStreamSynchronize(h0->stream));
  return worst;
}

extern "C" nle_status nle_batch_solve(int count, nle_t *hs, int p, double tol, int max_newton, int max_pcg,
                                      const double *const *X0s, double *const *lambdas, double *const *Vs,
                                      nle_status *per_problem) {
  if (count < 1 || !hs || !lambdas || !Vs) return fail(nullptr, NLE_ERR_ARG, "bad nle_batch_solve arguments");
  for (int b = 0; b < count; b++) {
    if (!hs[b]) return fail(nullptr, NLE_ERR_ARG, "NULL handle in the batch");
    if (!hs[b]->factored) return fail(hs[b], NLE_ERR_STATE, "nle_factor_ic has not been called");
    if (hs[b]->opt.precision != hs[0]->opt.precision || hs[b]->device != hs[0]->device)
      return fail(hs[b], NLE_ERR_ARG, "all handles of a batch need the same precision and device");
    if (hs[b]->chain != hs[0]->chain)
      return fail(hs[b], NLE_ERR_ARG,
                  "all handles of a batch need the same triangular-solve schedule (set nle_options.trsv_schedule)");
    if (hs[b]->grid > 8)
      return fail(hs[b], NLE_ERR_ARG, "batched handles must be factored for at most 8 CTAs (nle_options.grid_ctas <= 8)");
    if (p < 1 || p >= hs[b]->n || p > NLE_MAX_P || !lambdas[b] || !Vs[b])
      return fail(hs[b], NLE_ERR_ARG, "bad p or output pointer");
  }
  if (!(tol > 0) || max_newton < 0 || max_pcg < 1) return fail(hs[0], NLE_ERR_ARG, "bad tolerance or iteration caps");
  cudaSetDevice(hs[0]->device);
  return mixed(hs[0]) ? batch_impl<float>(count, hs, p, tol, max_newton, max_pcg, X0s, lambdas, Vs, per_problem)
                      : batch_impl<double>(count, hs, p, tol, max_newton, max_pcg, X0s, lambdas, Vs, per_problem);
}
