// Allocation-free application of the incomplete-Cholesky preconditioner,
// c = (L L^T)^{-1} g, for callers that must not allocate device memory.
//
// All temporary storage of this entry point lives in one file-scope device
// array (nle_noalloc_scratch): the intermediate vector z = L^{-1} g and an
// error word.  Host code never uses the array's name as an address; it asks
// the runtime for the array's device address once per device.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/nle.h"
#include "nle_device.cuh"

namespace {

constexpr int64_t kMaxN = NLE_NOALLOC_MAX_N;
constexpr int kMaxDevices = 64;

// z (kMaxN doubles) followed by a small control block (error word).
static __device__ __align__(256) double nle_noalloc_scratch[kMaxN + 32];

std::mutex g_mu;
double *g_scratch[kMaxDevices] = {nullptr};

// Set z and c to the not-yet-computed marker and clear the error word.
__global__ void k_na_fill(double *z, double *c, int64_t n, int *err) {
  const double sent = nle::sentinel<double>();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    z[i] = sent;
    c[i] = sent;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
}

// One warp per row, rows taken round-robin in order (ascending for the lower
// factor, descending for the upper one): a row only waits for rows owned by
// other warps that are resident (cooperative launch), so every wait ends.
// Entries whose column is not strictly below (above) the row, or outside
// [0, n), are skipped and reported; every wait is bounded.
template <bool LOWER>
__global__ void __launch_bounds__(256) k_na_solve(int64_t n, const int32_t *rp, const int32_t *col,
                                                  const double *val, const double *diag, const double *rhs,
                                                  double *x, int *err, long long lim_cycles) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = w; it < n; it += nw) {
    const int64_t r = LOWER ? it : n - 1 - it;
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    double acc = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const int64_t c = __ldg(col + e);
      const bool ok = LOWER ? (c >= 0 && c < r) : (c > r && c < n);
      if (!ok) {
        atomicCAS(err, 0, (int)NLE_ERR_CSR);
        continue;
      }
      double xv = nle::ld_relaxed(x + c);
      if (nle::is_sent(xv)) {
        const long long c0 = clock64();
        while (nle::is_sent(xv)) {
          xv = nle::ld_relaxed(x + c);
          if (nle::is_sent(xv) && clock64() - c0 > lim_cycles) {
            atomicCAS(err, 0, (int)NLE_ERR_TIMEOUT);
            xv = 0.0;
          }
        }
      }
      acc += __ldg(val + e) * xv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) nle::st_relaxed(x + r, (__ldg(rhs + r) - acc) / __ldg(diag + r));
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, nle_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

namespace nle {
void set_global_error(const std::string &msg);
}

extern "C" nle_status nle_ic_apply_noalloc(int64_t n, const int32_t *Lrp, const int32_t *Lcol, const double *Lval,
                                           const int32_t *Urp, const int32_t *Ucol, const double *Uval,
                                           const double *diag, const double *g, double *c, void *stream) {
  if (n < 1 || n > kMaxN) {
    char buf[160];
    snprintf(buf, sizeof buf, "nle_ic_apply_noalloc: n = %lld is outside 1..%lld (the size of its fixed scratch)",
             (long long)n, (long long)kMaxN);
    nle::set_global_error(buf);
    return NLE_ERR_ARG;
  }
  if (!Lrp || !Lcol || !Lval || !Urp || !Ucol || !Uval || !diag || !g || !c) {
    nle::set_global_error("nle_ic_apply_noalloc: NULL pointer");
    return NLE_ERR_ARG;
  }
  {
    // c is written (with the not-yet-computed marker) before g is read, so
    // the two may not share memory
    const uintptr_t g0 = (uintptr_t)g, c0 = (uintptr_t)c, nb = (uintptr_t)n * sizeof(double);
    if (g0 < c0 + nb && c0 < g0 + nb) {
      nle::set_global_error("nle_ic_apply_noalloc: g and c overlap (in-place application is not supported)");
      return NLE_ERR_ARG;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *z = nullptr;
  cudaError_t e = scratch_address(&z);
  if (e != cudaSuccess) {
    nle::set_global_error(std::string("nle_ic_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return NLE_ERR_CUDA;
  }
  int *err = reinterpret_cast<int *>(z + kMaxN);
  int dev = 0, nsm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) {
    nle::set_global_error("nle_ic_apply_noalloc: device lacks cooperative launch");
    return NLE_ERR_CUDA;
  }
  const long long lim = (long long)(2.0 * 2.1e9);  // ~2 s at the maximum SM clock
  // clear a launch error left pending by earlier work of the caller, so
  // that the check below reports this call's own launches
  (void)cudaGetLastError();
  k_na_fill<<<256, 256, 0, s>>>(z, c, n, err);
  e = cudaGetLastError();
  int64_t nn = n;
  const double *zc = z;
  void *fa[] = {&nn, (void *)&Lrp, (void *)&Lcol, (void *)&Lval, (void *)&diag, (void *)&g, (void *)&z, (void *)&err,
                (void *)&lim};
  void *ba[] = {&nn, (void *)&Urp, (void *)&Ucol, (void *)&Uval, (void *)&diag, (void *)&zc, (void *)&c, (void *)&err,
                (void *)&lim};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((void *)k_na_solve<true>, dim3(nsm), dim3(256), fa, 0, s);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((void *)k_na_solve<false>, dim3(nsm), dim3(256), ba, 0, s);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    nle::set_global_error(std::string("nle_ic_apply_noalloc: ") + cudaGetErrorString(e));
    return NLE_ERR_CUDA;
  }
  if (herr != 0) {
    nle::set_global_error(herr == NLE_ERR_CSR ? "nle_ic_apply_noalloc: an entry is not strictly triangular"
                                              : "nle_ic_apply_noalloc: a device wait ran out");
    return (nle_status)herr;
  }
  return NLE_OK;
}
