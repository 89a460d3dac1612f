// Device IC(lfil, tau_IC) factor: launch interface (kernel in nle_ict.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace nle {

constexpr int ICT_WARPS = 32;     // warps per CTA, one column per warp at a time
constexpr int ICT_LFIL_MAX = 31;  // a column's record (diagonal + lfil rows) fits one warp

enum { ICT_OK = 0, ICT_ERR_NOT_SPD = 1, ICT_ERR_CAPACITY = 2, ICT_ERR_TIMEOUT = 3 };

// Error word of one factor launch (zeroed by the host before the launch).
struct IctError {
  int code;       // ICT_*
  int pad;
  long long col;  // column at which it happened
};

// Dynamic shared memory of one CTA, and the largest co-resident grid.
int ict_smem_bytes();
int ict_max_grid(int nsm);

// Factor the n x n matrix (CSR on the device, both triangles, rows sorted)
// into records of lfil + 1 slots per column: crow/cval[j*(lfil+1) + t]
// (t = 0: the diagonal; then the kept rows ascending) and cnt[j] = entries
// of column j.  cnt, crow, cval must be filled with 0xFF bytes before the
// launch (count -1, row -1, value NaN: "not written yet").  Cooperative
// launch of `grid` CTAs (at most ict_max_grid).
cudaError_t ict_launch(int grid, int64_t n, const int64_t *rp, const int32_t *ci, const double *va, int lfil,
                       double tau, int *cnt, int *crow, double *cval, IctError *err, long long spin_ns,
                       cudaStream_t stream);

}  // namespace nle
