// COO-Row SpMV that allocates no device memory.
//
// Some callers cannot allocate device memory when they multiply: solvers that
// reserve all of their memory up front (a fixed arena owned by a host
// framework) and must not grow it afterwards, and latency-critical loops in
// which an allocation may block on the driver or fail under memory pressure
// between two iterations. spmv_apply on a COO-Row handle takes a small
// temporary buffer (the partial sums of rows that cross tile boundaries) from
// the library's pool on every call; this entry point uses a fixed array in
// device memory instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (SPMV_NOALLOC_SCRATCH_BYTES) until the process exits. All
// calls share it, so calls whose kernels overlap on a device (different
// streams, or several host threads) race on it and must be ordered by the
// caller. Its contents survive from call to call; nothing in it has to start
// at zero, because each call writes every slot it later reads.
#include <mutex>

#include "common.cuh"
#include "spmvat.h"

using namespace spmvat;

namespace {

constexpr size_t kScratchBytes = SPMV_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_coo_carry_scratch[kScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[64] = {};  // device address of the array, per device

// Host code may not use g_coo_carry_scratch as a device pointer (on the host
// it names a stand-in object). Its device address is looked up once per
// device, with that device current, and kept: it stays valid as long as the
// device's primary context lives, so a cudaDeviceReset (which destroys that
// context) makes it stale, and the header tells callers not to call this
// entry point after one.
spmv_status scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SPMV_ERR_CUDA; }
    if (dev < 0 || dev >= 64) return SPMV_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_coo_carry_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SPMV_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SPMV_OK;
}

}  // namespace

extern "C" spmv_status spmv_apply_coo_row_noalloc(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                                  const int32_t *irow, const int32_t *icol, const double *val,
                                                  const double *x, double *y, spmv_stream_t stream) {
    if (n_rows <= 0 || n_cols <= 0 || nnz < 0) return SPMV_ERR_INVALID_ARG;
    if (nnz > SPMV_NOALLOC_COO_MAX_NNZ || coo_row_scratch_bytes(nnz) > kScratchBytes) return SPMV_ERR_UNSUPPORTED;
    if (!x || !y || (nnz > 0 && (!irow || !icol || !val))) return SPMV_ERR_INVALID_ARG;
    void *scratch = nullptr;
    spmv_status st = scratch_for_current_device(&scratch);
    if (st != SPMV_OK) return st;
    if (launch_spmv_coo_row(irow, icol, val, nnz, n_rows, n_cols, x, y, scratch, nullptr,
                            reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return SPMV_ERR_CUDA;
    }
    return SPMV_OK;
}
