// Host-side internals shared by the C-ABI translation units: library-owned
// device buffers (through the caller's allocator hook or a private
// stream-ordered pool) and the status plumbing.
#pragma once

#include <cuda_runtime.h>

#include <memory>

#include "spmvat.h"

namespace spmvat {

struct Hooks {
    spmv_alloc_fn alloc = nullptr;
    spmv_free_fn free = nullptr;
    void *ctx = nullptr;
};

// One device allocation; freed on the stream it was made on when the last
// owner lets go of it.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    Hooks hooks;
    ~DevBuf() {
        if (!p) return;
        if (hooks.free) hooks.free(p, bytes, hooks.ctx, stream);
        else if (cudaFreeAsync(p, stream) != cudaSuccess) cudaGetLastError();
    }
};
using BufPtr = std::shared_ptr<DevBuf>;

// Stream-ordered allocation of at least `bytes` (rounded up to 256).
spmv_status alloc_buf(size_t bytes, cudaStream_t s, BufPtr *out);
// Device status word (ST_* bits) to an ABI status.
spmv_status status_from_dev(int st);

}  // namespace spmvat

#define CK(call)                                                               \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) { cudaGetLastError(); return SPMV_ERR_CUDA; }    \
    } while (0)
#define CKS(call)                                                              \
    do {                                                                       \
        spmv_status s_ = (call);                                               \
        if (s_ != SPMV_OK) return s_;                                          \
    } while (0)
