// Tr(A*B) without any device allocation.
//
// Some callers may not allocate device memory while they call into the
// library: a host application that hands the whole GPU memory to its own arena,
// code that records work into a CUDA graph and must not insert allocations into
// it, or a loop that cannot afford the allocator's bookkeeping.  For them this
// file provides a variant of dbcsr_trace_product whose scratch (one partial sum
// per block of A, then the per-CTA partials of the fixed reduction tree) lives in
// a file-scope device array instead of stream-ordered allocations.  The kernels,
// launch shapes and summation order are the ones dbcsr_trace_product uses, so
// the two return the same value.
#include <mutex>

#include "common.cuh"

namespace dbg {
namespace {

// Largest A the variant accepts: one partial per block.
constexpr int64_t kNoAllocMaxBlocks = 1 << 20;
constexpr int kMaxDevices = 64;

// 8 MB + 8 KB per device that loads the library, held until the process exits.
// Every word a call reads is written earlier by the same call, so nothing needs
// clearing between calls.
static __device__ __align__(256) double g_trace_scratch[kNoAllocMaxBlocks + kDetSumPartials];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_trace_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
double* scratch_of_current_device() {
    int dev = 0;
    DBG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(DBCSR_ECAPACITY, "trace_product_noalloc: device ordinal beyond 64");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_trace_scratch);
        if (e != cudaSuccess)
            fail(DBCSR_ECUDA, std::string("trace_product_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    return g_scratch_addr[dev];
}

}  // namespace
}  // namespace dbg

extern "C" dbcsr_status dbcsr_trace_product_noalloc(dbcsr_matrix A, dbcsr_matrix B, double* out_dev) {
    try {
        dbg::check_finalized(A);
        dbg::check_finalized(B);
        if (!out_dev) dbg::fail(DBCSR_EINVAL, "trace_product_noalloc: null output");
        if (A->h_bs != B->h_bs) dbg::fail(DBCSR_EINVAL, "trace_product_noalloc: block sizes differ");
        if (A->stream != B->stream) dbg::fail(DBCSR_EINVAL, "trace_product_noalloc: A and B must share a stream");
        if (A->nnzb > dbg::kNoAllocMaxBlocks)
            dbg::fail(DBCSR_ECAPACITY, "trace_product_noalloc: A has " + std::to_string(A->nnzb) +
                                           " blocks; at most 1048576 are supported");
        double* scratch = dbg::scratch_of_current_device();
        dbg::trace_product_parts_into(A, B, scratch, A->stream);
        dbg::det_sum_into(scratch, A->nnzb, scratch + dbg::kNoAllocMaxBlocks, out_dev, A->stream);
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        dbg::set_last_error(e.what());
        return DBCSR_EINVAL;
    }
}
