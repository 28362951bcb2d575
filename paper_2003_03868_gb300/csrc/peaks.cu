// FP64 rate microbenchmarks (no counterpart in the paper; they measure the
// pipes that bound the FP64 block products), the launch counter, and the self-test of the
// bounded device-side waits.
#include <atomic>

#include "common.cuh"
#include "dbcsr_gb_bench.h"
#include "tc05.cuh"

namespace dbg {

std::atomic<int64_t> g_launches{0};

namespace {

constexpr int kChains = 8;

__global__ void k_peak_dfma(int iters, double seed, double* sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-9 + c;
    const double b = 0.999999999, d = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == 12345.678) sink[blockIdx.x] = s;   // never true; keeps the loop alive
}

__global__ void k_peak_dmma(int iters, double seed, double* sink) {
    const double a = seed + threadIdx.x * 1e-9, b = 0.5 + threadIdx.x * 1e-9;
    double c[kChains / 2][2];
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) c[i][0] = c[i][1] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains / 2; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[i][0]), "+d"(c[i][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) s += c[i][0] + c[i][1];
    if (s == 12345.678) sink[blockIdx.x] = s;
}

}  // namespace

double bench_peak(int kind, int iters, int blocks, int threads) {
    if (iters < 1 || blocks < 1 || blocks > 65535 || threads < 32 || threads > 1024 || threads % 32)
        fail(DBCSR_EINVAL, "bench_peak: bad launch shape");
    if (kind != DBCSR_PEAK_DFMA && kind != DBCSR_PEAK_DMMA) fail(DBCSR_EINVAL, "bench_peak: unknown kind");
    cudaStream_t s = nullptr;
    DBuf<double> sink;
    sink.alloc(blocks, s);
    cudaEvent_t e0, e1;
    DBG_CK(cudaEventCreate(&e0));
    DBG_CK(cudaEventCreate(&e1));
    auto launch = [&](int it) {
        if (kind == DBCSR_PEAK_DFMA) k_peak_dfma<<<blocks, threads, 0, s>>>(it, 1.0, sink.p);
        else k_peak_dmma<<<blocks, threads, 0, s>>>(it, 1.0, sink.p);
        DBG_LAUNCH_CK();
    };
    launch(std::max(1, iters / 10));   // warm-up
    DBG_CK(cudaEventRecord(e0, s));
    launch(iters);
    DBG_CK(cudaEventRecord(e1, s));
    DBG_CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    DBG_CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double ops = (kind == DBCSR_PEAK_DFMA)
                           ? 2.0 * kChains * (double)iters * threads * blocks
                           : 512.0 * (kChains / 2) * (double)iters * (threads / 32) * blocks;
    return ops / (ms * 1e-3) * 1e-9;
}

// One warp: an mbarrier of count 1, thread 0 arrives first when `arrive`, then every lane
// waits (bounded, as the library's kernels do) for the first phase.  out[0] = 1 if the wait
// completed, out[1] = the cycles lane 0 waited.  No asynchronous copy or TMEM is involved,
// so giving up leaves nothing in flight.
__global__ void k_wait_selftest(long long limit, int arrive, int64_t* out) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) tc::mbar_arrive(&bar);
    const long long t0 = clock64();
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&bar, 0, limit));
    if (threadIdx.x == 0) {
        out[0] = ok ? 1 : 0;
        out[1] = clock64() - t0;
    }
}

}  // namespace dbg

extern "C" {

double dbcsr_bench_peak(int32_t kind, int32_t iters, int32_t blocks, int32_t threads) {
    try {
        return dbg::bench_peak(kind, iters, blocks, threads);
    } catch (const std::exception&) {
        return -1.0;
    }
}

int64_t dbcsr_launch_count(void) { return dbg::g_launches.load(); }

int32_t dbcsr_wait_selftest(int64_t limit_cycles, int32_t arrive, int64_t* waited) {
    try {
        if (limit_cycles < 0) dbg::fail(DBCSR_EINVAL, "wait_selftest: negative limit");
        int64_t* d = nullptr;
        DBG_CK(cudaMalloc(&d, 2 * sizeof(int64_t)));
        dbg::k_wait_selftest<<<1, 32>>>((long long)limit_cycles, arrive, d);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        int64_t h[2] = {0, 0};
        if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
        cudaFree(d);
        DBG_CK(e);
        if (waited) *waited = h[1];
        if (!h[0]) dbg::fail(DBCSR_ETIMEOUT, "wait_selftest: the wait ran out");
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

int32_t dbcsr_pool_usage(int64_t* used_now, int64_t* used_high, int32_t reset_high) {
    try {
        cudaMemPool_t pool = dbg::library_pool();
        uint64_t v = 0;
        if (used_now) {
            DBG_CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
            *used_now = (int64_t)v;
        }
        if (used_high) {
            DBG_CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v));
            *used_high = (int64_t)v;
        }
        if (reset_high) {
            uint64_t zero = 0;
            DBG_CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
        }
        dbg::set_last_error("");
        return DBCSR_OK;
    } catch (const dbg::Error& e) {
        dbg::set_last_error(e.what());
        return e.code;
    }
}

}  // extern "C"
