// FP64 rate microbenchmarks (no counterpart in the paper; they measure the
// pipes that bound the FP64 block products) and the launch counter.
#include <atomic>

#include "common.cuh"
#include "dbcsr_gb_bench.h"

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
